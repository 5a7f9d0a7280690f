// Batched persistent sweep kernels for double population storage, one per (VEC, BLOCK) shape
// the autotuner may choose.
#include "lbm_batch.cuh"
#include "lbm_internal.h"

namespace lbm {
const void* batch_kernel_f64(int vec, int block) {
    if (vec == 2 && block == 256) return (const void*)batch_kernel<double, 2, 256>;
    return nullptr;
}
}  // namespace lbm
