// Batched persistent sweep kernels for float population storage, one per (VEC, BLOCK) shape
// the autotuner may choose.
#include "lbm_batch.cuh"
#include "lbm_internal.h"

namespace lbm {
const void* batch_kernel_f32(int vec, int block) {
    if (vec == 4 && block == 256) return (const void*)batch_kernel<float, 4, 256>;
    if (vec == 4 && block == 128) return (const void*)batch_kernel<float, 4, 128>;
    if (vec == 4 && block == 512) return (const void*)batch_kernel<float, 4, 512>;
    if (vec == 2 && block == 256) return (const void*)batch_kernel<float, 2, 256>;
    if (vec == 2 && block == 128) return (const void*)batch_kernel<float, 2, 128>;
    if (vec == 2 && block == 512) return (const void*)batch_kernel<float, 2, 512>;
    return nullptr;
}
}  // namespace lbm
