// Batched persistent sweep kernels for __nv_bfloat16 population storage, one per (VEC, BLOCK) shape
// the autotuner may choose.
#include "lbm_batch.cuh"
#include "lbm_internal.h"

namespace lbm {
const void* batch_kernel_bf16(int vec, int block) {
    if (vec == 8 && block == 256) return (const void*)batch_kernel<__nv_bfloat16, 8, 256>;
    if (vec == 8 && block == 128) return (const void*)batch_kernel<__nv_bfloat16, 8, 128>;
    if (vec == 4 && block == 256) return (const void*)batch_kernel<__nv_bfloat16, 4, 256>;
    if (vec == 4 && block == 128) return (const void*)batch_kernel<__nv_bfloat16, 4, 128>;
    return nullptr;
}
}  // namespace lbm
