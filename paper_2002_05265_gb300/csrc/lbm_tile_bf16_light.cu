// Bulk-copy staged step kernels for __nv_bfloat16 population storage, light form (BGK, RM, HM, PR).
#include "lbm_tile_table.cuh"
#include "lbm_internal.h"

namespace lbm {
const void* tile_kernel_bf16_light(bool shifted, int stages) { return tile_kernel_table<__nv_bfloat16, 1>(shifted, stages); }
}  // namespace lbm
