// Bulk-copy staged step kernels for __nv_bfloat16 population storage, light form (BGK, RM, HM, PR).
#include "lbm_tile_table.cuh"

namespace lbm {
bool tile_kernel_bf16_light(bool shifted, int stages, TileKernelInfo* out) {
    return tile_kernel_info<__nv_bfloat16, 1>(shifted, stages, out);
}
}  // namespace lbm
