// Bulk-copy staged step kernels for __half population storage, light form (BGK, RM, HM, PR).
#include "lbm_tile_table.cuh"

namespace lbm {
bool tile_kernel_f16_light(bool shifted, int stages, TileKernelInfo* out) {
    return tile_kernel_info<__half, 1>(shifted, stages, out);
}
}  // namespace lbm
