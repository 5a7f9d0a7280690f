// Bulk-copy staged step kernels for float population storage, light form (BGK, RM, HM, PR).
#include "lbm_tile_table.cuh"

namespace lbm {
bool tile_kernel_f32_light(bool shifted, int stages, TileKernelInfo* out) {
    return tile_kernel_info<float, 1>(shifted, stages, out);
}
}  // namespace lbm
