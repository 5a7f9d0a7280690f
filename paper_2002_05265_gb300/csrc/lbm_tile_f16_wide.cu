// Bulk-copy staged step kernels for __half population storage, wide form (16 consumer warps,
// one CTA per SM; one-step launches).
#include "lbm_tile_table.cuh"

namespace lbm {
bool tile_kernel_f16_wide(bool shifted, int stages, TileKernelInfo* out) {
    return tile_kernel_info<__half, 2>(shifted, stages, out);
}
}  // namespace lbm
