// Bulk-copy staged step kernels for __nv_bfloat16 population storage, wide form (16 consumer warps,
// one CTA per SM; one-step launches).
#include "lbm_tile_table.cuh"

namespace lbm {
bool tile_kernel_bf16_wide(bool shifted, int stages, TileKernelInfo* out) {
    return tile_kernel_info<__nv_bfloat16, 2>(shifted, stages, out);
}
}  // namespace lbm
