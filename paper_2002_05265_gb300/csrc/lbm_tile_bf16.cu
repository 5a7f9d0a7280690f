// Bulk-copy staged step kernels for __nv_bfloat16 population storage, general form (the light
// and wide forms are in lbm_tile_bf16_light.cu and lbm_tile_bf16_wide.cu, compiled in parallel).
#include "lbm_tile_table.cuh"

namespace lbm {
bool tile_kernel_bf16_light(bool shifted, int stages, TileKernelInfo* out);
bool tile_kernel_bf16_wide(bool shifted, int stages, TileKernelInfo* out);
bool tile_kernel_bf16(bool shifted, int stages, int form, TileKernelInfo* out) {
    switch (form) {
        case 0: return tile_kernel_info<__nv_bfloat16, 0>(shifted, stages, out);
        case 1: return tile_kernel_bf16_light(shifted, stages, out);
        case 2: return tile_kernel_bf16_wide(shifted, stages, out);
        default: return false;
    }
}
}  // namespace lbm
