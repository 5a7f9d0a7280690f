// Bulk-copy staged step kernels for double population storage (general form only).
#include "lbm_tile_table.cuh"

namespace lbm {
bool tile_kernel_f64(bool shifted, int stages, int form, TileKernelInfo* out) {
    return form == 0 && tile_kernel_info<double, 0>(shifted, stages, out);
}
}  // namespace lbm
