// Bulk-copy staged step kernels for double population storage.
#include "lbm_tile_table.cuh"
#include "lbm_internal.h"

namespace lbm {
const void* tile_kernel_f64(bool shifted, int stages, bool) { return tile_kernel_table<double, 0>(shifted, stages); }
}  // namespace lbm
