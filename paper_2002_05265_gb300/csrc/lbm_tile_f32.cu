// Bulk-copy staged step kernels for float population storage.
#include "lbm_tile_table.cuh"
#include "lbm_internal.h"

namespace lbm {
const void* tile_kernel_f32(bool shifted, int stages, bool) { return tile_kernel_table<float, 0>(shifted, stages); }
}  // namespace lbm
