// Bulk-copy staged step kernels for float population storage, light form (BGK, RM, HM, PR).
#include "lbm_tile_table.cuh"
#include "lbm_internal.h"

namespace lbm {
const void* tile_kernel_f32_light(bool shifted, int stages) { return tile_kernel_table<float, 1>(shifted, stages); }
}  // namespace lbm
