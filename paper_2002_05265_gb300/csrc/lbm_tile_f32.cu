// Bulk-copy staged step kernels for float population storage (general form; the light form
// is in lbm_tile_f32_light.cu).
#include "lbm_tile_table.cuh"
#include "lbm_internal.h"

namespace lbm {
const void* tile_kernel_f32_light(bool shifted, int stages);
const void* tile_kernel_f32(bool shifted, int stages, bool light) {
    return light ? tile_kernel_f32_light(shifted, stages) : tile_kernel_table<float, 0>(shifted, stages);
}
}  // namespace lbm
