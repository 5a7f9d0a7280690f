// Bulk-copy staged step kernels for __half population storage (general form; the light form is in lbm_tile_f16_light.cu).
#include "lbm_tile_table.cuh"
#include "lbm_internal.h"

namespace lbm {
const void* tile_kernel_f16_light(bool shifted, int stages);
const void* tile_kernel_f16(bool shifted, int stages, bool light) {
    return light ? tile_kernel_f16_light(shifted, stages) : tile_kernel_table<__half, 0>(shifted, stages);
}
}  // namespace lbm
