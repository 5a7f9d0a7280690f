// Bulk-copy staged step kernels for __half population storage.
#include "lbm_tile_table.cuh"
#include "lbm_internal.h"

namespace lbm {
const void* tile_kernel_f16(bool shifted, int stages) { return tile_kernel_table<__half>(shifted, stages); }
}  // namespace lbm
