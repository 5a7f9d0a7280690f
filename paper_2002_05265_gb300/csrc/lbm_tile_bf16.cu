// Bulk-copy staged step kernels for __nv_bfloat16 population storage.
#include "lbm_tile_table.cuh"
#include "lbm_internal.h"

namespace lbm {
const void* tile_kernel_bf16(bool shifted, int stages) { return tile_kernel_table<__nv_bfloat16>(shifted, stages); }
}  // namespace lbm
