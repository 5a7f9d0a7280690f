// Step kernels (all collision models) for __half population storage.
#include "lbm_step_table.cuh"
#include "lbm_internal.h"

namespace lbm {
const void* step_kernel_f16(int model, int eq_order, bool shifted) {
    return step_kernel_table<__half>(model, eq_order, shifted);
}
const void* group_kernel_f16(bool shifted) { return group_kernel_table<__half>(shifted); }
}  // namespace lbm
