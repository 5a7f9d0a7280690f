// Step kernels (all collision models) for float population storage.
#include "lbm_step_table.cuh"
#include "lbm_internal.h"

namespace lbm {
const void* step_kernel_f32(int model, int eq_order, bool shifted) {
    return step_kernel_table<float>(model, eq_order, shifted);
}
const void* group_kernel_f32(bool shifted) { return group_kernel_table<float>(shifted); }
}  // namespace lbm
