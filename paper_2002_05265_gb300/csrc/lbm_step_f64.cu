// Step kernels (all collision models) for double population storage.
#include "lbm_step_table.cuh"
#include "lbm_internal.h"

namespace lbm {
const void* step_kernel_f64(int model, int eq_order, bool shifted) {
    return step_kernel_table<double>(model, eq_order, shifted);
}
const void* group_kernel_f64(bool shifted) { return group_kernel_table<double>(shifted); }
}  // namespace lbm
