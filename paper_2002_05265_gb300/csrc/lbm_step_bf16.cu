// Step kernels (all collision models) for __nv_bfloat16 population storage.
#include "lbm_step_table.cuh"
#include "lbm_internal.h"

namespace lbm {
const void* step_kernel_bf16(int model, int eq_order, bool shifted) {
    return step_kernel_table<__nv_bfloat16>(model, eq_order, shifted);
}
const void* group_kernel_bf16(bool shifted) { return group_kernel_table<__nv_bfloat16>(shifted); }
}  // namespace lbm
