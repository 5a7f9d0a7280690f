// Instantiates the step kernels of every collision model for one storage type.
#pragma once
#include "lbm_device.cuh"

namespace lbm {
template <typename S, bool SH>
static const void* step_kernel_table_sh(int model, int eq_order) {
    if (eq_order == 2) return (model == BGK && !SH) ? (const void*)step_kernel<BGK, 2, S, false> : nullptr;
    if (eq_order == 3) return (model == BGK && !SH) ? (const void*)step_kernel<BGK, 3, S, false> : nullptr;
    if (eq_order != 4) return nullptr;
    switch (model) {
        case BGK: return (const void*)step_kernel<BGK, 4, S, SH>;
        case RM:  return (const void*)step_kernel<RM, 4, S, SH>;
        case HM:  return (const void*)step_kernel<HM, 4, S, SH>;
        case CM:  return (const void*)step_kernel<CM, 4, S, SH>;
        case CHM: return (const void*)step_kernel<CHM, 4, S, SH>;
        case CUM: return (const void*)step_kernel<CUM, 4, S, SH>;
        case PR:  return (const void*)step_kernel<PR, 4, S, SH>;
        case RR:  return (const void*)step_kernel<RR, 4, S, SH>;
        default:  return nullptr;
    }
}
template <typename S>
static const void* step_kernel_table(int model, int eq_order, bool shifted) {
    return shifted ? step_kernel_table_sh<S, true>(model, eq_order) : step_kernel_table_sh<S, false>(model, eq_order);
}
template <typename S>
static const void* group_kernel_table(bool shifted) {
    return shifted ? (const void*)group_step_kernel<S, true> : (const void*)group_step_kernel<S, false>;
}
}  // namespace lbm
