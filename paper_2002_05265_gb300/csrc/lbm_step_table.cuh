// Instantiates the step kernel of every collision model for one storage type.
#pragma once
#include "lbm_device.cuh"

namespace lbm {
template <typename S>
static const void* step_kernel_table(int model, int eq_order) {
    if (eq_order == 2) return model == BGK ? (const void*)step_kernel<BGK, 2, S> : nullptr;
    if (eq_order != 4) return nullptr;
    switch (model) {
        case BGK: return (const void*)step_kernel<BGK, 4, S>;
        case RM:  return (const void*)step_kernel<RM, 4, S>;
        case HM:  return (const void*)step_kernel<HM, 4, S>;
        case CM:  return (const void*)step_kernel<CM, 4, S>;
        case CHM: return (const void*)step_kernel<CHM, 4, S>;
        case CUM: return (const void*)step_kernel<CUM, 4, S>;
        case PR:  return (const void*)step_kernel<PR, 4, S>;
        case RR:  return (const void*)step_kernel<RR, 4, S>;
        default:  return nullptr;
    }
}
}  // namespace lbm
