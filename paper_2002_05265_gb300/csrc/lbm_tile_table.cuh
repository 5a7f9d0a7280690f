// Instantiates the bulk-copy staged step kernel for one storage type (stages 2, 3, 4).
#pragma once
#include "lbm_tile.cuh"

namespace lbm {
template <typename S>
static const void* tile_kernel_table(bool shifted, int stages) {
    switch (stages) {
        case 2: return shifted ? (const void*)tile_step_kernel<S, true, 2> : (const void*)tile_step_kernel<S, false, 2>;
        case 3: return shifted ? (const void*)tile_step_kernel<S, true, 3> : (const void*)tile_step_kernel<S, false, 3>;
        case 4: return shifted ? (const void*)tile_step_kernel<S, true, 4> : (const void*)tile_step_kernel<S, false, 4>;
        default: return nullptr;
    }
}
}  // namespace lbm
