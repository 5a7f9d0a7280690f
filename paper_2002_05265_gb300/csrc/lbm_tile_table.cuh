// Instantiates the bulk-copy staged step kernel for one storage type (stages 2, 3, 4; form 0
// general, form 1 the light 16-bit form).
#pragma once
#include "lbm_tile.cuh"

namespace lbm {
template <typename S, int FORM>
static const void* tile_kernel_table(bool shifted, int stages) {
    switch (stages) {
        case 2: return shifted ? (const void*)tile_step_kernel<S, true, 2, FORM> : (const void*)tile_step_kernel<S, false, 2, FORM>;
        case 3: return shifted ? (const void*)tile_step_kernel<S, true, 3, FORM> : (const void*)tile_step_kernel<S, false, 3, FORM>;
        case 4: return shifted ? (const void*)tile_step_kernel<S, true, 4, FORM> : (const void*)tile_step_kernel<S, false, 4, FORM>;
        default: return nullptr;
    }
}
}  // namespace lbm
