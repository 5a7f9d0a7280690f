// Instantiates the bulk-copy staged step kernel for one storage type and kernel form (stages
// 2, 3, 4; both shift families) and describes it to the host.
#pragma once
#include "lbm_tile.cuh"
#include "lbm_internal.h"

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
template <typename S, int FORM>
static bool tile_kernel_info(bool shifted, int stages, TileKernelInfo* out) {
    out->kernel = tile_kernel_table<S, FORM>(shifted, stages);
    out->threads = TileForm<S, FORM>::THREADS;
    out->width = Tile<S, TileForm<S, FORM>::CW>::W;
    out->smem = tile_smem_bytes<S, FORM>(stages);
    return out->kernel != nullptr;
}
}  // namespace lbm
