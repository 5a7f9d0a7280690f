// Host-side declarations shared by the library's translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>

namespace lbm {

struct StepArgs;

// Step kernel entry for (storage, model, equilibrium order); nullptr if not instantiated.
const void* step_kernel_f64(int model, int eq_order);
const void* step_kernel_f32(int model, int eq_order);
const void* step_kernel_f16(int model, int eq_order);
const void* step_kernel_bf16(int model, int eq_order);

// Vector width (nodes per thread) of the step kernel for a storage type.
int storage_vec(int storage);
// Bytes per stored population.
int storage_bytes(int storage);

// Auxiliary kernels (lbm_aux.cu).  Pointers are device pointers; fields are dense [ny][nx].
struct FieldArgs {
    int nx, ny, pitch;
    long long plane;
    double rho0;
};
// f(x) = f^eq(rho(x), u(x)) (eq_order 2 or 4), scattered so the next pull gathers it.
cudaError_t launch_init_eq(int storage, void* buf, const FieldArgs& a, int eq_order,
                           const double* rho, const double* ux, const double* uy, cudaStream_t s);
// Write the canonical populations f[9][ny][nx] (FP64, unshifted) into the buffer.
cudaError_t launch_scatter(int storage, void* buf, const FieldArgs& a, const double* f, cudaStream_t s);
// Gather the pre-collision state: populations (f != nullptr) and/or moments (each optional).
cudaError_t launch_gather(int storage, const void* buf, const FieldArgs& a, double* f,
                          double* rho, double* ux, double* uy, double* pxx, double* pxy, double* pyy,
                          cudaStream_t s);
// FP64 reductions: pass 1 writes `blocks` x 8 partials, pass 2 folds them into out[8] and
// applies the blow-up criterion to status[0] (int) / blowup_step[0].
struct CheckArgs {
    double ke_ref, ke_factor, uref_x, uref_y;
    long long step;
    int apply;       // evaluate the criterion
};
int reduce_blocks();
cudaError_t launch_reduce(int storage, const void* buf, const FieldArgs& a, double* partials,
                          double* out8, int* status, long long* blowup_step, const CheckArgs& c,
                          cudaStream_t s);

}  // namespace lbm
