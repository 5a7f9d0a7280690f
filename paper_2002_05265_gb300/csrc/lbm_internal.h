// Host-side declarations shared by the library's translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>

namespace lbm {

struct StepArgs;

// Step kernel entry for (storage, model, equilibrium order, non-default shift); nullptr if not
// instantiated.
const void* step_kernel_f64(int model, int eq_order, bool shifted);
const void* step_kernel_f32(int model, int eq_order, bool shifted);
const void* step_kernel_f16(int model, int eq_order, bool shifted);
const void* step_kernel_bf16(int model, int eq_order, bool shifted);
// Multi-lattice step kernel (group_step_kernel<S>, one GroupArgs parameter) per storage.
const void* group_kernel_f64(bool shifted);
const void* group_kernel_f32(bool shifted);
const void* group_kernel_f16(bool shifted);
const void* group_kernel_bf16(bool shifted);

// Bulk-copy staged step kernel (tile_step_kernel<S, shifted, stages, form>, one TileArgs
// parameter) per storage; stages 2-4; form 0 general (every model, several CTAs per SM),
// 1 light (lattices that all run BGK, RM, HM or PR; one-step launches), 2 wide (every model,
// one CTA per SM; one-step launches).  FP64 has form 0 only.  False if not instantiated.
struct TileKernelInfo {
    const void* kernel;
    int threads;   // CTA size
    int width;     // nodes per tile (W)
    int smem;      // dynamic shared memory bytes
};
bool tile_kernel_f64(bool shifted, int stages, int form, TileKernelInfo* out);
bool tile_kernel_f32(bool shifted, int stages, int form, TileKernelInfo* out);
bool tile_kernel_f16(bool shifted, int stages, int form, TileKernelInfo* out);
bool tile_kernel_bf16(bool shifted, int stages, int form, TileKernelInfo* out);

// Batched persistent sweep kernel for (vector width, CTA size); nullptr if not instantiated.
const void* batch_kernel_f64(int vec, int block);
const void* batch_kernel_f32(int vec, int block);
const void* batch_kernel_f16(int vec, int block);
const void* batch_kernel_bf16(int vec, int block);

// Vector width (nodes per thread) of the step kernel for a storage type.
int storage_vec(int storage);
// Bytes per stored population.
int storage_bytes(int storage);

// Auxiliary kernels (lbm_aux.cu).  Pointers are device pointers; fields are dense [ny][nx].
struct FieldArgs {
    int nx, ny, pitch;
    long long plane;
    double rho0;         // shift s_i = rho0 phi(u_ref,x) phi(u_ref,y)
    double urx, ury;
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
// applies the blow-up criterion to status[0] (int) / blowup_step[0].  With a completion
// counter (zero before the first launch; each launch leaves it zero) the last block of pass 1
// runs pass 2 itself; without one, pass 2 is a second launch.
struct CheckArgs {
    double ke_ref, ke_factor, uref_x, uref_y;
    long long step;
    int apply;       // evaluate the criterion
};
int reduce_blocks();
// bytes of a context's reduction scratch: the partials, then the counter at offset
// 8 * 8 * reduce_blocks()
size_t reduce_scratch_bytes();
cudaError_t launch_reduce(int storage, const void* buf, const FieldArgs& a, double* partials, unsigned* counter,
                          double* out8, int* status, long long* blowup_step, const CheckArgs& c,
                          cudaStream_t s);
// The fused checks (with completion counters) of up to kReduceGroupMax lattices of one
// storage type, 16-byte aligned rows, in one launch; each job's results are those of its own
// launch_reduce up to the rounding of the FP64 sums (fewer blocks per job, a fixed fold order).
// cudaErrorInvalidValue for an unaligned job or a missing counter.
constexpr int kReduceGroupMax = 16;
struct ReduceJob {
    const void* buf;
    FieldArgs a;
    double* partials;
    unsigned* counter;
    double* out;
    int* status;
    long long* blowup_step;
    CheckArgs c;
};
struct ReduceGroupArgs {
    int n;
    ReduceJob j[kReduceGroupMax];
};
cudaError_t launch_reduce_group(int storage, const ReduceGroupArgs& g, cudaStream_t s);

// Halo rows of a y-slab (lbm_halo_pack / lbm_halo_unpack): messages of [3][nx] raw storage
// elements; pack reads rows ny - 2 (planes 2, 5, 6 -> up) and 1 (planes 4, 7, 8 -> down), unpack
// writes up into row 0 (planes 2, 5, 6) and down into row ny - 1 (planes 4, 7, 8).
cudaError_t launch_halo(int storage, void* buf, const FieldArgs& a, void* up, void* down, bool pack, cudaStream_t s);

// Discrete adjoint (lbm_adjoint.cu).
struct AdjArgs {
    int nx, ny, pitch, nseg;
    long long plane;
    double w_nu, w3, w4, rho0;
    double urx, ury;     // storage shift velocity
    double cd[18];       // collision constants as in StepArgs (fill_consts), FP64 and FP32
    float cf[18];
};
struct AdjointPlan {
    int storage;            // LBM_F64 or LBM_F32 (lambda kept in the collision precision)
    AdjArgs a;
    const void* step_fwd;   // forward step kernel (src, dst, StepArgs), default shift
    const void* step_adj;   // adjoint step kernel of the model
    int grid_fwd, grid_adj, block;
    const void* step_fused; // adjoint step + next segment's forward step in one launch
    int grid_fused, nadj_fused;   // its grid and adjoint blocks (0: not available)
};
int adjoint_plan(int storage, int model, int kread, int nx, int ny, int pitch, long long plane, double w, double w3,
                 double w4, double rho0, double urx, double ury, AdjointPlan* p);
cudaError_t adjoint_launch_fwd(const AdjointPlan& p, const StepArgs& sa, const void* src, void* dst, cudaStream_t s);
cudaError_t adjoint_launch_step(const AdjointPlan& p, const void* state, const void* lam_in, void* lam_out,
                                double* rate_part, cudaStream_t s);
// One adjoint step (state, lam_in -> lam_out) and one forward step (fsrc -> fdst) in one launch.
cudaError_t adjoint_launch_fused(const AdjointPlan& p, const void* state, const void* lam_in, void* lam_out,
                                 double* rate_part, const StepArgs& sa, const void* fsrc, void* fdst, cudaStream_t s);
int adjoint_seed_blocks();
cudaError_t adjoint_launch_seed(const AdjointPlan& p, const void* state, int loss, const double* uxt,
                                const double* uyt, void* lam, double* loss_part, cudaStream_t s);
cudaError_t adjoint_launch_init(const AdjointPlan& p, const void* state0, const void* lam, double* gux, double* guy,
                                cudaStream_t s);

}  // namespace lbm
