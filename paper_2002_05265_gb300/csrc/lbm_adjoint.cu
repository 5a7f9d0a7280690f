// Discrete adjoint of the stream-and-collide iteration (lbm_adjoint_run in include/lbm.h).
//
// With f^{n+1}_i(x + xi_i) = C_i(f^n(x)) (Eq. StreamCollide) and a loss L(f^N), the adjoint
// lambda^n = dL/df^n obeys
//     lambda^n_j(x) = sum_i lambda^{n+1}_i(x + xi_i) dC_i/df_j(f^n(x))
// (reverse streaming, then the transposed per-node collision Jacobian of App. A), and the
// rate sensitivities are dL/domega_k = sum_n sum_x sum_i lambda^{n+1}_i(x + xi_i) dC_i/domega_k.
// The initial velocity enters through f^0 = f^eq(rho0, u0):
//     dL/du0_a(x) = sum_i lambda^0_i(x) df^eq_i/du_a(rho0(x), u0(x)).
//
// Memory: the forward run stores a checkpoint of the state every K steps (K ~ sqrt(N)); the
// backward sweep restores each segment's checkpoint, recomputes the K states of the segment
// into a ring of buffers, then runs the K adjoint steps backwards.  lambda is stored densely
// per node (canonical layout, same row pitch as the populations) in the collision precision.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <vector>

#include "lbm.h"
#include "lbm_adjoint.cuh"
#include "lbm_internal.h"

namespace lbm {
namespace {

constexpr int kAdjBlock = 256;
// Resident 256-thread blocks per SM the compiler must allow, which sets its register budget:
// 2 (at most 128 registers a thread) for the FP32 and 16-bit kernels, whose register
// allocation then runs the 512 x 512 adjoint 2-10 % faster than with the budget unstated
// or capped at 80; unstated for FP64.
#ifndef LBM_ADJ_MIN_BLOCKS
#define LBM_ADJ_MIN_BLOCKS 2
#endif
template <typename S> constexpr int kAdjMinBlocks = sizeof(S) == 8 ? 0 : LBM_ADJ_MIN_BLOCKS;

// Nodes per thread of the adjoint step: it holds the populations and the adjoints of every
// node it handles, so it uses half the vector width of the forward kernel (FP32: 2 nodes,
// FP64: 1 node) to keep its registers, and so its occupancy, close to the forward kernel's.
#ifndef LBM_ADJ_VEC_DIV
#define LBM_ADJ_VEC_DIV 2
#endif
template <typename S> struct AdjVec {
    static constexpr int value = DefaultVec<S>::value / LBM_ADJ_VEC_DIV > 0 ? DefaultVec<S>::value / LBM_ADJ_VEC_DIV : 1;
};

template <typename T> __device__ __forceinline__ const T* adj_consts(const AdjArgs& a);
template <> __device__ __forceinline__ const float* adj_consts<float>(const AdjArgs& a) { return a.cf; }
template <> __device__ __forceinline__ const double* adj_consts<double>(const AdjArgs& a) { return a.cd; }

// One adjoint step: lam_out = J^T (reverse-streamed lam_in) at every node, done by `nblk`
// blocks of which this is block `blk`; the rate sensitivities are accumulated into this
// block's FP64 slot of `rate_part` (3 per block).
template <int MODEL, typename S>
__device__ __forceinline__ void adjoint_body(const S* __restrict__ state, const typename Conv<S>::T* __restrict__ lam_in,
                                             typename Conv<S>::T* __restrict__ lam_out, const AdjArgs& a,
                                             double* __restrict__ rate_part, unsigned blk, unsigned nblk) {
    using T = typename Conv<S>::T;
    constexpr int VEC = AdjVec<S>::value;
    const int lane = threadIdx.x & 31;
    const int nseg = (a.nx + VEC - 1) / VEC;
    const unsigned total = (unsigned)a.ny * (unsigned)nseg;
    const unsigned stride = nblk * blockDim.x;
    // constants precomputed on the host in both precisions (no FP64 set-up in the kernel)
    const T* ct = adj_consts<T>(a);
    VjpConsts<T> vc;
    vc.w = ct[0]; vc.w3 = ct[1]; vc.w4 = ct[2]; vc.rho0 = ct[3]; vc.urx = ct[4]; vc.ury = ct[5];
    vc.Xr = ct[12]; vc.Yr = ct[13];
    vc.kap = ct[16]; vc.kapw = ct[17];
    // per-thread sums in the collision precision (a thread handles a few nodes), FP64 from
    // the block fold on
    T acc[3] = {T(0), T(0), T(0)};
    for (unsigned base = blk * blockDim.x + (threadIdx.x & ~31u); base < total; base += stride) {
        const unsigned s = base + lane;
        const bool active = s < total;
        const unsigned sc = active ? s : total - 1;
        const int y = (int)(sc / (unsigned)nseg);
        const int seg = (int)(sc - (unsigned)y * (unsigned)nseg);
        const int x0 = seg * VEC;
        const int nvalid = min(VEC, a.nx - x0);
        T f[9][VEC], l[9][VEC];
        gather_pull<S, VEC, 1>(state, a.nx, a.ny, a.pitch, a.plane, y, seg, nseg, x0, nvalid, lane, f);
        gather_pull<T, VEC, -1>(lam_in, a.nx, a.ny, a.pitch, a.plane, y, seg, nseg, x0, nvalid, lane, l);
        T out[9][VEC];
#pragma unroll
        for (int j = 0; j < VEC; ++j) {
            T g[9], v[9], gb[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) { g[i] = f[i][j]; v[i] = l[i][j]; }
            T wb, w3b, w4b;
            collide_vjp<MODEL, T>(g, v, gb, vc, wb, w3b, w4b);
#pragma unroll
            for (int i = 0; i < 9; ++i) out[i][j] = gb[i];
            if (active && j < nvalid) {
                acc[0] += wb;
                acc[1] += w3b;
                acc[2] += w4b;
            }
        }
        if (active) {
#pragma unroll
            for (int i = 0; i < 9; ++i)
                vstore<T, VEC>(lam_out + (long long)i * a.plane + (long long)y * a.pitch + x0, out[i]);
        }
    }
    // warp sums in the collision precision (32 per-thread sums of a few nodes), FP64 from the
    // block fold on: GB300's FP64 pipe is narrow, per-thread FP64 work would dominate
    __shared__ double sh[kAdjBlock / 32][3];
    const int warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        T x = acc[k];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) sh[warp][k] = (double)x;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double x = 0.0;
        for (int w2 = 0; w2 < kAdjBlock / 32; ++w2) x += sh[w2][threadIdx.x];
        rate_part[blk * 3 + threadIdx.x] += x;
    }
}

template <int MODEL, typename S>
__global__ void __launch_bounds__(kAdjBlock, kAdjMinBlocks<S>) adjoint_step_kernel(const S* __restrict__ state,
                                                                 const typename Conv<S>::T* __restrict__ lam_in,
                                                                 typename Conv<S>::T* __restrict__ lam_out,
                                                                 AdjArgs a, double* __restrict__ rate_part) {
    adjoint_body<MODEL, S>(state, lam_in, lam_out, a, rate_part, blockIdx.x, gridDim.x);
}

// One adjoint step of one checkpoint segment and, in the same launch, one recomputed forward
// step of the next segment (independent work: the next segment's states go to the other
// ring of buffers).  Blocks [0, nadj) run the adjoint step, the others the forward step, so
// the two latency-bound passes share the SMs instead of following one another.
template <int MODEL, typename S, bool SHIFT>
__global__ void __launch_bounds__(kAdjBlock, kAdjMinBlocks<S>) adjoint_fused_kernel(const S* __restrict__ state,
                                                                  const typename Conv<S>::T* __restrict__ lam_in,
                                                                  typename Conv<S>::T* __restrict__ lam_out,
                                                                  AdjArgs a, double* __restrict__ rate_part,
                                                                  unsigned nadj, const S* __restrict__ fsrc,
                                                                  S* __restrict__ fdst, StepArgs sa) {
    if (blockIdx.x < nadj) {
        adjoint_body<MODEL, S>(state, lam_in, lam_out, a, rate_part, blockIdx.x, nadj);
        return;
    }
    using T = typename Conv<S>::T;
    constexpr int VEC = DefaultVec<S>::value;
    const int lane = threadIdx.x & 31;
    const unsigned total = (unsigned)sa.ny * (unsigned)sa.nseg;
    const unsigned stride = (gridDim.x - nadj) * blockDim.x;
    const Consts<T> c = make_consts<T>(sa);
    Diag dg;
    for (unsigned base = (blockIdx.x - nadj) * blockDim.x + (threadIdx.x & ~31u); base < total; base += stride)
        step_segment<MODEL, 4, S, VEC, false, SHIFT>(fsrc, fdst, sa, c, base + lane, total, lane, dg);
}

__device__ __forceinline__ int wrapi(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

// lambda^N_i(x) = dL/df^N_i(x) and the loss, per block in FP64:
//   misfit  L = 1/2 sum |u - u*|^2:   lambda_i = sum_a (u_a - u*_a)(xi_ia - u_a) / rho
//   kinetic L = 1/2 sum rho |u|^2:    lambda_i = u . xi_i - |u|^2 / 2
template <typename S>
__global__ void __launch_bounds__(kAdjBlock) adjoint_seed_kernel(const S* __restrict__ state, AdjArgs a, int loss,
                                                                 const double* __restrict__ uxt,
                                                                 const double* __restrict__ uyt,
                                                                 typename Conv<S>::T* __restrict__ lam,
                                                                 double* __restrict__ loss_part) {
    using T = typename Conv<S>::T;
    const long long n = (long long)a.nx * a.ny;
    double acc = 0.0;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(k / a.nx), x = (int)(k - (long long)y * a.nx);
        double dr = 0.0, jx = 0.0, jy = 0.0;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const double gi = Conv<S>::to_double(
                state[(long long)i * a.plane + (long long)wrapi(y - ey_of(i), a.ny) * a.pitch + wrapi(x - ex_of(i), a.nx)]);
            dr += gi; jx += ex_of(i) * gi; jy += ey_of(i) * gi;
        }
        jx += a.rho0 * a.urx;
        jy += a.rho0 * a.ury;
        const double rho = a.rho0 + dr, ux = jx / rho, uy = jy / rho;
        double lv[9];
        if (loss == 0) {
            const double dx = ux - uxt[k], dy = uy - uyt[k];
            acc += 0.5 * (dx * dx + dy * dy);
#pragma unroll
            for (int i = 0; i < 9; ++i) lv[i] = (dx * (ex_of(i) - ux) + dy * (ey_of(i) - uy)) / rho;
        } else {
            acc += 0.5 * rho * (ux * ux + uy * uy);
#pragma unroll
            for (int i = 0; i < 9; ++i) lv[i] = ux * ex_of(i) + uy * ey_of(i) - 0.5 * (ux * ux + uy * uy);
        }
#pragma unroll
        for (int i = 0; i < 9; ++i) lam[(long long)i * a.plane + (long long)y * a.pitch + x] = (T)lv[i];
    }
    __shared__ double sh[kAdjBlock];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int s = kAdjBlock / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) loss_part[blockIdx.x] = sh[0];
}

// dL/du0 from lambda^0 and the initial state f^0 = f^eq(rho0, u0) (Eq. extendedFeq):
// d f^eq_(a,b) / du_x = rho phi_a'(u_x) phi_b(u_y), phi_0' = -2u, phi_+-1' = u +- 1/2.
template <typename S>
__global__ void adjoint_init_kernel(const S* __restrict__ state0, AdjArgs a,
                                    const typename Conv<S>::T* __restrict__ lam, double* gux, double* guy) {
    const long long n = (long long)a.nx * a.ny;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(k / a.nx), x = (int)(k - (long long)y * a.nx);
        double dr = 0.0, jx = 0.0, jy = 0.0;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const double gi = Conv<S>::to_double(
                state0[(long long)i * a.plane + (long long)wrapi(y - ey_of(i), a.ny) * a.pitch + wrapi(x - ex_of(i), a.nx)]);
            dr += gi; jx += ex_of(i) * gi; jy += ey_of(i) * gi;
        }
        jx += a.rho0 * a.urx;
        jy += a.rho0 * a.ury;
        const double rho = a.rho0 + dr, ux = jx / rho, uy = jy / rho;
        double gx = 0.0, gy = 0.0;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const int sx = ex_of(i), sy = ey_of(i);
            const double px = phi1d(sx, ux), py = phi1d(sy, uy);
            const double dpx = sx == 0 ? -2.0 * ux : ux + 0.5 * sx;
            const double dpy = sy == 0 ? -2.0 * uy : uy + 0.5 * sy;
            const double li = (double)lam[(long long)i * a.plane + (long long)y * a.pitch + x];
            gx += li * rho * dpx * py;
            gy += li * rho * px * dpy;
        }
        gux[k] = gx;
        guy[k] = gy;
    }
}

template <typename S, bool SH>
const void* adjoint_fused_for(int model) {
    switch (model) {
        case BGK: return (const void*)adjoint_fused_kernel<BGK, S, SH>;
        case RM: return (const void*)adjoint_fused_kernel<RM, S, SH>;
        case HM: return (const void*)adjoint_fused_kernel<HM, S, SH>;
        case CM: return (const void*)adjoint_fused_kernel<CM, S, SH>;
        case CHM: return (const void*)adjoint_fused_kernel<CHM, S, SH>;
        case CUM: return (const void*)adjoint_fused_kernel<CUM, S, SH>;
        case PR: return (const void*)adjoint_fused_kernel<PR, S, SH>;
        case RR: return (const void*)adjoint_fused_kernel<RR, S, SH>;
        default: return nullptr;
    }
}

template <typename S>
const void* adjoint_kernel_for(int model) {
    switch (model) {
        case BGK: return (const void*)adjoint_step_kernel<BGK, S>;
        case RM: return (const void*)adjoint_step_kernel<RM, S>;
        case HM: return (const void*)adjoint_step_kernel<HM, S>;
        case CM: return (const void*)adjoint_step_kernel<CM, S>;
        case CHM: return (const void*)adjoint_step_kernel<CHM, S>;
        case CUM: return (const void*)adjoint_step_kernel<CUM, S>;
        case PR: return (const void*)adjoint_step_kernel<PR, S>;
        case RR: return (const void*)adjoint_step_kernel<RR, S>;
        default: return nullptr;
    }
}

}  // namespace

int adjoint_plan(int storage, int model, int kread, int nx, int ny, int pitch, long long plane, double w, double w3,
                 double w4, double rho0, double urx, double ury, AdjointPlan* p) {
    static_assert(kNumConsts <= (int)(sizeof(AdjArgs::cf) / sizeof(float)), "AdjArgs constant table too small");
    if (storage != LBM_F64 && storage != LBM_F32) return LBM_ERR_UNSUPPORTED;
    const int vec = storage_vec(storage);
    p->storage = storage;
    p->a.nx = nx; p->a.ny = ny; p->a.pitch = pitch; p->a.nseg = (nx + vec - 1) / vec; p->a.plane = plane;
    p->a.w_nu = w; p->a.w3 = w3; p->a.w4 = w4; p->a.rho0 = rho0; p->a.urx = urx; p->a.ury = ury;
    {
        StepArgs t{};
        t.w_nu = w; t.w3 = w3; t.w4 = w4; t.rho0 = rho0; t.urx = urx; t.ury = ury; t.kread = kread;
        fill_consts(t);
        for (int k = 0; k < kNumConsts; ++k) { p->a.cd[k] = t.cd[k]; p->a.cf[k] = t.cf[k]; }
    }
    const bool shifted = urx != 0.0 || ury != 0.0;
    p->step_adj = storage == LBM_F64 ? adjoint_kernel_for<double>(model) : adjoint_kernel_for<float>(model);
    p->step_fwd = storage == LBM_F64 ? step_kernel_f64(model, 4, shifted) : step_kernel_f32(model, 4, shifted);
    if (!p->step_adj || !p->step_fwd) return LBM_ERR_UNSUPPORTED;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    p->block = kAdjBlock;
    const int avec = std::max(1, vec / LBM_ADJ_VEC_DIV);
    const long long warps_f = ((long long)ny * p->a.nseg + 31) / 32;
    const long long warps_a = ((long long)ny * ((nx + avec - 1) / avec) + 31) / 32;
    const long long need_f = (warps_f * 32 + kAdjBlock - 1) / kAdjBlock;
    const long long need_a = (warps_a * 32 + kAdjBlock - 1) / kAdjBlock;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, p->step_adj, kAdjBlock, 0);
    p->grid_adj = (int)std::min<long long>(need_a, (long long)sms * std::max(per_sm, 1));
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, p->step_fwd, kAdjBlock, 0);
    p->grid_fwd = (int)std::min<long long>(need_f, (long long)sms * std::max(per_sm, 1));
    if (p->grid_adj < 1) p->grid_adj = 1;
    if (p->grid_fwd < 1) p->grid_fwd = 1;
    // fused adjoint + recompute launches: the resident blocks split about 2 : 1 (the adjoint
    // step costs about twice the forward step); the adjoint part never exceeds grid_adj,
    // which sizes the per-block rate partials
    p->step_fused = storage == LBM_F64
                        ? (shifted ? adjoint_fused_for<double, true>(model) : adjoint_fused_for<double, false>(model))
                        : (shifted ? adjoint_fused_for<float, true>(model) : adjoint_fused_for<float, false>(model));
    p->grid_fused = 0;
    p->nadj_fused = 0;
    if (p->step_fused &&
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, p->step_fused, kAdjBlock, 0) == cudaSuccess &&
        per_sm >= 1) {
        const long long R = (long long)sms * per_sm;
        const long long nadj = std::min<long long>(std::max<long long>(1, (2 * R) / 3), p->grid_adj);
        const long long nfwd = std::min<long long>(std::max<long long>(1, R - nadj), need_f);
        p->nadj_fused = (int)nadj;
        p->grid_fused = (int)(nadj + nfwd);
    } else {
        cudaGetLastError();
    }
    return LBM_OK;
}

cudaError_t adjoint_launch_fused(const AdjointPlan& p, const void* state, const void* lam_in, void* lam_out,
                                 double* rate_part, const StepArgs& sa, const void* fsrc, void* fdst, cudaStream_t s) {
    AdjArgs a = p.a;
    StepArgs f = sa;
    unsigned nadj = (unsigned)p.nadj_fused;
    void* args[] = {(void*)&state, (void*)&lam_in, (void*)&lam_out, (void*)&a, (void*)&rate_part,
                    (void*)&nadj, (void*)&fsrc, (void*)&fdst, (void*)&f};
    return cudaLaunchKernel(p.step_fused, dim3(p.grid_fused), dim3(p.block), args, 0, s);
}

cudaError_t adjoint_launch_fwd(const AdjointPlan& p, const StepArgs& sa, const void* src, void* dst, cudaStream_t s) {
    void* args[] = {(void*)&src, (void*)&dst, (void*)&sa};
    return cudaLaunchKernel(p.step_fwd, dim3(p.grid_fwd), dim3(p.block), args, 0, s);
}

cudaError_t adjoint_launch_step(const AdjointPlan& p, const void* state, const void* lam_in, void* lam_out,
                                double* rate_part, cudaStream_t s) {
    AdjArgs a = p.a;
    void* args[] = {(void*)&state, (void*)&lam_in, (void*)&lam_out, (void*)&a, (void*)&rate_part};
    return cudaLaunchKernel(p.step_adj, dim3(p.grid_adj), dim3(p.block), args, 0, s);
}

int adjoint_seed_blocks() { return 608; }

cudaError_t adjoint_launch_seed(const AdjointPlan& p, const void* state, int loss, const double* uxt,
                                const double* uyt, void* lam, double* loss_part, cudaStream_t s) {
    if (p.storage == LBM_F64)
        adjoint_seed_kernel<double><<<adjoint_seed_blocks(), kAdjBlock, 0, s>>>((const double*)state, p.a, loss, uxt,
                                                                                uyt, (double*)lam, loss_part);
    else
        adjoint_seed_kernel<float><<<adjoint_seed_blocks(), kAdjBlock, 0, s>>>((const float*)state, p.a, loss, uxt,
                                                                               uyt, (float*)lam, loss_part);
    return cudaGetLastError();
}

cudaError_t adjoint_launch_init(const AdjointPlan& p, const void* state0, const void* lam, double* gux, double* guy,
                                cudaStream_t s) {
    const long long n = (long long)p.a.nx * p.a.ny;
    const int grid = (int)std::min<long long>((n + 255) / 256, 152 * 16);
    if (p.storage == LBM_F64)
        adjoint_init_kernel<double><<<grid, 256, 0, s>>>((const double*)state0, p.a, (const double*)lam, gux, guy);
    else
        adjoint_init_kernel<float><<<grid, 256, 0, s>>>((const float*)state0, p.a, (const float*)lam, gux, guy);
    return cudaGetLastError();
}

}  // namespace lbm
