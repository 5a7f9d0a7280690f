// Auxiliary kernels: equilibrium initialisation, population scatter / gather, moments and
// the FP64 global reductions behind the blow-up check.  None of these is on the per-step
// hot path except the reduction, which runs every `check_every` steps.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <mutex>

#include "lbm.h"

#include "lbm_device.cuh"
#include "lbm_internal.h"

namespace lbm {

namespace {

constexpr int kBlock = 256;
constexpr int kReduceBlocks = 608;   // 4 x 152 SMs; fixed, so the fold order is deterministic
#ifndef LBM_REDUCE_GROUP_BLOCKS
#define LBM_REDUCE_GROUP_BLOCKS 76   // least blocks per lattice in a group's check launch
#endif
static_assert(LBM_REDUCE_GROUP_BLOCKS >= 1 && LBM_REDUCE_GROUP_BLOCKS <= kReduceBlocks,
              "a group check's partials must fit a context's kReduceBlocks slots");
constexpr int kReduceThreads = 128;  // threads of a reduction block (fewer threads, less FP64 folding)
constexpr int kReduceValues = 8;
constexpr int kReduceFlush = 4;      // row segments summed in the collision precision per FP64 add

__device__ __forceinline__ int wrap(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

// offset of the slot that node (x, y) reads its population i from in a pull step
__device__ __forceinline__ long long src_offset(int i, int x, int y, const FieldArgs& a) {
    const int xs = wrap(x - ex_of(i), a.nx), ys = wrap(y - ey_of(i), a.ny);
    return (long long)i * a.plane + (long long)ys * a.pitch + xs;
}

template <typename S>
__global__ void init_eq_kernel(S* buf, FieldArgs a, int eq_order, const double* __restrict__ rho,
                               const double* __restrict__ ux, const double* __restrict__ uy) {
    const long long n = (long long)a.nx * a.ny;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(k / a.nx), x = (int)(k - (long long)y * a.nx);
        const double r = rho[k], vx = ux[k], vy = uy[k];
        const double dr = r - a.rho0;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const int sx = ex_of(i), sy = ey_of(i);
            double g;
            if (eq_order >= 3) {
                // Eq. extendedFeq in product form minus the shift s_i = rho0 P_sx P_sy, with
                // P_s = phi_s(u_ref) and D_s = phi_s(u) - phi_s(u_ref) written as differences
                const double Px = phi1d(sx, a.urx), Py = phi1d(sy, a.ury);
                const double dux = vx - a.urx, sux = vx + a.urx, duy = vy - a.ury, suy = vy + a.ury;
                const double Dx = sx ? 0.5 * dux * (sux + sx) : -dux * sux;
                const double Dy = sy ? 0.5 * duy * (suy + sy) : -duy * suy;
                g = Px * Py * dr + r * (Px * Dy + Dx * (Py + Dy));
                // partial third order (u_ref = 0): minus rho u_x^2 u_y^2 times the populations
                // of a unit M_22 (Eq. Q9postCollVDF_RM: 1 at rest, -1/2 on the axes, 1/4 on
                // the diagonals)
                if (eq_order == 3) g -= r * (vx * vx) * (vy * vy) * (sx ? -0.5 : 1.0) * (sy ? -0.5 : 1.0);
            } else {
                const double wi = weight_of(i);
                const double eu = 3.0 * (sx * vx + sy * vy);
                g = wi * dr + wi * r * (eu + 0.5 * eu * eu - 1.5 * (vx * vx + vy * vy));
            }
            buf[src_offset(i, x, y, a)] = Conv<S>::from_double(g);
        }
    }
}

template <typename S>
__global__ void scatter_kernel(S* buf, FieldArgs a, const double* __restrict__ f) {
    const long long n = (long long)a.nx * a.ny;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(k / a.nx), x = (int)(k - (long long)y * a.nx);
#pragma unroll
        for (int i = 0; i < 9; ++i)
            buf[src_offset(i, x, y, a)] = Conv<S>::from_double(f[i * n + k] - shift_of(i, a.rho0, a.urx, a.ury));
    }
}

template <typename S>
__global__ void gather_kernel(const S* buf, FieldArgs a, double* f, double* rho, double* ux, double* uy,
                              double* pxx, double* pxy, double* pyy) {
    const long long n = (long long)a.nx * a.ny;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(k / a.nx), x = (int)(k - (long long)y * a.nx);
        double g[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) g[i] = Conv<S>::to_double(buf[src_offset(i, x, y, a)]);
        if (f) {
#pragma unroll
            for (int i = 0; i < 9; ++i) f[i * n + k] = g[i] + shift_of(i, a.rho0, a.urx, a.ury);
        }
        if (rho || ux || uy || pxx || pxy || pyy) {
            double dr = 0, jx = 0, jy = 0, sxx = 0, sxy = 0, syy = 0;
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                const int sx = ex_of(i), sy = ey_of(i);
                dr += g[i]; jx += sx * g[i]; jy += sy * g[i];
                sxx += sx * sx * g[i]; sxy += sx * sy * g[i]; syy += sy * sy * g[i];
            }
            // moments of the shift: sum s = rho0, sum xi s = rho0 u_ref,
            // sum xi_a xi_b s = rho0 (u_ref,a u_ref,b + c_s^2 delta_ab)
            const double r = a.rho0 + dr;
            jx += a.rho0 * a.urx;
            jy += a.rho0 * a.ury;
            if (rho) rho[k] = r;
            if (ux) ux[k] = jx / r;
            if (uy) uy[k] = jy / r;
            if (pxx) pxx[k] = sxx + a.rho0 * (a.urx * a.urx + 1.0 / 3.0);
            if (pxy) pxy[k] = sxy + a.rho0 * a.urx * a.ury;
            if (pyy) pyy[k] = syy + a.rho0 * (a.ury * a.ury + 1.0 / 3.0);
        }
    }
}

__device__ __forceinline__ double fold_op(int slot, double x, double y) { return slot == 6 ? fmin(x, y) : x + y; }

// Folds the eight values of the 32 lanes of a warp (slot 6 by min, the others by sum) with
// nine FP64 operations a lane: in the rounds xor 16, 8 and 4 every lane keeps half of the
// slots it still holds and adds its partner's copy of them, then the rounds xor 2 and 1 fold
// the one slot left.  Lane l ends with the warp's value of slot
// 4 * bit4(l) + 2 * bit3(l) + bit2(l); *slot_out is that slot.
__device__ __forceinline__ double warp_fold8(const double (&a)[kReduceValues], int lane, int* slot_out) {
    const bool h16 = lane & 16, h8 = lane & 8, h4 = lane & 4;
    const int base = h16 ? 4 : 0;
    double b[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const double recv = __shfl_xor_sync(0xffffffffu, h16 ? a[j] : a[j + 4], 16);
        b[j] = fold_op(base + j, h16 ? a[j + 4] : a[j], recv);
    }
    const int base2 = base + (h8 ? 2 : 0);
    double c[2];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const double recv = __shfl_xor_sync(0xffffffffu, h8 ? b[j] : b[j + 2], 8);
        c[j] = fold_op(base2 + j, h8 ? b[j + 2] : b[j], recv);
    }
    const int slot = base2 + (h4 ? 1 : 0);
    double d = fold_op(slot, h4 ? c[1] : c[0], __shfl_xor_sync(0xffffffffu, h4 ? c[0] : c[1], 4));
    d = fold_op(slot, d, __shfl_xor_sync(0xffffffffu, d, 2));
    d = fold_op(slot, d, __shfl_xor_sync(0xffffffffu, d, 1));
    *slot_out = slot;
    return d;
}

// Folds the per-thread values acc[0..7] of a block of kReduceThreads threads in a fixed order
// (the warp fold above, then the warps in order); thread v < 8 returns the block's value v,
// the other threads return 0.
__device__ __forceinline__ double block_fold(const double (&acc)[kReduceValues]) {
    __shared__ double sh[kReduceThreads / 32][kReduceValues];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int slot;
    const double w = warp_fold8(acc, lane, &slot);
    if ((lane & 3) == 0) sh[warp][slot] = w;
    __syncthreads();
    double x = 0.0;
    if (threadIdx.x < kReduceValues) {
        const int v = threadIdx.x;
        x = sh[0][v];
        for (int k = 1; k < kReduceThreads / 32; ++k) x = fold_op(v, x, sh[k][v]);
    }
    return x;
}

// Pass 2: folds nparts partials (fixed order: thread t takes parts t, t + 128, ..., then the
// block fold), forms the outputs and applies the blow-up criterion.  Partials are read through
// L2 (they may come from other blocks of the same launch).
__device__ void finish_fold(const double* partials, int nparts, const FieldArgs& a, double* out, int* status,
                            long long* blowup_step, const CheckArgs& c) {
    double acc[kReduceValues] = {0, 0, 0, 0, 0, 0, 1e300, 0};
    // nparts <= kReduceBlocks: a fixed trip count, so the loads of every round issue together
    constexpr int kRounds = (kReduceBlocks + kReduceThreads - 1) / kReduceThreads;
    double part[kRounds][kReduceValues];
#pragma unroll
    for (int k = 0; k < kRounds; ++k) {
        const int b = threadIdx.x + k * kReduceThreads;
#pragma unroll
        for (int v = 0; v < kReduceValues; ++v)
            part[k][v] = b < nparts ? __ldcg(&partials[b * kReduceValues + v]) : acc[v];
    }
#pragma unroll
    for (int k = 0; k < kRounds; ++k) {
#pragma unroll
        for (int v = 0; v < kReduceValues; ++v) acc[v] = fold_op(v, acc[v], part[k][v]);
    }
    __shared__ double tot[kReduceValues];
    const double x = block_fold(acc);
    if (threadIdx.x < kReduceValues) tot[threadIdx.x] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        const double n = (double)a.nx * (double)a.ny;
        double o[kReduceValues];
        o[0] = n * a.rho0 + tot[0];
        o[1] = tot[1];
        o[2] = tot[2];
        o[3] = tot[3];
        o[4] = tot[4] / n;
        o[5] = tot[5] / n;
        o[6] = a.rho0 + tot[6];
        o[7] = tot[7];
        for (int v = 0; v < kReduceValues; ++v) out[v] = o[v];
        if (c.apply && status && *status == 0) {
            const bool blown = (o[7] > 0.0) || !(o[6] > 0.0) ||
                               (c.ke_ref > 0.0 && o[4] > c.ke_factor * c.ke_ref);
            if (blown) {
                *status = -4;   // LBM_ERR_BLOWUP
                *blowup_step = c.step;
            }
        }
    }
}

// Pass 1 arithmetic.  Per node: rho, j = sum xi f (+ rho0 u_ref) and u = j / rho in the
// collision precision T.  The finite nodes' contributions are summed in T over kReduceFlush
// successive row segments of a thread's grid-stride loop (in node order), then added to the
// thread's FP64 accumulators.  Slots: 0 sum drho, 1 sum rho ux, 2 sum rho uy, 3 sum rho|u|^2/2, 4 sum |u|^2,
// 5 sum |u-uref|^2, 6 min rho (as drho), 7 non-finite count.  Both pass-1 kernels visit the
// same segments in the same per-thread order, so their partials are bitwise equal.
template <typename T> __device__ __forceinline__ T div_rho(T j, T ir, T r);
template <> __device__ __forceinline__ float div_rho(float j, float ir, float) { return j * ir; }
template <> __device__ __forceinline__ double div_rho(double j, double, double r) { return j / r; }

template <typename T> struct SegSums {
    T dr = 0, jx = 0, jy = 0, ke = 0, u2 = 0, w2 = 0, mn = T(INFINITY);
    int good = 0, bad = 0;
};

template <typename T, int VEC>
__device__ __forceinline__ void segment_add(const T (&f)[9][VEC], int nvalid, T rho0, T jx0, T jy0, T urefx,
                                            T urefy, SegSums<T>& p) {
#pragma unroll
    for (int j = 0; j < VEC; ++j) {
        if (j >= nvalid) continue;
        T dr = 0, jx = 0, jy = 0;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            dr += f[i][j];
            jx += T(ex_of(i)) * f[i][j];
            jy += T(ey_of(i)) * f[i][j];
        }
        jx += jx0;
        jy += jy0;
        const T r = rho0 + dr;
        const T ir = recip(r);
        const T vx = div_rho(jx, ir, r), vy = div_rho(jy, ir, r);
        if (isfinite(r) && isfinite(vx) && isfinite(vy)) {
            const T u2 = vx * vx + vy * vy;
            const T wx = vx - urefx, wy = vy - urefy;
            p.dr += dr;
            p.jx += jx;
            p.jy += jy;
            p.ke += r * u2;
            p.u2 += u2;
            p.w2 += wx * wx + wy * wy;
            p.mn = fmin(p.mn, dr);
            ++p.good;
        } else {
            ++p.bad;
        }
    }
}

template <typename T>
__device__ __forceinline__ void segment_flush(SegSums<T>& p, double (&acc)[kReduceValues]) {
    if (p.good) {
        acc[0] += (double)p.dr;
        acc[1] += (double)p.jx;
        acc[2] += (double)p.jy;
        acc[3] += 0.5 * (double)p.ke;
        acc[4] += (double)p.u2;
        acc[5] += (double)p.w2;
        acc[6] = fmin(acc[6], (double)p.mn);
    }
    const int bad = p.bad;
    p = SegSums<T>();
    p.bad = bad;
}

// End of pass 1: the block's partials; with a completion counter (FUSED), the last block to
// finish also runs pass 2 and resets the counter for the next launch.
template <bool FUSED>
__device__ __forceinline__ void reduce_epilogue(double (&acc)[kReduceValues], double* partials, unsigned* counter,
                                                const FieldArgs& a, double* out, int* status,
                                                long long* blowup_step, const CheckArgs& c) {
    const double x = block_fold(acc);
    if (threadIdx.x < kReduceValues) partials[blockIdx.x * kReduceValues + threadIdx.x] = x;
    if (!FUSED) return;
    __shared__ bool last;
    __threadfence();   // this block's partials before its count
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(counter, 1u) == gridDim.x - 1;
    __syncthreads();
    if (last) {        // uniform over the block
        __threadfence();   // every block's partials after the count
        finish_fold(partials, gridDim.x, a, out, status, blowup_step, c);
        if (threadIdx.x == 0) *counter = 0u;
    }
}

// Pass 1, scalar-load form for layouts whose rows are not 16-byte aligned (caller-owned
// buffers of lbm_reduce_noalloc may have any pitch): the same row segments as the vectorised
// form, one segment per thread and iteration.
template <typename S, bool FUSED>
__global__ void __launch_bounds__(kReduceThreads) reduce_kernel_scalar(const S* buf, FieldArgs a, double* partials,
                                                                       unsigned* counter, double* out, int* status,
                                                                       long long* blowup_step, CheckArgs c) {
    using T = typename Conv<S>::T;
    constexpr int VEC = DefaultVec<S>::value;
    const int nseg = (a.nx + VEC - 1) / VEC;
    const long long total = (long long)a.ny * nseg;
    const T jx0 = T(a.rho0 * a.urx), jy0 = T(a.rho0 * a.ury);
    double acc[kReduceValues] = {0, 0, 0, 0, 0, 0, 1e300, 0};
    SegSums<T> p;
    int it = 0;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < total; k += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(k / nseg), seg = (int)(k - (long long)y * nseg);
        const int x0 = seg * VEC;
        const int nvalid = min(VEC, a.nx - x0);
        T f[9][VEC];
#pragma unroll
        for (int j = 0; j < VEC; ++j) {
#pragma unroll
            for (int i = 0; i < 9; ++i)
                f[i][j] = j < nvalid ? Conv<S>::to_T(buf[src_offset(i, x0 + j, y, a)]) : T(0);
        }
        segment_add<T, VEC>(f, nvalid, T(a.rho0), jx0, jy0, T(c.uref_x), T(c.uref_y), p);
        if (++it == kReduceFlush) {
            segment_flush(p, acc);
            it = 0;
        }
    }
    segment_flush(p, acc);
    acc[7] = (double)p.bad;
    reduce_epilogue<FUSED>(acc, partials, counter, a, out, status, blowup_step, c);
}

// Pass 1: the same vectorised pull gather as the step kernel, one row segment per thread and
// iteration.
template <typename S, bool FUSED>
__device__ __forceinline__ void reduce_pass1(const S* buf, const FieldArgs& a, double* partials, unsigned* counter,
                                             double* out, int* status, long long* blowup_step, const CheckArgs& c) {
    using T = typename Conv<S>::T;
    constexpr int VEC = DefaultVec<S>::value;
    const int lane = threadIdx.x & 31;
    const int nseg = (a.nx + VEC - 1) / VEC;
    const unsigned total = (unsigned)a.ny * (unsigned)nseg;
    const unsigned stride = gridDim.x * blockDim.x;
    const T jx0 = T(a.rho0 * a.urx), jy0 = T(a.rho0 * a.ury);
    double acc[kReduceValues] = {0, 0, 0, 0, 0, 0, 1e300, 0};
    SegSums<T> p;
    int it = 0;
    for (unsigned base = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < total; base += stride) {
        const unsigned s = base + lane;
        const bool active = s < total;
        const unsigned sc = active ? s : total - 1;
        const int y = (int)(sc / (unsigned)nseg);
        const int seg = (int)(sc - (unsigned)y * (unsigned)nseg);
        const int x0 = seg * VEC;
        const int nvalid = min(VEC, a.nx - x0);
        T f[9][VEC];
        gather_pull<S, VEC, 1>(buf, a.nx, a.ny, a.pitch, a.plane, y, seg, nseg, x0, nvalid, lane, f);
        if (active) {
            segment_add<T, VEC>(f, nvalid, T(a.rho0), jx0, jy0, T(c.uref_x), T(c.uref_y), p);
            if (++it == kReduceFlush) {
                segment_flush(p, acc);
                it = 0;
            }
        }
    }
    segment_flush(p, acc);
    acc[7] = (double)p.bad;
    reduce_epilogue<FUSED>(acc, partials, counter, a, out, status, blowup_step, c);
}
template <typename S, bool FUSED>
__global__ void __launch_bounds__(kReduceThreads) reduce_kernel(const S* buf, FieldArgs a, double* partials,
                                                                unsigned* counter, double* out, int* status,
                                                                long long* blowup_step, CheckArgs c) {
    reduce_pass1<S, FUSED>(buf, a, partials, counter, out, status, blowup_step, c);
}

// The checks of several lattices of one storage type in one launch: grid row blockIdx.y runs
// job blockIdx.y's check (the code of reduce_kernel<S, true>) with kReduceBlocks / n blocks
// (at least LBM_REDUCE_GROUP_BLOCKS) instead of kReduceBlocks: the jobs' blocks together fill
// the SMs about as one lattice's check does, and fewer threads, each summing more row
// segments, spend fewer FP64 folds, which bound the check (GB300's FP64 pipe).  The fold order
// is fixed for a given group size, so a lattice's figures are reproducible; they differ from
// its single-launch check only in the rounding of the FP64 sums.  Measured on eight 1024^2
// FP32 lattices (the benchmark's step time outside the step kernel, per check of the eight):
// 76 blocks each 82 us, 152: 90 us, 304: 94 us, 608: 104 us, 38: 120 us, 19: 210 us; each
// block running every job in turn 155 us.
template <typename S>
__global__ void __launch_bounds__(kReduceThreads) reduce_group_kernel(const __grid_constant__ ReduceGroupArgs g) {
    const ReduceJob& J = g.j[blockIdx.y];
    reduce_pass1<S, true>(static_cast<const S*>(J.buf), J.a, J.partials, J.counter, J.out, J.status, J.blowup_step,
                          J.c);
}

// Pass 2 as its own launch (the allocation-free entry point, which keeps no counter).
__global__ void __launch_bounds__(kReduceThreads) reduce_finish_kernel(const double* partials, int nparts, FieldArgs a,
                                                                       double* out, int* status, long long* blowup_step,
                                                                       CheckArgs c) {
    finish_fold(partials, nparts, a, out, status, blowup_step, c);
}

int grid_for(long long n) {
    long long g = (n + kBlock - 1) / kBlock;
    if (g > 152 * 16) g = 152 * 16;
    if (g < 1) g = 1;
    return (int)g;
}

// Halo rows of a y-slab.  Messages are [3][nx] elements: `up` holds the planes with xi_y = +1
// (i = 2, 5, 6) of one row, `down` those with xi_y = -1 (i = 4, 7, 8).  pack: up <- row ny - 2
// (the slab's last own row), down <- row 1 (its first own row).  unpack: row 0 (the ghost row
// below) <- up, row ny - 1 (the ghost row above) <- down.  Raw storage elements are copied.
template <typename E>
__global__ void halo_kernel(E* buf, FieldArgs a, E* up, E* down, int pack) {
    const int n = 3 * a.nx;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < 2 * n; k += gridDim.x * blockDim.x) {
        const bool top = k < n;
        const int j = top ? k : k - n;
        const int q = j / a.nx, x = j - q * a.nx;
        const int i = top ? (q == 0 ? 2 : (q == 1 ? 5 : 6)) : (q == 0 ? 4 : (q == 1 ? 7 : 8));
        E* msg = top ? up : down;
        const int row = pack ? (top ? a.ny - 2 : 1) : (top ? 0 : a.ny - 1);
        E* slot = buf + (long long)i * a.plane + (long long)row * a.pitch + x;
        if (pack) msg[j] = *slot;
        else *slot = msg[j];
    }
}

template <typename S>
cudaError_t init_t(void* buf, const FieldArgs& a, int eq, const double* r, const double* x, const double* y, cudaStream_t s) {
    init_eq_kernel<S><<<grid_for((long long)a.nx * a.ny), kBlock, 0, s>>>((S*)buf, a, eq, r, x, y);
    return cudaGetLastError();
}
template <typename S>
cudaError_t scatter_t(void* buf, const FieldArgs& a, const double* f, cudaStream_t s) {
    scatter_kernel<S><<<grid_for((long long)a.nx * a.ny), kBlock, 0, s>>>((S*)buf, a, f);
    return cudaGetLastError();
}
template <typename S>
cudaError_t gather_t(const void* buf, const FieldArgs& a, double* f, double* r, double* x, double* y,
                     double* pxx, double* pxy, double* pyy, cudaStream_t s) {
    gather_kernel<S><<<grid_for((long long)a.nx * a.ny), kBlock, 0, s>>>((const S*)buf, a, f, r, x, y, pxx, pxy, pyy);
    return cudaGetLastError();
}
template <typename S>
cudaError_t reduce_t(const void* buf, const FieldArgs& a, double* partials, unsigned* counter, double* out8,
                     int* status, long long* blowup_step, const CheckArgs& c, cudaStream_t s) {
    // the vectorised gather needs every row start 16-byte aligned
    const bool aligned = ((size_t)a.pitch * sizeof(S)) % 16 == 0 && ((uintptr_t)buf % 16) == 0;
    const S* p = (const S*)buf;
    if (counter) {
        if (aligned)
            reduce_kernel<S, true><<<kReduceBlocks, kReduceThreads, 0, s>>>(p, a, partials, counter, out8, status,
                                                                          blowup_step, c);
        else
            reduce_kernel_scalar<S, true><<<kReduceBlocks, kReduceThreads, 0, s>>>(p, a, partials, counter, out8,
                                                                                 status, blowup_step, c);
        return cudaGetLastError();
    }
    if (aligned)
        reduce_kernel<S, false><<<kReduceBlocks, kReduceThreads, 0, s>>>(p, a, partials, nullptr, out8, status,
                                                                       blowup_step, c);
    else
        reduce_kernel_scalar<S, false><<<kReduceBlocks, kReduceThreads, 0, s>>>(p, a, partials, nullptr, out8,
                                                                              status, blowup_step, c);
    reduce_finish_kernel<<<1, kReduceThreads, 0, s>>>(partials, kReduceBlocks, a, out8, status, blowup_step, c);
    return cudaGetLastError();
}

}  // namespace

template <typename S>
cudaError_t reduce_group_t(const ReduceGroupArgs& g, cudaStream_t s) {
    for (int e = 0; e < g.n; ++e) {
        const ReduceJob& J = g.j[e];
        if (((size_t)J.a.pitch * sizeof(S)) % 16 != 0 || ((uintptr_t)J.buf % 16) != 0 || !J.counter)
            return cudaErrorInvalidValue;
    }
    const int blocks = std::max(LBM_REDUCE_GROUP_BLOCKS, kReduceBlocks / g.n);
    reduce_group_kernel<S><<<dim3(blocks, g.n), kReduceThreads, 0, s>>>(g);
    return cudaGetLastError();
}

int reduce_blocks() { return kReduceBlocks; }
size_t reduce_scratch_bytes() { return sizeof(double) * kReduceValues * kReduceBlocks + 16; }

#define LBM_DISPATCH(storage, call)                                     \
    switch (storage) {                                                  \
        case 0: { using S = double; return call; }                      \
        case 1: { using S = float; return call; }                       \
        case 2: { using S = __half; return call; }                      \
        case 3: { using S = __nv_bfloat16; return call; }               \
        default: return cudaErrorInvalidValue;                          \
    }

cudaError_t launch_init_eq(int storage, void* buf, const FieldArgs& a, int eq_order,
                           const double* rho, const double* ux, const double* uy, cudaStream_t s) {
    LBM_DISPATCH(storage, init_t<S>(buf, a, eq_order, rho, ux, uy, s));
}
cudaError_t launch_scatter(int storage, void* buf, const FieldArgs& a, const double* f, cudaStream_t s) {
    LBM_DISPATCH(storage, scatter_t<S>(buf, a, f, s));
}
cudaError_t launch_gather(int storage, const void* buf, const FieldArgs& a, double* f, double* rho, double* ux,
                          double* uy, double* pxx, double* pxy, double* pyy, cudaStream_t s) {
    LBM_DISPATCH(storage, gather_t<S>(buf, a, f, rho, ux, uy, pxx, pxy, pyy, s));
}
cudaError_t launch_reduce(int storage, const void* buf, const FieldArgs& a, double* partials, unsigned* counter,
                          double* out8, int* status, long long* blowup_step, const CheckArgs& c, cudaStream_t s) {
    LBM_DISPATCH(storage, reduce_t<S>(buf, a, partials, counter, out8, status, blowup_step, c, s));
}

cudaError_t launch_reduce_group(int storage, const ReduceGroupArgs& g, cudaStream_t s) {
    if (g.n < 1 || g.n > kReduceGroupMax) return cudaErrorInvalidValue;
    LBM_DISPATCH(storage, reduce_group_t<S>(g, s));
}

cudaError_t launch_halo(int storage, void* buf, const FieldArgs& a, void* up, void* down, bool pack, cudaStream_t s) {
    const int grid = grid_for(6LL * a.nx);
    switch (storage_bytes(storage)) {
        case 8: halo_kernel<unsigned long long><<<grid, kBlock, 0, s>>>((unsigned long long*)buf, a,
                                                (unsigned long long*)up, (unsigned long long*)down, pack); break;
        case 4: halo_kernel<unsigned><<<grid, kBlock, 0, s>>>((unsigned*)buf, a, (unsigned*)up, (unsigned*)down, pack);
            break;
        case 2: halo_kernel<unsigned short><<<grid, kBlock, 0, s>>>((unsigned short*)buf, a, (unsigned short*)up,
                                                                   (unsigned short*)down, pack); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

int storage_vec(int storage) {
    switch (storage) {
        case 0: return DefaultVec<double>::value;
        case 1: return DefaultVec<float>::value;
        case 2: return DefaultVec<__half>::value;
        case 3: return DefaultVec<__nv_bfloat16>::value;
        default: return 0;
    }
}
int storage_bytes(int storage) {
    switch (storage) {
        case 0: return 8;
        case 1: return 4;
        case 2: case 3: return 2;
        default: return 0;
    }
}

}  // namespace lbm

// ---------------------------------------------------------------------------------------
// Self-test of the FP32 reciprocal behind u = j / rho (lbm_selftest_recip in include/lbm.h).
namespace lbm {
namespace {
__global__ void selftest_recip_kernel(const float* __restrict__ x, float* __restrict__ approx,
                                      float* __restrict__ rounded, long long n) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const float v = x[k];
        approx[k] = recip(v);
        rounded[k] = __frcp_rn(v);
    }
}
}  // namespace
}  // namespace lbm

extern "C" int lbm_selftest_recip(const float* x, float* approx, float* rounded, long long n, void* cuda_stream) {
    using namespace lbm;
    if (!x || !approx || !rounded || n < 0) return LBM_ERR_INVALID_ARG;
    if (n == 0) return LBM_OK;
    selftest_recip_kernel<<<grid_for(n), kBlock, 0, (cudaStream_t)cuda_stream>>>(x, approx, rounded, n);
    return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}

// ---------------------------------------------------------------------------------------
// Allocation-free reductions (lbm_reduce_noalloc in include/lbm.h).
//
// The two reduction passes above need a scratch array for the per-block partial sums.  For
// callers that cannot allocate device memory, that scratch lives in this file-scope device
// array instead: 608 blocks x 8 doubles = 38,912 bytes, allocated by the CUDA runtime when
// the library's module loads on a device and held by every device that loads it until the
// process exits.  Its host-side name is not a device address: host code obtains the device
// address once per device with cudaGetSymbolAddress, while that device is current, and passes
// that address to the kernels.
namespace lbm {
namespace {
constexpr int kNoallocMaxDevices = 64;
static __device__ __align__(256) double g_noalloc_partials[kReduceBlocks * kReduceValues];
std::mutex g_noalloc_mutex;
double* g_noalloc_ptr[kNoallocMaxDevices] = {nullptr};

// Device memory of device `dev` (the current one), or managed memory.  Device memory of
// another GPU is rejected: the kernels run on the current device, and reading another GPU's
// memory without peer access enabled is an illegal access.
bool noalloc_is_device_ptr(const void* p, int dev) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (at.type == cudaMemoryTypeManaged) return true;
    return at.type == cudaMemoryTypeDevice && at.device == dev;
}
}  // namespace

}  // namespace lbm

extern "C" int lbm_reduce_noalloc(const void* populations, int storage, int nx, int ny, int pitch, double rho0,
                                  double uref_x, double uref_y, double* out8, void* cuda_stream) {
    using namespace lbm;
    if (!populations || !out8) return LBM_ERR_INVALID_ARG;
    if (storage < LBM_F64 || storage > LBM_BF16) return LBM_ERR_INVALID_ARG;
    if (nx < 3 || ny < 3 || pitch < nx) return LBM_ERR_INVALID_ARG;
    // the largest lattice accepted: 2^31 nodes, as for lbm_create
    if ((long long)nx * (long long)ny > (1LL << 31)) return LBM_ERR_INVALID_ARG;
    if (!(rho0 > 0.0) || !std::isfinite(rho0) || !std::isfinite(uref_x) || !std::isfinite(uref_y))
        return LBM_ERR_INVALID_ARG;
    const size_t esize = (size_t)storage_bytes(storage);
    if (((uintptr_t)populations % esize) != 0 || ((uintptr_t)out8 % sizeof(double)) != 0) return LBM_ERR_INVALID_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoallocMaxDevices) return LBM_ERR_CUDA;
    if (!noalloc_is_device_ptr(populations, dev) || !noalloc_is_device_ptr(out8, dev)) return LBM_ERR_INVALID_ARG;

    double* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mutex);
        if (!g_noalloc_ptr[dev]) {
            void* p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
            if (e != cudaSuccess || !p) {
                cudaGetLastError();
                return LBM_ERR_CUDA;
            }
            g_noalloc_ptr[dev] = static_cast<double*>(p);
        }
        scratch = g_noalloc_ptr[dev];
    }
    FieldArgs a;
    a.nx = nx; a.ny = ny; a.pitch = pitch; a.plane = (long long)ny * pitch; a.rho0 = rho0;
    a.urx = 0.0; a.ury = 0.0;
    CheckArgs c;
    c.ke_ref = 0.0; c.ke_factor = 1.0; c.uref_x = uref_x; c.uref_y = uref_y; c.step = 0; c.apply = 0;
    // pass 1 overwrites every partial slot before pass 2 reads it (same stream), so nothing in
    // the shared array needs clearing between calls
    cudaError_t e = launch_reduce(storage, populations, a, scratch, nullptr, out8, nullptr, nullptr, c,
                                  (cudaStream_t)cuda_stream);
    return e == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}
