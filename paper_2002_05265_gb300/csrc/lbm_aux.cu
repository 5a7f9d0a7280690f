// Auxiliary kernels: equilibrium initialisation, population scatter / gather, moments and
// the FP64 global reductions behind the blow-up check.  None of these is on the per-step
// hot path except the reduction, which runs every `check_every` steps.
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
constexpr int kReduceValues = 8;

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
            if (eq_order == 4) {
                // Eq. extendedFeq in product form minus the shift s_i = rho0 P_sx P_sy, with
                // P_s = phi_s(u_ref) and D_s = phi_s(u) - phi_s(u_ref) written as differences
                const double Px = phi1d(sx, a.urx), Py = phi1d(sy, a.ury);
                const double dux = vx - a.urx, sux = vx + a.urx, duy = vy - a.ury, suy = vy + a.ury;
                const double Dx = sx ? 0.5 * dux * (sux + sx) : -dux * sux;
                const double Dy = sy ? 0.5 * duy * (suy + sy) : -duy * suy;
                g = Px * Py * dr + r * (Px * Dy + Dx * (Py + Dy));
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

// Folds the per-thread accumulators of a block in a fixed order into its partial slot.
__device__ __forceinline__ void block_fold_partials(double (&acc)[kReduceValues], double* partials) {
    __shared__ double sh[kBlock / 32][kReduceValues];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int v = 0; v < kReduceValues; ++v) {
        double x = acc[v];
        for (int o = 16; o > 0; o >>= 1) {
            const double y2 = __shfl_down_sync(0xffffffffu, x, o);
            x = (v == 6) ? fmin(x, y2) : x + y2;
        }
        if (lane == 0) sh[warp][v] = x;
    }
    __syncthreads();
    if (threadIdx.x < kReduceValues) {
        const int v = threadIdx.x;
        double x = sh[0][v];
        for (int w = 1; w < kBlock / 32; ++w) x = (v == 6) ? fmin(x, sh[w][v]) : x + sh[w][v];
        partials[blockIdx.x * kReduceValues + v] = x;
    }
}

// Pass 1, per-node form: the same sums for layouts whose rows are not 16-byte aligned
// (caller-owned buffers of lbm_reduce_noalloc may have any pitch); one node per thread,
// scalar loads.
template <typename S>
__global__ void __launch_bounds__(kBlock) reduce_kernel_scalar(const S* buf, FieldArgs a, double* partials,
                                                               double urefx, double urefy) {
    using T = typename Conv<S>::T;
    const long long n = (long long)a.nx * a.ny;
    const T jx0 = T(a.rho0 * a.urx), jy0 = T(a.rho0 * a.ury);
    double acc[kReduceValues] = {0, 0, 0, 0, 0, 0, 1e300, 0};
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(k / a.nx), x = (int)(k - (long long)y * a.nx);
        T dr = 0, jx = 0, jy = 0;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const T g = Conv<S>::to_T(buf[src_offset(i, x, y, a)]);
            dr += g;
            jx += T(ex_of(i)) * g;
            jy += T(ey_of(i)) * g;
        }
        jx += jx0;
        jy += jy0;
        const T r = T(a.rho0) + dr;
        const T vx = jx / r, vy = jy / r;
        if (isfinite(r) && isfinite(vx) && isfinite(vy)) {
            const T u2 = vx * vx + vy * vy;
            const T wx = vx - T(urefx), wy = vy - T(urefy);
            acc[0] += (double)dr;
            acc[1] += (double)jx;
            acc[2] += (double)jy;
            acc[3] += 0.5 * (double)(r * u2);
            acc[4] += (double)u2;
            acc[5] += (double)(wx * wx + wy * wy);
            acc[6] = fmin(acc[6], (double)dr);
        } else {
            acc[7] += 1.0;
        }
    }
    block_fold_partials(acc, partials);
}

// Pass 1: per-node rho, u in the collision precision T from the same vectorised pull gather
// as the step kernel, accumulated per thread in FP64, then folded per block in a fixed
// order.  Slots: 0 sum drho, 1 sum rho ux, 2 sum rho uy, 3 sum rho|u|^2/2, 4 sum |u|^2,
// 5 sum |u-uref|^2, 6 min rho (as drho), 7 non-finite count.
template <typename S>
__global__ void __launch_bounds__(kBlock) reduce_kernel(const S* buf, FieldArgs a, double* partials,
                                                        double urefx, double urefy) {
    using T = typename Conv<S>::T;
    constexpr int VEC = DefaultVec<S>::value;
    const int lane = threadIdx.x & 31;
    const int nseg = (a.nx + VEC - 1) / VEC;
    const unsigned total = (unsigned)a.ny * (unsigned)nseg;
    const unsigned stride = gridDim.x * blockDim.x;
    const T jx0 = T(a.rho0 * a.urx), jy0 = T(a.rho0 * a.ury);
    double acc[kReduceValues] = {0, 0, 0, 0, 0, 0, 1e300, 0};
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
#pragma unroll
        for (int j = 0; j < VEC; ++j) {
            if (!active || j >= nvalid) continue;
            T dr = 0, jx = 0, jy = 0;
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                dr += f[i][j];
                jx += T(ex_of(i)) * f[i][j];
                jy += T(ey_of(i)) * f[i][j];
            }
            jx += jx0;
            jy += jy0;
            const T r = T(a.rho0) + dr;
            const T vx = jx / r, vy = jy / r;
            if (isfinite(r) && isfinite(vx) && isfinite(vy)) {
                const T u2 = vx * vx + vy * vy;
                const T wx = vx - T(urefx), wy = vy - T(urefy);
                acc[0] += (double)dr;
                acc[1] += (double)jx;
                acc[2] += (double)jy;
                acc[3] += 0.5 * (double)(r * u2);
                acc[4] += (double)u2;
                acc[5] += (double)(wx * wx + wy * wy);
                acc[6] = fmin(acc[6], (double)dr);
            } else {
                acc[7] += 1.0;
            }
        }
    }
    block_fold_partials(acc, partials);
}

// Pass 2: one block folds the partials (fixed order), forms the outputs and applies the
// blow-up criterion.
__global__ void __launch_bounds__(kBlock) reduce_finish_kernel(const double* partials, int nparts, FieldArgs a,
                                                               double* out, int* status, long long* blowup_step,
                                                               CheckArgs c) {
    __shared__ double sh[kBlock][kReduceValues];
    double acc[kReduceValues] = {0, 0, 0, 0, 0, 0, 1e300, 0};
    for (int b = threadIdx.x; b < nparts; b += blockDim.x) {
#pragma unroll
        for (int v = 0; v < kReduceValues; ++v) {
            const double x = partials[b * kReduceValues + v];
            acc[v] = (v == 6) ? fmin(acc[v], x) : acc[v] + x;
        }
    }
#pragma unroll
    for (int v = 0; v < kReduceValues; ++v) sh[threadIdx.x][v] = acc[v];
    __syncthreads();
    for (int s = kBlock / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) {
#pragma unroll
            for (int v = 0; v < kReduceValues; ++v)
                sh[threadIdx.x][v] = (v == 6) ? fmin(sh[threadIdx.x][v], sh[threadIdx.x + s][v])
                                              : sh[threadIdx.x][v] + sh[threadIdx.x + s][v];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double n = (double)a.nx * (double)a.ny;
        const double* t = sh[0];
        double o[kReduceValues];
        o[0] = n * a.rho0 + t[0];
        o[1] = t[1];
        o[2] = t[2];
        o[3] = t[3];
        o[4] = t[4] / n;
        o[5] = t[5] / n;
        o[6] = a.rho0 + t[6];
        o[7] = t[7];
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

int grid_for(long long n) {
    long long g = (n + kBlock - 1) / kBlock;
    if (g > 152 * 16) g = 152 * 16;
    if (g < 1) g = 1;
    return (int)g;
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
cudaError_t reduce_t(const void* buf, const FieldArgs& a, double* partials, double* out8, int* status,
                     long long* blowup_step, const CheckArgs& c, cudaStream_t s) {
    // the vectorised gather needs every row start 16-byte aligned
    const bool aligned = ((size_t)a.pitch * sizeof(S)) % 16 == 0 && ((uintptr_t)buf % 16) == 0;
    if (aligned)
        reduce_kernel<S><<<kReduceBlocks, kBlock, 0, s>>>((const S*)buf, a, partials, c.uref_x, c.uref_y);
    else
        reduce_kernel_scalar<S><<<kReduceBlocks, kBlock, 0, s>>>((const S*)buf, a, partials, c.uref_x, c.uref_y);
    reduce_finish_kernel<<<1, kBlock, 0, s>>>(partials, kReduceBlocks, a, out8, status, blowup_step, c);
    return cudaGetLastError();
}

}  // namespace

int reduce_blocks() { return kReduceBlocks; }

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
cudaError_t launch_reduce(int storage, const void* buf, const FieldArgs& a, double* partials, double* out8,
                          int* status, long long* blowup_step, const CheckArgs& c, cudaStream_t s) {
    LBM_DISPATCH(storage, reduce_t<S>(buf, a, partials, out8, status, blowup_step, c, s));
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

bool noalloc_is_device_ptr(const void* p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
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
    if (!noalloc_is_device_ptr(populations) || !noalloc_is_device_ptr(out8)) return LBM_ERR_INVALID_ARG;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoallocMaxDevices) return LBM_ERR_CUDA;
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
    cudaError_t e = launch_reduce(storage, populations, a, scratch, out8, nullptr, nullptr, c,
                                  (cudaStream_t)cuda_stream);
    return e == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}
