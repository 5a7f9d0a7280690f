// Device code of the D2Q9 stream-and-collide kernels: storage traits, the per-node collision
// of every model of App. B written in non-equilibrium form, and the fused pull kernel.
//
// Layout in HBM (one lattice): nine SoA planes g_i[y][x], row pitch `pitch` elements
// (multiple of 32, so every row starts 128-byte aligned), plane = ny * pitch elements.
// Stored values are shifted populations g_i = f_i - w_i rho0 in the storage type.
// Two such buffers alternate: a step reads buffer A and writes buffer B.
//
// Buffer semantics: A_i(z) holds the post-collision population f*_i(z, t-1) emitted by node z,
// so node x gathers its pre-collision populations as f_i(x, t) = A_i(x - xi_i) (pull form of
// Eq. StreamCollide), collides them, and writes f*_i(x, t) to B_i(x).
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace lbm {

enum Model { BGK = 0, RM = 1, HM = 2, CM = 3, CHM = 4, CUM = 5, PR = 6, RR = 7 };

// D2Q9 velocities in the library's index order.
__host__ __device__ constexpr int ex_of(int i) {
    return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0);
}
__host__ __device__ constexpr int ey_of(int i) {
    return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
}
// D2Q9 weights w_i = W(ex) W(ey), W(0) = 2/3, W(+-1) = 1/6.
__host__ __device__ constexpr double weight_of(int i) {
    return (i == 0) ? 4.0 / 9.0 : ((i <= 4) ? 1.0 / 9.0 : 1.0 / 36.0);
}

struct StepArgs {
    int nx, ny;          // lattice size
    int pitch;           // row pitch in elements
    int nseg;            // vector segments per row = ceil(nx / VEC)
    long long plane;     // elements per population plane
    double w_nu, w3, w4; // relaxation frequencies of orders 2, 3, 4
    double rho0;         // shift reference density
};

// ---------------------------------------------------------------------------------------
// Storage traits: VEC consecutive x-nodes move as one 16-byte vector.
template <typename S> struct Store;

template <> struct Store<double> {
    using T = double;
    static constexpr int VEC = 2;
    __device__ static __forceinline__ void load(const double* p, T (&v)[VEC]) {
        const double2 t = *reinterpret_cast<const double2*>(p);
        v[0] = t.x; v[1] = t.y;
    }
    __device__ static __forceinline__ void store(double* p, const T (&v)[VEC]) {
        *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
    }
    __device__ static __forceinline__ T load1(const double* p) { return *p; }
    __device__ static __forceinline__ double to_double(double s) { return s; }
    __device__ static __forceinline__ double from_double(double d) { return d; }
};

template <> struct Store<float> {
    using T = float;
    static constexpr int VEC = 4;
    __device__ static __forceinline__ void load(const float* p, T (&v)[VEC]) {
        const float4 t = *reinterpret_cast<const float4*>(p);
        v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
    }
    __device__ static __forceinline__ void store(float* p, const T (&v)[VEC]) {
        *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
    }
    __device__ static __forceinline__ T load1(const float* p) { return *p; }
    __device__ static __forceinline__ double to_double(float s) { return (double)s; }
    __device__ static __forceinline__ float from_double(double d) { return __double2float_rn(d); }
};

template <> struct Store<__half> {
    using T = float;
    static constexpr int VEC = 8;
    __device__ static __forceinline__ void load(const __half* p, T (&v)[VEC]) {
        const uint4 t = *reinterpret_cast<const uint4*>(p);
        const uint32_t w[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            __half2 h = *reinterpret_cast<const __half2*>(&w[k]);
            const float2 f = __half22float2(h);
            v[2 * k] = f.x; v[2 * k + 1] = f.y;
        }
    }
    __device__ static __forceinline__ void store(__half* p, const T (&v)[VEC]) {
        uint32_t w[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            __half2 h = __floats2half2_rn(v[2 * k], v[2 * k + 1]);
            w[k] = *reinterpret_cast<uint32_t*>(&h);
        }
        *reinterpret_cast<uint4*>(p) = make_uint4(w[0], w[1], w[2], w[3]);
    }
    __device__ static __forceinline__ T load1(const __half* p) { return __half2float(*p); }
    __device__ static __forceinline__ double to_double(__half s) { return (double)__half2float(s); }
    __device__ static __forceinline__ __half from_double(double d) { return __double2half(d); }
};

template <> struct Store<__nv_bfloat16> {
    using T = float;
    static constexpr int VEC = 8;
    __device__ static __forceinline__ void load(const __nv_bfloat16* p, T (&v)[VEC]) {
        const uint4 t = *reinterpret_cast<const uint4*>(p);
        const uint32_t w[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            __nv_bfloat162 h = *reinterpret_cast<const __nv_bfloat162*>(&w[k]);
            const float2 f = __bfloat1622float2(h);
            v[2 * k] = f.x; v[2 * k + 1] = f.y;
        }
    }
    __device__ static __forceinline__ void store(__nv_bfloat16* p, const T (&v)[VEC]) {
        uint32_t w[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * k], v[2 * k + 1]);
            w[k] = *reinterpret_cast<uint32_t*>(&h);
        }
        *reinterpret_cast<uint4*>(p) = make_uint4(w[0], w[1], w[2], w[3]);
    }
    __device__ static __forceinline__ T load1(const __nv_bfloat16* p) { return __bfloat162float(*p); }
    __device__ static __forceinline__ double to_double(__nv_bfloat16 s) { return (double)__bfloat162float(s); }
    __device__ static __forceinline__ __nv_bfloat16 from_double(double d) { return __double2bfloat16(d); }
};

// ---------------------------------------------------------------------------------------
// Per-node collision (App. B) on shifted populations g_i = f_i - w_i rho0.
//
// Every model of App. B relaxes the moments of f towards those of f^eq with the same rho
// and u, through a transform that is linear in f for the node's u.  So each model can be
// written as f* = f^eq + T(u)^-1 [ (1 - omega_n) T(u) f^neq ] with f^neq = f - f^eq, where
// the conserved (order 0 and 1) non-equilibrium moments are exactly zero.  Working with
// f^neq and the deviation g^eq = f^eq - w rho0 keeps every intermediate small, which is what
// makes FP32 arithmetic on FP16-stored populations accurate.  The cumulant model adds the
// C22 product terms, the recursive regularized model the recursion of Eq. RRformulas_D2Q9.
template <int MODEL, int EQ, typename T>
__device__ __forceinline__ void collide(const T (&g)[9], T (&o)[9], T w, T w3, T w4, T rho0) {
    const T cs2 = T(1) / T(3);
    // density and velocity (Sec. 1): sums of the shifted populations
    const T drho = ((g[0] + g[1]) + (g[2] + g[3])) + ((g[4] + g[5]) + (g[6] + g[7])) + g[8];
    const T rho = rho0 + drho;
    const T jx = (g[1] - g[3]) + ((g[5] - g[7]) + (g[8] - g[6]));
    const T jy = (g[2] - g[4]) + ((g[5] - g[7]) + (g[6] - g[8]));
    const T irho = T(1) / rho;
    const T ux = jx * irho, uy = jy * irho;
    const T uxx = ux * ux, uyy = uy * uy;

    // g^eq_i = f^eq_i - w_i rho0
    T geq[9];
    if (EQ == 4) {
        // Eq. extendedFeq, product form: f^eq_(sx,sy) = rho phi_sx(u_x) phi_sy(u_y) with
        // phi_s = W_s + d_s: W_0 = 2/3, W_+-1 = 1/6, d_0 = -u^2, d_+-1 = (u^2 +- u)/2.
        const T W0 = T(2) / T(3), W1 = T(1) / T(6);
        const T dx0 = -uxx, dxp = T(0.5) * (uxx + ux), dxm = T(0.5) * (uxx - ux);
        const T dy0 = -uyy, dyp = T(0.5) * (uyy + uy), dym = T(0.5) * (uyy - uy);
        // rho * (W_a d_b + d_a W_b + d_a d_b) + W_a W_b drho
#define LBM_GEQ(Wa, da, Wb, db) ((Wa) * (Wb) * drho + rho * ((Wa) * (db) + (da) * ((Wb) + (db))))
        geq[0] = LBM_GEQ(W0, dx0, W0, dy0);
        geq[1] = LBM_GEQ(W1, dxp, W0, dy0);
        geq[2] = LBM_GEQ(W0, dx0, W1, dyp);
        geq[3] = LBM_GEQ(W1, dxm, W0, dy0);
        geq[4] = LBM_GEQ(W0, dx0, W1, dym);
        geq[5] = LBM_GEQ(W1, dxp, W1, dyp);
        geq[6] = LBM_GEQ(W1, dxm, W1, dyp);
        geq[7] = LBM_GEQ(W1, dxm, W1, dym);
        geq[8] = LBM_GEQ(W1, dxp, W1, dym);
#undef LBM_GEQ
    } else {
        // second-order equilibrium (Sec. 2, Hermite reading):
        // f^eq_i = w_i rho (1 + 3 xi.u + 4.5 (xi.u)^2 - 1.5 u^2)
        const T usq = T(1.5) * (uxx + uyy);
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const T wi = T(weight_of(i));
            const T eu = T(3) * (T(ex_of(i)) * ux + T(ey_of(i)) * uy);
            geq[i] = wi * drho + wi * rho * (eu + T(0.5) * eu * eu - usq);
        }
    }

    T fn[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) fn[i] = g[i] - geq[i];

    if (MODEL == BGK) {
        const T c = T(1) - w;
#pragma unroll
        for (int i = 0; i < 9; ++i) o[i] = geq[i] + c * fn[i];
        return;
    }

    // raw moments of f^neq (App. B, M_pq = sum xi_x^p xi_y^q f), x sums then y sums
    const T a0p = (fn[6] + fn[2]) + fn[5], a1p = fn[5] - fn[6], a2p = fn[5] + fn[6];
    const T a0m = (fn[7] + fn[4]) + fn[8], a1m = fn[8] - fn[7], a2m = fn[8] + fn[7];
    const T a2z = fn[1] + fn[3];
    const T m20 = (a2m + a2z) + a2p, m02 = a0p + a0m, m11 = a1p - a1m;
    const T m21 = a2p - a2m, m12 = a1p + a1m, m22 = a2p + a2m;

    const T c2 = T(1) - w, c3 = T(1) - w3, c4 = T(1) - w4;
    T M20, M02, M11, M21, M12, M22;   // post-collision non-equilibrium raw moments
    if (MODEL == RM) {
        // Eq. RMcoll
        M20 = c2 * m20; M02 = c2 * m02; M11 = c2 * m11;
        M21 = c3 * m21; M12 = c3 * m12; M22 = c4 * m22;
    } else if (MODEL == HM || MODEL == PR) {
        // Hermite moments: A_2 = M_2, A_21 = M_21, A_12 = M_12 (conserved parts vanish),
        // A_22 = M_22 - c_s^2 (M_20 + M_02); back with Eq. HM2RM_Q9
        M20 = c2 * m20; M02 = c2 * m02; M11 = c2 * m11;
        if (MODEL == HM) {
            M21 = c3 * m21; M12 = c3 * m12;
            M22 = c4 * (m22 - cs2 * (m20 + m02)) + cs2 * (M20 + M02);
        } else {   // PR: omega3 = omega4 = 1
            M21 = T(0); M12 = T(0);
            M22 = cs2 * (M20 + M02);
        }
    } else if (MODEL == RR) {
        // Eqs. HMColl_Q9, RRformulas_D2Q9: third/fourth-order A^neq from the recursion
        const T a21 = uy * m20 + T(2) * ux * m11;
        const T a12 = ux * m02 + T(2) * uy * m11;
        const T a22 = uyy * m20 + uxx * m02 + T(4) * ux * uy * m11;
        M20 = c2 * m20; M02 = c2 * m02; M11 = c2 * m11;
        M21 = c3 * a21; M12 = c3 * a12;
        M22 = c4 * a22 + cs2 * (M20 + M02);
    } else {
        // central moments of f^neq: binomial shift by -u (first-order parts vanish)
        const T k20 = m20, k02 = m02, k11 = m11;
        const T k21 = m21 - T(2) * ux * m11 - uy * m20;
        const T k12 = m12 - T(2) * uy * m11 - ux * m02;
        const T k22 = m22 - T(2) * ux * m12 - T(2) * uy * m21 + uxx * m02 + uyy * m20 + T(4) * ux * uy * m11;
        const T K20 = c2 * k20, K02 = c2 * k02, K11 = c2 * k11;
        const T K21 = c3 * k21, K12 = c3 * k12;
        T K22;
        if (MODEL == CM) {
            K22 = c4 * k22;
        } else if (MODEL == CHM) {
            // central Hermite: A~_22 = K~_22 - c_s^2 (K~_20 + K~_02)   (Eqs. CHpoly, CHMcoll)
            K22 = c4 * (k22 - cs2 * (k20 + k02)) + cs2 * (K20 + K02);
        } else {
            // cumulants: C22 = K22 - (K20 K02 + 2 K11^2)/rho relaxes to 0; rebuilt with the
            // post-collision second-order central moments (written for deviations from
            // the equilibrium central moments rho c_s^2, 0, rho c_s^4)
            const T C22 = k22 - cs2 * (k20 + k02) - (k20 * k02 + T(2) * k11 * k11) * irho;
            K22 = c4 * C22 + cs2 * (K20 + K02) + (K20 * K02 + T(2) * K11 * K11) * irho;
        }
        // back to raw moments: binomial shift by +u
        M20 = K20; M02 = K02; M11 = K11;
        M21 = K21 + T(2) * ux * K11 + uy * K20;
        M12 = K12 + T(2) * uy * K11 + ux * K02;
        M22 = K22 + T(2) * ux * K12 + T(2) * uy * K21 + uxx * K02 + uyy * K20 + T(4) * ux * uy * K11;
    }

    // Eq. Q9postCollVDF_RM with M00 = M10 = M01 = 0 (non-equilibrium part), added to g^eq
    const T h = T(0.5), q = T(0.25);
    o[0] = geq[0] + (M22 - (M20 + M02));
    o[1] = geq[1] + h * ((M20 - M22) - M12);
    o[3] = geq[3] + h * ((M20 - M22) + M12);
    o[2] = geq[2] + h * ((M02 - M22) - M21);
    o[4] = geq[4] + h * ((M02 - M22) + M21);
    o[5] = geq[5] + q * ((M22 + M11) + (M12 + M21));
    o[6] = geq[6] + q * ((M22 - M11) + (M21 - M12));
    o[7] = geq[7] + q * ((M22 + M11) - (M12 + M21));
    o[8] = geq[8] + q * ((M22 - M11) + (M12 - M21));
}

// ---------------------------------------------------------------------------------------
// Fused pull step: gather (periodic) -> collide -> store, one thread per VEC consecutive
// x-nodes of one row.  Loads and stores are aligned 16-byte vectors; the x-shifted planes
// take their edge element from the neighbouring lane with a warp shuffle, or with one scalar
// load at warp and row edges (where the periodic wrap is applied).  Warps walk the lattice
// with a grid-stride loop (the grid is sized to the resident CTAs of the GPU).
template <int MODEL, int EQ, typename S>
__global__ void __launch_bounds__(256) step_kernel(const S* __restrict__ src, S* __restrict__ dst, StepArgs a) {
    using St = Store<S>;
    using T = typename St::T;
    constexpr int VEC = St::VEC;
    const int lane = threadIdx.x & 31;
    const unsigned total = (unsigned)a.ny * (unsigned)a.nseg;
    const unsigned stride = gridDim.x * blockDim.x;
    const T w = (T)a.w_nu, w3 = (T)a.w3, w4 = (T)a.w4, rho0 = (T)a.rho0;

    for (unsigned base = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < total; base += stride) {
        const unsigned s = base + lane;
        const bool active = s < total;
        const unsigned sc = active ? s : total - 1;
        const int y = (int)(sc / (unsigned)a.nseg);
        const int seg = (int)(sc - (unsigned)y * (unsigned)a.nseg);
        const int x0 = seg * VEC;
        const int nvalid = min(VEC, a.nx - x0);
        const int ym = (y == 0) ? a.ny - 1 : y - 1;
        const int yp = (y == a.ny - 1) ? 0 : y + 1;
        const bool left_from_lane = (lane > 0) && (seg > 0);
        const bool right_from_lane = (lane < 31) && (seg < a.nseg - 1);
        const int xl = (x0 == 0) ? a.nx - 1 : x0 - 1;           // source of xi_x = +1 at j = 0
        const int xr = (x0 + nvalid >= a.nx) ? 0 : x0 + VEC;     // source of xi_x = -1 at j = nvalid-1

        T f[9][VEC];
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const int ex = ex_of(i), ey = ey_of(i);
            const int row = (ey == 1) ? ym : ((ey == -1) ? yp : y);
            const S* p = src + (long long)i * a.plane + (long long)row * a.pitch;
            T v[VEC];
            St::load(p + x0, v);
            if (ex == 0) {
#pragma unroll
                for (int j = 0; j < VEC; ++j) f[i][j] = v[j];
            } else if (ex == 1) {
                T left = __shfl_up_sync(0xffffffffu, v[VEC - 1], 1);
                if (!left_from_lane) left = St::load1(p + xl);
                f[i][0] = left;
#pragma unroll
                for (int j = 1; j < VEC; ++j) f[i][j] = v[j - 1];
            } else {
                T right = __shfl_down_sync(0xffffffffu, v[0], 1);
                if (!right_from_lane) right = St::load1(p + xr);
#pragma unroll
                for (int j = 0; j < VEC - 1; ++j) f[i][j] = (j + 1 < nvalid) ? v[j + 1] : right;
                f[i][VEC - 1] = right;
            }
        }

        T out[9][VEC];
#pragma unroll
        for (int j = 0; j < VEC; ++j) {
            T gin[9], gout[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) gin[i] = f[i][j];
            collide<MODEL, EQ, T>(gin, gout, w, w3, w4, rho0);
#pragma unroll
            for (int i = 0; i < 9; ++i) out[i][j] = gout[i];
        }
        if (active) {
#pragma unroll
            for (int i = 0; i < 9; ++i)
                St::store(dst + (long long)i * a.plane + (long long)y * a.pitch + x0, out[i]);
        }
    }
}

}  // namespace lbm
