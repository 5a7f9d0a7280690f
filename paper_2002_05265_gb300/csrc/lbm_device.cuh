// Device code of the D2Q9 stream-and-collide kernels: storage conversions, the per-node
// collision of every model of App. B written in non-equilibrium form, the per-segment pull
// step shared by all stepping kernels, and the single-lattice and multi-lattice step kernels.
//
// Layout in HBM (one lattice): nine SoA planes g_i[y][x], row pitch `pitch` elements (rows
// 32-byte aligned or better), plane = ny * pitch elements.  Stored values are shifted
// populations g_i = f_i - s_i in the storage type, where the shift s_i = f^eq_i(rho0, u_ref)
// is the extended equilibrium at a reference state; with u_ref = 0 (the default) it is
// s_i = w_i rho0.  Two such buffers alternate: a step reads buffer A and writes buffer B.
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
// One-dimensional factor of the extended equilibrium (Eq. extendedFeq, product form):
// phi_0(u) = 2/3 - u^2, phi_+-1(u) = (u^2 +- u + 1/3) / 2.
__host__ __device__ inline double phi1d(int s, double u) {
    return s == 0 ? 2.0 / 3.0 - u * u : 0.5 * (u * u + s * u + 1.0 / 3.0);
}
// Shift s_i = rho0 phi_ex(urx) phi_ey(ury) (= w_i rho0 when u_ref = 0).
__host__ __device__ inline double shift_of(int i, double rho0, double urx, double ury) {
    return rho0 * phi1d(ex_of(i), urx) * phi1d(ey_of(i), ury);
}

// Collision constants, computed once on the host in both precisions (kernels then do no
// FP64 set-up work, which GB300's narrow FP64 pipe would make costly):
// [w_nu, w3, w4, rho0, urx, ury, Px0, Px+, Px-, Py0, Py+, Py-, urx^2 + cs^2, ury^2 + cs^2,
//  ka, kb, kappa, dkappa/dw_nu] -- ka, kb the cumulant model's coefficients
// cs^2 (c4 - kappa), c4 - kappa^2 (c4 = 1 - w4; kappa = 1 - w_nu, 1 or 0 for the
// post-collision, pre-collision or equilibrium rebuild of K~22, field `kread`).
constexpr int kNumConsts = 18;

struct StepArgs {
    int nx, ny;          // lattice size
    int pitch;           // row pitch in elements
    int nseg;            // vector segments per row = ceil(nx / VEC)
    long long plane;     // elements per population plane
    double w_nu, w3, w4; // relaxation frequencies of orders 2, 3, 4
    double rho0;         // shift reference density
    double urx, ury;     // shift reference velocity
    int kread;           // cumulant rebuild: 0 post-collision, 1 pre-collision, 2 equilibrium
    double cd[kNumConsts];   // the constants above, FP64 (filled by fill_consts)
    float cf[kNumConsts];    // the same, rounded to FP32
};

// Second-order central moments of the cumulant model's rebuild of K~22, as a multiple kappa
// of the non-equilibrium ones n: post-collision (1 - w_nu) n, pre-collision n, equilibrium 0.
__host__ __device__ inline double cumulant_kappa(int kread, double w_nu) {
    return kread == 1 ? 1.0 : (kread == 2 ? 0.0 : 1.0 - w_nu);
}

// Fills the constant tables of a StepArgs from its rates, rho0 and shift velocity.
__host__ __device__ inline void fill_consts(StepArgs& a) {
    const double kap = cumulant_kappa(a.kread, a.w_nu), c4 = 1.0 - a.w4;
    const double v[kNumConsts] = {a.w_nu, a.w3, a.w4, a.rho0, a.urx, a.ury,
                                  phi1d(0, a.urx), phi1d(1, a.urx), phi1d(-1, a.urx),
                                  phi1d(0, a.ury), phi1d(1, a.ury), phi1d(-1, a.ury),
                                  a.urx * a.urx + 1.0 / 3.0, a.ury * a.ury + 1.0 / 3.0,
                                  (c4 - kap) / 3.0, c4 - kap * kap, kap, a.kread == 0 ? -1.0 : 0.0};
    for (int k = 0; k < kNumConsts; ++k) {
        a.cd[k] = v[k];
        a.cf[k] = (float)v[k];
    }
}

// ---------------------------------------------------------------------------------------
// Element conversions between the storage type S and the collision type T.
template <typename S> struct Conv;
template <> struct Conv<double> {
    using T = double;
    __device__ static __forceinline__ T to_T(double s) { return s; }
    __device__ static __forceinline__ double from_T(T v) { return v; }
    __device__ static __forceinline__ double to_double(double s) { return s; }
    __device__ static __forceinline__ double from_double(double d) { return d; }
};
template <> struct Conv<float> {
    using T = float;
    __device__ static __forceinline__ T to_T(float s) { return s; }
    __device__ static __forceinline__ float from_T(T v) { return v; }
    __device__ static __forceinline__ double to_double(float s) { return (double)s; }
    __device__ static __forceinline__ float from_double(double d) { return __double2float_rn(d); }
};
template <> struct Conv<__half> {
    using T = float;
    __device__ static __forceinline__ T to_T(__half s) { return __half2float(s); }
    __device__ static __forceinline__ __half from_T(T v) { return __float2half_rn(v); }
    __device__ static __forceinline__ double to_double(__half s) { return (double)__half2float(s); }
    __device__ static __forceinline__ __half from_double(double d) { return __double2half(d); }
};
template <> struct Conv<__nv_bfloat16> {
    using T = float;
    __device__ static __forceinline__ T to_T(__nv_bfloat16 s) { return __bfloat162float(s); }
    __device__ static __forceinline__ __nv_bfloat16 from_T(T v) { return __float2bfloat16_rn(v); }
    __device__ static __forceinline__ double to_double(__nv_bfloat16 s) { return (double)__bfloat162float(s); }
    __device__ static __forceinline__ __nv_bfloat16 from_double(double d) { return __double2bfloat16(d); }
};

// Default vector width: VEC consecutive x-nodes of one row move as one access of
// VEC * sizeof(S) bytes: 16 bytes for FP64 and FP32; for the 16-bit types LBM_HALF_VEC
// nodes (8 = 16-byte accesses, 4 = 8-byte accesses and about half the registers).
#ifndef LBM_HALF_VEC
#define LBM_HALF_VEC 8
#endif
template <typename S> struct DefaultVec {
    static constexpr int value = (sizeof(S) == 2) ? LBM_HALF_VEC : 16 / (int)sizeof(S);
};

template <int BYTES> struct Raw;
template <> struct Raw<4> { using type = uint32_t; };
template <> struct Raw<8> { using type = uint2; };
template <> struct Raw<16> { using type = uint4; };

// aligned vector load / store of VEC elements (VEC * sizeof(S) in {4, 8, 16} bytes)
template <typename S, int VEC>
__device__ __forceinline__ void vload(const S* p, typename Conv<S>::T (&v)[VEC]) {
    using R = typename Raw<VEC * (int)sizeof(S)>::type;
    const R r = *reinterpret_cast<const R*>(p);
    S e[VEC];
    memcpy(e, &r, sizeof(R));
#pragma unroll
    for (int j = 0; j < VEC; ++j) v[j] = Conv<S>::to_T(e[j]);
}
// pairs of floats rounded to a packed pair of 16-bit values in one conversion
__device__ __forceinline__ uint32_t pack2(__half, float a, float b) {
    const __half2 h = __floats2half2_rn(a, b);
    uint32_t u;
    memcpy(&u, &h, 4);
    return u;
}
__device__ __forceinline__ uint32_t pack2(__nv_bfloat16, float a, float b) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    uint32_t u;
    memcpy(&u, &h, 4);
    return u;
}
template <typename S, int VEC>
__device__ __forceinline__ void vstore(S* p, const typename Conv<S>::T (&v)[VEC]) {
    using R = typename Raw<VEC * (int)sizeof(S)>::type;
    R r;
    if constexpr (sizeof(S) == 2) {
        uint32_t w[VEC / 2];
#pragma unroll
        for (int k = 0; k < VEC / 2; ++k) w[k] = pack2(S(), v[2 * k], v[2 * k + 1]);
        memcpy(&r, w, sizeof(R));
    } else {
        S e[VEC];
#pragma unroll
        for (int j = 0; j < VEC; ++j) e[j] = Conv<S>::from_T(v[j]);
        memcpy(&r, e, sizeof(R));
    }
    *reinterpret_cast<R*>(p) = r;
}

// 1/x.  FP32: the hardware approximation (rcp.approx) refined by one Newton-Raphson step,
// r' = r + r (1 - x r), two FMAs; within an ulp of the rounded quotient and free of any
// data-dependent branch, so a lattice that has blown up (non-finite populations) steps as fast
// as a healthy one.  FP64: the correctly rounded reciprocal intrinsic.
__device__ __forceinline__ float recip(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return fmaf(r, fmaf(-x, r, 1.0f), r);
}
__device__ __forceinline__ double recip(double x) { return __drcp_rn(x); }

// Per-launch constants of the collision in the collision precision.
template <typename T> struct Consts {
    T w, w3, w4, rho0, urx, ury;
    T Px[3], Py[3];      // phi_s(u_ref) for s = 0, +1, -1 (shift factors)
    T Xr, Yr;            // mu_2(u_ref) = u_ref^2 + c_s^2 per axis
    T ka, kb;            // cumulant coefficients (see kNumConsts)
};
template <typename T> __device__ __forceinline__ const T* const_table(const StepArgs& a);
template <> __device__ __forceinline__ const float* const_table<float>(const StepArgs& a) { return a.cf; }
template <> __device__ __forceinline__ const double* const_table<double>(const StepArgs& a) { return a.cd; }

template <typename T>
__device__ __forceinline__ Consts<T> make_consts(const StepArgs& a) {
    const T* t = const_table<T>(a);
    Consts<T> c;
    c.w = t[0]; c.w3 = t[1]; c.w4 = t[2]; c.rho0 = t[3]; c.urx = t[4]; c.ury = t[5];
    c.Px[0] = t[6]; c.Px[1] = t[7]; c.Px[2] = t[8];
    c.Py[0] = t[9]; c.Py[1] = t[10]; c.Py[2] = t[11];
    c.Xr = t[12]; c.Yr = t[13];
    c.ka = t[14]; c.kb = t[15];
    return c;
}

// ---------------------------------------------------------------------------------------
// Per-node collision (App. B) on shifted populations g_i = f_i - s_i.
//
// Every model of App. B relaxes the moments of f towards those of f^eq with the same rho
// and u, through a transform that is linear in f for the node's u, and keeps the conserved
// moments (order 0 and 1).  So each model is f* = f - T(u)^-1 D with D = n - n*: n the
// non-equilibrium moments M(f) - M^eq(rho, u), n* their post-collision values, and D's
// conserved components exactly zero.  The kernels compute that directly on the stored
// g = f - s: the nine raw moments of g by x-then-y partial sums; n = M(g) - (M^eq - M(s)),
// where M^eq_pq = rho mu_p(u_x) mu_q(u_y) and M_pq(s) = rho0 mu_p(ur_x) mu_q(ur_y) are the
// product-form moments of Eq. extendedFeq (mu_0 = 1, mu_1 = u, mu_2 = u^2 + c_s^2), their
// difference written without cancellation; the model's relaxation of n (raw, Hermite,
// central, central-Hermite, cumulant, recursive); and g* = g - (back-transform of D, Eq.
// Q9postCollVDF_RM with D_00 = D_10 = D_01 = 0).  BGK is the raw-moment relaxation with one
// rate for every order (exact for the D2Q9 moment basis).  Every intermediate is small, which
// is what makes FP32 arithmetic on FP16-stored populations accurate, and the stored mass and
// momentum change only by the rounding of D.  rho, ux, uy of the pre-collision state are
// returned for diagnostics.  SHIFT = false is the default shift s = w rho0 (u_ref = 0), which
// keeps the shift constants out of the arithmetic.  EQ = 2 (BGK only) uses the second-order
// equilibrium of Sec. 2 in population space; EQ = 3 (BGK only) the partial third-order one of
// Fig. 4 (Hermite A^eq_22 = 0: M^eq_22 without its rho u_x^2 u_y^2 term).
template <int MODEL, int EQ, typename T, bool SHIFT>
__device__ __forceinline__ void collide(const T (&g)[9], T (&o)[9], const Consts<T>& c, T& rho_out, T& ux_out,
                                        T& uy_out) {
    const T cs2 = T(1) / T(3);
    const T w = c.w, w3 = c.w3, w4 = c.w4;
    // x-sums of each row of the velocity set (xi_y = +1, 0, -1) with weights 1, xi_x, xi_x^2
    const T a0p = (g[6] + g[2]) + g[5], a1p = g[5] - g[6], a2p = g[5] + g[6];
    const T a0z = (g[3] + g[0]) + g[1], a1z = g[1] - g[3], a2z = g[1] + g[3];
    const T a0m = (g[7] + g[4]) + g[8], a1m = g[8] - g[7], a2m = g[8] + g[7];
    // raw moments of g (App. B, M_pq = sum xi_x^p xi_y^q g); sum s = rho0, sum xi s = rho0 u_ref
    const T drho = (a0p + a0z) + a0m;
    T jx = (a1p + a1z) + a1m;
    T jy = a0p - a0m;
    const T m20 = (a2p + a2z) + a2m, m02 = a0p + a0m, m11 = a1p - a1m;
    const T m21 = a2p - a2m, m12 = a1p + a1m, m22 = a2p + a2m;
    const T rho = c.rho0 + drho;
    if (SHIFT) {
        jx += c.rho0 * c.urx;
        jy += c.rho0 * c.ury;
    }
    const T irho = recip(rho);
    const T ux = jx * irho, uy = jy * irho;
    const T uxx = ux * ux, uyy = uy * uy;
    rho_out = rho; ux_out = ux; uy_out = uy;

    if (EQ == 2) {
        // second-order equilibrium (Sec. 2, Hermite reading), shift s = w rho0 (u_ref = 0):
        // f^eq_i = w_i rho (1 + 3 xi.u + 4.5 (xi.u)^2 - 1.5 u^2); BGK in population space
        const T usq = T(1.5) * (uxx + uyy);
        const T cc = T(1) - w;
        T fn[9], geq[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const T wi = T(weight_of(i));
            const T eu = T(3) * (T(ex_of(i)) * ux + T(ey_of(i)) * uy);
            geq[i] = wi * drho + wi * rho * (eu + T(0.5) * eu * eu - usq);
            fn[i] = g[i] - geq[i];
        }
        // f^neq carries the rounding of the conserved moments, which (1 - omega) would feed
        // back with a factor ~1 at low viscosity: remove it (populations carrying exactly the
        // residual mass and momentum), the map is unchanged
        const T e0 = ((fn[0] + fn[1]) + (fn[2] + fn[3])) + ((fn[4] + fn[5]) + (fn[6] + fn[7])) + fn[8];
        const T hx = T(0.5) * ((fn[1] - fn[3]) + ((fn[5] - fn[7]) + (fn[8] - fn[6])));
        const T hy = T(0.5) * ((fn[2] - fn[4]) + ((fn[5] - fn[7]) + (fn[6] - fn[8])));
        fn[0] -= e0;
        fn[1] -= hx; fn[3] += hx;
        fn[2] -= hy; fn[4] += hy;
#pragma unroll
        for (int i = 0; i < 9; ++i) o[i] = geq[i] + cc * fn[i];
        return;
    }

    // non-equilibrium raw moments n = M(g) - (M^eq(rho, u) - M(s)) (Eq. extendedFeq)
    T n20, n02, n11, n21, n12, n22;
    if (SHIFT) {
        const T X = uxx + cs2, Y = uyy + cs2;                   // mu_2(u_x), mu_2(u_y)
        const T dx = ux - c.urx, dy = uy - c.ury;               // mu_1(u) - mu_1(u_ref)
        const T dX = dx * (ux + c.urx), dY = dy * (uy + c.ury); // mu_2(u) - mu_2(u_ref)
        const T r0 = c.rho0;
        n20 = m20 - (drho * X + r0 * dX);
        n02 = m02 - (drho * Y + r0 * dY);
        n11 = m11 - (drho * (ux * uy) + r0 * (dx * uy + c.urx * dy));
        n21 = m21 - (drho * (X * uy) + r0 * (dX * uy + c.Xr * dy));
        n12 = m12 - (drho * (ux * Y) + r0 * (dx * Y + c.urx * dY));
        n22 = m22 - (drho * (X * Y) + r0 * (dX * Y + c.Xr * dY));
    } else {
        const T Y = uyy + cs2;
        const T rX = rho * (uxx + cs2);
        n20 = m20 - (cs2 * drho + rho * uxx);
        n02 = m02 - (cs2 * drho + rho * uyy);
        n11 = m11 - rho * (ux * uy);
        n21 = m21 - rX * uy;
        n12 = m12 - (rho * ux) * Y;
        n22 = m22 - (drho * ((uxx + cs2) * Y) + c.rho0 * (uxx * Y + cs2 * uyy));
    }
    if (EQ == 3) n22 += rho * (uxx * uyy);   // M^eq_22 of the partial third-order equilibrium

    // D = n - n* (the moments the collision removes), per model
    T D20, D02, D11, D21, D12, D22;
    if (MODEL == BGK || MODEL == RM) {
        // Eq. RMcoll (BGK: one rate for every order)
        const T r3 = (MODEL == BGK) ? w : w3, r4 = (MODEL == BGK) ? w : w4;
        D20 = w * n20; D02 = w * n02; D11 = w * n11;
        D21 = r3 * n21; D12 = r3 * n12; D22 = r4 * n22;
    } else if (MODEL == HM || MODEL == PR) {
        // Hermite moments: A_2 = n_2, A_21 = n_21, A_12 = n_12 (conserved parts vanish),
        // A_22 = n_22 - c_s^2 (n_20 + n_02); relaxed, back with Eq. HM2RM_Q9
        D20 = w * n20; D02 = w * n02; D11 = w * n11;
        if (MODEL == HM) {
            D21 = w3 * n21; D12 = w3 * n12;
            D22 = w4 * (n22 - cs2 * (n20 + n02)) + cs2 * (D20 + D02);
        } else {   // PR: omega3 = omega4 = 1
            D21 = n21; D12 = n12;
            D22 = (n22 - cs2 * (n20 + n02)) + cs2 * (D20 + D02);
        }
    } else if (MODEL == RR) {
        // Eqs. HMColl_Q9, RRformulas_D2Q9: third/fourth-order A^neq from the recursion,
        // A* = A^eq + (1 - omega) A^neq_rec, so D = A^neq - (1 - omega) A^neq_rec
        const T a21 = uy * n20 + T(2) * ux * n11;
        const T a12 = ux * n02 + T(2) * uy * n11;
        const T a22 = uyy * n20 + uxx * n02 + T(4) * ux * uy * n11;
        const T c3 = T(1) - w3, c4 = T(1) - w4;
        D20 = w * n20; D02 = w * n02; D11 = w * n11;
        D21 = n21 - c3 * a21; D12 = n12 - c3 * a12;
        D22 = (n22 - cs2 * (n20 + n02)) - c4 * a22 + cs2 * (D20 + D02);
    } else {
        // central moments k = S(-u) n of f^neq (binomial shift, first-order parts vanish),
        // relaxed by order (d = rates . k), shifted back D = S(u) d.  The three linear steps are
        // folded into one expression in n: with a21 = 2 ux n11 + uy n20, a12 = 2 uy n11 + ux n02,
        // R = 2 (ux n12 + uy n21) and Q = ux^2 n02 + uy^2 n20 + 4 ux uy n11 one has
        // k21 = n21 - a21, k12 = n12 - a12, k22 = n22 - R + Q, and
        //   D21 = w3 n21 + (w - w3) a21,   D12 = w3 n12 + (w - w3) a12,
        //   D22 = w4 n22 + (w3 - w4) R + (w - 2 w3 + w4) Q + (model terms),
        // the model terms being d22 - w4 k22 (zero for CM).
        const T uxy = ux * uy;
        const T a21 = T(2) * ux * n11 + uy * n20, a12 = T(2) * uy * n11 + ux * n02;
        const T R = T(2) * (ux * n12 + uy * n21);
        const T Q = uxx * n02 + uyy * n20 + T(4) * uxy * n11;
        D20 = w * n20; D02 = w * n02; D11 = w * n11;
        D21 = w3 * n21 + (w - w3) * a21;
        D12 = w3 * n12 + (w - w3) * a12;
        T D22c = w4 * n22 + (w3 - w4) * R + (w - T(2) * w3 + w4) * Q;
        if (MODEL == CHM) {
            // central Hermite: A~_22 = K~_22 - c_s^2 (K~_20 + K~_02) relaxed with w4, the
            // second order with w (Eqs. CHpoly, CHMcoll): d22 = w4 A~_22 + c_s^2 (d20 + d02)
            // = w4 k22 + c_s^2 (w - w4) (n20 + n02)
            D22c += (cs2 * (w - w4)) * (n20 + n02);
        } else if (MODEL != CM) {
            // cumulants: C22 = K22 - (K20 K02 + 2 K11^2)/rho relaxes to 0 and K22* is rebuilt
            // with second-order central moments kappa n (written for deviations from the
            // equilibrium central moments rho c_s^2, 0, rho c_s^4): kappa = 1 - w for the
            // post-collision values (the paper's K), 1 or 0 for the pre-collision / equilibrium
            // readings.  With S = n20 + n02, P = n20 n02 + 2 n11^2 and c4 = 1 - w4:
            // C22 = k22 - c_s^2 S - P / rho, K22* = c4 C22 + c_s^2 kappa S + kappa^2 P / rho, so
            // d22 = k22 - K22* = w4 k22 + ka S + kb P / rho with the per-launch constants
            // ka = c_s^2 (c4 - kappa), kb = c4 - kappa^2
            const T P = n20 * n02 + T(2) * n11 * n11;
            D22c += c.ka * (n20 + n02) + (c.kb * irho) * P;
        }
        D22 = D22c;
    }

    // g* = g - (Eq. Q9postCollVDF_RM applied to D, with D_00 = D_10 = D_01 = 0)
    const T h = T(0.5), q = T(0.25);
    o[0] = g[0] - (D22 - (D20 + D02));
    o[1] = g[1] - h * ((D20 - D22) - D12);
    o[3] = g[3] - h * ((D20 - D22) + D12);
    o[2] = g[2] - h * ((D02 - D22) - D21);
    o[4] = g[4] - h * ((D02 - D22) + D21);
    o[5] = g[5] - q * ((D22 + D11) + (D12 + D21));
    o[6] = g[6] - q * ((D22 - D11) + (D21 - D12));
    o[7] = g[7] - q * ((D22 + D11) - (D12 + D21));
    o[8] = g[8] - q * ((D22 - D11) + (D12 - D21));
}

// Per-thread FP64 accumulators of the blow-up diagnostics (used by the batched sweep).
struct Diag {
    double pert;      // sum |u - u_ref|^2
    double ke;        // sum |u|^2
    double rho_min;   // min rho
    double nonfinite; // count of nodes with a non-finite rho or u
};

// ---------------------------------------------------------------------------------------
// Gather of the nine planes of one vector segment (VEC consecutive x-nodes of row y) at the
// periodic offsets -SIGN * xi_i: SIGN = +1 gives the populations that node x collides,
// f_i(x) = A_i(x - xi_i) (pull); SIGN = -1 gives lambda_i(x + xi_i) (reverse streaming of the
// adjoint).  All 32 lanes call it together with consecutive segments; loads are aligned
// vectors, the x-shifted element comes from the neighbouring lane by a warp shuffle, or from
// one scalar load at warp and row edges (where the periodic wrap is applied).
template <typename S, int VEC, int SIGN>
__device__ __forceinline__ void gather_pull(const S* __restrict__ src, int nx, int ny, int pitch, long long plane,
                                            int y, int seg, int nseg, int x0, int nvalid, int lane,
                                            typename Conv<S>::T (&f)[9][VEC]) {
    using T = typename Conv<S>::T;
    const int ym = (y == 0) ? ny - 1 : y - 1;
    const int yp = (y == ny - 1) ? 0 : y + 1;
    const bool left_from_lane = (lane > 0) && (seg > 0);
    const bool right_from_lane = (lane < 31) && (seg < nseg - 1);
    const int xl = (x0 == 0) ? nx - 1 : x0 - 1;           // source of an x-offset of -1 at j = 0
    const int xr = (x0 + nvalid >= nx) ? 0 : x0 + VEC;     // source of an x-offset of +1 at j = nvalid-1
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int ex = SIGN * ex_of(i), ey = SIGN * ey_of(i);
        const int row = (ey == 1) ? ym : ((ey == -1) ? yp : y);
        const S* p = src + (long long)i * plane + (long long)row * pitch;
        T v[VEC];
        vload<S, VEC>(p + x0, v);
        if (ex == 0) {
#pragma unroll
            for (int j = 0; j < VEC; ++j) f[i][j] = v[j];
        } else if (ex == 1) {
            T left = __shfl_up_sync(0xffffffffu, v[VEC - 1], 1);
            if (!left_from_lane) left = Conv<S>::to_T(p[xl]);
            f[i][0] = left;
#pragma unroll
            for (int j = 1; j < VEC; ++j) f[i][j] = v[j - 1];
        } else {
            T right = __shfl_down_sync(0xffffffffu, v[0], 1);
            if (!right_from_lane) right = Conv<S>::to_T(p[xr]);
#pragma unroll
            for (int j = 0; j < VEC - 1; ++j) f[i][j] = (j + 1 < nvalid) ? v[j + 1] : right;
            f[i][VEC - 1] = right;
        }
    }
}

// ---------------------------------------------------------------------------------------
// One pull step of one vector segment (VEC consecutive x-nodes of one row): gather
// (periodic) -> collide -> store.  All 32 lanes of the warp call it together with
// consecutive segment indices s = base + lane (base a multiple of 32); lanes with s >= total
// take part in the shuffles and store nothing.
template <int MODEL, int EQ, typename S, int VEC, bool DIAG, bool SHIFT>
__device__ __forceinline__ void step_segment(const S* __restrict__ src, S* __restrict__ dst, const StepArgs& a,
                                             const Consts<typename Conv<S>::T>& c, unsigned s, unsigned total,
                                             int lane, Diag& dg) {
    using T = typename Conv<S>::T;
    const bool active = s < total;
    const unsigned sc = active ? s : total - 1;
    const int y = (int)(sc / (unsigned)a.nseg);
    const int seg = (int)(sc - (unsigned)y * (unsigned)a.nseg);
    const int x0 = seg * VEC;
    const int nvalid = min(VEC, a.nx - x0);
    T f[9][VEC];
    gather_pull<S, VEC, 1>(src, a.nx, a.ny, a.pitch, a.plane, y, seg, a.nseg, x0, nvalid, lane, f);

    T out[9][VEC];
#pragma unroll
    for (int j = 0; j < VEC; ++j) {
        T gin[9], gout[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) gin[i] = f[i][j];
        T rho, ux, uy;
        collide<MODEL, EQ, T, SHIFT>(gin, gout, c, rho, ux, uy);
#pragma unroll
        for (int i = 0; i < 9; ++i) out[i][j] = gout[i];
        if (DIAG) {
            if (active && j < nvalid) {
                if (isfinite(rho) && isfinite(ux) && isfinite(uy)) {
                    const T wx = ux - c.urx, wy = uy - c.ury;
                    dg.pert += (double)(wx * wx + wy * wy);
                    dg.ke += (double)(ux * ux + uy * uy);
                    dg.rho_min = fmin(dg.rho_min, (double)rho);
                } else {
                    dg.nonfinite += 1.0;
                }
            }
        }
    }
    if (active) {
#pragma unroll
        for (int i = 0; i < 9; ++i) vstore<S, VEC>(dst + (long long)i * a.plane + (long long)y * a.pitch + x0, out[i]);
    }
}

// ---------------------------------------------------------------------------------------
// Single-lattice step: warps walk the lattice with a grid-stride loop (the grid is sized to
// the resident CTAs of the GPU).
template <int MODEL, int EQ, typename S, bool SHIFT>
__global__ void __launch_bounds__(256) step_kernel(const S* __restrict__ src, S* __restrict__ dst, StepArgs a) {
    using T = typename Conv<S>::T;
    constexpr int VEC = DefaultVec<S>::value;
    const int lane = threadIdx.x & 31;
    const unsigned total = (unsigned)a.ny * (unsigned)a.nseg;
    const unsigned stride = gridDim.x * blockDim.x;
    const Consts<T> c = make_consts<T>(a);
    Diag dg;
    for (unsigned base = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < total; base += stride)
        step_segment<MODEL, EQ, S, VEC, false, SHIFT>(src, dst, a, c, base + lane, total, lane, dg);
}

// ---------------------------------------------------------------------------------------
// Multi-lattice step: one launch advances every lattice of a group by one time step.  The
// lattices' segment ranges, each padded to a multiple of 32, are concatenated; a warp finds
// its lattice from the warp-aligned base index and runs that lattice's collision model.
// One launch per time step instead of one per lattice removes the per-launch ramp and the
// gaps between graph nodes that dominate small (<= 1024^2) lattices.
constexpr int kGroupMax = 16;

struct GroupEntry {
    const void* src;    // buffers of the storage type of the launch
    void* dst;
    StepArgs a;
    int model;          // lbm::Model
    int eq_order;       // 4, or 2 / 3 (BGK only)
    unsigned begin;     // first padded segment index of this lattice
    unsigned total;     // ny * nseg (unpadded)
};
struct GroupArgs {
    int n;
    unsigned padded_total;
    GroupEntry e[kGroupMax];
};

template <typename S, bool SH>
__device__ __forceinline__ void group_segment(const GroupEntry& e, const Consts<typename Conv<S>::T>& c,
                                              unsigned local, int lane) {
    constexpr int VEC = DefaultVec<S>::value;
    Diag dg;
    const unsigned s = local + lane;
    const S* src = static_cast<const S*>(e.src);
    S* dst = static_cast<S*>(e.dst);
    switch (e.model) {
        case BGK:
            if (e.eq_order == 2) step_segment<BGK, 2, S, VEC, false, SH>(src, dst, e.a, c, s, e.total, lane, dg);
            else if (e.eq_order == 3) step_segment<BGK, 3, S, VEC, false, SH>(src, dst, e.a, c, s, e.total, lane, dg);
            else step_segment<BGK, 4, S, VEC, false, SH>(src, dst, e.a, c, s, e.total, lane, dg);
            break;
        case RM: step_segment<RM, 4, S, VEC, false, SH>(src, dst, e.a, c, s, e.total, lane, dg); break;
        case HM: step_segment<HM, 4, S, VEC, false, SH>(src, dst, e.a, c, s, e.total, lane, dg); break;
        case CM: step_segment<CM, 4, S, VEC, false, SH>(src, dst, e.a, c, s, e.total, lane, dg); break;
        case CHM: step_segment<CHM, 4, S, VEC, false, SH>(src, dst, e.a, c, s, e.total, lane, dg); break;
        case CUM: step_segment<CUM, 4, S, VEC, false, SH>(src, dst, e.a, c, s, e.total, lane, dg); break;
        case PR: step_segment<PR, 4, S, VEC, false, SH>(src, dst, e.a, c, s, e.total, lane, dg); break;
        default: step_segment<RR, 4, S, VEC, false, SH>(src, dst, e.a, c, s, e.total, lane, dg); break;
    }
}

template <typename S, bool SHIFT>
__global__ void __launch_bounds__(256) group_step_kernel(const __grid_constant__ GroupArgs g) {
    using T = typename Conv<S>::T;
    const int lane = threadIdx.x & 31;
    const unsigned stride = gridDim.x * blockDim.x;
    for (unsigned base = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < g.padded_total; base += stride) {
        int k = 0;
        while (k + 1 < g.n && base >= g.e[k + 1].begin) ++k;
        group_segment<S, SHIFT>(g.e[k], make_consts<T>(g.e[k].a), base - g.e[k].begin, lane);
    }
}

}  // namespace lbm
