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
// [w_nu, w3, w4, rho0, urx, ury, Px0, Px+, Px-, Py0, Py+, Py-].
constexpr int kNumConsts = 12;

struct StepArgs {
    int nx, ny;          // lattice size
    int pitch;           // row pitch in elements
    int nseg;            // vector segments per row = ceil(nx / VEC)
    long long plane;     // elements per population plane
    double w_nu, w3, w4; // relaxation frequencies of orders 2, 3, 4
    double rho0;         // shift reference density
    double urx, ury;     // shift reference velocity
    double cd[kNumConsts];   // the constants above, FP64 (filled by fill_consts)
    float cf[kNumConsts];    // the same, rounded to FP32
};

// Fills the constant tables of a StepArgs from its rates, rho0 and shift velocity.
__host__ __device__ inline void fill_consts(StepArgs& a) {
    const double v[kNumConsts] = {a.w_nu, a.w3, a.w4, a.rho0, a.urx, a.ury,
                                  phi1d(0, a.urx), phi1d(1, a.urx), phi1d(-1, a.urx),
                                  phi1d(0, a.ury), phi1d(1, a.ury), phi1d(-1, a.ury)};
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

// Correctly rounded reciprocal (the reciprocal intrinsic instead of a full division).
__device__ __forceinline__ float recip(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double recip(double x) { return __drcp_rn(x); }

// Per-launch constants of the collision in the collision precision.
template <typename T> struct Consts {
    T w, w3, w4, rho0, urx, ury;
    T Px[3], Py[3];      // phi_s(u_ref) for s = 0, +1, -1 (shift factors)
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
    return c;
}

// ---------------------------------------------------------------------------------------
// Per-node collision (App. B) on shifted populations g_i = f_i - s_i.
//
// Every model of App. B relaxes the moments of f towards those of f^eq with the same rho
// and u, through a transform that is linear in f for the node's u.  So each model can be
// written as f* = f^eq + T(u)^-1 [ (1 - omega_n) T(u) f^neq ] with f^neq = f - f^eq, where
// the conserved (order 0 and 1) non-equilibrium moments are exactly zero.  Working with
// f^neq and the deviation g^eq = f^eq - s keeps every intermediate small, which is what
// makes FP32 arithmetic on FP16-stored populations accurate.  The cumulant model adds the
// C22 product terms, the recursive regularized model the recursion of Eq. RRformulas_D2Q9.
// rho, ux, uy of the pre-collision state are returned for diagnostics.  SHIFT = false is the
// default shift s = w rho0 (u_ref = 0) with compile-time weights, which keeps the shift
// constants out of registers.
template <int MODEL, int EQ, typename T, bool SHIFT>
__device__ __forceinline__ void collide(const T (&g)[9], T (&o)[9], const Consts<T>& c, T& rho_out, T& ux_out,
                                        T& uy_out) {
    const T cs2 = T(1) / T(3);
    const T w = c.w, w3 = c.w3, w4 = c.w4;
    // density and velocity (Sec. 1): sum s_i = rho0, sum xi_i s_i = rho0 u_ref
    const T drho = ((g[0] + g[1]) + (g[2] + g[3])) + ((g[4] + g[5]) + (g[6] + g[7])) + g[8];
    const T rho = c.rho0 + drho;
    T jx = (g[1] - g[3]) + ((g[5] - g[7]) + (g[8] - g[6]));
    T jy = (g[2] - g[4]) + ((g[5] - g[7]) + (g[6] - g[8]));
    if (SHIFT) {
        jx += c.rho0 * c.urx;
        jy += c.rho0 * c.ury;
    }
    const T irho = recip(rho);
    const T ux = jx * irho, uy = jy * irho;
    const T uxx = ux * ux, uyy = uy * uy;
    rho_out = rho; ux_out = ux; uy_out = uy;

    // g^eq_i = f^eq_i - s_i
    T geq[9];
    if (EQ == 4) {
        // Eq. extendedFeq, product form: f^eq_(sx,sy) = rho phi_sx(u_x) phi_sy(u_y), written as
        // phi_s(u) = P_s + D_s with P_s = phi_s(u_ref) and the difference
        // D_0 = -(u - ur)(u + ur), D_+-1 = (u - ur)((u + ur) +- 1) / 2:
        // f^eq - s = drho P_a P_b + rho (P_a D_b + D_a (P_b + D_b))
        T Dx0, Dxp, Dxm, Dy0, Dyp, Dym, Px0, Pxp, Pxm, Py0, Pyp, Pym;
        if (SHIFT) {
            const T dux = ux - c.urx, sux = ux + c.urx, duy = uy - c.ury, suy = uy + c.ury;
            Dx0 = -dux * sux; Dxp = T(0.5) * (dux * (sux + T(1))); Dxm = T(0.5) * (dux * (sux - T(1)));
            Dy0 = -duy * suy; Dyp = T(0.5) * (duy * (suy + T(1))); Dym = T(0.5) * (duy * (suy - T(1)));
            Px0 = c.Px[0]; Pxp = c.Px[1]; Pxm = c.Px[2];
            Py0 = c.Py[0]; Pyp = c.Py[1]; Pym = c.Py[2];
        } else {
            Dx0 = -uxx; Dxp = T(0.5) * (uxx + ux); Dxm = T(0.5) * (uxx - ux);
            Dy0 = -uyy; Dyp = T(0.5) * (uyy + uy); Dym = T(0.5) * (uyy - uy);
            Px0 = Py0 = T(2) / T(3);
            Pxp = Pxm = Pyp = Pym = T(1) / T(6);
        }
        // f^eq - s = drho P_a P_b + P_a (rho D_b) + (rho D_a)(P_b + D_b)
        const T Ex0 = rho * Dx0, Exp = rho * Dxp, Exm = rho * Dxm;
        const T Ey0 = rho * Dy0, Eyp = rho * Dyp, Eym = rho * Dym;
        const T Hy0 = Py0 + Dy0, Hyp = Pyp + Dyp, Hym = Pym + Dym;
#define LBM_GEQ(Pa, Ea, Pb, Eb, Hb) (((Pa) * (Pb)) * drho + (Pa) * (Eb) + (Ea) * (Hb))
        geq[0] = LBM_GEQ(Px0, Ex0, Py0, Ey0, Hy0);
        geq[1] = LBM_GEQ(Pxp, Exp, Py0, Ey0, Hy0);
        geq[2] = LBM_GEQ(Px0, Ex0, Pyp, Eyp, Hyp);
        geq[3] = LBM_GEQ(Pxm, Exm, Py0, Ey0, Hy0);
        geq[4] = LBM_GEQ(Px0, Ex0, Pym, Eym, Hym);
        geq[5] = LBM_GEQ(Pxp, Exp, Pyp, Eyp, Hyp);
        geq[6] = LBM_GEQ(Pxm, Exm, Pyp, Eyp, Hyp);
        geq[7] = LBM_GEQ(Pxm, Exm, Pym, Eym, Hym);
        geq[8] = LBM_GEQ(Pxp, Exp, Pym, Eym, Hym);
#undef LBM_GEQ
    } else {
        // second-order equilibrium (Sec. 2, Hermite reading), shift s = w rho0 (u_ref = 0):
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
        // f^neq has no mass or momentum in exact arithmetic; in finite precision it carries
        // their rounding, which f* = f^eq + (1 - omega) f^neq would feed back with a factor
        // |1 - omega| ~ 1 at low viscosity.  Remove it (the moment-space models drop the same
        // components), i.e. subtract the populations (e0, ex/2, -ex/2, ey/2, -ey/2) that carry
        // exactly those moments and nothing else: the map is unchanged, its FP32 rounding is
        // that of the moment-space models.
        const T e0 = ((fn[0] + fn[1]) + (fn[2] + fn[3])) + ((fn[4] + fn[5]) + (fn[6] + fn[7])) + fn[8];
        const T hx = T(0.5) * ((fn[1] - fn[3]) + ((fn[5] - fn[7]) + (fn[8] - fn[6])));
        const T hy = T(0.5) * ((fn[2] - fn[4]) + ((fn[5] - fn[7]) + (fn[6] - fn[8])));
        fn[0] -= e0;
        fn[1] -= hx; fn[3] += hx;
        fn[2] -= hy; fn[4] += hy;
        const T cc = T(1) - w;
#pragma unroll
        for (int i = 0; i < 9; ++i) o[i] = geq[i] + cc * fn[i];
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
    int eq_order;       // 4, or 2 (BGK only)
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
