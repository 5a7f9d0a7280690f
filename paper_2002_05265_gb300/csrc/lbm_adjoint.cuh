// Hand-written reverse mode of the per-node collision (the transpose of the collision
// Jacobian J_ij = dC_i/df_j of App. A, Eq. Perturbed_Collision, evaluated at the node's own
// state rather than at a uniform flow), for every model, in the non-equilibrium form used by
// the forward kernels (extended equilibrium, storage shift s_i = rho0 P_a P_b with
// P = phi(u_ref); u_ref = 0 gives the weights).
//
// Given the pre-collision populations g (shifted) of a node and the adjoint v_i of its
// post-collision populations, collide_vjp returns gbar_j = sum_i v_i dC_i/df_j and the rate
// sensitivities sum_i v_i dC_i/domega for omega_nu, omega3, omega4.  The primal is recomputed
// line by line and each line is then differentiated in reverse order.
#pragma once

#include "lbm_device.cuh"

namespace lbm {

template <int MODEL, typename T>
__device__ __forceinline__ void collide_vjp(const T (&g)[9], const T (&v)[9], T (&gb)[9], T w, T w3, T w4, T rho0,
                                            const T (&Px)[3], const T (&Py)[3], T urx, T ury, T& wb, T& w3b,
                                            T& w4b) {
    const T cs2 = T(1) / T(3);
    // ---------------- primal ----------------
    const T drho = ((g[0] + g[1]) + (g[2] + g[3])) + ((g[4] + g[5]) + (g[6] + g[7])) + g[8];
    const T rho = rho0 + drho;
    const T jx = ((g[1] - g[3]) + ((g[5] - g[7]) + (g[8] - g[6]))) + rho0 * urx;
    const T jy = ((g[2] - g[4]) + ((g[5] - g[7]) + (g[6] - g[8]))) + rho0 * ury;
    const T irho = T(1) / rho;
    const T ux = jx * irho, uy = jy * irho;
    const T uxx = ux * ux, uyy = uy * uy;
    // 1D factors of the extended equilibrium: phi_s(u) = P_s + D_s with P_s = phi_s(u_ref),
    // D_0 = -(u - ur)(u + ur), D_+-1 = (u - ur)(u + ur +- 1)/2 (dD_0/du = -2u, dD_+-1/du = u +- 1/2)
    const T dux = ux - urx, sux = ux + urx, duy = uy - ury, suy = uy + ury;
    const T Dx[3] = {-dux * sux, T(0.5) * (dux * (sux + T(1))), T(0.5) * (dux * (sux - T(1)))};
    const T Dy[3] = {-duy * suy, T(0.5) * (duy * (suy + T(1))), T(0.5) * (duy * (suy - T(1)))};
    // index of the 1D factor for xi component e: 0 -> 0, +1 -> 1, -1 -> 2
#define LBM_K1(e) ((e) == 0 ? 0 : ((e) == 1 ? 1 : 2))
    T geq[9], fn[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int a = LBM_K1(ex_of(i)), b = LBM_K1(ey_of(i));
        geq[i] = Px[a] * Py[b] * drho + rho * (Px[a] * Dy[b] + Dx[a] * (Py[b] + Dy[b]));
        fn[i] = g[i] - geq[i];
    }
    // ---------------- reverse ----------------
    T geqb[9], fnb[9];
    T uxb = T(0), uyb = T(0), irhob = T(0);
    wb = T(0); w3b = T(0); w4b = T(0);
    if (MODEL == BGK) {
        const T c = T(1) - w;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            geqb[i] = v[i];
            fnb[i] = c * v[i];
            wb -= v[i] * fn[i];
        }
    } else {
        // raw moments of f^neq
        const T m20 = fn[1] + fn[3] + fn[5] + fn[6] + fn[7] + fn[8];
        const T m02 = fn[2] + fn[4] + fn[5] + fn[6] + fn[7] + fn[8];
        const T m11 = fn[5] - fn[6] + fn[7] - fn[8];
        const T m21 = fn[5] + fn[6] - fn[7] - fn[8];
        const T m12 = fn[5] - fn[6] - fn[7] + fn[8];
        const T m22 = fn[5] + fn[6] + fn[7] + fn[8];
        const T c2 = T(1) - w, c3 = T(1) - w3, c4 = T(1) - w4;
        // d = B M (Eq. Q9postCollVDF_RM without the conserved moments): M-bar = B^T d-bar
        const T h = T(0.5), q = T(0.25);
        const T Mb20 = -v[0] + h * (v[1] + v[3]);
        const T Mb02 = -v[0] + h * (v[2] + v[4]);
        const T Mb22 = v[0] - h * (v[1] + v[3] + v[2] + v[4]) + q * (v[5] + v[6] + v[7] + v[8]);
        const T Mb12 = h * (v[3] - v[1]) + q * (v[5] - v[6] - v[7] + v[8]);
        const T Mb21 = h * (v[4] - v[2]) + q * (v[5] + v[6] - v[7] - v[8]);
        const T Mb11 = q * (v[5] - v[6] + v[7] - v[8]);
        T mb20 = T(0), mb02 = T(0), mb11 = T(0), mb21 = T(0), mb12 = T(0), mb22 = T(0);
        if (MODEL == RM) {
            mb20 = c2 * Mb20; mb02 = c2 * Mb02; mb11 = c2 * Mb11;
            mb21 = c3 * Mb21; mb12 = c3 * Mb12; mb22 = c4 * Mb22;
            wb -= Mb20 * m20 + Mb02 * m02 + Mb11 * m11;
            w3b -= Mb21 * m21 + Mb12 * m12;
            w4b -= Mb22 * m22;
        } else if (MODEL == HM || MODEL == PR) {
            // M22 = c4 (m22 - cs2 (m20 + m02)) + cs2 (M20 + M02)   (PR: c3 = c4 = 0)
            const T Mb20t = Mb20 + cs2 * Mb22, Mb02t = Mb02 + cs2 * Mb22;
            mb20 = c2 * Mb20t; mb02 = c2 * Mb02t; mb11 = c2 * Mb11;
            wb -= Mb20t * m20 + Mb02t * m02 + Mb11 * m11;
            if (MODEL == HM) {
                const T a22 = m22 - cs2 * (m20 + m02);
                const T ab22 = c4 * Mb22;
                mb22 = ab22;
                mb20 -= cs2 * ab22;
                mb02 -= cs2 * ab22;
                w4b -= Mb22 * a22;
                mb21 = c3 * Mb21; mb12 = c3 * Mb12;
                w3b -= Mb21 * m21 + Mb12 * m12;
            }
        } else if (MODEL == RR) {
            const T a21 = uy * m20 + T(2) * ux * m11;
            const T a12 = ux * m02 + T(2) * uy * m11;
            const T a22 = uyy * m20 + uxx * m02 + T(4) * ux * uy * m11;
            const T Mb20t = Mb20 + cs2 * Mb22, Mb02t = Mb02 + cs2 * Mb22;
            const T ab21 = c3 * Mb21, ab12 = c3 * Mb12, ab22 = c4 * Mb22;
            w3b -= Mb21 * a21 + Mb12 * a12;
            w4b -= Mb22 * a22;
            wb -= Mb20t * m20 + Mb02t * m02 + Mb11 * m11;
            mb20 = c2 * Mb20t + uy * ab21 + uyy * ab22;
            mb02 = c2 * Mb02t + ux * ab12 + uxx * ab22;
            mb11 = c2 * Mb11 + T(2) * ux * ab21 + T(2) * uy * ab12 + T(4) * ux * uy * ab22;
            uxb += T(2) * m11 * ab21 + m02 * ab12 + (T(2) * ux * m02 + T(4) * uy * m11) * ab22;
            uyb += m20 * ab21 + T(2) * m11 * ab12 + (T(2) * uy * m20 + T(4) * ux * m11) * ab22;
        } else {
            // central moments (binomial shift by -u)
            const T k20 = m20, k02 = m02, k11 = m11;
            const T k21 = m21 - T(2) * ux * m11 - uy * m20;
            const T k12 = m12 - T(2) * uy * m11 - ux * m02;
            const T k22 = m22 - T(2) * ux * m12 - T(2) * uy * m21 + uxx * m02 + uyy * m20 + T(4) * ux * uy * m11;
            const T K20 = c2 * k20, K02 = c2 * k02, K11 = c2 * k11, K21 = c3 * k21, K12 = c3 * k12;
            // back-transform (shift by +u): M = K + ...
            T Kb22 = Mb22;
            const T Kb21 = Mb21 + T(2) * uy * Mb22;
            const T Kb12 = Mb12 + T(2) * ux * Mb22;
            T Kb11 = Mb11 + T(2) * ux * Mb21 + T(2) * uy * Mb12 + T(4) * ux * uy * Mb22;
            T Kb20 = Mb20 + uy * Mb21 + uyy * Mb22;
            T Kb02 = Mb02 + ux * Mb12 + uxx * Mb22;
            uxb += T(2) * K11 * Mb21 + K02 * Mb12 + (T(2) * K12 + T(2) * ux * K02 + T(4) * uy * K11) * Mb22;
            uyb += K20 * Mb21 + T(2) * K11 * Mb12 + (T(2) * K21 + T(2) * uy * K20 + T(4) * ux * K11) * Mb22;
            T kb20 = T(0), kb02 = T(0), kb11 = T(0), kb22 = T(0);
            if (MODEL == CM) {
                kb22 = c4 * Kb22;
                w4b -= Kb22 * k22;
            } else if (MODEL == CHM) {
                const T a = k22 - cs2 * (k20 + k02);
                kb22 = c4 * Kb22;
                kb20 -= cs2 * c4 * Kb22;
                kb02 -= cs2 * c4 * Kb22;
                w4b -= Kb22 * a;
                Kb20 += cs2 * Kb22;
                Kb02 += cs2 * Kb22;
            } else {
                // K22 = c4 C22 + cs2 (K20 + K02) + (K20 K02 + 2 K11^2) irho
                const T C22 = k22 - cs2 * (k20 + k02) - (k20 * k02 + T(2) * k11 * k11) * irho;
                const T Cb22 = c4 * Kb22;
                w4b -= Kb22 * C22;
                Kb20 += (cs2 + K02 * irho) * Kb22;
                Kb02 += (cs2 + K20 * irho) * Kb22;
                Kb11 += T(4) * K11 * irho * Kb22;
                irhob += (K20 * K02 + T(2) * K11 * K11) * Kb22;
                kb22 += Cb22;
                kb20 += (-cs2 - k02 * irho) * Cb22;
                kb02 += (-cs2 - k20 * irho) * Cb22;
                kb11 += T(-4) * k11 * irho * Cb22;
                irhob -= (k20 * k02 + T(2) * k11 * k11) * Cb22;
            }
            kb20 += c2 * Kb20;
            kb02 += c2 * Kb02;
            kb11 += c2 * Kb11;
            const T kb21 = c3 * Kb21, kb12 = c3 * Kb12;
            wb -= Kb20 * k20 + Kb02 * k02 + Kb11 * k11;
            w3b -= Kb21 * k21 + Kb12 * k12;
            // central -> raw (reverse of the shift by -u)
            mb22 = kb22;
            mb12 = kb12 - T(2) * ux * kb22;
            mb21 = kb21 - T(2) * uy * kb22;
            mb11 = kb11 - T(2) * ux * kb21 - T(2) * uy * kb12 + T(4) * ux * uy * kb22;
            mb20 = kb20 - uy * kb21 + uyy * kb22;
            mb02 = kb02 - ux * kb12 + uxx * kb22;
            uxb += -T(2) * m11 * kb21 - m02 * kb12 + (-T(2) * m12 + T(2) * ux * m02 + T(4) * uy * m11) * kb22;
            uyb += -m20 * kb21 - T(2) * m11 * kb12 + (-T(2) * m21 + T(2) * uy * m20 + T(4) * ux * m11) * kb22;
        }
        // f^neq-bar = A^T m-bar
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const T ex = T(ex_of(i)), ey = T(ey_of(i));
            const T ex2 = ex * ex, ey2 = ey * ey;
            fnb[i] = ex2 * mb20 + ey2 * mb02 + ex * ey * mb11 + ex2 * ey * mb21 + ex * ey2 * mb12 + ex2 * ey2 * mb22;
            geqb[i] = v[i];
        }
    }
    // fn = g - geq;  o = geq + d
    T drhob = T(0), rhob = T(0);
    T Dxb[3] = {T(0), T(0), T(0)}, Dyb[3] = {T(0), T(0), T(0)};
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        gb[i] = fnb[i];
        const T gq = geqb[i] - fnb[i];
        const int a = LBM_K1(ex_of(i)), b = LBM_K1(ey_of(i));
        drhob += Px[a] * Py[b] * gq;
        rhob += (Px[a] * Dy[b] + Dx[a] * (Py[b] + Dy[b])) * gq;
        Dyb[b] += rho * (Px[a] + Dx[a]) * gq;
        Dxb[a] += rho * (Py[b] + Dy[b]) * gq;
    }
#undef LBM_K1
    uxb += -T(2) * ux * Dxb[0] + (ux + T(0.5)) * Dxb[1] + (ux - T(0.5)) * Dxb[2];
    uyb += -T(2) * uy * Dyb[0] + (uy + T(0.5)) * Dyb[1] + (uy - T(0.5)) * Dyb[2];
    // u = j irho, irho = 1/rho, rho = rho0 + drho
    const T jxb = uxb * irho, jyb = uyb * irho;
    irhob += uxb * jx + uyb * jy;
    rhob -= irhob * irho * irho;
    drhob += rhob;
#pragma unroll
    for (int i = 0; i < 9; ++i) gb[i] += drhob + T(ex_of(i)) * jxb + T(ey_of(i)) * jyb;
}

}  // namespace lbm
