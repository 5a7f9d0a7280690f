// Hand-written reverse mode of the per-node collision (the transpose of the collision
// Jacobian J_ij = dC_i/df_j of App. A, Eq. Perturbed_Collision, evaluated at the node's own
// state rather than at a uniform flow), for every model, in the moment-space form of the
// forward kernels: g* = g - B D(n(g), u, rho), with the raw moments m of the stored g, the
// non-equilibrium moments n = m - (M^eq(rho, u) - M(s)) of Eq. extendedFeq (product form,
// storage shift s = f^eq(rho0, u_ref)), the model's removed moments D and the back-transform
// B of Eq. Q9postCollVDF_RM.
//
// Given the pre-collision populations g (shifted) of a node and the adjoint v_i of its
// post-collision populations, collide_vjp returns gbar_j = sum_i v_i dC_i/df_j and the rate
// sensitivities sum_i v_i dC_i/domega for omega_nu, omega3, omega4.  The primal is recomputed,
// then each step is differentiated in reverse: D-bar = -B^T v; through the model to n-bar (and
// to u, 1/rho where the model depends on them); through n = m - E(rho, u) to m-bar, rho-bar,
// u-bar; through u = j / rho; and back to populations with the transposed moment matrix.
#pragma once

#include "lbm_device.cuh"

namespace lbm {

// Collision constants of the reverse pass (from the host-filled table of StepArgs / AdjArgs).
template <typename T> struct VjpConsts {
    T w, w3, w4, rho0, urx, ury, Xr, Yr;   // rates, shift density and velocity, mu_2(u_ref)
    T kap, kapw;                           // cumulant rebuild: kappa and dkappa/dw (kNumConsts)
};

template <int MODEL, typename T>
__device__ __forceinline__ void collide_vjp(const T (&g)[9], const T (&v)[9], T (&gb)[9], const VjpConsts<T>& c,
                                            T& wb, T& w3b, T& w4b) {
    const T cs2 = T(1) / T(3);
    const T w = c.w, w3 = c.w3, w4 = c.w4;
    // ---------------- primal (as the forward kernels) ----------------
    const T a0p = (g[6] + g[2]) + g[5], a1p = g[5] - g[6], a2p = g[5] + g[6];
    const T a0z = (g[3] + g[0]) + g[1], a1z = g[1] - g[3], a2z = g[1] + g[3];
    const T a0m = (g[7] + g[4]) + g[8], a1m = g[8] - g[7], a2m = g[8] + g[7];
    const T drho = (a0p + a0z) + a0m;
    const T jx = ((a1p + a1z) + a1m) + c.rho0 * c.urx;
    const T jy = (a0p - a0m) + c.rho0 * c.ury;
    const T m20 = (a2p + a2z) + a2m, m02 = a0p + a0m, m11 = a1p - a1m;
    const T m21 = a2p - a2m, m12 = a1p + a1m, m22 = a2p + a2m;
    const T rho = c.rho0 + drho;
    const T irho = recip(rho);
    const T ux = jx * irho, uy = jy * irho;
    const T uxx = ux * ux, uyy = uy * uy;
    const T X = uxx + cs2, Y = uyy + cs2;   // mu_2(u_x), mu_2(u_y)
    // n = m - (rho mu_p(u_x) mu_q(u_y) - rho0 mu_p(ur_x) mu_q(ur_y)), without cancellation
    const T dx = ux - c.urx, dy = uy - c.ury;
    const T dX = dx * (ux + c.urx), dY = dy * (uy + c.ury);
    const T r0 = c.rho0;
    const T n20 = m20 - (drho * X + r0 * dX);
    const T n02 = m02 - (drho * Y + r0 * dY);
    const T n11 = m11 - (drho * (ux * uy) + r0 * (dx * uy + c.urx * dy));
    const T n21 = m21 - (drho * (X * uy) + r0 * (dX * uy + c.Xr * dy));
    const T n12 = m12 - (drho * (ux * Y) + r0 * (dx * Y + c.urx * dY));
    const T n22 = m22 - (drho * (X * Y) + r0 * (dX * Y + c.Xr * dY));

    // ---------------- reverse ----------------
    // g* = g - B D: g-bar = v, D-bar = -B^T v
    const T h = T(0.5), q = T(0.25);
    const T Db20 = v[0] - h * (v[1] + v[3]);
    const T Db02 = v[0] - h * (v[2] + v[4]);
    const T Db22 = -v[0] + h * ((v[1] + v[3]) + (v[2] + v[4])) - q * ((v[5] + v[6]) + (v[7] + v[8]));
    const T Db12 = h * (v[1] - v[3]) - q * ((v[5] - v[6]) + (v[8] - v[7]));
    const T Db21 = h * (v[2] - v[4]) - q * ((v[5] + v[6]) - (v[7] + v[8]));
    const T Db11 = -q * ((v[5] - v[6]) + (v[7] - v[8]));

    T nb20 = T(0), nb02 = T(0), nb11 = T(0), nb21 = T(0), nb12 = T(0), nb22 = T(0);
    T uxb = T(0), uyb = T(0), irhob = T(0);
    wb = T(0); w3b = T(0); w4b = T(0);
    if (MODEL == BGK || MODEL == RM) {
        // D = (w n20, w n02, w n11, r3 n21, r3 n12, r4 n22), BGK: r3 = r4 = w
        const T r3 = (MODEL == BGK) ? w : w3, r4 = (MODEL == BGK) ? w : w4;
        nb20 = w * Db20; nb02 = w * Db02; nb11 = w * Db11;
        nb21 = r3 * Db21; nb12 = r3 * Db12; nb22 = r4 * Db22;
        const T s2 = (Db20 * n20 + Db02 * n02) + Db11 * n11, s3 = Db21 * n21 + Db12 * n12, s4 = Db22 * n22;
        if (MODEL == BGK) {
            wb = (s2 + s3) + s4;
        } else {
            wb = s2; w3b = s3; w4b = s4;
        }
    } else if (MODEL == HM || MODEL == PR) {
        // D22 = r4 A + cs2 (D20 + D02), A = n22 - cs2 (n20 + n02); PR: r3 = r4 = 1
        const T A = n22 - cs2 * (n20 + n02);
        const T Dt20 = Db20 + cs2 * Db22, Dt02 = Db02 + cs2 * Db22;
        const T r3 = (MODEL == PR) ? T(1) : w3, r4 = (MODEL == PR) ? T(1) : w4;
        const T Ab = r4 * Db22;
        nb20 = w * Dt20 - cs2 * Ab;
        nb02 = w * Dt02 - cs2 * Ab;
        nb11 = w * Db11;
        nb21 = r3 * Db21; nb12 = r3 * Db12; nb22 = Ab;
        wb = (Dt20 * n20 + Dt02 * n02) + Db11 * n11;
        if (MODEL == HM) {
            w3b = Db21 * n21 + Db12 * n12;
            w4b = Db22 * A;
        }
    } else if (MODEL == RR) {
        // D21 = n21 - c3 a21, D12 = n12 - c3 a12, D22 = A - c4 a22 + cs2 (D20 + D02)
        const T c3 = T(1) - w3, c4 = T(1) - w4;
        const T a21 = uy * n20 + T(2) * ux * n11;
        const T a12 = ux * n02 + T(2) * uy * n11;
        const T a22 = uyy * n20 + uxx * n02 + T(4) * ux * uy * n11;
        const T Dt20 = Db20 + cs2 * Db22, Dt02 = Db02 + cs2 * Db22;
        const T ab21 = -c3 * Db21, ab12 = -c3 * Db12, ab22 = -c4 * Db22;   // adjoints of a21, a12, a22
        nb20 = w * Dt20 - cs2 * Db22 + uy * ab21 + uyy * ab22;
        nb02 = w * Dt02 - cs2 * Db22 + ux * ab12 + uxx * ab22;
        nb11 = w * Db11 + T(2) * (ux * ab21 + uy * ab12) + T(4) * ux * uy * ab22;
        nb21 = Db21; nb12 = Db12; nb22 = Db22;
        uxb = T(2) * n11 * ab21 + n02 * ab12 + (T(2) * ux * n02 + T(4) * uy * n11) * ab22;
        uyb = n20 * ab21 + T(2) * n11 * ab12 + (T(2) * uy * n20 + T(4) * ux * n11) * ab22;
        wb = (Dt20 * n20 + Dt02 * n02) + Db11 * n11;
        w3b = Db21 * a21 + Db12 * a12;
        w4b = Db22 * a22;
    } else {
        // central moments k of the non-equilibrium part (binomial shift by -u) ...
        const T k21 = n21 - T(2) * ux * n11 - uy * n20;
        const T k12 = n12 - T(2) * uy * n11 - ux * n02;
        const T k22 = n22 - T(2) * ux * n12 - T(2) * uy * n21 + uxx * n02 + uyy * n20 + T(4) * ux * uy * n11;
        const T d20 = w * n20, d02 = w * n02, d11 = w * n11, d21 = w3 * k21, d12 = w3 * k12;
        // ... removed central moments d, shifted back by +u: D = S(u) d
        const T db22 = Db22;
        const T db21 = Db21 + T(2) * uy * Db22;
        const T db12 = Db12 + T(2) * ux * Db22;
        const T db11 = Db11 + T(2) * ux * Db21 + T(2) * uy * Db12 + T(4) * ux * uy * Db22;
        T db20 = Db20 + uy * Db21 + uyy * Db22;
        T db02 = Db02 + ux * Db12 + uxx * Db22;
        T kb22 = T(0);
        T xb20 = T(0), xb02 = T(0), xb11 = T(0);   // direct n-bar contributions of d22
        if (MODEL == CM) {
            kb22 = w4 * db22;
            w4b = db22 * k22;
        } else if (MODEL == CHM) {
            // d22 = w4 (k22 - cs2 (n20 + n02)) + cs2 (d20 + d02)
            kb22 = w4 * db22;
            xb20 = -cs2 * kb22;
            xb02 = -cs2 * kb22;
            w4b = db22 * (k22 - cs2 * (n20 + n02));
            db20 += cs2 * db22;
            db02 += cs2 * db22;
        } else {
            // d22 = k22 - K22*, K22* = c4 C22 + cs2 (K20 + K02) + (K20 K02 + 2 K11^2) / rho,
            // C22 = k22 - cs2 (n20 + n02) - (n20 n02 + 2 n11^2) / rho, K = kappa n (order 2):
            // kappa = 1 - w for the post-collision rebuild, 1 or 0 for the other readings
            const T kap = c.kap, c4 = T(1) - w4;
            const T K20 = kap * n20, K02 = kap * n02, K11 = kap * n11;
            const T C22 = k22 - cs2 * (n20 + n02) - (n20 * n02 + T(2) * n11 * n11) * irho;
            const T Kb = -db22;                       // adjoint of K22*
            const T Cb = c4 * Kb;                     // adjoint of C22
            w4b = -C22 * Kb;
            const T Kb20 = Kb * (cs2 + K02 * irho), Kb02 = Kb * (cs2 + K20 * irho), Kb11 = Kb * (T(4) * K11 * irho);
            irhob = Kb * (K20 * K02 + T(2) * K11 * K11) - Cb * (n20 * n02 + T(2) * n11 * n11);
            kb22 = db22 + Cb;
            xb20 = kap * Kb20 - Cb * (cs2 + n02 * irho);
            xb02 = kap * Kb02 - Cb * (cs2 + n20 * irho);
            xb11 = kap * Kb11 - Cb * (T(4) * n11 * irho);
            wb = c.kapw * ((Kb20 * n20 + Kb02 * n02) + Kb11 * n11);
        }
        // u enters S(u): D21 = d21 + 2 ux d11 + uy d20, D12 = d12 + 2 uy d11 + ux d02,
        // D22 = d22 + 2 ux d12 + 2 uy d21 + ux^2 d02 + uy^2 d20 + 4 ux uy d11
        uxb = T(2) * d11 * Db21 + d02 * Db12 + (T(2) * d12 + T(2) * ux * d02 + T(4) * uy * d11) * Db22;
        uyb = d20 * Db21 + T(2) * d11 * Db12 + (T(2) * d21 + T(2) * uy * d20 + T(4) * ux * d11) * Db22;
        // d = rates * (n, k)
        wb += (db20 * n20 + db02 * n02) + db11 * n11;
        w3b = db21 * k21 + db12 * k12;
        const T kb21 = w3 * db21, kb12 = w3 * db12;
        nb20 = w * db20 + xb20;
        nb02 = w * db02 + xb02;
        nb11 = w * db11 + xb11;
        // k = S(-u) n
        nb22 = kb22;
        nb12 = kb12 - T(2) * ux * kb22;
        nb21 = kb21 - T(2) * uy * kb22;
        nb11 += -T(2) * (ux * kb21 + uy * kb12) + T(4) * ux * uy * kb22;
        nb20 += -uy * kb21 + uyy * kb22;
        nb02 += -ux * kb12 + uxx * kb22;
        uxb += -T(2) * n11 * kb21 - n02 * kb12 + (-T(2) * n12 + T(2) * ux * n02 + T(4) * uy * n11) * kb22;
        uyb += -n20 * kb21 - T(2) * n11 * kb12 + (-T(2) * n21 + T(2) * uy * n20 + T(4) * ux * n11) * kb22;
    }

    // n = m - E, E_pq = rho mu_p(u_x) mu_q(u_y) - rho0 mu_p(ur_x) mu_q(ur_y):
    // dE/d(drho) = mu_p mu_q, dE/du_x = rho mu_p' mu_q, dE/du_y = rho mu_p mu_q'
    const T drhob_n =
        -(((nb20 * X + nb02 * Y) + nb11 * (ux * uy)) + ((nb21 * X) * uy + (nb12 * ux) * Y) + nb22 * (X * Y));
    uxb -= rho * (T(2) * ux * (nb20 + nb21 * uy + nb22 * Y) + nb11 * uy + nb12 * Y);
    uyb -= rho * (T(2) * uy * (nb02 + nb12 * ux + nb22 * X) + nb11 * ux + nb21 * X);
    // u = j / rho
    const T jxb = uxb * irho, jyb = uyb * irho;
    irhob += uxb * jx + uyb * jy;
    const T drhob = drhob_n - irhob * irho * irho;
    // back to populations: g-bar_i = v_i + [1, xi_x, xi_y, xi_x^2, xi_y^2, xi_x xi_y, xi_x^2 xi_y,
    // xi_x xi_y^2, xi_x^2 xi_y^2] . (drho-bar, jx-bar, jy-bar, n-bar), by rows of xi_y
    const T tp0 = drhob + jyb + nb02, tp1 = jxb + nb11 + nb12, tp2 = nb20 + nb21 + nb22;   // xi_y = +1
    const T tz0 = drhob, tz1 = jxb, tz2 = nb20;                                               // xi_y = 0
    const T tm0 = drhob - jyb + nb02, tm1 = jxb - nb11 + nb12, tm2 = nb20 - nb21 + nb22;   // xi_y = -1
    gb[0] = v[0] + tz0;
    gb[1] = v[1] + tz0 + tz1 + tz2;
    gb[3] = v[3] + tz0 - tz1 + tz2;
    gb[2] = v[2] + tp0;
    gb[5] = v[5] + tp0 + tp1 + tp2;
    gb[6] = v[6] + tp0 - tp1 + tp2;
    gb[4] = v[4] + tm0;
    gb[8] = v[8] + tm0 + tm1 + tm2;
    gb[7] = v[7] + tm0 - tm1 + tm2;
}

}  // namespace lbm
