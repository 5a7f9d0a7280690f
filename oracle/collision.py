"""Collision models of App. B: post-collision populations f* from pre-collision f.

Every function takes f with shape (9, ...) and the relaxation frequencies of Sec. 4c:
omega_nu for second-order quantities (viscous), omega3 and omega4 for third- and
fourth-order quantities.  All second-order quantities, including the trace, relax with
omega_nu (the paper's isothermal D2Q9 has bulk viscosity nu_b = nu, Sec. 3b, and Sec. 4c
names no separate bulk rate).  Zeroth- and first-order moments are kept (mass and momentum
conservation, App. B after Eq. RMcoll).

Models:
  bgk  f* = f - omega_nu (f - f^eq)                                (Sec. 1; Eq. StreamCollide)
  rm   raw moments relaxed by order                                (Eqs. RMcoll, Q9postCollVDF_RM)
  hm   Hermite moments relaxed by order, HM -> RM                  (App. B text; Eq. HM2RM_Q9)
  cm   central moments relaxed by order, CM -> RM (binomial)       (App. B text)
  chm  central Hermite moments                                     (Eqs. CHpoly, CHMcoll, CHM2HM_Q9, HM2RM_Q9)
  k    cumulants, nonlinear fourth-order cumulant                  (Sec. 4c; reading below)
  rr   recursive regularized                                       (Eqs. HMColl_Q9, RRformulas_D2Q9)
  pr   standard regularized = HM with omega3 = omega4 = 1          (Sec. 5c; App. C)

Readings (where the paper defers the definition or is ambiguous):
  * hm, cm: their equilibrium moments are the moments of f^eq in the same space
    (the definition of an equilibrium moment); the paper lists closed forms only for
    RM and CHM.
  * k: the cumulant transform of moments.cumulants_from_central; equilibrium cumulants are
    the cumulants of f^eq; cumulants of order 2, 3, 4 relax with omega_nu, omega3, omega4;
    the fourth-order central moment is rebuilt from the relaxed C_22 with the
    post-collision second-order central moments.
  * rr: in Eq. HMColl_Q9 the moments A_pq of order >= 3 are taken as
    A^eq_pq + A^neq_pq with A^neq_pq from the recursion Eq. RRformulas_D2Q9; this is the
    reading under which REG-RR reduces to the standard regularized model as stated in
    Sec. 5c.
  * pr: the paper identifies the standard regularized model with REG-HM (Sec. 5c, App. C);
    the rates omega3, omega4 passed in are ignored and 1 is used.
"""

import numpy as np

from .d2q9 import XI, Q
from .equilibrium import feq, raw_equilibrium_moments
from .moments import (raw_moments, populations_from_raw, hermite_moments, raw_from_hermite,
                      central_moments, raw_from_central, central_hermite_moments,
                      hermite_from_central_hermite, cumulants_from_central,
                      central_from_cumulants)

MODELS = ("bgk", "rm", "hm", "cm", "chm", "k", "pr", "rr")


def macroscopic(f):
    """rho = sum_i f_i, rho u = sum_i xi_i f_i (Sec. 1)."""
    rho = sum(f[i] for i in range(Q))
    jx = sum(float(XI[i, 0]) * f[i] for i in range(Q))
    jy = sum(float(XI[i, 1]) * f[i] for i in range(Q))
    return rho, jx / rho, jy / rho


def _order_rate(p, q, w_nu, w3, w4):
    n = p + q
    return {2: w_nu, 3: w3, 4: w4}[n]


def _relax_by_order(X, Xeq, w_nu, w3, w4):
    """X*_pq = (1 - omega_n) X_pq + omega_n X^eq_pq for orders n = 2, 3, 4; orders 0 and 1
    are set to their (conserved) equilibrium values (Eq. RMcoll; same pattern in
    Eq. CHMcoll)."""
    Xs = {}
    for (p, q) in X:
        if p + q <= 1:
            Xs[p, q] = Xeq[p, q]
        else:
            w = _order_rate(p, q, w_nu, w3, w4)
            Xs[p, q] = (1.0 - w) * X[p, q] + w * Xeq[p, q]
    return Xs


def bgk(f, w_nu, w3=None, w4=None, eq_order=4):
    """BGK: f*_i = f_i - omega_nu (f_i - f^eq_i)."""
    rho, ux, uy = macroscopic(f)
    fe = feq(rho, ux, uy, eq_order)
    return np.array([f[i] - w_nu * (f[i] - fe[i]) for i in range(Q)])


def rm(f, w_nu, w3, w4, eq_order=4):
    """Raw-moment model: Eq. RMcoll then Eq. Q9postCollVDF_RM."""
    rho, ux, uy = macroscopic(f)
    M = raw_moments(f)
    Meq = raw_equilibrium_moments(rho, ux, uy, eq_order)
    Ms = _relax_by_order(M, Meq, w_nu, w3, w4)
    return np.array(populations_from_raw(Ms))


def hm(f, w_nu, w3, w4, eq_order=4):
    """Hermite-moment model: relax A_pq by order, back to RMs with Eq. HM2RM_Q9, then
    Eq. Q9postCollVDF_RM."""
    rho, ux, uy = macroscopic(f)
    A = hermite_moments(f)
    Aeq = hermite_moments(feq(rho, ux, uy, eq_order))
    As = _relax_by_order(A, Aeq, w_nu, w3, w4)
    return np.array(populations_from_raw(raw_from_hermite(As)))


def cm(f, w_nu, w3, w4, eq_order=4):
    """Central-moment model: relax K~_pq by order, back to RMs with the binomial identity,
    then Eq. Q9postCollVDF_RM."""
    rho, ux, uy = macroscopic(f)
    K = central_moments(f, ux, uy)
    Keq = central_moments(feq(rho, ux, uy, eq_order), ux, uy)
    Ks = _relax_by_order(K, Keq, w_nu, w3, w4)
    return np.array(populations_from_raw(raw_from_central(Ks, ux, uy)))


def chm(f, w_nu, w3, w4, eq_order=4):
    """Central-Hermite-moment model, App. B step by step: CHMs (Eq. CHpoly), equilibrium
    CHMs (all zero but A~_00 = rho), relaxation (Eq. CHMcoll), CHM -> HM (Eq. CHM2HM_Q9),
    HM -> RM (Eq. HM2RM_Q9), RM -> f (Eq. Q9postCollVDF_RM)."""
    if eq_order != 4:
        raise ValueError("the CHM equilibrium of App. B is the extended one")
    rho, ux, uy = macroscopic(f)
    At = central_hermite_moments(f, ux, uy)
    zero = 0.0 * rho
    Ateq = {pq: zero for pq in At}
    Ateq[0, 0] = rho
    Ats = _relax_by_order(At, Ateq, w_nu, w3, w4)
    A = hermite_from_central_hermite(Ats, rho, ux, uy)
    return np.array(populations_from_raw(raw_from_hermite(A)))


def k_reading(f, w_nu, w3, w4, eq_order=4, rebuild="post"):
    """Cumulant model with a choice of the second-order central moments in the rebuild of
    K~_22 from the relaxed C_22 (the step the paper defers to an external reference):
      "post"  K~*_22 = C*_22 + (K~*_20 K~*_02 + 2 K~*_11^2) / rho   (post-collision values;
              the oracle's reading, `k` below)
      "pre"   the same with the pre-collision K~_20, K~_02, K~_11
      "eq"    the same with their equilibrium values (rho c_s^2, rho c_s^2, 0), i.e.
              K~*_22 = C*_22 + rho c_s^4
    The alternatives exist to test the reading against the paper's statements about K."""
    if eq_order != 4:
        raise ValueError("the cumulant model is defined with the extended equilibrium")
    rho, ux, uy = macroscopic(f)
    K = central_moments(f, ux, uy)
    C = cumulants_from_central(K)
    Keq = central_moments(feq(rho, ux, uy, 4), ux, uy)
    Ceq = cumulants_from_central(Keq)
    Cs = _relax_by_order(C, Ceq, w_nu, w3, w4)
    if rebuild == "post":
        Ks = central_from_cumulants(Cs)
    else:
        src = K if rebuild == "pre" else Keq
        if rebuild not in ("pre", "eq"):
            raise ValueError(rebuild)
        Ks = dict(Cs)
        Ks[2, 2] = Cs[2, 2] + (src[2, 0] * src[0, 2] + 2.0 * src[1, 1] * src[1, 1]) / rho
    return np.array(populations_from_raw(raw_from_central(Ks, ux, uy)))


def k(f, w_nu, w3, w4, eq_order=4):
    """Cumulant model (reading in the module docstring)."""
    return k_reading(f, w_nu, w3, w4, eq_order, "post")


def rr(f, w_nu, w3, w4, eq_order=4):
    """Recursive regularized model: second-order A^neq_pq = sum_i H_pq (f_i - f^eq_i),
    third/fourth-order A^neq from Eq. RRformulas_D2Q9, post-collision HMs from
    Eq. HMColl_Q9 (reading in the module docstring), then Eqs. HM2RM_Q9 and
    Q9postCollVDF_RM."""
    rho, ux, uy = macroscopic(f)
    fe = feq(rho, ux, uy, eq_order)
    Aeq = hermite_moments(fe)
    Aneq = hermite_moments(f - fe)
    a20, a02, a11 = Aneq[2, 0], Aneq[0, 2], Aneq[1, 1]
    a21 = uy * a20 + 2.0 * ux * a11
    a12 = ux * a02 + 2.0 * uy * a11
    a22 = uy * uy * a20 + ux * ux * a02 + 4.0 * ux * uy * a11
    As = {}
    As[0, 0] = rho
    As[1, 0] = rho * ux
    As[0, 1] = rho * uy
    As[1, 1] = (Aeq[1, 1] + a11) - w_nu * a11
    As[2, 0] = (Aeq[2, 0] + a20) - w_nu * a20
    As[0, 2] = (Aeq[0, 2] + a02) - w_nu * a02
    As[2, 1] = (Aeq[2, 1] + a21) - w3 * a21
    As[1, 2] = (Aeq[1, 2] + a12) - w3 * a12
    As[2, 2] = (Aeq[2, 2] + a22) - w4 * a22
    return np.array(populations_from_raw(raw_from_hermite(As)))


def pr(f, w_nu, w3=None, w4=None, eq_order=4):
    """Standard regularized model = REG-HM (Sec. 5c, App. C)."""
    return hm(f, w_nu, 1.0, 1.0, eq_order)


COLLIDE = {"bgk": bgk, "rm": rm, "hm": hm, "cm": cm, "chm": chm, "k": k, "pr": pr, "rr": rr,
           # the two alternative readings of the cumulant rebuild (see k_reading)
           "k_pre": lambda f, w_nu, w3, w4, eq_order=4: k_reading(f, w_nu, w3, w4, eq_order, "pre"),
           "k_eq": lambda f, w_nu, w3, w4, eq_order=4: k_reading(f, w_nu, w3, w4, eq_order, "eq")}


def collide(model, f, w_nu, w3, w4, eq_order=4):
    return COLLIDE[model](f, w_nu, w3, w4, eq_order)
