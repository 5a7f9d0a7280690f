"""Pins of the oracle's moment transforms (App. B) against their definitions and exact
symbolic derivatives."""

import numpy as np
import pytest
import sympy as sp

from oracle import d2q9, moments
from oracle.collision import macroscopic


def _random_f(shape=(4, 3), seed=7):
    g = np.random.default_rng(seed)
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    return w[:, None, None] * (1.0 + 0.4 * g.uniform(-1, 1, (9,) + shape))


def _close(a, b, tol=1e-15):
    for pq in d2q9.PQ:
        np.testing.assert_allclose(a[pq], b[pq], rtol=0, atol=tol)


def test_populations_from_raw_inverts_raw_moments():
    """Eq. Q9postCollVDF_RM is the inverse of the nine raw moments."""
    f = _random_f()
    np.testing.assert_allclose(np.array(moments.populations_from_raw(moments.raw_moments(f))), f, atol=2e-16)


def test_hm2rm_holds_for_any_distribution():
    """Eq. HM2RM_Q9 maps the Hermite moments of any f to its raw moments."""
    f = _random_f()
    _close(moments.raw_from_hermite(moments.hermite_moments(f)), moments.raw_moments(f))


def test_chm2hm_holds_with_the_corrected_polynomial():
    """Eq. CHM2HM_Q9 maps the CHMs of f (Eq. CHpoly, H~_12 read as H~_10 H~_02) to its
    HMs, for any f with u = j / rho."""
    f = _random_f()
    rho, ux, uy = macroscopic(f)
    At = moments.central_hermite_moments(f, ux, uy)
    _close(moments.hermite_from_central_hermite(At, rho, ux, uy), moments.hermite_moments(f), 3e-16)


def test_chm_polynomial_as_printed_breaks_chm2hm():
    """The H~_12 printed in Eq. CHpoly, (xi_y - u_y)[(xi_y - u_y)^2 - c_s^2], is
    inconsistent with Eq. CHM2HM_Q9: the identity fails, so the printed form is a typo."""
    f = _random_f()
    rho, ux, uy = macroscopic(f)
    At = moments.central_hermite_moments(f, ux, uy)
    At[1, 2] = sum(((d2q9.XI[i, 1] - uy) * ((d2q9.XI[i, 1] - uy) ** 2 - d2q9.CS2)) * f[i] for i in range(9))
    A = moments.hermite_from_central_hermite(At, rho, ux, uy)
    assert np.max(np.abs(A[1, 2] - moments.hermite_moments(f)[1, 2])) > 1e-3


def test_central_to_raw_binomial():
    f = _random_f()
    rho, ux, uy = macroscopic(f)
    _close(moments.raw_from_central(moments.central_moments(f, ux, uy), ux, uy), moments.raw_moments(f), 3e-16)


def test_central_moments_conserved_entries():
    """With u = j / rho the first central moments vanish and K~_00 = rho."""
    f = _random_f()
    rho, ux, uy = macroscopic(f)
    K = moments.central_moments(f, ux, uy)
    np.testing.assert_allclose(K[0, 0], rho, atol=1e-16)
    np.testing.assert_allclose(K[1, 0], 0, atol=1e-16)
    np.testing.assert_allclose(K[0, 1], 0, atol=1e-16)


def test_cumulant_roundtrip():
    f = _random_f()
    rho, ux, uy = macroscopic(f)
    K = moments.central_moments(f, ux, uy)
    _close(moments.central_from_cumulants(moments.cumulants_from_central(K)), K, 1e-16)


def test_cumulants_equal_log_mgf_derivatives_exactly():
    """C_pq = rho * d^{p+q} ln Z / dX^p dY^q at 0, with Z(X, Y) = sum_i f_i exp(X xi_ix +
    Y xi_iy): the definition of cumulants, differentiated symbolically in exact rational
    arithmetic and compared with the oracle's closed form."""
    X, Y = sp.symbols("X Y")
    g = np.random.default_rng(11)
    fr = [sp.Rational(int(v), 10000) for v in g.integers(100, 5000, 9)]
    Z = sum(fr[i] * sp.exp(X * int(d2q9.XI[i, 0]) + Y * int(d2q9.XI[i, 1])) for i in range(9))
    lnZ = sp.log(Z)
    rho = sum(fr)
    f = np.array([float(v) for v in fr])[:, None]
    r, ux, uy = macroscopic(f)
    C = moments.cumulants_from_central(moments.central_moments(f, ux, uy))
    for (p, q) in [(2, 0), (0, 2), (1, 1), (2, 1), (1, 2), (2, 2)]:
        d = lnZ
        if p:
            d = sp.diff(d, X, p)
        if q:
            d = sp.diff(d, Y, q)
        exact = float(rho * d.subs({X: 0, Y: 0}))
        assert C[p, q][0] == pytest.approx(exact, rel=1e-12, abs=1e-15), (p, q)
