"""Pins of the oracle's lattice and equilibria against what the paper and textbooks fix."""

import json
import os
from fractions import Fraction

import numpy as np
import pytest
from numpy.polynomial.hermite_e import hermegauss

from oracle import d2q9, equilibrium, moments

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def _fields(shape=(6, 5), seed=3, umax=0.3):
    g = np.random.default_rng(seed)
    rho = 1.0 + 0.1 * g.uniform(-1, 1, shape)
    ux = umax * g.uniform(-1, 1, shape)
    uy = umax * g.uniform(-1, 1, shape)
    return rho, ux, uy


def test_rest_weights_match_textbook():
    """Eq. extendedFeq at u = 0 reduces to the D2Q9 weights 4/9, 1/9, 1/36."""
    f = equilibrium.feq(np.array(1.0), np.array(0.0), np.array(0.0))
    w = GOLDEN["d2q9_rest_weights"]["values"]
    for i in range(9):
        sx, sy = d2q9.XI[i]
        key = "(0,0)" if sx == 0 and sy == 0 else ("(+-1,0)" if sy == 0 else ("(0,+-1)" if sx == 0 else "(+-1,+-1)"))
        assert f[i] == pytest.approx(float(Fraction(w[key])), abs=1e-16)
    assert float(Fraction(GOLDEN["cs2"]["value"])) == d2q9.CS2


def _maxwellian_moment(rho, ux, uy, p, q):
    """int xi_x^p xi_y^q f^MB d xi for the Maxwellian of Eq. eqMB with T_0 = c_s^2, by
    Gauss-Hermite quadrature (exact for polynomial integrands of this degree)."""
    x, w = hermegauss(12)                     # weight exp(-x^2/2), sum w = sqrt(2 pi)
    s = np.sqrt(d2q9.CS2)
    w = w / np.sqrt(2 * np.pi)
    mx = sum(wk * (ux + s * xk) ** p for xk, wk in zip(x, w))
    my = sum(wk * (uy + s * xk) ** q for xk, wk in zip(x, w))
    return rho * mx * my


def test_extended_equilibrium_matches_nine_maxwellian_moments():
    """Eq. MatchingCondition holds for all p, q <= 2 with the extended equilibrium
    (Sec. 2, text after Eq. extendedFeq)."""
    rho, ux, uy = _fields()
    f = equilibrium.feq(rho, ux, uy, 4)
    for (p, q) in d2q9.PQ:
        lhs = sum(d2q9.XI[i, 0] ** p * d2q9.XI[i, 1] ** q * f[i] for i in range(9))
        rhs = _maxwellian_moment(rho, ux, uy, p, q)
        np.testing.assert_allclose(lhs, rhs, rtol=0, atol=1e-15)


def test_second_order_equilibrium_is_the_textbook_polynomial():
    """Reading of 'standard second-order equilibrium' (Sec. 2): the polynomial
    w_i rho (1 + xi.u/c_s^2 + (xi.u)^2/(2 c_s^4) - u^2/(2 c_s^2))."""
    rho, ux, uy = _fields()
    f = equilibrium.feq(rho, ux, uy, 2)
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    cs2 = 1.0 / 3.0
    for i in range(9):
        xu = d2q9.XI[i, 0] * ux + d2q9.XI[i, 1] * uy
        ref = w[i] * rho * (1 + xu / cs2 + xu * xu / (2 * cs2 * cs2) - (ux * ux + uy * uy) / (2 * cs2))
        np.testing.assert_allclose(f[i], ref, rtol=0, atol=2e-16)


def test_second_order_equilibrium_matches_only_low_moments():
    """The second-order equilibrium keeps the matching conditions for p + q <= 2 and
    loses M_21, M_12 (the source of Eq. RemainingErrors)."""
    rho, ux, uy = _fields()
    f = equilibrium.feq(rho, ux, uy, 2)
    for (p, q) in d2q9.PQ:
        lhs = sum(d2q9.XI[i, 0] ** p * d2q9.XI[i, 1] ** q * f[i] for i in range(9))
        rhs = _maxwellian_moment(rho, ux, uy, p, q)
        if p + q <= 2:
            np.testing.assert_allclose(lhs, rhs, atol=1e-15)
        if (p, q) == (2, 1):
            assert np.max(np.abs(lhs - rhs)) > 1e-3


def test_third_order_equilibrium_matches_all_moments_but_m22():
    """Partial third order (Fig. 4, middle): the matching conditions of every p, q <= 2 but
    (2, 2) hold -- M_21 and M_12 included, which correct the off-diagonal viscous stress
    (Sec. 2) -- and M_22 misses the Maxwellian's by exactly rho u_x^2 u_y^2."""
    rho, ux, uy = _fields()
    f = equilibrium.feq(rho, ux, uy, 3)
    for (p, q) in d2q9.PQ:
        lhs = sum(d2q9.XI[i, 0] ** p * d2q9.XI[i, 1] ** q * f[i] for i in range(9))
        rhs = _maxwellian_moment(rho, ux, uy, p, q)
        if (p, q) == (2, 2):
            np.testing.assert_allclose(rhs - lhs, rho * ux ** 2 * uy ** 2, rtol=0, atol=1e-15)
        else:
            np.testing.assert_allclose(lhs, rhs, rtol=0, atol=1e-15)


def test_third_order_equilibrium_is_the_truncated_hermite_expansion():
    """The D2Q9 Hermite expansion of the Maxwellian truncated after the mixed third-order
    terms, written out from the tensor Hermite polynomials:
    w_i [rho + rho xi.u / c_s^2 + (H2 : rho u u) / (2 c_s^4) + (H_xxy a_xxy + H_xyy a_xyy) / (2 c_s^6)]
    with a_xxy = rho u_x^2 u_y, a_xyy = rho u_x u_y^2 (3!/(3! c_s^6) times three equal
    permutations gives 1/(2 c_s^6)); its fourth-order Hermite moment is zero."""
    rho, ux, uy = _fields()
    f = equilibrium.feq(rho, ux, uy, 3)
    cs2 = d2q9.CS2
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    for i in range(9):
        x, y = d2q9.XI[i]
        h2 = (x * x - cs2) * ux * ux + 2 * x * y * ux * uy + (y * y - cs2) * uy * uy
        hxxy, hxyy = (x * x - cs2) * y, x * (y * y - cs2)
        ref = w[i] * rho * (1 + (x * ux + y * uy) / cs2 + h2 / (2 * cs2 ** 2)
                            + (hxxy * ux * ux * uy + hxyy * ux * uy * uy) / (2 * cs2 ** 3))
        np.testing.assert_allclose(f[i], ref, rtol=0, atol=2e-16)
    a22 = sum((d2q9.XI[i, 0] ** 2 - cs2) * (d2q9.XI[i, 1] ** 2 - cs2) * f[i] for i in range(9))
    np.testing.assert_allclose(a22, 0.0, atol=1e-16)


def test_equilibria_differ_by_their_truncated_hermite_terms():
    """Extended - third order = rho u_x^2 u_y^2 times the population vector of a unit M_22
    (Eq. Q9postCollVDF_RM: +1 at rest, -1/2 on the axes, +1/4 on the diagonals); all three
    orders coincide at rest (w_i rho)."""
    rho, ux, uy = _fields()
    d = equilibrium.feq(rho, ux, uy, 4) - equilibrium.feq(rho, ux, uy, 3)
    beta = {0: 1.0, 1: -0.5, -1: -0.5}
    for i in range(9):
        x, y = (int(v) for v in d2q9.XI[i])
        np.testing.assert_allclose(d[i], rho * ux ** 2 * uy ** 2 * beta[x] * beta[y], rtol=0, atol=2e-16)
    z = np.zeros(3)
    r = np.array([0.9, 1.0, 1.1])
    for order in (2, 3):
        np.testing.assert_allclose(equilibrium.feq(r, z, z, order), equilibrium.feq(r, z, z, 4), rtol=0, atol=1e-16)


def test_product_form_equals_moment_form():
    """The two equalities of Eq. extendedFeq agree."""
    rho, ux, uy = _fields()
    np.testing.assert_allclose(equilibrium.feq(rho, ux, uy), equilibrium.feq_product_form(rho, ux, uy),
                               rtol=0, atol=2e-16)


def test_central_hermite_equilibrium_closed_form():
    """App. B: all equilibrium CHMs vanish except A~_00 = rho."""
    rho, ux, uy = _fields()
    At = moments.central_hermite_moments(equilibrium.feq(rho, ux, uy), ux, uy)
    for pq, v in At.items():
        np.testing.assert_allclose(v, rho if pq == (0, 0) else 0.0, atol=2e-16)


def test_equilibrium_raw_moments_roundtrip():
    """Raw moments of the equilibrium populations equal the closed forms listed after
    Eq. RMcoll."""
    rho, ux, uy = _fields()
    for order in (2, 4):
        M = moments.raw_moments(equilibrium.feq(rho, ux, uy, order))
        Meq = equilibrium.raw_equilibrium_moments(rho, ux, uy, order)
        for pq in d2q9.PQ:
            np.testing.assert_allclose(M[pq], Meq[pq], atol=3e-16)


def test_d2q9_hermite_polynomials_are_orthogonal():
    """Textbook property of the D2Q9 Hermite basis: sum_i w_i H_pq H_rs = 0 for
    (p,q) != (r,s) and c_s^{2(p+q)} p! q! otherwise (p, q <= 2)."""
    w = equilibrium.feq(np.array(1.0), np.array(0.0), np.array(0.0))
    from math import factorial
    basis = {}
    for (p, q) in d2q9.PQ:
        e = {pq: 0.0 for pq in d2q9.PQ}
        basis[p, q] = []
        for i in range(9):
            f = np.zeros(9)
            f[i] = 1.0
            basis[p, q].append(moments.hermite_moments(f)[p, q])
    for a in d2q9.PQ:
        for b in d2q9.PQ:
            s = sum(w[i] * basis[a][i] * basis[b][i] for i in range(9))
            ref = d2q9.CS2 ** (a[0] + a[1]) * factorial(a[0]) * factorial(a[1]) if a == b else 0.0
            assert s == pytest.approx(ref, abs=1e-15)
