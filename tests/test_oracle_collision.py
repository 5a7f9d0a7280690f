"""Pins of the oracle's collision models (App. B) against the identities the paper states
and against each model's own moment definition."""

import numpy as np
import pytest

from oracle import collision, equilibrium, lbm, moments, d2q9
from oracle.collision import macroscopic
from paper_2002_05265_gb300 import flows

MODELS = collision.MODELS


def _offeq(shape=(5, 4), seed=5, amp=0.05, umax=0.2):
    g = np.random.default_rng(seed)
    rho = 1.0 + 0.05 * g.uniform(-1, 1, shape)
    ux = umax * g.uniform(-1, 1, shape)
    uy = umax * g.uniform(-1, 1, shape)
    fe = equilibrium.feq(rho, ux, uy)
    return fe * (1.0 + amp * g.uniform(-1, 1, fe.shape))


@pytest.mark.parametrize("model", MODELS)
@pytest.mark.parametrize("rates", [(1.9, 1.9, 1.9), (1.9, 1.0, 1.0), (1.3, 0.7, 1.6)])
def test_equilibrium_is_a_fixed_point(model, rates):
    g = np.random.default_rng(1)
    rho = 1.0 + 0.05 * g.uniform(-1, 1, (4, 4))
    ux, uy = 0.3 * g.uniform(-1, 1, (2, 4, 4))
    fe = equilibrium.feq(rho, ux, uy)
    np.testing.assert_allclose(collision.collide(model, fe, *rates), fe, rtol=0, atol=1e-15)


def test_bgk_second_order_fixed_point():
    g = np.random.default_rng(2)
    rho = 1.0 + 0.05 * g.uniform(-1, 1, (4, 4))
    ux, uy = 0.3 * g.uniform(-1, 1, (2, 4, 4))
    fe = equilibrium.feq(rho, ux, uy, 2)
    np.testing.assert_allclose(collision.bgk(fe, 1.7, eq_order=2), fe, atol=1e-15)


@pytest.mark.parametrize("model", MODELS)
def test_collision_conserves_mass_and_momentum(model):
    f = _offeq()
    fs = collision.collide(model, f, 1.8, 1.2, 0.6)
    r0, x0, y0 = macroscopic(f)
    r1, x1, y1 = macroscopic(fs)
    np.testing.assert_allclose(r1, r0, atol=1e-15)
    np.testing.assert_allclose(r1 * x1, r0 * x0, atol=1e-15)
    np.testing.assert_allclose(r1 * y1, r0 * y0, atol=1e-15)


@pytest.mark.parametrize("model", ["rm", "hm", "cm", "chm"])
def test_srt_moment_models_reduce_to_bgk(model):
    """Sec. 4c and 5c: with omega3 = omega4 = omega_nu, RM, HM, CM and CHM are BGK."""
    f = _offeq()
    w = 1.97
    np.testing.assert_allclose(collision.collide(model, f, w, w, w), collision.bgk(f, w), rtol=0, atol=1e-15)


@pytest.mark.parametrize("model", ["k", "rr"])
def test_srt_k_and_rr_differ_from_bgk(model):
    """Sec. 4c and 5c: SRT-K and SRT-RR do not reduce to BGK."""
    f = _offeq()
    w = 1.97
    assert np.max(np.abs(collision.collide(model, f, w, w, w) - collision.bgk(f, w))) > 1e-6


def test_reg_identities():
    """Sec. 5c: REG-HM = REG-RR = PR and REG-CHM = SRT-RR."""
    f = _offeq()
    w = 1.93
    pr = collision.pr(f, w)
    np.testing.assert_allclose(collision.hm(f, w, 1.0, 1.0), pr, atol=1e-15)
    np.testing.assert_allclose(collision.rr(f, w, 1.0, 1.0), pr, atol=1e-15)
    np.testing.assert_allclose(collision.chm(f, w, 1.0, 1.0), collision.rr(f, w, w, w), atol=1e-15)
    np.testing.assert_allclose(collision.pr(f, w, 0.3, 1.7), pr, atol=0)


def test_bgk_with_unit_rate_returns_equilibrium():
    f = _offeq()
    rho, ux, uy = macroscopic(f)
    np.testing.assert_allclose(collision.bgk(f, 1.0), equilibrium.feq(rho, ux, uy), atol=1e-16)


RATES = (1.6, 0.7, 1.3)


def _relaxed(X, Xeq, pq):
    w = {2: RATES[0], 3: RATES[1], 4: RATES[2]}[pq[0] + pq[1]]
    return (1 - w) * X[pq] + w * Xeq[pq]


def _check_space(model, transform, eq_transform):
    f = _offeq()
    fs = collision.collide(model, f, *RATES)
    rho, ux, uy = macroscopic(f)
    X, Xs, Xeq = transform(f, ux, uy), transform(fs, ux, uy), eq_transform(rho, ux, uy)
    for pq in d2q9.PQ:
        ref = X[pq] if pq[0] + pq[1] <= 1 else _relaxed(X, Xeq, pq)
        np.testing.assert_allclose(Xs[pq], ref, rtol=0, atol=1e-15, err_msg=str(pq))


def test_rm_relaxes_raw_moments():
    _check_space("rm", lambda f, ux, uy: moments.raw_moments(f),
                 lambda r, ux, uy: equilibrium.raw_equilibrium_moments(r, ux, uy))


def test_hm_relaxes_hermite_moments():
    _check_space("hm", lambda f, ux, uy: moments.hermite_moments(f),
                 lambda r, ux, uy: moments.hermite_moments(equilibrium.feq(r, ux, uy)))


def test_cm_relaxes_central_moments():
    _check_space("cm", moments.central_moments,
                 lambda r, ux, uy: moments.central_moments(equilibrium.feq(r, ux, uy), ux, uy))


def test_chm_relaxes_central_hermite_moments():
    """Post-collision CHMs of f* equal Eq. CHMcoll (checks Eqs. CHM2HM_Q9, HM2RM_Q9 and
    Q9postCollVDF_RM end to end against the forward definition Eq. CHpoly)."""
    _check_space("chm", moments.central_hermite_moments,
                 lambda r, ux, uy: {pq: (r if pq == (0, 0) else 0 * r) for pq in d2q9.PQ})


def test_k_relaxes_cumulants():
    """Cumulants of f* (computed from its own central moments) are the relaxed cumulants."""
    cum = lambda f, ux, uy: moments.cumulants_from_central(moments.central_moments(f, ux, uy))
    _check_space("k", cum, lambda r, ux, uy: cum(equilibrium.feq(r, ux, uy), ux, uy))


def test_rr_hermite_moments_follow_recursion():
    """HMs of the RR post-collision state: order 2 relaxed with omega_nu, orders 3-4 equal
    A^eq + (1 - omega_n) A^neq_rec with the recursion of Eq. RRformulas_D2Q9."""
    f = _offeq()
    w, w3, w4 = RATES
    fs = collision.rr(f, w, w3, w4)
    rho, ux, uy = macroscopic(f)
    fe = equilibrium.feq(rho, ux, uy)
    A, As, Aeq = moments.hermite_moments(f), moments.hermite_moments(fs), moments.hermite_moments(fe)
    n = {pq: A[pq] - Aeq[pq] for pq in A}
    rec = {(2, 1): uy * n[2, 0] + 2 * ux * n[1, 1], (1, 2): ux * n[0, 2] + 2 * uy * n[1, 1],
           (2, 2): uy * uy * n[2, 0] + ux * ux * n[0, 2] + 4 * ux * uy * n[1, 1]}
    for pq in [(2, 0), (0, 2), (1, 1)]:
        np.testing.assert_allclose(As[pq], Aeq[pq] + (1 - w) * n[pq], atol=1e-15)
    np.testing.assert_allclose(As[2, 1], Aeq[2, 1] + (1 - w3) * rec[2, 1], atol=1e-15)
    np.testing.assert_allclose(As[1, 2], Aeq[1, 2] + (1 - w3) * rec[1, 2], atol=1e-15)
    np.testing.assert_allclose(As[2, 2], Aeq[2, 2] + (1 - w4) * rec[2, 2], atol=1e-15)


@pytest.mark.parametrize("model", MODELS)
def test_run_conserves_mass_and_momentum(model):
    """Streaming is a permutation and collision conserves rho and rho u: totals drift only
    by rounding over many steps on the convected vortex."""
    rho, ux, uy = flows.vortex(24, Ma=0.3, noise=1e-8)
    f = lbm.init_equilibrium(rho, ux, uy)
    r0 = lbm.reductions(f)
    f = lbm.run(f, model, lbm.rates_from_nu(1e-4, "reg" if model in ("k", "chm") else "srt"), 150)
    r1 = lbm.reductions(f)
    assert abs(r1[0] - r0[0]) / r0[0] < 1e-13
    assert abs(r1[1] - r0[1]) / abs(r0[1]) < 1e-13
    assert abs(r1[2] - r0[2]) < 1e-13 * abs(r0[1])


@pytest.mark.parametrize("model", MODELS)
def test_uniform_flow_stays_uniform(model):
    rho, ux, uy = np.ones((6, 7)), np.full((6, 7), 0.2), np.full((6, 7), -0.1)
    f0 = lbm.init_equilibrium(rho, ux, uy)
    f = lbm.run(f0, model, (1.9, 1.2, 1.5), 20)
    np.testing.assert_allclose(f, f0, atol=2e-15)


def test_srt_identities_hold_along_a_run():
    """The SRT identities survive many steps on the convected vortex; K and RR drift away."""
    rho, ux, uy = flows.vortex(24, Ma=0.3, noise=1e-8)
    f0 = lbm.init_equilibrium(rho, ux, uy)
    r = lbm.rates_from_nu(1e-5, "srt")
    ref = lbm.run(f0, "bgk", r, 100)
    for m in ("rm", "hm", "cm", "chm"):
        np.testing.assert_allclose(lbm.run(f0, m, r, 100), ref, rtol=0, atol=1e-13)
    for m in ("k", "rr"):
        assert np.max(np.abs(lbm.run(f0, m, r, 100) - ref)) > 1e-10
