"""The oracle's pins are sensitive: plant a plausible mistake in the oracle (on the CPU,
through monkeypatching) and check that a pin fails.  Nothing here touches a GPU."""

import numpy as np
import pytest

import oracle.collision as collision
import oracle.lbm as lbm
import oracle.moments as moments
from oracle import d2q9
from paper_2002_05265_gb300 import flows

import test_oracle_collision as tc
import test_oracle_dynamics as td
import test_oracle_transforms as tt


def _expect_failure(fn, *args):
    with pytest.raises(AssertionError):
        fn(*args)


def test_wrong_sign_in_chm_to_hm_is_caught(monkeypatch):
    orig = moments.hermite_from_central_hermite

    def bad(At, rho, ux, uy):
        A = orig(At, rho, ux, uy)
        A[2, 1] = A[2, 1] - 2.0 * uy * At[2, 0]          # + u_y A~_20 turned into - u_y A~_20
        return A
    monkeypatch.setattr(moments, "hermite_from_central_hermite", bad)
    monkeypatch.setattr(collision, "hermite_from_central_hermite", bad)
    _expect_failure(tt.test_chm2hm_holds_with_the_corrected_polynomial)
    _expect_failure(tc.test_reg_identities)


def test_dropped_cs2_term_in_hm_to_rm_is_caught(monkeypatch):
    orig = moments.raw_from_hermite

    def bad(A):
        M = orig(A)
        M[2, 2] = M[2, 2] - d2q9.CS2 * A[0, 2]           # drops c_s^2 A_02 from M_22
        return M
    monkeypatch.setattr(moments, "raw_from_hermite", bad)
    monkeypatch.setattr(collision, "raw_from_hermite", bad)
    _expect_failure(tt.test_hm2rm_holds_for_any_distribution)
    _expect_failure(tc.test_srt_moment_models_reduce_to_bgk, "hm")


def test_transposed_cumulant_term_is_caught(monkeypatch):
    def bad(K):
        C = dict(K)
        C[2, 2] = K[2, 2] - (K[2, 0] * K[0, 2] + 2.0 * K[2, 0] * K[1, 1]) / K[0, 0]
        return C
    monkeypatch.setattr(moments, "cumulants_from_central", bad)
    _expect_failure(tt.test_cumulants_equal_log_mgf_derivatives_exactly)


def test_wrong_viscosity_relation_is_caught(monkeypatch):
    monkeypatch.setattr(lbm, "omega_from_nu", lambda nu: 1.0 / (nu / 0.5 + 0.5))   # c_s^2 taken as 1/2
    _expect_failure(td.test_shear_wave_decays_at_nu_k2, 1e-2, 200, 600)


def test_wrong_equilibrium_cross_term_is_caught(monkeypatch):
    import oracle.equilibrium as eq
    orig = eq.raw_equilibrium_moments

    def bad(rho, ux, uy, order=4):
        M = orig(rho, ux, uy, order)
        M[1, 2] = uy * M[0, 2]                            # u_x M02 with the wrong velocity
        return M
    monkeypatch.setattr(eq, "raw_equilibrium_moments", bad)
    import test_oracle_equilibrium as te
    _expect_failure(te.test_extended_equilibrium_matches_nine_maxwellian_moments)


def _vortex_core_x(f):
    rho, _, _ = collision.macroscopic(f)
    return float(np.argmin(rho.min(axis=0)))


def test_vortex_is_carried_downstream():
    """Sec. 5a: the vortex is transported by the mean flow u_0 along +x.  After t steps its
    density minimum has moved by u_0 t (nearest node)."""
    L, Ma, t = 48, 0.3, 120
    rho, ux, uy = flows.vortex(L, Ma=Ma)
    f = lbm.init_equilibrium(rho, ux, uy)
    x0 = _vortex_core_x(f)
    f = lbm.run(f, "bgk", lbm.rates_from_nu(1e-3), t)
    shift = (_vortex_core_x(f) - x0) % L
    assert abs(shift - Ma * np.sqrt(1 / 3) * t) <= 1.5


def test_reversed_streaming_is_caught(monkeypatch):
    def bad(fs):
        out = np.empty_like(fs)
        for i in range(9):
            out[i] = np.roll(fs[i], shift=(-int(d2q9.XI[i, 1]), -int(d2q9.XI[i, 0])), axis=(0, 1))
        return out
    monkeypatch.setattr(lbm, "stream", bad)
    _expect_failure(test_vortex_is_carried_downstream)


def test_pre_collision_cumulant_rebuild_is_caught(monkeypatch):
    """Planting the pre-collision rebuild of K~_22 (reading "pre" of
    oracle.collision.k_reading) into the oracle's K makes it grow at rest, which the
    flow-at-rest pin catches."""
    from functools import partial
    monkeypatch.setitem(collision.COLLIDE, "k", partial(collision.k_reading, rebuild="pre"))
    _expect_failure(td.test_flow_at_rest_is_linearly_stable, "k", "srt")
