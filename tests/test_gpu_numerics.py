"""GPU checks of two FP32 building blocks against FP64 or correctly rounded references.

* The reciprocal that forms u = j / rho (Sec. 1) in every FP32 kernel -- the hardware
  approximation plus one Newton-Raphson step -- against the correctly rounded reciprocal,
  exhaustively over the densities [0.5, 2) and on a logarithmic sweep of finite values.
* The blow-up / conservation reductions (Sec. 5b criterion; FP64 accumulation) for FP32 and
  FP16 storage: per node rho, j and u are formed in FP32 from the stored values and a few
  consecutive row segments are pre-summed in FP32 before each FP64 addition.  Their result is
  compared with the FP64 oracle's reductions of the same stored state against a first-order
  worst-case rounding bound derived below.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_2002_05265_gb300 import flows  # noqa: E402
import oracle.lbm as olbm  # noqa: E402
from oracle.d2q9 import XI  # noqa: E402

U32 = 2.0 ** -24          # unit roundoff of FP32


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2002_05265_gb300 import build, lbm
    build.build_library()
    lbm.load_library()
    return lbm


def _ulp_distance(a, b):
    """Distance in units in the last place between float32 arrays of the same sign (ordered
    integer representation)."""
    ia = a.view(np.int32).astype(np.int64)
    ib = b.view(np.int32).astype(np.int64)
    return np.abs(ia - ib)


def _recip(L, x):
    xd = torch.from_numpy(x).cuda()
    a, r = torch.empty_like(xd), torch.empty_like(xd)
    L.lbm_selftest_recip(xd, a, r)
    torch.cuda.synchronize()
    return a.cpu().numpy(), r.cpu().numpy()


def test_fp32_reciprocal_within_one_ulp_on_every_density_in_half_to_two(L):
    """Every float in [0.5, 2) (2^24 values): the library's reciprocal is within 1 ulp of the
    correctly rounded one, and equal to it for most inputs."""
    lo = np.float32(0.5).view(np.int32)
    hi = np.float32(2.0).view(np.int32)
    x = np.arange(lo, hi, dtype=np.int32).view(np.float32)
    a, r = _recip(L, x)
    d = _ulp_distance(a, r)
    assert d.max() <= 1, (d.max(), x[np.argmax(d)])
    assert (d == 0).mean() > 0.5


def test_fp32_reciprocal_on_a_wide_sweep_and_non_finite_inputs(L):
    g = np.random.default_rng(11)
    # finite values whose reciprocals are normal floats, both signs
    mag = np.exp(g.uniform(np.log(1e-36), np.log(1e36), 2_000_000)).astype(np.float32)
    x = np.concatenate([mag, -mag]).astype(np.float32)
    a, r = _recip(L, x)
    assert np.all(np.isfinite(a))
    assert _ulp_distance(a, r).max() <= 1
    # zero, infinities and NaN give NaN (documented in lbm.h): a node with such a density is
    # classified non-finite by the blow-up check in both arithmetics
    special = np.array([0.0, -0.0, np.inf, -np.inf, np.nan], dtype=np.float32)
    a, _ = _recip(L, special)
    assert np.all(np.isnan(a))


def _presum_bound(f, uref, nodes_per_flush):
    """First-order worst-case bound on |GPU - FP64| of each of the first six reduction slots
    for the stored state f (FP64 values that the stored FP32/FP16 numbers represent exactly).

    Per node, in FP32 with unit roundoff u: drho = sum of 9 stored values and j = sum of 6
    signed ones (any order): |err| <= 8 u S with S = sum_i |g_i|, g_i = f_i - w_i; rho =
    1 + drho adds u|rho|; 1/rho (one Newton step on the hardware approximation) is within one
    ulp; u_a = j_a (1/rho): err(u_a) <= err(j_a)/rho + |u_a| (err(rho)/rho + 3u); |u|^2 and
    rho |u|^2 add 2|u_a| err(u_a) terms and a few u of relative rounding.  The per-node values
    are then summed in FP32 over at most `nodes_per_flush` nodes before each FP64 addition:
    err <= (nodes_per_flush - 1) u sum |x|.  FP64 accumulation adds ~1e-16 relative."""
    u = U32
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)[:, None, None]
    S = np.abs(f - w).sum(axis=0)
    rho = f.sum(axis=0)
    jx = sum(float(XI[i, 0]) * f[i] for i in range(9))
    jy = sum(float(XI[i, 1]) * f[i] for i in range(9))
    ux, uy = jx / rho, jy / rho
    e_dr = 8 * u * S
    e_rho = e_dr + u * np.abs(rho)
    e_j = 8 * u * S
    e_ux = e_j / rho + np.abs(ux) * (e_rho / rho + 3 * u)
    e_uy = e_j / rho + np.abs(uy) * (e_rho / rho + 3 * u)
    u2 = ux * ux + uy * uy
    e_u2 = 2 * np.abs(ux) * e_ux + 2 * np.abs(uy) * e_uy + 3 * u * u2
    e_ke = rho * e_u2 + u2 * e_rho + 2 * u * rho * u2
    wx, wy = ux - uref[0], uy - uref[1]
    w2 = wx * wx + wy * wy
    e_w2 = 2 * np.abs(wx) * (e_ux + u * np.abs(ux)) + 2 * np.abs(wy) * (e_uy + u * np.abs(uy)) + 3 * u * w2
    k = (nodes_per_flush - 1) * u
    n = rho.size
    return np.array([
        e_dr.sum() + k * np.abs(rho - 1).sum(),
        e_j.sum() + k * np.abs(jx).sum(),
        e_j.sum() + k * np.abs(jy).sum(),
        0.5 * (e_ke.sum() + k * (rho * u2).sum()),
        (e_u2.sum() + k * u2.sum()) / n,
        (e_w2.sum() + k * w2.sum()) / n,
    ])


@pytest.mark.parametrize("storage,vec", [("f32", 4), ("f16", 8)])
def test_presummed_reductions_within_rounding_bound_of_fp64(L, storage, vec):
    """A 256 x 200 double shear layer (CHM, REG, nu = 1e-4) after 300 steps in FP32 / FP16
    storage: lbm_reduce against the oracle's FP64 reductions of the same stored populations
    (read back exactly with lbm_get_populations), slot by slot within the derived bound
    (4 row segments of `vec` nodes pre-summed per FP64 addition); min rho within its per-node
    bound; the non-finite count exact."""
    nx, ny = 256, 200
    fields = flows.double_shear_layer(nx, ny, Ma=0.1, width_frac=0.1)
    lat = L.Lattice(nx, ny, L.LBM_CHM, olbm.rates_from_nu(1e-4, "reg"), storage=L.STORAGES[storage])
    lat.init_equilibrium(*[torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in fields])
    lat.step(300)
    uref = (0.05, 0.01)
    lat.set_check(0, uref=uref)
    red = torch.empty(8, dtype=torch.float64, device="cuda")
    lat.reduce(red)
    f = np.empty((9, ny, nx))
    lat.get_populations(f)
    lat.close()
    got = red.cpu().numpy()
    ref = olbm.reductions(f, uref)
    bound = _presum_bound(f, uref, 4 * vec)
    err = np.abs(got[:6] - ref[:6])
    assert np.all(err <= bound), (err, bound)
    # the bound is not vacuous: small against the total mass, the momentum magnitudes (the
    # signed totals of this flow nearly cancel) and the energies
    rho = f.sum(axis=0)
    jx = sum(float(XI[i, 0]) * f[i] for i in range(9))
    jy = sum(float(XI[i, 1]) * f[i] for i in range(9))
    assert bound[0] / ref[0] < 1e-6
    assert bound[1] / np.abs(jx).sum() < 1e-4 and bound[2] / np.abs(jy).sum() < 1e-4
    assert np.all(bound[3:6] / ref[3:6] < 1e-4)
    # min rho: the minimum of per-node FP32 densities, each within 8 u S of the FP64 one
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)[:, None, None]
    assert abs(got[6] - ref[6]) <= 8 * U32 * np.abs(f - w).sum(axis=0).max() + 1e-15
    assert got[7] == ref[7] == 0
