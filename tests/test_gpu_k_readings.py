"""GPU checks of the two alternative readings of the cumulant rebuild (LBM_K_PRE, LBM_K_EQ:
the fourth-order central moment rebuilt with the pre-collision / equilibrium second-order
central moments), which run the K kernels with other per-launch constants: FP64 stepping,
the batched sweep, the exact collision Jacobian of the linear stability tool and the adjoint
against the oracle's oracle.collision.k_reading."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_2002_05265_gb300 import flows  # noqa: E402
import oracle.lbm as olbm  # noqa: E402
import oracle.lsa as olsa  # noqa: E402
from oracle import adjoint as oadj  # noqa: E402

READINGS = ["k_pre", "k_eq"]
CS = 1.0 / np.sqrt(3.0)


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2002_05265_gb300 import build, lbm
    build.build_library()
    lbm.load_library()
    return lbm


def _run(L, fields, model, rates, steps, path):
    rho, ux, uy = fields
    ny, nx = rho.shape
    lat = L.Lattice(nx, ny, L.MODELS[model], rates, storage=L.LBM_F64)
    lat.set_kernel_path(path)
    lat.init_equilibrium(*[torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in fields])
    lat.step(steps)
    f = torch.empty((9, ny, nx), dtype=torch.float64, device="cuda")
    lat.get_populations(f)
    lat.close()
    return f.cpu().numpy()


@pytest.mark.parametrize("model", READINGS)
@pytest.mark.parametrize("preset", ["srt", "reg"])
@pytest.mark.parametrize("path", ["vector", "bulk"])
def test_readings_fp64_match_the_oracle(L, model, preset, path):
    """64 x 37 vortex, 6 steps, both kernel families: populations within 1e-12 relative of the
    oracle.  The readings amplify every perturbation, rounding differences between the two
    arithmetics included, by up to e^0.63 per step (their growth rate at rest), so the runs are
    short: ~1e-15 of per-step rounding grows by e^3.8 ~ 44 over 6 steps (12 steps reached
    1.4e-12, the e^7.6 ~ 2000 of that growth)."""
    fields = flows.vortex(64, 37, Ma=0.2, noise=1e-6, seed=5)
    rates = olbm.rates_from_nu(1e-3, preset)
    got = _run(L, fields, model, rates, 6, {"vector": L.LBM_PATH_VECTOR, "bulk": L.LBM_PATH_BULK}[path])
    ref = olbm.run(olbm.init_equilibrium(*fields), model, rates, 6)
    assert float(np.max(np.abs(got - ref) / np.abs(ref))) <= 1e-12


def test_readings_in_the_batched_sweep(L):
    """Batch instances of both readings (FP64, 6 steps: short for the reason above) equal the
    oracle within 1e-12."""
    descs, fields = [], []
    for k, (m, preset) in enumerate([(m, p) for m in READINGS for p in ("srt", "reg")]):
        nx, ny = 40 + 3 * k, 33 + 2 * k
        descs.append(dict(nx=nx, ny=ny, model=m, rates=olbm.rates_from_nu(1e-2, preset), ux_ref=0.1 * CS, uy_ref=0.0))
        fields.append(flows.uniform_noise(nx, ny, Ma=0.1, amp=1e-6, seed=50 + k))
    b = L.lbm_batch_create(descs, storage=L.LBM_F64)
    cat = [np.ascontiguousarray(np.concatenate([f[i].ravel() for f in fields])) for i in range(3)]
    L.lbm_batch_init_equilibrium(b, *cat)
    L.lbm_batch_run(b, 6, check_every=3, growth=1e300)
    for k, (d, f) in enumerate(zip(descs, fields)):
        got = np.empty((9, d["ny"], d["nx"]))
        L.lbm_batch_get_populations(b, k, got)
        ref = olbm.run(olbm.init_equilibrium(*f), d["model"], d["rates"], 6)
        assert float(np.max(np.abs(got - ref) / np.abs(ref))) <= 1e-12, (k, d["model"])
    L.lbm_batch_destroy(b)


@pytest.mark.parametrize("model", READINGS)
@pytest.mark.parametrize("preset", ["srt", "reg"])
def test_readings_jacobian_and_growth_at_rest(L, model, preset):
    """lbm_lsa_growth's exact Jacobian of each reading equals the oracle's complex-step one
    (1e-12, three base flows), and at rest (nu = 1e-6) the reading's largest growth rate
    matches the oracle's: e^0.63 / e^0.51 per step for "pre", e^0.33 for SRT "eq", none for
    REG "eq" -- the linear instability at rest of Sec. 4b that these readings reproduce."""
    rates = olbm.rates_from_nu(1e-6, preset)
    fl = np.array([[1.0, 0.0, 0.0], [1.03, 0.1, -0.05], [0.97, -0.2, 0.15]])
    k1 = np.linspace(-np.pi, np.pi, 33)
    ks = np.array([(a, b) for a in k1 for b in k1])
    flt = torch.from_numpy(fl).cuda()
    kk = torch.from_numpy(ks).cuda()
    growth = torch.empty((3, len(ks)), dtype=torch.float64, device="cuda")
    jac = torch.empty((3, 9, 9), dtype=torch.float64, device="cuda")
    L.lbm_lsa_growth(model, rates, flt, kk, growth, jac=jac)
    for j in range(3):
        G = olsa.collision_map_jacobian(model, fl[j, 0], fl[j, 1], fl[j, 2], rates)
        np.testing.assert_allclose(jac[j].cpu().numpy(), G, atol=1e-12)
    G0 = olsa.collision_map_jacobian(model, 1.0, 0.0, 0.0, rates)
    ref = olsa.max_growth_rate(G0, k1, k1)
    got = float(growth[0].max())
    if model == "k_eq" and preset == "reg":
        assert got < 1e-12 and ref < 1e-12
    else:
        assert got == pytest.approx(ref, rel=1e-9) and got > 0.3


@pytest.mark.parametrize("model", READINGS)
def test_readings_adjoint_matches_complex_step(L, model):
    """FP64 adjoint of an 8-step misfit run (22 x 18 vortex): the u0 directional derivative
    and the three rate derivatives equal the oracle's complex-step derivatives to 1e-9."""
    rho, ux, uy = flows.vortex(22, 18, Ma=0.25, noise=1e-3, seed=3)
    tx = np.roll(ux, 2, axis=1) + flows.gaussian_noise(ux.shape, 1e-3, 4)
    ty = np.roll(uy, 2, axis=1) + flows.gaussian_noise(uy.shape, 1e-3, 5)
    rates, n = (1.8, 1.3, 0.7), 8
    lat = L.Lattice(22, 18, L.MODELS[model], rates, storage=L.LBM_F64)
    lat.init_equilibrium(*[np.ascontiguousarray(a) for a in (rho, ux, uy)])
    gx, gy = np.zeros_like(ux), np.zeros_like(uy)
    val, gr, _ = L.lbm_adjoint_run(lat.ctx, n, 0, np.ascontiguousarray(tx), np.ascontiguousarray(ty), gx, gy, 3)
    lat.close()
    assert val == pytest.approx(oadj.run_loss(rho, ux, uy, model, rates, n, "misfit", tx, ty), rel=1e-12)
    g = np.random.default_rng(6)
    dx, dy = g.standard_normal(ux.shape), g.standard_normal(uy.shape)
    ref = oadj.directional_derivative(rho, ux, uy, model, rates, n, "misfit", tx, ty, dux=dx, duy=dy)
    assert float((gx * dx).sum() + (gy * dy).sum()) == pytest.approx(ref, rel=1e-9)
    for k in range(3):
        d = [0.0, 0.0, 0.0]
        d[k] = 1.0
        ref = oadj.directional_derivative(rho, ux, uy, model, rates, n, "misfit", tx, ty, drates=d)
        assert gr[k] == pytest.approx(ref, rel=1e-9, abs=1e-14), k
