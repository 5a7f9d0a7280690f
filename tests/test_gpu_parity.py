"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the same seeded
inputs.  Tolerances: FP64 populations <= 1e-12 relative; FP32 velocity <= 1e-5 absolute
after 1000 steps (both stated targets of the method's specification); FP16 storage shifted
at the reference state (rho0, mean flow) <= 1e-3 normalised L2 on the vortex velocity (the
stated FP16 target, reading of "shifted storage" recorded in the design notes); FP16 / BF16
storage shifted by w_i rho0 within twice the random-walk estimate of the storage rounding
(storage_walk_error); FP32 conservation within six standard deviations of the same rounding
walk (conservation_walk_bound)."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_2002_05265_gb300 import flows  # noqa: E402
import oracle.lbm as olbm  # noqa: E402
from oracle.collision import macroscopic  # noqa: E402
from storage_bounds import WALK_FACTOR, conservation_walk_bound, storage_walk_error  # noqa: E402

MODELS = ["bgk", "rm", "hm", "cm", "chm", "k", "pr", "rr"]


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2002_05265_gb300 import build, lbm
    build.build_library()
    lbm.load_library()
    return lbm


def _dev(*arrs):
    return [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrs]


def _run_gpu(L, fields, model, rates, storage, steps, eq_order=4):
    rho, ux, uy = fields
    ny, nx = rho.shape
    lat = L.Lattice(nx, ny, L.MODELS[model], rates, storage=storage, eq_order=eq_order)
    lat.init_equilibrium(*_dev(rho, ux, uy))
    lat.step(steps)
    f = torch.empty((9, ny, nx), dtype=torch.float64, device="cuda")
    lat.get_populations(f)
    out = f.cpu().numpy()
    lat.close()
    return out


def _rel(a, b):
    return float(np.max(np.abs(a - b) / np.abs(b)))


def test_vortex_128_bgk_fp64_1000_steps(L):
    """Convected vortex, 128 x 128, Ma = 0.1, nu = 1e-4, seeded 1e-8 velocity noise, BGK with
    the extended equilibrium, FP64, 1000 steps: populations within 1e-12 relative."""
    fields = flows.vortex(128, Ma=0.1, noise=1e-8, seed=1)
    rates = olbm.rates_from_nu(1e-4, "srt")
    got = _run_gpu(L, fields, "bgk", rates, L.LBM_F64, 1000)
    ref = olbm.run(olbm.init_equilibrium(*fields), "bgk", rates, 1000)
    assert _rel(got, ref) <= 1e-12


@pytest.mark.parametrize("model", MODELS)
@pytest.mark.parametrize("preset", ["srt", "reg"])
def test_every_model_fp64_ragged(L, model, preset):
    """67 x 37 (ragged against every vector width and warp), Ma = 0.3 vortex, 150 steps."""
    fields = flows.vortex(67, 37, Ma=0.3, noise=1e-6, seed=2)
    rates = olbm.rates_from_nu(1e-3, preset)
    got = _run_gpu(L, fields, model, rates, L.LBM_F64, 150)
    ref = olbm.run(olbm.init_equilibrium(*fields), model, rates, 150)
    assert _rel(got, ref) <= 1e-12


@pytest.mark.parametrize("eq_order", [2, 3])
def test_truncated_equilibria_bgk_fp64(L, eq_order):
    """BGK with the second-order (Sec. 2) and the partial third-order (Fig. 4) equilibrium,
    48 x 40 Ma = 0.2 vortex, 100 steps: populations within 1e-12 relative."""
    fields = flows.vortex(48, 40, Ma=0.2, noise=1e-6, seed=3)
    rates = olbm.rates_from_nu(1e-3, "srt")
    got = _run_gpu(L, fields, "bgk", rates, L.LBM_F64, 100, eq_order=eq_order)
    ref = olbm.run(olbm.init_equilibrium(*fields, eq_order=eq_order), "bgk", rates, 100, eq_order=eq_order)
    assert _rel(got, ref) <= 1e-12


@pytest.mark.parametrize("model", MODELS)
def test_every_model_fp32_1000_steps(L, model):
    """Double shear layer resolved as in the 1024^2 workload (layer width 12.8 nodes), on a
    128 x 96 lattice (ragged for 4-wide vectors is covered elsewhere), Ma = 0.1, nu = 1e-5,
    FP32 shifted storage, 1000 steps: velocity within 1e-5 absolute of the FP64 oracle."""
    fields = flows.double_shear_layer(128, 96, Ma=0.1, width_frac=12.8 / 96)
    rates = olbm.rates_from_nu(1e-5, "srt" if model == "bgk" else "reg")
    got = _run_gpu(L, fields, model, rates, L.LBM_F32, 1000)
    ref = olbm.run(olbm.init_equilibrium(*fields), model, rates, 1000)
    _, gx, gy = macroscopic(got)
    _, rx, ry = macroscopic(ref)
    assert max(np.max(np.abs(gx - rx)), np.max(np.abs(gy - ry))) <= 1e-5


@pytest.mark.parametrize("model", MODELS)
def test_every_model_fp32_ragged_vortex(L, model):
    """FP32 on a lattice ragged against the 4-wide vectors and the warps (99 x 45)."""
    fields = flows.vortex(99, 45, Ma=0.2, noise=1e-8, seed=8)
    rates = olbm.rates_from_nu(1e-4, "srt" if model == "bgk" else "reg")
    got = _run_gpu(L, fields, model, rates, L.LBM_F32, 300)
    ref = olbm.run(olbm.init_equilibrium(*fields), model, rates, 300)
    _, gx, gy = macroscopic(got)
    _, rx, ry = macroscopic(ref)
    assert max(np.max(np.abs(gx - rx)), np.max(np.abs(gy - ry))) <= 1e-5


def _l2(got, ref):
    _, gx, gy = macroscopic(got)
    _, rx, ry = macroscopic(ref)
    return float(np.sqrt(((gx - rx) ** 2 + (gy - ry) ** 2).sum() / (rx ** 2 + ry ** 2).sum()))



# FP16 / BF16 storage of f - w rho0 on the 96^2, Ma = 0.1, nu = 1e-4 vortex, 1000 steps: the
# normalised L2 velocity error against the FP64 oracle is held to twice the random-walk
# estimate of storage_walk_error (the factor covers the spread of a sum of random kicks over
# ~10^4 nodes and the FP32 collision arithmetic, whose rounding is ~2^-13 of the storage's).
# The stated 1e-3 FP16 target is met with the shift at the mean flow (next test); with the
# w rho0 shift the populations themselves, not the perturbation, set the ulp.


@pytest.mark.parametrize("model", MODELS)
def test_fp16_shifted_vortex_error(L, model):
    fields = flows.vortex(96, Ma=0.1, noise=1e-8, seed=1)
    rates = olbm.rates_from_nu(1e-4, "srt" if model == "bgk" else "reg")
    got = _run_gpu(L, fields, model, rates, L.LBM_F16, 1000)
    f0 = olbm.init_equilibrium(*fields)
    ref = olbm.run(f0, model, rates, 1000)
    est = storage_walk_error(f0, "f16", 1000)
    assert _l2(got, ref) <= WALK_FACTOR * est, (_l2(got, ref), est)


@pytest.mark.parametrize("model", ["bgk", "chm", "k", "rr"])
def test_bf16_shifted_vortex_error(L, model):
    fields = flows.vortex(96, Ma=0.1, noise=1e-8, seed=1)
    rates = olbm.rates_from_nu(1e-4, "srt" if model == "bgk" else "reg")
    got = _run_gpu(L, fields, model, rates, L.LBM_BF16, 1000)
    f0 = olbm.init_equilibrium(*fields)
    ref = olbm.run(f0, model, rates, 1000)
    est = storage_walk_error(f0, "bf16", 1000)
    assert _l2(got, ref) <= WALK_FACTOR * est, (_l2(got, ref), est)


@pytest.mark.parametrize("model", MODELS)
def test_fp16_with_mean_flow_shift_vortex_error(L, model):
    """The same FP16 run with the storage shift taken at the mean flow, g = f - f^eq(1, u0):
    the stored deviations shrink to the vortex perturbation and the error falls below the
    1e-3 normalised L2 target."""
    fields = flows.vortex(96, Ma=0.1, noise=1e-8, seed=1)
    rates = olbm.rates_from_nu(1e-4, "srt" if model == "bgk" else "reg")
    lat = L.Lattice(96, 96, L.MODELS[model], rates, storage=L.LBM_F16)
    lat.set_shift_velocity(0.1 / np.sqrt(3.0), 0.0)
    lat.init_equilibrium(*_dev(*fields))
    lat.step(1000)
    f = np.empty((9, 96, 96))
    lat.get_populations(f)
    lat.close()
    ref = olbm.run(olbm.init_equilibrium(*fields), model, rates, 1000)
    assert _l2(f, ref) <= 1e-3


@pytest.mark.parametrize("model", ["bgk", "cm", "chm", "k", "rr"])
def test_shift_velocity_fp64_parity(L, model):
    """A non-zero shift velocity changes only the storage encoding: FP64 results still match
    the oracle to 1e-12, including a re-encoding in the middle of the run."""
    fields = flows.vortex(64, 48, Ma=0.3, noise=1e-6, seed=9)
    rates = olbm.rates_from_nu(1e-3, "reg")
    lat = L.Lattice(64, 48, L.MODELS[model], rates, storage=L.LBM_F64)
    lat.set_shift_velocity(0.17, -0.03)
    lat.init_equilibrium(*_dev(*fields))
    lat.step(60)
    lat.set_shift_velocity(-0.05, 0.08)
    lat.step(40)
    f = np.empty((9, 48, 64))
    lat.get_populations(f)
    lat.close()
    assert _rel(f, olbm.run(olbm.init_equilibrium(*fields), model, rates, 100)) <= 1e-12


def test_moments_and_reductions_match_oracle(L):
    fields = flows.vortex(40, 33, Ma=0.2, noise=1e-6, seed=4)
    rates = olbm.rates_from_nu(1e-3, "reg")
    lat = L.Lattice(40, 33, L.LBM_CHM, rates, storage=L.LBM_F64)
    lat.init_equilibrium(*_dev(*fields))
    lat.step(37)
    outs = [torch.empty((33, 40), dtype=torch.float64, device="cuda") for _ in range(6)]
    lat.moments(*outs)
    red = torch.empty(8, dtype=torch.float64, device="cuda")
    lat.set_check(0, uref=(0.1, -0.02))
    lat.reduce(red)
    ref_f = olbm.run(olbm.init_equilibrium(*fields), "chm", rates, 37)
    for g, r in zip(outs, olbm.moments_output(ref_f)):
        np.testing.assert_allclose(g.cpu().numpy(), r, rtol=0, atol=1e-13)
    np.testing.assert_allclose(red.cpu().numpy(), olbm.reductions(ref_f, (0.1, -0.02)), rtol=1e-12, atol=1e-14)
    lat.close()


def test_successive_checks_reset_the_completion_counter(L):
    """lbm_reduce runs its second pass in the last block of the first launch (a completion
    counter that every launch leaves at zero): 25 successive reductions of an evolving FP64
    lattice, three steps apart, each equal the oracle's reductions of the same populations."""
    fields = flows.vortex(40, 33, Ma=0.2, noise=1e-6, seed=8)
    rates = olbm.rates_from_nu(1e-3, "reg")
    lat = L.Lattice(40, 33, L.LBM_K, rates, storage=L.LBM_F64)
    lat.init_equilibrium(*_dev(*fields))
    lat.set_check(0, uref=(0.05, 0.01))
    red = torch.empty(8, dtype=torch.float64, device="cuda")
    f = torch.empty((9, 33, 40), dtype=torch.float64, device="cuda")
    for _ in range(25):
        lat.step(3)
        lat.reduce(red)
        lat.get_populations(f)
        np.testing.assert_allclose(red.cpu().numpy(), olbm.reductions(f.cpu().numpy(), (0.05, 0.01)),
                                   rtol=1e-12, atol=1e-14)
    lat.close()


def test_host_and_device_pointers_agree(L):
    fields = flows.vortex(32, Ma=0.2, noise=1e-6, seed=5)
    rates = olbm.rates_from_nu(1e-3)
    a = L.Lattice(32, 32, L.LBM_RR, rates, storage=L.LBM_F32)
    b = L.Lattice(32, 32, L.LBM_RR, rates, storage=L.LBM_F32)
    a.init_equilibrium(*[np.ascontiguousarray(x) for x in fields])          # host pointers
    b.init_equilibrium(*_dev(*fields))                                       # device pointers
    a.step(20)
    b.step(20)
    fa = np.empty((9, 32, 32))
    a.get_populations(fa)
    fb = torch.empty((9, 32, 32), dtype=torch.float64, device="cuda")
    b.get_populations(fb)
    np.testing.assert_array_equal(fa, fb.cpu().numpy())
    a.close()
    b.close()


def test_graph_replay_equals_single_launches(L):
    """lbm_step(n) replays recorded CUDA graphs; stepping one at a time gives identical bits."""
    fields = flows.vortex(50, 44, Ma=0.2, noise=1e-6, seed=6)
    rates = olbm.rates_from_nu(1e-3, "reg")
    a = L.Lattice(50, 44, L.LBM_K, rates, storage=L.LBM_F32)
    b = L.Lattice(50, 44, L.LBM_K, rates, storage=L.LBM_F32)
    for lat in (a, b):
        lat.init_equilibrium(*_dev(*fields))
    a.step(101)
    for _ in range(101):
        b.step(1)
    fa = torch.empty((9, 44, 50), dtype=torch.float64, device="cuda")
    fb = torch.empty_like(fa)
    a.get_populations(fa)
    b.get_populations(fb)
    assert torch.equal(fa, fb)
    a.close()
    b.close()


def test_group_stepping_equals_individual_stepping(L):
    fields = flows.double_shear_layer(64, 48)
    rates = olbm.rates_from_nu(1e-4, "srt")
    lats = [L.Lattice(64, 48, L.MODELS[m], rates, storage=L.LBM_F32) for m in ("bgk", "hm", "rr")]
    refs = [L.Lattice(64, 48, L.MODELS[m], rates, storage=L.LBM_F32) for m in ("bgk", "hm", "rr")]
    for lat in lats + refs:
        lat.init_equilibrium(*_dev(*fields))
    g = L.lbm_group_create([x.ctx for x in lats], graph_steps=8)
    L.lbm_group_step(g, 45)
    for r in refs:
        r.step(45)
    for x, r in zip(lats, refs):
        fa = torch.empty((9, 48, 64), dtype=torch.float64, device="cuda")
        fb = torch.empty_like(fa)
        x.get_populations(fa)
        r.get_populations(fb)
        assert torch.equal(fa, fb)
    L.lbm_group_destroy(g)
    for lat in lats + refs:
        lat.close()


def test_set_get_populations_roundtrip(L):
    g = np.random.default_rng(0)
    f = olbm.init_equilibrium(*flows.vortex(24, 20, Ma=0.2)) * (1 + 1e-3 * g.uniform(-1, 1, (9, 20, 24)))
    lat = L.Lattice(24, 20, L.LBM_BGK, (1.5, 1.5, 1.5), storage=L.LBM_F64)
    lat.set_populations(np.ascontiguousarray(f))
    back = np.empty_like(f)
    lat.get_populations(back)
    np.testing.assert_allclose(back, f, rtol=0, atol=1e-16)
    lat.step(3)
    lat.get_populations(back)
    np.testing.assert_allclose(back, olbm.run(f, "bgk", (1.5, 1.5, 1.5), 3), rtol=1e-14)
    lat.close()


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_conservation(L, storage):
    """Mass and momentum totals (FP64 reductions) over 2000 steps of a 128^2 double shear
    layer.  FP64: exact to 1e-14 relative (the moment-space collision keeps the conserved
    moments of the stored values; only their rounding moves them).  FP32: the drift stays
    within six standard deviations of the random walk of the per-step storage rounding
    (conservation_walk_bound: ~2e-5 absolute here, against the 1.6e-3 of a 1e-7 relative
    mass bound)."""
    fields = flows.double_shear_layer(128, 128, width_frac=0.1)
    lat = L.Lattice(128, 128, L.LBM_CHM, olbm.rates_from_nu(1e-5, "reg"), storage=L.STORAGES[storage])
    lat.init_equilibrium(*_dev(*fields))
    r0 = np.empty(8)
    lat.reduce(r0)
    lat.step(2000)
    r1 = np.empty(8)
    lat.reduce(r1)
    lat.close()
    drift = np.abs(r1[:3] - r0[:3])
    if storage == "f64":
        assert drift[0] / r0[0] < 1e-14 and drift[1] < 1e-14 * r0[0] and drift[2] < 1e-14 * r0[0]
    else:
        bound = conservation_walk_bound(olbm.init_equilibrium(*fields), "f32", 2000)
        assert np.all(drift <= bound), (drift, bound)


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_group_checks_equal_individual_checks(L, storage):
    """Blow-up checks of a group's lattices that fall due together run in one launch (each
    lattice's check with its own grid-wide fold over fewer blocks): five 32 x 32 lattices with
    check cadences 50, 50, 100, 0 and 50 (two unstable, Ma = 0.9; one with the kinetic-energy
    criterion), 1000 steps in graph chunks of 10, give the same status and blow-up step as
    each lattice stepped alone, and the stable ones the same populations."""
    n = 32
    specs = [("bgk", 0.9, 1e-6, 50, 0.0), ("rr", 0.1, 1e-2, 50, 0.0), ("chm", 0.1, 1e-3, 100, 0.0),
             ("k", 0.1, 1e-3, 0, 0.0), ("hm", 0.9, 1e-6, 50, 1e-3)]

    def make(m, ma, nu, every, ke):
        lat = L.Lattice(n, n, L.MODELS[m], olbm.rates_from_nu(nu), storage=L.STORAGES[storage])
        lat.init_equilibrium(*_dev(*flows.uniform_noise(n, Ma=ma, amp=1e-3, seed=3)))
        lat.set_check(every, ke_ref=ke)
        return lat

    grp = [make(*sp) for sp in specs]
    alone = [make(*sp) for sp in specs]
    g = L.lbm_group_create([x.ctx for x in grp], graph_steps=10)
    L.lbm_group_step(g, 1000)
    for a in alone:
        a.step(1000)
    blown = 0
    for x, a in zip(grp, alone):
        assert x.status() == a.status()
        if x.status()[0] == L.LBM_ERR_BLOWUP:
            blown += 1
            continue
        fa = torch.empty((9, n, n), dtype=torch.float64, device="cuda")
        fb = torch.empty_like(fa)
        x.get_populations(fa)
        a.get_populations(fb)
        assert torch.equal(fa, fb)
    assert blown >= 2
    L.lbm_group_destroy(g)
    for lat in grp + alone:
        lat.close()


def test_blowup_detection(L):
    """An unstable lattice (BGK, Ma = 0.9, nu = 1e-6) is flagged by the periodic check; a
    stable one is not; a NaN written from the host is caught at the next check."""
    n = 32
    unstable = L.Lattice(n, n, L.LBM_BGK, olbm.rates_from_nu(1e-6), storage=L.LBM_F32)
    unstable.init_equilibrium(*_dev(*flows.uniform_noise(n, Ma=0.9, amp=1e-3, seed=1)))
    unstable.set_check(50)
    unstable.step(3000)
    st, step, steps = unstable.status()
    assert st == L.LBM_ERR_BLOWUP and 0 < step <= 3000 and step % 50 == 0 and steps == 3000
    stable = L.Lattice(n, n, L.LBM_RR, olbm.rates_from_nu(1e-2), storage=L.LBM_F32)
    stable.init_equilibrium(*_dev(*flows.uniform_noise(n, Ma=0.1, amp=1e-6, seed=1)))
    stable.set_check(50)
    stable.step(1000)
    assert stable.status()[:2] == (0, -1)
    f = np.empty((9, n, n))
    stable.get_populations(f)
    f[3, 5, 7] = np.nan
    stable.set_populations(f)
    stable.step(50)
    assert stable.status()[:2] == (L.LBM_ERR_BLOWUP, 1050)
    unstable.close()
    stable.close()


@pytest.mark.parametrize("model", MODELS)
def test_full_size_double_shear_layer_sampled(L, model):
    """1024 x 1024 double shear layer (Ma = 0.1, nu = 1e-5, FP32, the benchmark's lattices):
    after k = 12 steps, 24 sampled nodes agree with the oracle run on the (2k+3)^2 patch around
    each node (the light cone of a stream-and-collide step is one node per step)."""
    N, k = 1024, 12
    fields = flows.double_shear_layer(N, Ma=0.1)
    rates = olbm.rates_from_nu(1e-5, "reg" if model in ("chm", "k") else "srt")
    lat = L.Lattice(N, N, L.MODELS[model], rates, storage=L.LBM_F32)
    lat.init_equilibrium(*_dev(*fields))
    lat.step(k)
    ux = torch.empty((N, N), dtype=torch.float64, device="cuda")
    uy = torch.empty_like(ux)
    lat.moments(None, ux, uy)
    ux, uy = ux.cpu().numpy(), uy.cpu().numpy()
    lat.close()
    g = np.random.default_rng(7)
    pts = list(zip(g.integers(0, N, 22), g.integers(0, N, 22))) + [(0, 0), (N - 1, N - 1)]
    P = 2 * k + 3
    for (y, x) in pts:
        ys = (np.arange(P) + y - P // 2) % N
        xs = (np.arange(P) + x - P // 2) % N
        patch = [a[np.ix_(ys, xs)] for a in fields]
        fr = olbm.run(olbm.init_equilibrium(*patch), model, rates, k)
        _, rx, ry = macroscopic(fr)
        assert abs(ux[y, x] - rx[P // 2, P // 2]) <= 1e-5
        assert abs(uy[y, x] - ry[P // 2, P // 2]) <= 1e-5


def test_benchmark_group_configuration_sampled(L):
    """The benchmark's own launch configuration: the eight 1024 x 1024 FP32 double-shear-layer
    lattices (one per model, nu = 1e-5, BGK SRT and the others REG) in one group with 100-step
    graph chunks, i.e. 100 copy-engine launches (wide form) each advancing all eight by one
    step.  After those
    100 steps, 2 sampled nodes per lattice (one at the periodic corner) agree with the oracle
    run on the (2k + 3)^2 light-cone patch around each node within 1e-5 on u."""
    N, k = 1024, 100
    fields = flows.double_shear_layer(N, Ma=0.1)
    dev = _dev(*fields)
    lats = []
    for m in MODELS:
        rates = olbm.rates_from_nu(1e-5, "srt" if m == "bgk" else "reg")
        lat = L.Lattice(N, N, L.MODELS[m], rates, storage=L.LBM_F32)
        lat.init_equilibrium(*dev)
        lats.append((m, rates, lat))
    g = L.lbm_group_create([x[2].ctx for x in lats], graph_steps=100)
    L.lbm_group_step(g, k)
    P = 2 * k + 3
    rng = np.random.default_rng(17)
    for m, rates, lat in lats:
        assert lat.status()[0] == L.LBM_OK
        ux = torch.empty((N, N), dtype=torch.float64, device="cuda")
        uy = torch.empty_like(ux)
        lat.moments(None, ux, uy)
        ux, uy = ux.cpu().numpy(), uy.cpu().numpy()
        pts = [(int(rng.integers(0, N)), int(rng.integers(0, N))), (0, N - 1)]
        for (y, x) in pts:
            ys = (np.arange(P) + y - P // 2) % N
            xs = (np.arange(P) + x - P // 2) % N
            patch = [a[np.ix_(ys, xs)] for a in fields]
            fr = olbm.run(olbm.init_equilibrium(*patch), m, rates, k)
            _, rx, ry = macroscopic(fr)
            assert abs(ux[y, x] - rx[P // 2, P // 2]) <= 1e-5, (m, y, x)
            assert abs(uy[y, x] - ry[P // 2, P // 2]) <= 1e-5, (m, y, x)
    L.lbm_group_destroy(g)
    for _, _, lat in lats:
        lat.close()
