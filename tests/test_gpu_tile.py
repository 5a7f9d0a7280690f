"""The two step-kernel families on lattices with several tiles per row and a short last tile:
the copy-engine staged kernel (LBM_PATH_BULK, cp.async.bulk into a ring of 2-4 shared-memory
stages) and the register-staged kernels (LBM_PATH_VECTOR), each against the FP64 oracle and
against each other.  Tile widths of the copy-engine kernel's forms: general 512 (FP64), 1024
(FP32), 2048 (FP16, BF16) nodes; light 512 (FP32), 2048 (16-bit); wide 2048 (FP32), 4096
(16-bit)."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_2002_05265_gb300 import flows  # noqa: E402
import oracle.lbm as olbm  # noqa: E402
from oracle.collision import macroscopic  # noqa: E402
from storage_bounds import WALK_FACTOR, storage_walk_error  # noqa: E402

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


def _run(L, fields, model, rates, storage, steps, path, stages=0, shift=None):
    rho, ux, uy = fields
    ny, nx = rho.shape
    lat = L.Lattice(nx, ny, L.MODELS[model], rates, storage=storage)
    lat.set_kernel_path(path, stages)
    if shift is not None:
        lat.set_shift_velocity(*shift)
    lat.init_equilibrium(*_dev(rho, ux, uy))
    lat.step(steps)
    st = lat.status()
    f = torch.empty((9, ny, nx), dtype=torch.float64, device="cuda")
    lat.get_populations(f)
    lat.close()
    assert st[0] == L.LBM_OK
    return f.cpu().numpy()


def _vel_err(got, ref):
    _, gx, gy = macroscopic(got)
    _, rx, ry = macroscopic(ref)
    return max(np.max(np.abs(gx - rx)), np.max(np.abs(gy - ry)))


def _l2(got, ref):
    _, gx, gy = macroscopic(got)
    _, rx, ry = macroscopic(ref)
    return float(np.sqrt(((gx - rx) ** 2 + (gy - ry) ** 2).sum() / (rx ** 2 + ry ** 2).sum()))


@pytest.mark.parametrize("stages", [2, 3, 4])
@pytest.mark.parametrize("model", MODELS)
def test_bulk_fp64_three_tiles_per_row(L, model, stages):
    """FP64, 1030 x 6 (tiles of 512, 512 and 6 nodes; periodic wrap in x and y at every
    tile edge), Ma = 0.3 vortex with noise, 40 steps: within 1e-12 of the oracle."""
    fields = flows.vortex(1030, 6, Ma=0.3, radius_frac=0.004, noise=1e-6, seed=21)
    rates = olbm.rates_from_nu(1e-3, "reg" if model in ("chm", "k") else "srt")
    got = _run(L, fields, model, rates, L.LBM_F64, 40, L.LBM_PATH_BULK, stages)
    ref = olbm.run(olbm.init_equilibrium(*fields), model, rates, 40)
    assert float(np.max(np.abs(got - ref) / np.abs(ref))) <= 1e-12


@pytest.mark.parametrize("model", MODELS)
def test_bulk_and_vector_fp32_agree_with_oracle(L, model):
    """FP32, 2060 x 5 (tiles of 1024, 1024 and 12 nodes), 200 steps: both kernel families
    within 1e-5 of the oracle's velocity, and within 1e-6 of each other's populations."""
    fields = flows.vortex(2060, 5, Ma=0.2, radius_frac=0.002, noise=1e-6, seed=22)
    rates = olbm.rates_from_nu(1e-4, "reg" if model in ("chm", "k") else "srt")
    bulk = _run(L, fields, model, rates, L.LBM_F32, 200, L.LBM_PATH_BULK)
    vec = _run(L, fields, model, rates, L.LBM_F32, 200, L.LBM_PATH_VECTOR)
    ref = olbm.run(olbm.init_equilibrium(*fields), model, rates, 200)
    assert _vel_err(bulk, ref) <= 1e-5
    assert _vel_err(vec, ref) <= 1e-5
    assert float(np.max(np.abs(bulk - vec))) <= 1e-6


@pytest.mark.parametrize("storage", ["f16", "bf16"])
@pytest.mark.parametrize("model", ["bgk", "cm", "k", "rr"])
def test_bulk_16bit_two_tiles_per_row(L, model, storage):
    """FP16 / BF16, 2072 x 4 (tiles of 2048 and 24 nodes), 300 steps, with and without a
    reference-velocity shift: both kernel families' velocity errors against the oracle, and
    their difference, stay within the storage-rounding bound (WALK_FACTOR times the random-walk
    estimate of the w rho0-shifted storage, which bounds the mean-flow shift too)."""
    st = L.LBM_F16 if storage == "f16" else L.LBM_BF16
    fields = flows.vortex(2072, 4, Ma=0.1, radius_frac=0.002, noise=1e-8, seed=23)
    rates = olbm.rates_from_nu(1e-4, "reg" if model in ("cm", "k") else "srt")
    f0 = olbm.init_equilibrium(*fields)
    bound = WALK_FACTOR * storage_walk_error(f0, storage, 300)
    ref = olbm.run(f0, model, rates, 300)
    for shift in (None, (0.1 / np.sqrt(3.0), 0.0)):
        bulk = _run(L, fields, model, rates, st, 300, L.LBM_PATH_BULK, shift=shift)
        vec = _run(L, fields, model, rates, st, 300, L.LBM_PATH_VECTOR, shift=shift)
        assert _l2(bulk, ref) <= bound
        assert _l2(vec, ref) <= bound
        assert _l2(bulk, vec) <= bound


@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
@pytest.mark.parametrize("model", ["bgk", "rm", "hm", "pr"])
def test_light_form_one_step_launches(L, model, storage):
    """The light kernel form (lattices of BGK, RM, HM or PR stepped one time step per launch:
    one CTA per SM, no row-completion counters) on 2072 x 5 (tiles of 1024 / 2048 nodes and a
    short last one), 200 steps, against the oracle and against the general form's multi-step
    launches: FP32 within 1e-5 of the oracle's velocity and 1e-6 of the general form's
    populations; 16-bit within the storage-rounding bound of both."""
    st = L.STORAGES[storage]
    fields = flows.vortex(2072, 5, Ma=0.1, radius_frac=0.002, noise=1e-8, seed=24)
    rates = olbm.rates_from_nu(1e-4, "srt")
    f0 = olbm.init_equilibrium(*fields)
    ref = olbm.run(f0, model, rates, 200)
    light = _run_shaped(L, fields, model, rates, st, 200, 1, L.LBM_ORDER_STEP)
    general = _run_shaped(L, fields, model, rates, st, 200, 10, L.LBM_ORDER_STEP)
    if storage == "f32":
        assert _vel_err(light, ref) <= 1e-5
        assert float(np.max(np.abs(light - general))) <= 1e-6
    else:
        bound = WALK_FACTOR * storage_walk_error(f0, storage, 200)
        assert _l2(light, ref) <= bound
        assert _l2(light, general) <= bound


def test_bulk_multi_lattice_group(L):
    """Three FP32 lattices of different sizes and models (1 to 3 tiles per row) advanced by
    one bulk-copy launch per step equal the same lattices stepped one by one."""
    shapes = [(2060, 7, "chm"), (1024, 9, "k"), (96, 40, "bgk")]
    rates = olbm.rates_from_nu(1e-4, "reg")
    lats, refs = [], []
    for nx, ny, m in shapes:
        fields = flows.vortex(nx, ny, Ma=0.2, radius_frac=0.01, noise=1e-6, seed=nx + ny)
        for group in (lats, refs):
            lat = L.Lattice(nx, ny, L.MODELS[m], rates, storage=L.LBM_F32)
            lat.set_kernel_path(L.LBM_PATH_BULK)
            lat.init_equilibrium(*_dev(*fields))
            group.append(lat)
    g = L.lbm_group_create([x.ctx for x in lats], graph_steps=8)
    L.lbm_group_step(g, 37)
    for r in refs:
        r.step(37)
    for (nx, ny, _), x, r in zip(shapes, lats, refs):
        fa = torch.empty((9, ny, nx), dtype=torch.float64, device="cuda")
        fb = torch.empty_like(fa)
        x.get_populations(fa)
        r.get_populations(fb)
        assert torch.equal(fa, fb)
        assert x.status()[0] == L.LBM_OK
    L.lbm_group_destroy(g)
    for lat in lats + refs:
        lat.close()


@pytest.mark.parametrize("eq_order", [2, 3])
def test_truncated_equilibria_every_kernel_family(L, eq_order):
    """BGK with the second-order or partial third-order equilibrium on a 1100 x 6 FP64 lattice
    (three tiles per row, the last short): the copy-engine and register-staged kernels within
    1e-12 of the oracle after 40 steps; in a group with a CHM lattice (the group kernel), the
    populations equal those of the lattice stepped alone."""
    fields = flows.vortex(1100, 6, Ma=0.2, radius_frac=0.01, noise=1e-6, seed=17 + eq_order)
    rates = olbm.rates_from_nu(1e-3, "srt")
    ref = olbm.run(olbm.init_equilibrium(*fields, eq_order=eq_order), "bgk", rates, 40, eq_order=eq_order)
    for path in (L.LBM_PATH_BULK, L.LBM_PATH_VECTOR):
        lat = L.Lattice(1100, 6, L.LBM_BGK, rates, storage=L.LBM_F64, eq_order=eq_order)
        lat.set_kernel_path(path)
        lat.init_equilibrium(*_dev(*fields))
        lat.step(40)
        f = torch.empty((9, 6, 1100), dtype=torch.float64, device="cuda")
        lat.get_populations(f)
        lat.close()
        got = f.cpu().numpy()
        assert np.max(np.abs(got - ref) / np.abs(ref)) <= 1e-12
    other = flows.vortex(64, 33, Ma=0.2, noise=1e-6, seed=5)
    lats = [L.Lattice(96, 40, L.LBM_BGK, rates, storage=L.LBM_F32, eq_order=eq_order),
            L.Lattice(64, 33, L.LBM_CHM, rates, storage=L.LBM_F32)]
    alone = L.Lattice(96, 40, L.LBM_BGK, rates, storage=L.LBM_F32, eq_order=eq_order)
    f96 = flows.vortex(96, 40, Ma=0.2, noise=1e-6, seed=6)
    for lat in (lats[0], alone):
        lat.set_kernel_path(L.LBM_PATH_VECTOR)
        lat.init_equilibrium(*_dev(*f96))
    lats[1].set_kernel_path(L.LBM_PATH_VECTOR)
    lats[1].init_equilibrium(*_dev(*other))
    g = L.lbm_group_create([x.ctx for x in lats], graph_steps=8)
    L.lbm_group_step(g, 24)
    alone.step(24)
    fa = torch.empty((9, 40, 96), dtype=torch.float64, device="cuda")
    fb = torch.empty_like(fa)
    lats[0].get_populations(fa)
    alone.get_populations(fb)
    assert torch.equal(fa, fb)
    L.lbm_group_destroy(g)
    for lat in lats + [alone]:
        lat.close()


def test_kernel_path_argument_checks(L):
    lat = L.Lattice(99, 10, L.LBM_BGK, (1.5, 1.5, 1.5), storage=L.LBM_F32)
    with pytest.raises(L.LBMError) as e:
        lat.set_kernel_path(L.LBM_PATH_BULK)          # 99 * 4 bytes is not a multiple of 16
    assert e.value.code == L.LBM_ERR_UNSUPPORTED
    for path, stages in ((3, 0), (-1, 0), (L.LBM_PATH_AUTO, 1), (L.LBM_PATH_AUTO, 5)):
        with pytest.raises(L.LBMError) as e:
            lat.set_kernel_path(path, stages)
        assert e.value.code == L.LBM_ERR_INVALID_ARG
    lat.set_kernel_path(L.LBM_PATH_AUTO)              # falls back to the register-staged kernels
    lat.close()


@pytest.mark.parametrize("model", MODELS)
@pytest.mark.parametrize("shape", [(70, 9), (64, 37), (96, 17)])
def test_bulk_fp64_row_block_tiles(L, model, shape):
    """FP64 lattices narrower than half a tile move as blocks of whole rows: 70 x 9 (pitch 96
    != nx: one copy per row; blocks of 7 and 2 rows), 64 x 37 (pitch == nx: consecutive rows
    in one copy, split at the periodic wrap; 8 rows per block, last block 5), 96 x 17.  Within
    1e-12 of the oracle after 30 steps."""
    nx, ny = shape
    fields = flows.vortex(nx, ny, Ma=0.3, radius_frac=0.1, noise=1e-6, seed=nx * ny)
    rates = olbm.rates_from_nu(1e-3, "reg" if model in ("chm", "k") else "srt")
    got = _run(L, fields, model, rates, L.LBM_F64, 30, L.LBM_PATH_BULK, 3)
    ref = olbm.run(olbm.init_equilibrium(*fields), model, rates, 30)
    assert float(np.max(np.abs(got - ref) / np.abs(ref))) <= 1e-12


@pytest.mark.parametrize("storage,shape", [("f32", (100, 23)), ("f32", (64, 37)), ("f16", (136, 17)),
                                           ("bf16", (64, 70))])
def test_bulk_row_block_tiles_reduced_precision(L, storage, shape):
    """Row-block tiles in FP32 (blocks of 10 rows with pitch 128 != nx = 100; blocks of 16
    dense rows) and 16-bit storage: the bulk-copy kernel agrees with the register-staged
    kernel (FP32: 1e-6 on populations) and with the oracle (FP32 1e-5 on u; FP16 / BF16 the
    storage-rounding bound of storage_bounds) after 200 steps, for the CHM model."""
    nx, ny = shape
    st = {"f32": L.LBM_F32, "f16": L.LBM_F16, "bf16": L.LBM_BF16}[storage]
    fields = flows.vortex(nx, ny, Ma=0.1, radius_frac=0.1, noise=1e-8, seed=nx + 7 * ny)
    rates = olbm.rates_from_nu(1e-4, "reg")
    bulk = _run(L, fields, "chm", rates, st, 200, L.LBM_PATH_BULK)
    vec = _run(L, fields, "chm", rates, st, 200, L.LBM_PATH_VECTOR)
    ref = olbm.run(olbm.init_equilibrium(*fields), "chm", rates, 200)
    if storage == "f32":
        assert _vel_err(bulk, ref) <= 1e-5
        assert float(np.max(np.abs(bulk - vec))) <= 1e-6
    else:
        bound = WALK_FACTOR * storage_walk_error(olbm.init_equilibrium(*fields), storage, 200)
        assert _l2(bulk, ref) <= bound
        assert _l2(bulk, vec) <= bound


def test_bulk_single_step_launches_large_lattice(L):
    """A lattice with many tiles per CTA (16384 x 2048 FP32: 32768 tiles per step) runs one
    time step per bulk-copy launch; smaller ones run many steps per launch with the
    row-completion counters (every other test here).  After 12 steps of the CHM model on the
    double shear layer: populations within 1e-6 of the register-staged kernels everywhere,
    and 16 sampled nodes within 1e-5 of the oracle run on the light cone of each node."""
    nx, ny, k = 16384, 2048, 12
    fields = flows.double_shear_layer(nx, ny, Ma=0.1, width_frac=1.0 / 80.0)
    rates = olbm.rates_from_nu(1e-5, "reg")
    outs = []
    for path in (L.LBM_PATH_BULK, L.LBM_PATH_VECTOR):
        lat = L.Lattice(nx, ny, L.LBM_CHM, rates, storage=L.LBM_F32)
        lat.set_kernel_path(path)
        lat.init_equilibrium(*_dev(*fields))
        lat.step(k)
        assert lat.status()[0] == L.LBM_OK
        ux = torch.empty((ny, nx), dtype=torch.float64, device="cuda")
        uy = torch.empty_like(ux)
        lat.moments(None, ux, uy)
        outs.append((ux.cpu().numpy(), uy.cpu().numpy()))
        lat.close()
    (bx, by), (vx, vy) = outs
    assert max(np.max(np.abs(bx - vx)), np.max(np.abs(by - vy))) <= 1e-6
    g = np.random.default_rng(11)
    pts = list(zip(g.integers(0, ny, 14), g.integers(0, nx, 14))) + [(0, 0), (ny - 1, nx - 1)]
    P = 2 * k + 3
    for (y, x) in pts:
        ys = (np.arange(P) + y - P // 2) % ny
        xs = (np.arange(P) + x - P // 2) % nx
        patch = [a[np.ix_(ys, xs)] for a in fields]
        fr = olbm.run(olbm.init_equilibrium(*patch), "chm", rates, k)
        _, rx, ry = macroscopic(fr)
        assert abs(bx[y, x] - rx[P // 2, P // 2]) <= 1e-5
        assert abs(by[y, x] - ry[P // 2, P // 2]) <= 1e-5


def _run_shaped(L, fields, model, rates, storage, steps, launch_steps, order):
    rho, ux, uy = fields
    ny, nx = rho.shape
    lat = L.Lattice(nx, ny, L.MODELS[model], rates, storage=storage)
    lat.set_kernel_path(L.LBM_PATH_BULK)
    lat.set_launch_shape(launch_steps, order)
    lat.init_equilibrium(*_dev(rho, ux, uy))
    lat.step(steps)
    assert lat.status()[0] == L.LBM_OK
    f = torch.empty((9, ny, nx), dtype=torch.float64, device="cuda")
    lat.get_populations(f)
    lat.close()
    return f.cpu().numpy()


@pytest.mark.parametrize("model", ["bgk", "chm", "k", "rr"])
@pytest.mark.parametrize("shape,launch_steps", [((1030, 6), 8), ((1030, 6), 3), ((64, 37), 7), ((70, 9), 16)])
def test_wavefront_order_fp64(L, model, shape, launch_steps):
    """Several time steps per launch in the wavefront order (steps interleaved a few rows
    apart, units visited in a rotated order per step, across the periodic wrap): segment tiles
    (1030 x 6) and row-block tiles (64 x 37, 70 x 9), 40 steps: within 1e-12 of the oracle."""
    nx, ny = shape
    fields = flows.vortex(nx, ny, Ma=0.3, radius_frac=0.05, noise=1e-6, seed=nx + ny + launch_steps)
    rates = olbm.rates_from_nu(1e-3, "reg" if model in ("chm", "k") else "srt")
    got = _run_shaped(L, fields, model, rates, L.LBM_F64, 40, launch_steps, L.LBM_ORDER_WAVE)
    ref = olbm.run(olbm.init_equilibrium(*fields), model, rates, 40)
    assert float(np.max(np.abs(got - ref) / np.abs(ref))) <= 1e-12


def test_launch_shapes_agree_bitwise(L):
    """The launch shape only reorders the same per-tile arithmetic: in the general kernel form,
    one step per launch, step order with 10 steps per launch, the wavefront with 16 steps per
    launch and the block order give identical FP32 populations (eight 256 x 160 lattices of all
    models in one group, 50 steps)."""
    rates = olbm.rates_from_nu(1e-4, "reg")
    fields = flows.double_shear_layer(256, 160, Ma=0.1, width_frac=0.05)
    results = []
    for steps, order in ((1, L.LBM_ORDER_STEP), (10, L.LBM_ORDER_STEP), (16, L.LBM_ORDER_WAVE),
                         (12, L.LBM_ORDER_BLOCK)):
        lats = []
        for m in MODELS:
            lat = L.Lattice(256, 160, L.MODELS[m], rates, storage=L.LBM_F32)
            lat.set_kernel_path(L.LBM_PATH_BULK)
            lat.set_launch_shape(steps, order)
            lat.set_tile_form(L.LBM_FORM_GENERAL)
            lat.init_equilibrium(*_dev(*fields))
            lats.append(lat)
        g = L.lbm_group_create([x.ctx for x in lats], graph_steps=8)
        L.lbm_group_step(g, 50)
        out = []
        for lat in lats:
            f = torch.empty((9, 160, 256), dtype=torch.float64, device="cuda")
            lat.get_populations(f)
            assert lat.status()[0] == L.LBM_OK
            out.append(f)
        results.append(torch.stack(out))
        L.lbm_group_destroy(g)
        for lat in lats:
            lat.close()
    for r in results[1:]:
        assert torch.equal(results[0], r)


def test_launch_shape_argument_checks(L):
    lat = L.Lattice(64, 64, L.LBM_BGK, (1.5, 1.5, 1.5), storage=L.LBM_F32)
    for steps, order in ((-1, 0), (0, 4), (0, -1)):
        with pytest.raises(L.LBMError) as e:
            lat.set_launch_shape(steps, order)
        assert e.value.code == L.LBM_ERR_INVALID_ARG
    lat.close()


@pytest.mark.parametrize("storage,tol", [("f16", 3e-4), ("bf16", 2e-3)])
def test_full_size_16384_reduced_precision_sampled(L, storage, tol):
    """The 16384² throughput workload in 16-bit storage (Ma = 0.2 vortex with 1e-8 seed noise,
    nu = 1e-6, REG-CHM, shift at the mean flow, the default kernel: one copy-engine launch per
    step): after 8 steps, 16 sampled nodes (half of them in the vortex core) match the oracle run
    on each node's light cone.  Bounds from the storage rounding: a population of size
    |g| ~ 0.03 rounds by 2^-12 (FP16) / 2^-9 (BF16) relative per step, about 2e-5 / 1e-4 of
    velocity per step, random-walking over 8 steps; the bounds leave a factor 5 or more."""
    n, k = 16384, 8
    fields = flows.vortex(n, Ma=0.2, noise=1e-8, seed=3)
    rates = olbm.rates_from_nu(1e-6, "reg")
    u0 = 0.2 / np.sqrt(3.0)
    lat = L.Lattice(n, n, L.LBM_CHM, rates, storage=L.STORAGES[storage])
    lat.set_shift_velocity(u0, 0.0)
    lat.init_equilibrium(*_dev(*fields))
    lat.step(k)
    assert lat.status()[0] == L.LBM_OK
    ux = torch.empty((n, n), dtype=torch.float64, device="cuda")
    uy = torch.empty_like(ux)
    lat.moments(None, ux, uy)
    lat.close()
    g = np.random.default_rng(23)
    R = int(0.1 * n)
    pts = list(zip(g.integers(0, n, 8), g.integers(0, n, 8)))
    pts += list(zip(g.integers(n // 2 - 2 * R, n // 2 + 2 * R, 8), g.integers(n // 2 - 2 * R, n // 2 + 2 * R, 8)))
    P = 2 * k + 3
    for (y, x) in pts:
        ys = (np.arange(P) + y - P // 2) % n
        xs = (np.arange(P) + x - P // 2) % n
        patch = [a[np.ix_(ys, xs)] for a in fields]
        fr = olbm.run(olbm.init_equilibrium(*patch), "chm", rates, k)
        _, rx, ry = macroscopic(fr)
        assert abs(float(ux[y, x]) - rx[P // 2, P // 2]) <= tol, (y, x)
        assert abs(float(uy[y, x]) - ry[P // 2, P // 2]) <= tol, (y, x)
    del ux, uy
    torch.cuda.empty_cache()


_GENERAL_CACHE = {}
_ORACLE_CACHE = {}


def _run_group(L, fields, models, rates, storage, steps, form, launch_steps):
    rho, ux, uy = fields
    ny, nx = rho.shape
    lats = []
    for m in models:
        lat = L.Lattice(nx, ny, L.MODELS[m], rates, storage=storage)
        lat.set_kernel_path(L.LBM_PATH_BULK)
        lat.set_launch_shape(launch_steps, L.LBM_ORDER_STEP)
        lat.set_tile_form(form)
        lat.init_equilibrium(*_dev(rho, ux, uy))
        lats.append(lat)
    g = L.lbm_group_create([x.ctx for x in lats], graph_steps=0)
    L.lbm_group_step(g, steps)
    out = {}
    for m, lat in zip(models, lats):
        assert lat.status()[0] == L.LBM_OK
        f = torch.empty((9, ny, nx), dtype=torch.float64, device="cuda")
        lat.get_populations(f)
        out[m] = f.cpu().numpy()
    L.lbm_group_destroy(g)
    for lat in lats:
        lat.close()
    return out


@pytest.mark.parametrize("launch_steps", [1, 6])
@pytest.mark.parametrize("shape", [(4120, 3), (136, 21)])
@pytest.mark.parametrize("form", ["light", "wide"])
@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
def test_kernel_forms_against_oracle_and_general_form(L, storage, form, shape, launch_steps):
    """The light form (BGK, RM, HM, PR; FP32: 4 consumer warps at 3 CTAs per SM, 16-bit: the
    packed 8-node pass) and the wide form (every model, 16 consumer warps at 1 CTA per SM) on a
    group of lattices: 4120 x 3 (segment tiles of every form's width with a short last tile of
    24 nodes) and 136 x 21 (row blocks of 3 to 30 rows, the last one short), one step per launch
    and 6 steps per launch (row-completion counters), 60 steps.  FP32: within 1e-5 of the
    oracle's velocity and within 1e-6 of the general form's populations; 16-bit: within the
    storage-rounding bound of both."""
    nx, ny = shape
    st = L.STORAGES[storage]
    models = ["bgk", "rm", "hm", "pr"] if form == "light" else MODELS
    fields = flows.vortex(nx, ny, Ma=0.1, radius_frac=0.02 if nx > 1000 else 0.1, noise=1e-8, seed=nx + ny)
    rates = olbm.rates_from_nu(1e-4, "srt")
    f0 = olbm.init_equilibrium(*fields)
    fm = L.LBM_FORM_LIGHT if form == "light" else L.LBM_FORM_WIDE
    got = _run_group(L, fields, models, rates, st, 60, fm, launch_steps)
    key = (storage, shape)
    if key not in _GENERAL_CACHE:
        _GENERAL_CACHE[key] = _run_group(L, fields, MODELS, rates, st, 60, L.LBM_FORM_GENERAL, 6)
    gen = _GENERAL_CACHE[key]
    bound = None if storage == "f32" else WALK_FACTOR * storage_walk_error(f0, storage, 60)
    for m in models:
        if (shape, m) not in _ORACLE_CACHE:
            _ORACLE_CACHE[(shape, m)] = olbm.run(f0, m, rates, 60)
        ref = _ORACLE_CACHE[(shape, m)]
        if storage == "f32":
            assert _vel_err(got[m], ref) <= 1e-5, m
            assert float(np.max(np.abs(got[m] - gen[m]))) <= 1e-6, m
        else:
            assert _l2(got[m], ref) <= bound, m
            assert _l2(got[m], gen[m]) <= bound, m


def test_tile_form_argument_checks(L):
    lat = L.Lattice(64, 64, L.LBM_CHM, (1.5, 1.5, 1.5), storage=L.LBM_F32)
    for form in (-1, 4):
        with pytest.raises(L.LBMError) as e:
            lat.set_tile_form(form)
        assert e.value.code == L.LBM_ERR_INVALID_ARG
    with pytest.raises(L.LBMError) as e:
        lat.set_tile_form(L.LBM_FORM_LIGHT)           # CHM is not a light model
    assert e.value.code == L.LBM_ERR_UNSUPPORTED
    lat.set_tile_form(L.LBM_FORM_WIDE)
    lat.close()
    lat = L.Lattice(64, 64, L.LBM_BGK, (1.5, 1.5, 1.5), storage=L.LBM_F64)
    for form in (L.LBM_FORM_LIGHT, L.LBM_FORM_WIDE):  # FP64 has the general form only
        with pytest.raises(L.LBMError) as e:
            lat.set_tile_form(form)
        assert e.value.code == L.LBM_ERR_UNSUPPORTED
    lat.set_tile_form(L.LBM_FORM_GENERAL)
    lat.close()


def test_default_kernel_form_choice(L):
    """The library's default form and launch shape for the configurations it was measured on
    (lbm_group_describe): the benchmark's eight 1024^2 FP32 lattices of all models run the
    wide form one step per launch; four of them (fewer than 24 wide tiles per CTA) the general
    form many steps per launch; a 4096^2 BGK lattice the light form; a 4096^2 CHM lattice the
    general form's 16-step wavefront launches; BF16 BGK lattices the wide form; FP64 the
    general form; a 64^2 lattice (fewer tiles than CTAs) the register-staged kernels."""
    rates = (1.5, 1.5, 1.5)

    def describe(specs, storage=None):
        st = L.LBM_F32 if storage is None else storage
        lats = [L.Lattice(n, n, L.MODELS[m], rates, storage=st) for n, m in specs]
        g = L.lbm_group_create([x.ctx for x in lats], graph_steps=0)
        d = L.lbm_group_describe(g)
        L.lbm_group_destroy(g)
        for lat in lats:
            lat.close()
        return d

    d = describe([(1024, m) for m in MODELS])
    assert (d["family"], d["form"], d["steps_per_launch"], d["tiles"], d["block"]) == \
        (L.LBM_PATH_BULK, L.LBM_FORM_WIDE, 1, 8 * 512, 576)
    d = describe([(1024, m) for m in MODELS[:4]])
    assert (d["family"], d["form"], d["block"]) == (L.LBM_PATH_BULK, L.LBM_FORM_GENERAL, 320)
    assert d["steps_per_launch"] > 1
    d = describe([(4096, "bgk")])
    assert (d["form"], d["steps_per_launch"], d["tiles"], d["block"]) == (L.LBM_FORM_LIGHT, 1, 4096 * 8, 192)
    d = describe([(4096, "chm")])
    assert (d["form"], d["steps_per_launch"]) == (L.LBM_FORM_GENERAL, 16)
    d = describe([(4096, "bgk"), (4096, "pr")], storage=L.LBM_BF16)
    assert (d["form"], d["steps_per_launch"]) == (L.LBM_FORM_WIDE, 1)
    d = describe([(4096, "bgk")], storage=L.LBM_F64)
    assert d["form"] == L.LBM_FORM_GENERAL
    d = describe([(4096, "bgk"), (4096, "hm")], storage=L.LBM_F16)
    assert (d["form"], d["steps_per_launch"], d["block"]) == (L.LBM_FORM_LIGHT, 1, 320)
    d = describe([(64, "bgk")])
    assert (d["family"], d["form"], d["tiles"]) == (L.LBM_PATH_VECTOR, L.LBM_FORM_AUTO, 0)


def test_forced_kernel_forms_are_honoured(L):
    """lbm_set_tile_form on the first context decides the group's form where its lattices
    allow it (and LBM_FORM_LIGHT on a group with a central-moment lattice falls back to the
    default choice)."""
    rates = (1.5, 1.5, 1.5)
    cases = [(L.LBM_FORM_GENERAL, ["bgk", "cm"], L.LBM_FORM_GENERAL, 320),
             (L.LBM_FORM_WIDE, ["bgk", "rm"], L.LBM_FORM_WIDE, 576),
             (L.LBM_FORM_LIGHT, ["bgk", "pr"], L.LBM_FORM_LIGHT, 192)]
    for form, models, want, block in cases:
        lats = [L.Lattice(2048, 2048, L.MODELS[m], rates, storage=L.LBM_F32) for m in models]
        lats[0].set_tile_form(form)
        g = L.lbm_group_create([x.ctx for x in lats], graph_steps=0)
        d = L.lbm_group_describe(g)
        L.lbm_group_destroy(g)
        assert (d["family"], d["form"], d["block"]) == (L.LBM_PATH_BULK, want, block), (form, d)
        lats.append(L.Lattice(2048, 2048, L.LBM_CHM, rates, storage=L.LBM_F32))
        g = L.lbm_group_create([x.ctx for x in lats], graph_steps=0)
        d = L.lbm_group_describe(g)
        L.lbm_group_destroy(g)
        if form == L.LBM_FORM_LIGHT:
            assert d["form"] != L.LBM_FORM_LIGHT
        else:
            assert d["form"] == want
        for lat in lats:
            lat.close()
