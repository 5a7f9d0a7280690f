"""GPU checks of the y-slab decomposition's halo calls (lbm_halo_pack / lbm_halo_unpack)
through the C ABI: one lattice split into 1 (periodic self-exchange), 2 and 3 slabs, all slabs
in one process on one GPU (paper_2002_05265_gb300.slab.step_slabs: host-ordered on one stream,
no kernel waits on another), against the same lattice stepped whole and against the oracle."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_2002_05265_gb300 import flows  # noqa: E402
import oracle.lbm as olbm  # noqa: E402
from oracle.collision import macroscopic  # noqa: E402


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2002_05265_gb300 import build, lbm
    build.build_library()
    lbm.load_library()
    return lbm


def _whole(L, fields, model, rates, storage, n, path):
    rho, ux, uy = fields
    ny, nx = rho.shape
    lat = L.Lattice(nx, ny, L.MODELS[model], rates, storage=storage)
    lat.set_kernel_path(path)
    lat.init_equilibrium(*[torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in fields])
    lat.step(n)
    out = [torch.empty((ny, nx), dtype=torch.float64, device="cuda") for _ in range(3)]
    lat.moments(*out)
    lat.close()
    return [o.cpu().numpy() for o in out]


def _slabs(L, fields, model, rates, storage, n, world, path):
    from paper_2002_05265_gb300 import slab
    rho, ux, uy = fields
    ny, nx = rho.shape
    slabs = [slab.SlabLattice(nx, ny, L.MODELS[model], rates, storage, r, world) for r in range(world)]
    dev = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in fields]
    for s in slabs:
        s.lat.set_kernel_path(path)
        s.init_equilibrium(*dev)
    if world == 1:
        slabs[0].step(n)            # advance() with the periodic self-exchange
    else:
        slab.step_slabs(slabs, n)
    out = [np.empty((ny, nx)) for _ in range(3)]
    for s in slabs:
        loc = [torch.empty((s.y1 - s.y0, nx), dtype=torch.float64, device="cuda") for _ in range(3)]
        s.moments(*loc)
        for o, t in zip(out, loc):
            o[s.y0:s.y1] = t.cpu().numpy()
        s.close()
    return out


@pytest.mark.parametrize("world", [1, 2, 3])
@pytest.mark.parametrize("storage,model", [("f64", "k"), ("f32", "chm"), ("f16", "k"), ("bf16", "rr")])
def test_slabs_equal_the_whole_lattice(L, world, storage, model):
    """64 x 47 vortex (uneven slabs for 2 and 3 ranks), 40 steps, register-staged kernel for
    both (the same compiled step kernel): rho and u of the slabs' rows bit for bit equal to
    the whole lattice's, for every storage width the halo messages carry."""
    fields = flows.vortex(64, 47, Ma=0.2, noise=1e-6, seed=world)
    rates = olbm.rates_from_nu(1e-3, "reg")
    st = L.STORAGES[storage]
    ref = _whole(L, fields, model, rates, st, 40, L.LBM_PATH_VECTOR)
    got = _slabs(L, fields, model, rates, st, 40, world, L.LBM_PATH_VECTOR)
    for g, r in zip(got, ref):
        np.testing.assert_array_equal(g, r)


@pytest.mark.parametrize("world", [1, 2])
def test_slabs_default_kernel_match_the_oracle(L, world):
    """The library's default kernel choice (copy-engine staged where the rows allow it), FP64,
    128 x 40 lattice in 1 / 2 slabs, 60 steps, CHM: populations' moments within 1e-12 of the
    FP64 oracle's whole-lattice run."""
    fields = flows.vortex(128, 40, Ma=0.25, noise=1e-6, seed=7)
    rates = olbm.rates_from_nu(1e-3, "reg")
    got = _slabs(L, fields, "chm", rates, L.LBM_F64, 60, world, L.LBM_PATH_AUTO)
    ref = olbm.run(olbm.init_equilibrium(*fields), "chm", rates, 60)
    rr, rx, ry = macroscopic(ref)
    np.testing.assert_allclose(got[0], rr, rtol=1e-12)
    np.testing.assert_allclose(got[1], rx, rtol=0, atol=1e-12)
    np.testing.assert_allclose(got[2], ry, rtol=0, atol=1e-12)


def test_halo_calls_reject_host_pointers(L):
    lat = L.Lattice(16, 8, L.LBM_BGK, (1.5, 1.5, 1.5), storage=L.LBM_F32)
    dev = torch.zeros(48, dtype=torch.float32, device="cuda")
    host = torch.zeros(48, dtype=torch.float32)
    with pytest.raises(L.LBMError) as e:
        L.lbm_halo_pack(lat.ctx, host, dev)
    assert e.value.code == L.LBM_ERR_INVALID_ARG
    with pytest.raises(L.LBMError) as e:
        L.lbm_halo_unpack(lat.ctx, dev, host)
    assert e.value.code == L.LBM_ERR_INVALID_ARG
    L.lbm_halo_pack(lat.ctx, dev, dev.clone())
    lat.synchronize()
    lat.close()
