"""GPU tests of the hand-written discrete adjoint (lbm_adjoint_run, LBMRun) against the
oracle's complex-step reference gradients and FP64 central finite differences."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_2002_05265_gb300 import flows  # noqa: E402
from oracle import adjoint as oadj  # noqa: E402

MODELS = ["bgk", "rm", "hm", "cm", "chm", "k", "pr", "rr"]


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2002_05265_gb300 import build, lbm
    build.build_library()
    lbm.load_library()
    return lbm


def _case(nx=22, ny=18, seed=3):
    rho, ux, uy = flows.vortex(nx, ny, Ma=0.25, noise=1e-3, seed=seed)
    tx = np.roll(ux, 2, axis=1) + flows.gaussian_noise(ux.shape, 1e-3, seed + 1)
    ty = np.roll(uy, 2, axis=1) + flows.gaussian_noise(uy.shape, 1e-3, seed + 2)
    return rho, ux, uy, tx, ty


def _gpu(L, rho, ux, uy, model, rates, storage, nsteps, loss, tx, ty, ckpt=0, shift=None):
    ny, nx = ux.shape
    lat = L.Lattice(nx, ny, L.MODELS[model], rates, storage=storage)
    if shift is not None:
        lat.set_shift_velocity(*shift)
    lat.init_equilibrium(*[np.ascontiguousarray(a) for a in (rho, ux, uy)])
    gx, gy = np.zeros_like(ux), np.zeros_like(uy)
    val, gr, times = L.lbm_adjoint_run(lat.ctx, nsteps, 0 if loss == "misfit" else 1,
                                       np.ascontiguousarray(tx), np.ascontiguousarray(ty), gx, gy, ckpt)
    lat.close()
    return val, gx, gy, gr


@pytest.mark.parametrize("model", MODELS)
def test_fp64_adjoint_matches_complex_step_oracle(L, model):
    """Misfit loss after 30 steps on a 22 x 18 vortex: the FP64 adjoint's rate gradients and
    its u0 gradient along two random directions match the oracle's complex-step derivatives
    to 1e-9 relative."""
    rho, ux, uy, tx, ty = _case()
    rates = (1.8, 1.3, 0.7)
    n = 30
    val, gx, gy, gr = _gpu(L, rho, ux, uy, model, rates, L.LBM_F64, n, "misfit", tx, ty, ckpt=7)
    assert val == pytest.approx(oadj.run_loss(rho, ux, uy, model, rates, n, "misfit", tx, ty), rel=1e-12)
    scale = np.abs(gx).max() + np.abs(gy).max()
    g = np.random.default_rng(11)
    for _ in range(2):
        dx, dy = g.standard_normal(ux.shape), g.standard_normal(uy.shape)
        ref = oadj.directional_derivative(rho, ux, uy, model, rates, n, "misfit", tx, ty, dux=dx, duy=dy)
        got = float((gx * dx).sum() + (gy * dy).sum())
        assert got == pytest.approx(ref, rel=1e-9, abs=1e-12 * scale * ux.size)
    for k in range(3):
        d = [0.0, 0.0, 0.0]
        d[k] = 1.0
        ref = oadj.directional_derivative(rho, ux, uy, model, rates, n, "misfit", tx, ty, drates=d)
        assert gr[k] == pytest.approx(ref, rel=1e-9, abs=1e-14), k


@pytest.mark.parametrize("model", ["bgk", "cm", "k", "rr"])
def test_fp64_adjoint_with_shift_velocity(L, model):
    """The adjoint of a run stored with a shift at a reference velocity is the same gradient
    (the shift changes only the encoding): complex-step oracle to 1e-9."""
    rho, ux, uy, tx, ty = _case(seed=4)
    rates = (1.8, 1.3, 0.7)
    val, gx, gy, gr = _gpu(L, rho, ux, uy, model, rates, L.LBM_F64, 30, "misfit", tx, ty, shift=(0.14, 0.02))
    g = np.random.default_rng(8)
    dx, dy = g.standard_normal(ux.shape), g.standard_normal(uy.shape)
    ref = oadj.directional_derivative(rho, ux, uy, model, rates, 30, "misfit", tx, ty, dux=dx, duy=dy)
    assert float((gx * dx).sum() + (gy * dy).sum()) == pytest.approx(ref, rel=1e-9)
    ref = oadj.directional_derivative(rho, ux, uy, model, rates, 30, "misfit", tx, ty, drates=(1.0, 0.0, 0.0))
    assert gr[0] == pytest.approx(ref, rel=1e-9)


def test_fp64_adjoint_kinetic_energy_loss(L):
    rho, ux, uy, tx, ty = _case(seed=5)
    rates = (1.6, 1.0, 1.0)
    val, gx, gy, gr = _gpu(L, rho, ux, uy, "chm", rates, L.LBM_F64, 25, "ke", tx, ty)
    assert val == pytest.approx(oadj.run_loss(rho, ux, uy, "chm", rates, 25, "ke"), rel=1e-12)
    g = np.random.default_rng(2)
    dx, dy = g.standard_normal(ux.shape), g.standard_normal(uy.shape)
    ref = oadj.directional_derivative(rho, ux, uy, "chm", rates, 25, "ke", dux=dx, duy=dy)
    assert float((gx * dx).sum() + (gy * dy).sum()) == pytest.approx(ref, rel=1e-9)
    ref = oadj.directional_derivative(rho, ux, uy, "chm", rates, 25, "ke", drates=(1.0, 0.0, 0.0))
    assert gr[0] == pytest.approx(ref, rel=1e-9)


@pytest.mark.parametrize("model", ["chm", "k", "rr"])
def test_fp32_adjoint_within_1e3(L, model):
    rho, ux, uy, tx, ty = _case(nx=40, ny=36, seed=7)
    rates = (1.9, 1.0, 1.0)
    n = 60
    val, gx, gy, gr = _gpu(L, rho, ux, uy, model, rates, L.LBM_F32, n, "misfit", tx, ty)
    g = np.random.default_rng(4)
    dx, dy = g.standard_normal(ux.shape), g.standard_normal(uy.shape)
    ref = oadj.directional_derivative(rho, ux, uy, model, rates, n, "misfit", tx, ty, dux=dx, duy=dy)
    assert float((gx * dx).sum() + (gy * dy).sum()) == pytest.approx(ref, rel=1e-3)
    ref = oadj.directional_derivative(rho, ux, uy, model, rates, n, "misfit", tx, ty, drates=(1.0, 0.0, 0.0))
    assert gr[0] == pytest.approx(ref, rel=1e-3)


def test_checkpoint_interval_does_not_change_the_gradient(L):
    rho, ux, uy, tx, ty = _case(seed=9)
    res = [_gpu(L, rho, ux, uy, "k", (1.7, 1.2, 1.1), L.LBM_F64, 40, "misfit", tx, ty, ckpt=c) for c in (1, 6, 40, 0)]
    for r in res[1:]:
        assert r[0] == res[0][0]
        np.testing.assert_array_equal(r[1], res[0][1])
        np.testing.assert_array_equal(r[3], res[0][3])


def test_autograd_function(L):
    from paper_2002_05265_gb300.adjoint import LBMRun
    rho, ux, uy, tx, ty = _case(seed=12)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    u0x = dev(ux).requires_grad_(True)
    u0y = dev(uy).requires_grad_(True)
    rates = torch.tensor([1.8, 1.0, 1.0], dtype=torch.float64, device="cuda", requires_grad=True)
    loss = LBMRun.apply(u0x, u0y, rates, dev(rho), 20, "rr", L.LBM_F64, 0, dev(tx), dev(ty), 0)
    (3.0 * loss).backward()
    _, gx, gy, gr = _gpu(L, rho, ux, uy, "rr", (1.8, 1.0, 1.0), L.LBM_F64, 20, "misfit", tx, ty)
    np.testing.assert_allclose(u0x.grad.cpu().numpy(), 3.0 * gx, rtol=1e-12, atol=1e-18)
    np.testing.assert_allclose(rates.grad.cpu().numpy(), 3.0 * gr, rtol=1e-12)


@pytest.mark.parametrize("model", ["chm", "k"])
def test_full_size_adjoint_vs_fp64_central_differences(L, model):
    """512 x 512 vortex, 4000 steps, REG rates, misfit to the translated vortex plus Gaussian
    noise (sigma = 1e-3 u0): FP32 and FP64 adjoint gradients against FP64 central finite
    differences of GPU FP64 forward runs (h = 1e-6): the rate omega_nu, two smooth random
    u0 directions (Fourier modes up to k = 8) and, for FP64, one white-noise u0 direction."""
    N, n = 512, 4000
    Ma = 0.1
    u0 = Ma / np.sqrt(3.0)
    rho, ux, uy = flows.vortex(N, Ma=Ma, noise=0.0)
    _, tx, ty = flows.vortex(N, Ma=Ma, center=((N / 2 + u0 * n) % N, N / 2))
    tx = tx + flows.gaussian_noise(tx.shape, 1e-3 * u0, 21)
    ty = ty + flows.gaussian_noise(ty.shape, 1e-3 * u0, 22)
    w = 1.0 / (3e-4 + 0.5)          # nu = 1e-4
    rates = (w, 1.0, 1.0)

    def loss64(r, dx=None, dy=None, h=0.0):
        lat = L.Lattice(N, N, L.MODELS[model], r, storage=L.LBM_F64)
        x = ux if dx is None else ux + h * dx
        y = uy if dy is None else uy + h * dy
        lat.init_equilibrium(*[torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (rho, x, y)])
        lat.step(n)
        mx = torch.empty((N, N), dtype=torch.float64, device="cuda")
        my = torch.empty_like(mx)
        lat.moments(None, mx, my)
        lat.close()
        mx, my = mx.cpu().numpy(), my.cpu().numpy()
        return 0.5 * (((mx - tx) ** 2) + ((my - ty) ** 2)).sum()

    h = 1e-6
    fd_w = (loss64((w + h, 1.0, 1.0)) - loss64((w - h, 1.0, 1.0))) / (2 * h)
    dirs = [(flows.smooth_random_field(N, N, 8, 31 + 2 * k), flows.smooth_random_field(N, N, 8, 32 + 2 * k))
            for k in range(2)]
    g = np.random.default_rng(31)
    noise = (g.standard_normal(ux.shape), g.standard_normal(uy.shape))
    fd_u = [(loss64(rates, dx, dy, h) - loss64(rates, dx, dy, -h)) / (2 * h) for dx, dy in dirs]
    fd_noise = (loss64(rates, *noise, h) - loss64(rates, *noise, -h)) / (2 * h)
    # The stated tolerances: FP64 adjoint 1e-7, FP32 adjoint 1e-3 relative against FP64
    # central differences, for the rate and both u0 directions (with the moment-space collision
    # the FP32 trajectory's rounding stays ~1e-6 of the misfit residual; the FP32 directional
    # derivatives agree with the FP64 adjoint's to ~1e-6).  The FP32 model's own central
    # differences (h = 3e-4 along a smooth direction, truncation ~1e-4 of it) are held to 5e-3.
    for storage, shift, tol_w, tol_u in ((L.LBM_F64, None, 1e-7, 1e-7), (L.LBM_F32, (u0, 0.0), 1e-3, 1e-3),
                                         (L.LBM_F32, None, 1e-3, 1e-3)):
        _, gx, gy, gr = _gpu(L, rho, ux, uy, model, rates, storage, n, "misfit", tx, ty, shift=shift)
        assert gr[0] == pytest.approx(fd_w, rel=tol_w)
        for (dx, dy), ref in zip(dirs, fd_u):
            assert float((gx * dx).sum() + (gy * dy).sum()) == pytest.approx(ref, rel=tol_u)
        if storage == L.LBM_F64:
            assert float((gx * noise[0]).sum() + (gy * noise[1]).sum()) == pytest.approx(fd_noise, rel=tol_u)
        else:
            def loss32(sign):
                dx, dy = dirs[0]
                lat = L.Lattice(N, N, L.MODELS[model], rates, storage=L.LBM_F32)
                if shift is not None:
                    lat.set_shift_velocity(*shift)
                lat.init_equilibrium(*[torch.from_numpy(np.ascontiguousarray(a)).cuda()
                                       for a in (rho, ux + sign * 3e-4 * dx, uy + sign * 3e-4 * dy)])
                lat.step(n)
                mx = torch.empty((N, N), dtype=torch.float64, device="cuda")
                my = torch.empty_like(mx)
                lat.moments(None, mx, my)
                lat.close()
                mx, my = mx.cpu().numpy(), my.cpu().numpy()
                return 0.5 * (((mx - tx) ** 2) + ((my - ty) ** 2)).sum()
            fd32 = (loss32(1.0) - loss32(-1.0)) / (2 * 3e-4)
            got = float((gx * dirs[0][0]).sum() + (gy * dirs[0][1]).sum())
            assert got == pytest.approx(fd32, rel=5e-3)
