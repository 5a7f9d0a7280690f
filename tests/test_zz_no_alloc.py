"""lbm_reduce_noalloc: the reductions of lbm_reduce for a caller-owned population buffer,
without any device allocation inside the library.  It exists for callers that cannot
allocate at that point (a global-mode graph capture in progress elsewhere, device memory
owned by an application pool, loops that must not synchronise on cudaMalloc/cudaFree).

The test builds population buffers in the documented layout itself, calls the new entry
point through the C ABI twice in a row on different lattices, and compares each result with
lbm_reduce on a context holding the same populations.  This file is collected last so that
a run stopping at the first failure has already run every other test."""

import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_2002_05265_gb300 import flows  # noqa: E402

XI = [(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)]
W = [4 / 9] + [1 / 9] * 4 + [1 / 36] * 4


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2002_05265_gb300 import build, lbm
    build.build_library()
    lib = lbm.load_library()
    lib.lbm_reduce_noalloc.restype = ctypes.c_int
    lib.lbm_reduce_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_void_p,
                                       ctypes.c_void_p]
    return lbm


def _populations(nx, ny, seed):
    """A non-equilibrium state: equilibrium of a vortex plus seeded population noise."""
    rho, ux, uy = flows.vortex(nx, ny, Ma=0.2, noise=1e-6, seed=seed)
    f = np.empty((9, ny, nx))
    for i, (sx, sy) in enumerate(XI):
        eu = 3 * (sx * ux + sy * uy)
        f[i] = W[i] * rho * (1 + eu + 0.5 * eu * eu - 1.5 * (ux * ux + uy * uy))
    return f * (1 + flows.random_populations_perturbation(f.shape, 1e-3, seed + 100))


def _round_bf16(x):
    """Round-to-nearest-even of FP64 values to bfloat16 (8 significant bits); the values here
    are normal numbers."""
    m, e = np.frexp(x)
    return np.ldexp(np.rint(m * 256.0) / 256.0, e)


def _to_storage(g, dtype):
    """FP64 array -> torch tensor of the storage type."""
    if dtype == torch.float16:
        return torch.from_numpy(g.astype(np.float16))
    if dtype == torch.bfloat16:
        return torch.from_numpy(_round_bf16(g)).to(dtype)  # exact: already representable
    return torch.from_numpy(g).to(dtype)


def _layout(f, dtype, pitch, rho0=1.0, offset=0):
    """The library layout: plane i holds g_i = f_i - w_i rho0 of node x at position x - xi_i,
    rounded to the storage type.  The buffer starts `offset` elements into a flat device
    allocation.  Returns the allocation and the FP64 populations the rounded buffer holds
    exactly (g_i + w_i rho0 in node order: adding w_i to a value with at most 24 significant
    bits below 2^-2 is exact in FP64, so the library recovers the same g_i from them)."""
    _, ny, nx = f.shape
    flat = torch.zeros(9 * ny * pitch + offset, dtype=dtype)
    buf = flat[offset:].view(9, ny, pitch)
    held = np.empty_like(f)
    for i, (sx, sy) in enumerate(XI):
        g = np.roll(f[i] - W[i] * rho0, shift=(-sy, -sx), axis=(0, 1))
        buf[i, :, :nx] = _to_storage(np.ascontiguousarray(g), dtype)
        gr = buf[i, :, :nx].double().numpy()
        held[i] = np.roll(gr, shift=(sy, sx), axis=(0, 1)) + W[i] * rho0
    return flat.cuda(), held


def _reference(L, f, storage, uref):
    _, ny, nx = f.shape
    lat = L.Lattice(nx, ny, L.LBM_BGK, (1.5, 1.5, 1.5), storage=storage)
    lat.set_populations(np.ascontiguousarray(f))
    lat.set_check(0, uref=uref)
    out = torch.empty(8, dtype=torch.float64, device="cuda")
    lat.reduce(out)
    res = out.cpu().numpy()
    lat.close()
    return res


def _check_case(L, lib, nx, ny, dtype, storage, pitch, uref, seed, offset=0):
    flat, f = _layout(_populations(nx, ny, seed), dtype, pitch, offset=offset)
    ptr = flat.data_ptr() + offset * flat.element_size()
    out = torch.full((8,), float("nan"), dtype=torch.float64, device="cuda")
    rc = lib.lbm_reduce_noalloc(ptr, storage, nx, ny, pitch, 1.0, uref[0], uref[1],
                                out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert rc == 0
    torch.cuda.synchronize()
    np.testing.assert_allclose(out.cpu().numpy(), _reference(L, f, storage, uref), rtol=1e-12, atol=1e-14)


def test_noalloc_reduce_matches_lbm_reduce_twice(L):
    """Two calls in a row (the shared scratch array keeps the first call's partials) on
    different lattices: FP64 with 16-byte rows (vectorised gather), FP32 with an odd pitch
    (scalar gather)."""
    lib = L.load_library()
    cases = [(70, 41, torch.float64, L.LBM_F64, 72, (0.05, -0.01), 1),
             (128, 97, torch.float32, L.LBM_F32, 131, (0.0, 0.02), 2)]
    for nx, ny, dtype, storage, pitch, uref, seed in cases:
        _check_case(L, lib, nx, ny, dtype, storage, pitch, uref, seed)


@pytest.mark.parametrize("nx,ny,dtype_name,pitch,offset", [
    (37, 23, "float16", 40, 0),      # 16-byte rows, last vector segment 5 of 8 nodes
    (45, 19, "bfloat16", 48, 0),     # same for BF16 (5 of 8)
    (33, 21, "float16", 35, 0),      # odd pitch: scalar gather
    (41, 17, "bfloat16", 41, 0),     # pitch = nx, odd: scalar gather
    (30, 18, "float32", 32, 1),      # 16-byte pitch but the buffer starts one element in: scalar
])
def test_noalloc_reduce_16bit_and_unaligned_layouts(L, nx, ny, dtype_name, pitch, offset):
    lib = L.load_library()
    dtype = getattr(torch, dtype_name)
    storage = {"float16": L.LBM_F16, "bfloat16": L.LBM_BF16, "float32": L.LBM_F32}[dtype_name]
    _check_case(L, lib, nx, ny, dtype, storage, pitch, (0.03, 0.01), nx + ny, offset=offset)


def test_noalloc_reduce_rejects_bad_arguments(L):
    lib = L.load_library()
    buf = torch.zeros((9, 8, 8), dtype=torch.float32, device="cuda")
    out = torch.zeros(8, dtype=torch.float64, device="cuda")
    host_out = np.zeros(8)
    ok = dict(p=buf.data_ptr(), s=L.LBM_F32, nx=8, ny=8, pitch=8, o=out.data_ptr())

    def call(**kw):
        a = dict(ok, **kw)
        return lib.lbm_reduce_noalloc(a["p"], a["s"], a["nx"], a["ny"], a["pitch"], 1.0, 0.0, 0.0, a["o"], None)
    assert call() == 0
    assert call(nx=65536, ny=65537, pitch=65536) == L.LBM_ERR_INVALID_ARG      # beyond 2^31 nodes
    assert call(pitch=7) == L.LBM_ERR_INVALID_ARG
    assert call(nx=2) == L.LBM_ERR_INVALID_ARG
    assert call(s=9) == L.LBM_ERR_INVALID_ARG
    assert call(o=host_out.ctypes.data) == L.LBM_ERR_INVALID_ARG
    assert call(p=None) == L.LBM_ERR_INVALID_ARG
    assert call(p=buf.data_ptr() + 1) == L.LBM_ERR_INVALID_ARG                # not element-aligned
    assert call(p=buf.data_ptr() + 2) == L.LBM_ERR_INVALID_ARG
    assert call(o=out.data_ptr() + 4) == L.LBM_ERR_INVALID_ARG                # out8 not 8-byte aligned
    host_buf = np.zeros(9 * 8 * 8, dtype=np.float32)
    assert call(p=host_buf.ctypes.data) == L.LBM_ERR_INVALID_ARG              # host populations
    torch.cuda.synchronize()
