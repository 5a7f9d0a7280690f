"""CPU checks of the C-ABI library: it builds for sm_103a, loads without a GPU, exports every
function include/lbm.h declares, and rejects invalid arguments before touching the GPU."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2002_05265_gb300 import build, lbm
    build.build_library()
    return lbm.load_library()


def _declared_functions():
    names = set()
    inc = os.path.join(ROOT, "include")
    for fn in os.listdir(inc):
        if fn.endswith(".h"):
            text = open(os.path.join(inc, fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(lbm_[a-z0-9_]+)\s*\(", text, re.M):
                names.add(m.group(1))
    return names


def test_every_declared_symbol_is_exported(lib):
    names = _declared_functions()
    assert len(names) >= 20
    for n in sorted(names):
        assert hasattr(lib, n), n


def test_library_is_built_for_sm_103a():
    from paper_2002_05265_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in " ".join(build.ARCH)


def test_rates_from_nu(lib):
    from paper_2002_05265_gb300 import lbm
    r = lbm.lbm_rates_from_nu(1e-4, lbm.LBM_PRESET_SRT)
    assert r.omega_nu == pytest.approx(1.0 / (3e-4 + 0.5), rel=1e-15)
    assert r.omega3 == r.omega_nu and r.omega4 == r.omega_nu
    r = lbm.lbm_rates_from_nu(1e-4, lbm.LBM_PRESET_REG)
    assert (r.omega3, r.omega4) == (1.0, 1.0)
    with pytest.raises(lbm.LBMError):
        lbm.lbm_rates_from_nu(-1.0)
    with pytest.raises(lbm.LBMError):
        lbm.lbm_rates_from_nu(1e-3, 7)


@pytest.mark.parametrize("kw,code", [
    (dict(nx=2), -1), (dict(ny=1), -1), (dict(model=10), -1), (dict(model=-1), -1), (dict(storage=4), -1),
    (dict(rates=(2.0, 1.0, 1.0)), -1), (dict(rates=(1.0, 0.0, 1.0)), -1), (dict(rates=(1.0, 1.0, float("nan"))), -1),
    (dict(eq_order=5), -1), (dict(eq_order=1), -1), (dict(rho0=0.0), -1), (dict(periodic=0), -2),
    (dict(model=4, eq_order=2), -2), (dict(model=1, eq_order=3), -2),
])
def test_create_rejects_invalid_arguments(lib, kw, code):
    """Validation happens on the host before any CUDA call, so it runs without a GPU."""
    from paper_2002_05265_gb300 import lbm
    args = dict(nx=16, ny=16, periodic=1, model=0, rates=(1.5, 1.5, 1.5), eq_order=4, storage=1, rho0=1.0)
    args.update(kw)
    h = ctypes.c_void_p()
    rc = lib.lbm_create(ctypes.byref(h), args["nx"], args["ny"], args["periodic"], args["model"],
                        lbm.lbm_rates(*args["rates"]), args["eq_order"], args["storage"], args["rho0"], None)
    assert rc == code
    assert h.value is None


def test_error_strings(lib):
    from paper_2002_05265_gb300 import lbm
    assert lbm.load_library().lbm_error_string(-4) == b"blow-up detected"
    assert b"sm_103a" in lib.lbm_version()


def test_null_handles_are_rejected(lib):
    """The launch-shape calls check their handles on the host (no GPU needed)."""
    n = ctypes.c_int(7)
    assert lib.lbm_set_tile_form(None, 0) == -1
    assert lib.lbm_set_launch_shape(None, 0, 0) == -1
    assert lib.lbm_group_describe(None, ctypes.byref(n), None, None, None, None, None) == -1
    assert n.value == 7
