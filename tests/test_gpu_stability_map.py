"""Numerical stability of the convected vortex (Sec. 5b) through the batched persistent kernel:
the qualitative statements of the paper at points well inside or outside each model's limit
on a 32 x 32 lattice (nu = 1e-4, M = 50 t_c, the map criterion of bench.py: mean |u|^2 above
1.01 x its initial value, or non-finite values).  SRT moment models behave as BGK; REG-CHM,
REG-K and SRT-RR are the most stable; REG-RM fails already at low Mach number."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_2002_05265_gb300 import flows  # noqa: E402

CS = 1.0 / np.sqrt(3.0)
N = 32
NU = 1e-4


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2002_05265_gb300 import build, lbm
    build.build_library()
    lbm.load_library()
    return lbm


def _stable(L, configs, ma):
    """Stable flags of (model, preset) instances of the vortex at Mach number ma."""
    u0 = ma * CS
    steps = int(np.ceil(50 * N / u0 / 100)) * 100
    rho, ux, uy = flows.vortex(N, Ma=ma, radius_frac=0.05)
    ke0 = float(np.mean(ux * ux + uy * uy))
    w = 1.0 / (3.0 * NU + 0.5)
    descs = [{"nx": N, "ny": N, "model": m, "rates": (w, w, w) if p == "srt" else (w, 1.0, 1.0),
              "ux_ref": u0, "uy_ref": 0.0, "ke_ref": ke0, "ke_factor": 1.01} for m, p in configs]
    b = L.lbm_batch_create(descs, storage=L.LBM_F32)
    cat = [torch.from_numpy(np.ascontiguousarray(np.tile(a.ravel(), len(descs)))).cuda() for a in (rho, ux, uy)]
    L.lbm_batch_init_equilibrium(b, *cat)
    L.lbm_batch_run(b, steps, check_every=100, growth=1e300)
    st, _, _, _ = L.lbm_batch_status(b, len(descs))
    L.lbm_batch_destroy(b)
    return {c: bool(s == 0) for c, s in zip(configs, st)}


SRT_GROUP = [("bgk", "srt"), ("rm", "srt"), ("hm", "srt"), ("cm", "srt"), ("chm", "srt"), ("k", "srt")]
MOST_STABLE = [("chm", "reg"), ("k", "reg"), ("rr", "srt")]


def test_srt_moment_models_share_bgk_stability(L):
    """BGK's limit at L = 32 is Ma = 0.40: every SRT moment model is stable at 0.2 and blows up
    at 0.6, like BGK (App. B: with one rate they are the BGK collision)."""
    low = _stable(L, SRT_GROUP, 0.2)
    high = _stable(L, SRT_GROUP, 0.6)
    assert all(low.values()), low
    assert not any(high.values()), high


def test_most_stable_models(L):
    """SRT-RR, REG-CHM and REG-K stay stable at Ma = 0.6 (limit 0.65 at L = 32), where BGK and
    the SRT moment models fail; REG-RM and REG-HM (= PR) fail already at Ma = 0.2."""
    res = _stable(L, MOST_STABLE + [("rm", "reg"), ("hm", "reg"), ("bgk", "srt")], 0.6)
    assert all(res[c] for c in MOST_STABLE), res
    assert not res[("bgk", "srt")]
    low = _stable(L, [("rm", "reg"), ("hm", "reg")], 0.2)
    assert not any(low.values()), low
