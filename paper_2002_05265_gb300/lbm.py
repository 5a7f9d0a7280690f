"""ctypes binding of liblbm.so (C ABI in include/lbm.h).  Argument marshalling only: every
step of the method runs in the CUDA library.  If the library is missing or cannot be loaded
the calls raise; there is no fallback.

Field arguments may be torch tensors (CUDA or CPU, float64, contiguous), numpy float64
arrays, or raw integer addresses.  Streams may be a torch.cuda.Stream, an int handle or None
(legacy default stream).
"""

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblbm.so")

LBM_BGK, LBM_RM, LBM_HM, LBM_CM, LBM_CHM, LBM_K, LBM_PR, LBM_RR, LBM_K_PRE, LBM_K_EQ = range(10)
LBM_F64, LBM_F32, LBM_F16, LBM_BF16 = range(4)
LBM_PRESET_SRT, LBM_PRESET_REG = 0, 1
LBM_PATH_AUTO, LBM_PATH_VECTOR, LBM_PATH_BULK = 0, 1, 2
LBM_ORDER_AUTO, LBM_ORDER_STEP, LBM_ORDER_WAVE, LBM_ORDER_BLOCK = 0, 1, 2, 3
LBM_FORM_AUTO, LBM_FORM_GENERAL, LBM_FORM_LIGHT, LBM_FORM_WIDE = 0, 1, 2, 3
LBM_OK, LBM_ERR_INVALID_ARG, LBM_ERR_UNSUPPORTED, LBM_ERR_CUDA, LBM_ERR_BLOWUP, LBM_ERR_TIMEOUT, LBM_ERR_NOMEM = \
    0, -1, -2, -3, -4, -5, -6

MODELS = {"bgk": LBM_BGK, "rm": LBM_RM, "hm": LBM_HM, "cm": LBM_CM, "chm": LBM_CHM, "k": LBM_K,
          "pr": LBM_PR, "rr": LBM_RR, "k_pre": LBM_K_PRE, "k_eq": LBM_K_EQ}
STORAGES = {"f64": LBM_F64, "f32": LBM_F32, "f16": LBM_F16, "bf16": LBM_BF16}
STORAGE_BYTES = {LBM_F64: 8, LBM_F32: 4, LBM_F16: 2, LBM_BF16: 2}


class lbm_rates(ctypes.Structure):
    _fields_ = [("omega_nu", ctypes.c_double), ("omega3", ctypes.c_double), ("omega4", ctypes.c_double)]

    def as_tuple(self):
        return (self.omega_nu, self.omega3, self.omega4)


class lbm_instance_desc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("model", ctypes.c_int), ("rates", lbm_rates),
                ("ux_ref", ctypes.c_double), ("uy_ref", ctypes.c_double),
                ("ke_ref", ctypes.c_double), ("ke_factor", ctypes.c_double)]


class LBMError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"liblbm error {code}: {msg}")
        self.code = code


_lib = None

_P = ctypes.c_void_p
_I = ctypes.c_int
_LL = ctypes.c_longlong
_D = ctypes.c_double

_SIGNATURES = {
    "lbm_rates_from_nu": (_I, [_D, _I, ctypes.POINTER(lbm_rates)]),
    "lbm_create": (_I, [ctypes.POINTER(_P), _I, _I, _I, _I, lbm_rates, _I, _I, _D, _P]),
    "lbm_destroy": (None, [_P]),
    "lbm_set_rates": (_I, [_P, lbm_rates]),
    "lbm_init_equilibrium": (_I, [_P, _P, _P, _P]),
    "lbm_step": (_I, [_P, _LL]),
    "lbm_moments": (_I, [_P, _P, _P, _P, _P, _P, _P]),
    "lbm_reduce": (_I, [_P, _P]),
    "lbm_get_populations": (_I, [_P, _P]),
    "lbm_set_populations": (_I, [_P, _P]),
    "lbm_set_check": (_I, [_P, _LL, _D, _D, _D, _D]),
    "lbm_status": (_I, [_P, ctypes.POINTER(_I), ctypes.POINTER(_LL), ctypes.POINTER(_LL)]),
    "lbm_synchronize": (_I, [_P]),
    "lbm_get_layout": (_I, [_P, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "lbm_set_kernel_path": (_I, [_P, _I, _I]),
    "lbm_set_launch_shape": (_I, [_P, _I, _I]),
    "lbm_set_tile_form": (_I, [_P, _I]),
    "lbm_group_describe": (_I, [_P] + [ctypes.POINTER(_I)] * 6),
    "lbm_group_create": (_I, [ctypes.POINTER(_P), ctypes.POINTER(_P), _I, _I]),
    "lbm_group_step": (_I, [_P, _LL]),
    "lbm_group_destroy": (None, [_P]),
    "lbm_group_set_timing": (_I, [_P, _I]),
    "lbm_group_timing": (_I, [_P, ctypes.POINTER(_D), ctypes.POINTER(_LL), ctypes.POINTER(_LL)]),
    "lbm_set_shift_velocity": (_I, [_P, _D, _D]),
    "lbm_adjoint_run": (_I, [_P, _LL, _I, _P, _P, _I, _P, _P, _P, _P, _P]),
    "lbm_batch_create": (_I, [ctypes.POINTER(_P), _I, ctypes.POINTER(lbm_instance_desc), _I, _D, _P]),
    "lbm_batch_destroy": (None, [_P]),
    "lbm_batch_nodes": (_LL, [_P]),
    "lbm_batch_init_equilibrium": (_I, [_P, _P, _P, _P]),
    "lbm_batch_run": (_I, [_P, _LL, _I, _D]),
    "lbm_batch_status": (_I, [_P, _P, _P, _P, _P]),
    "lbm_batch_get_populations": (_I, [_P, _I, _P]),
    "lbm_batch_set_shape": (_I, [_P, _I, _I]),
    "lbm_batch_get_shape": (_I, [_P, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "lbm_batch_autotune": (_I, [_P, _LL, _I, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_D)]),
    "lbm_batch_last_error": (ctypes.c_char_p, [_P]),
    "lbm_last_error": (ctypes.c_char_p, [_P]),
    "lbm_error_string": (ctypes.c_char_p, [_I]),
    "lbm_version": (ctypes.c_char_p, []),
    "lbm_lsa_growth": (_I, [_I, lbm_rates, _I, _P, _I, _P, _I, _P, _P, _P, _P]),
    "lbm_selftest_recip": (_I, [_P, _P, _P, _LL, _P]),
    "lbm_halo_pack": (_I, [_P, _P, _P]),
    "lbm_halo_unpack": (_I, [_P, _P, _P]),
}


def load_library(path=LIB_PATH):
    """Load liblbm.so (raises if it is absent: build it with paper_2002_05265_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing; build it with `python -m paper_2002_05265_gb300.build`")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _addr(x):
    """Address of a field argument (torch tensor, numpy array, int or None)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        import torch
        if x.dtype != torch.float64 or not x.is_contiguous():
            raise TypeError("fields must be contiguous float64 tensors")
        return x.data_ptr()
    if hasattr(x, "__array_interface__"):
        import numpy as np
        if x.dtype != np.float64 or not x.flags["C_CONTIGUOUS"]:
            raise TypeError("fields must be C-contiguous float64 arrays")
        return x.__array_interface__["data"][0]
    raise TypeError(f"unsupported field argument {type(x)}")


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _check(rc, ctx=None):
    if rc != LBM_OK:
        lib = load_library()
        msg = lib.lbm_last_error(ctx).decode() if ctx else lib.lbm_error_string(rc).decode()
        raise LBMError(rc, msg or lib.lbm_error_string(rc).decode())


def lbm_rates_from_nu(nu, preset=LBM_PRESET_SRT):
    r = lbm_rates()
    _check(load_library().lbm_rates_from_nu(nu, preset, ctypes.byref(r)))
    return r


def lbm_create(nx, ny, model, rates, storage=LBM_F32, eq_order=4, rho0=1.0, stream=None, periodic=1):
    if isinstance(model, str):
        model = MODELS[model]
    if isinstance(storage, str):
        storage = STORAGES[storage]
    if not isinstance(rates, lbm_rates):
        rates = lbm_rates(*rates)
    h = _P()
    _check(load_library().lbm_create(ctypes.byref(h), nx, ny, periodic, model, rates, eq_order, storage, rho0,
                                     _stream(stream)))
    return h.value


def lbm_destroy(ctx):
    load_library().lbm_destroy(ctx)


def lbm_set_rates(ctx, rates):
    if not isinstance(rates, lbm_rates):
        rates = lbm_rates(*rates)
    _check(load_library().lbm_set_rates(ctx, rates), ctx)


def lbm_init_equilibrium(ctx, rho, ux, uy):
    _check(load_library().lbm_init_equilibrium(ctx, _addr(rho), _addr(ux), _addr(uy)), ctx)


def lbm_step(ctx, n):
    _check(load_library().lbm_step(ctx, n), ctx)


def lbm_moments(ctx, rho=None, ux=None, uy=None, pxx=None, pxy=None, pyy=None):
    _check(load_library().lbm_moments(ctx, _addr(rho), _addr(ux), _addr(uy), _addr(pxx), _addr(pxy), _addr(pyy)), ctx)


def lbm_reduce(ctx, out8):
    _check(load_library().lbm_reduce(ctx, _addr(out8)), ctx)


def lbm_get_populations(ctx, f):
    _check(load_library().lbm_get_populations(ctx, _addr(f)), ctx)


def lbm_set_populations(ctx, f):
    _check(load_library().lbm_set_populations(ctx, _addr(f)), ctx)


def lbm_set_check(ctx, every, ke_ref=0.0, ke_factor=1.0, uref=(0.0, 0.0)):
    _check(load_library().lbm_set_check(ctx, every, ke_ref, ke_factor, uref[0], uref[1]), ctx)


def lbm_status(ctx):
    st, bs, n = _I(), _LL(), _LL()
    _check(load_library().lbm_status(ctx, ctypes.byref(st), ctypes.byref(bs), ctypes.byref(n)), ctx)
    return st.value, bs.value, n.value


def lbm_synchronize(ctx):
    _check(load_library().lbm_synchronize(ctx), ctx)


def lbm_get_layout(ctx):
    p, g, b = _I(), _I(), _I()
    _check(load_library().lbm_get_layout(ctx, ctypes.byref(p), ctypes.byref(g), ctypes.byref(b)), ctx)
    return p.value, g.value, b.value


def lbm_set_kernel_path(ctx, path, stages=0):
    _check(load_library().lbm_set_kernel_path(ctx, path, stages), ctx)


def lbm_set_launch_shape(ctx, steps_per_launch=0, order=LBM_ORDER_AUTO):
    _check(load_library().lbm_set_launch_shape(ctx, steps_per_launch, order), ctx)


def lbm_set_tile_form(ctx, form=LBM_FORM_AUTO):
    _check(load_library().lbm_set_tile_form(ctx, form), ctx)


def lbm_group_describe(g):
    """How a group is advanced: dict of family (LBM_PATH_*), form (LBM_FORM_*),
    steps_per_launch, tiles, grid, block."""
    vals = [ctypes.c_int(0) for _ in range(6)]
    rc = load_library().lbm_group_describe(g, *[ctypes.byref(v) for v in vals])
    if rc != LBM_OK:
        raise LBMError(rc, "lbm_group_describe failed")
    keys = ("family", "form", "steps_per_launch", "tiles", "grid", "block")
    return {k: v.value for k, v in zip(keys, vals)}


def lbm_group_create(ctxs, graph_steps=64):
    arr = (_P * len(ctxs))(*ctxs)
    h = _P()
    _check(load_library().lbm_group_create(ctypes.byref(h), arr, len(ctxs), graph_steps), ctxs[0])
    return h.value


def lbm_group_step(group, n, ctx_for_errors=None):
    _check(load_library().lbm_group_step(group, n), ctx_for_errors)


def lbm_group_destroy(group):
    load_library().lbm_group_destroy(group)


def lbm_group_set_timing(group, enable=True):
    _check(load_library().lbm_group_set_timing(group, 1 if enable else 0))


def lbm_group_timing(group):
    """(summed replay ms, lattice time steps, step-kernel launches) of the timed replays."""
    ms, n, k = _D(), _LL(), _LL()
    _check(load_library().lbm_group_timing(group, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(k)))
    return ms.value, n.value, k.value


def lbm_set_shift_velocity(ctx, ux_ref, uy_ref):
    _check(load_library().lbm_set_shift_velocity(ctx, ux_ref, uy_ref), ctx)


def lbm_adjoint_run(ctx, nsteps, loss, ux_target, uy_target, grad_ux0, grad_uy0, checkpoint_every=0):
    """Runs N steps forward with checkpoints and the discrete adjoint backwards; fills
    grad_ux0 / grad_uy0 and returns (loss, [dL/domega_nu, dL/domega3, dL/domega4],
    (forward_ms, backward_ms))."""
    import numpy as np
    gr = np.zeros(3)
    L = np.zeros(1)
    t = np.zeros(2)
    _check(load_library().lbm_adjoint_run(ctx, nsteps, loss, _addr(ux_target), _addr(uy_target), checkpoint_every,
                                          _addr(grad_ux0), _addr(grad_uy0), gr.ctypes.data, L.ctypes.data,
                                          t.ctypes.data), ctx)
    return float(L[0]), gr, (float(t[0]), float(t[1]))


def _bcheck(rc, b=None):
    if rc != LBM_OK:
        lib = load_library()
        msg = lib.lbm_batch_last_error(b).decode() if b else lib.lbm_error_string(rc).decode()
        raise LBMError(rc, msg or lib.lbm_error_string(rc).decode())


def lbm_batch_create(descs, storage=LBM_F32, rho0=1.0, stream=None):
    """descs: sequence of dicts with nx, ny, model, rates (3-tuple or lbm_rates), ux_ref,
    uy_ref and optional ke_ref, ke_factor."""
    if isinstance(storage, str):
        storage = STORAGES[storage]
    arr = (lbm_instance_desc * len(descs))()
    for k, d in enumerate(descs):
        r = d["rates"] if isinstance(d["rates"], lbm_rates) else lbm_rates(*d["rates"])
        m = d["model"] if not isinstance(d["model"], str) else MODELS[d["model"]]
        arr[k] = lbm_instance_desc(d["nx"], d["ny"], m, r, d.get("ux_ref", 0.0), d.get("uy_ref", 0.0),
                                   d.get("ke_ref", 0.0), d.get("ke_factor", 1.0))
    h = _P()
    _bcheck(load_library().lbm_batch_create(ctypes.byref(h), len(descs), arr, storage, rho0, _stream(stream)))
    return h.value


def lbm_batch_destroy(b):
    load_library().lbm_batch_destroy(b)


def lbm_batch_nodes(b):
    return load_library().lbm_batch_nodes(b)


def lbm_batch_init_equilibrium(b, rho, ux, uy):
    _bcheck(load_library().lbm_batch_init_equilibrium(b, _addr(rho), _addr(ux), _addr(uy)), b)


def lbm_batch_run(b, target_steps, check_every=100, growth=1e4):
    _bcheck(load_library().lbm_batch_run(b, target_steps, check_every, growth), b)


def lbm_batch_status(b, n):
    """(status[n], blowup_step[n], steps[n], diag[n, 4]) as numpy arrays."""
    import numpy as np
    st = np.zeros(n, dtype=np.int32)
    bs = np.zeros(n, dtype=np.int64)
    steps = np.zeros(n, dtype=np.int64)
    diag = np.zeros((n, 4))
    _bcheck(load_library().lbm_batch_status(b, st.ctypes.data, bs.ctypes.data, steps.ctypes.data, diag.ctypes.data), b)
    return st, bs, steps, diag


def lbm_batch_get_populations(b, index, f):
    _bcheck(load_library().lbm_batch_get_populations(b, index, _addr(f)), b)


def lbm_batch_set_shape(b, vec, block):
    _bcheck(load_library().lbm_batch_set_shape(b, vec, block), b)


def lbm_batch_get_shape(b):
    v, k, g = _I(), _I(), _I()
    _bcheck(load_library().lbm_batch_get_shape(b, ctypes.byref(v), ctypes.byref(k), ctypes.byref(g)), b)
    return v.value, k.value, g.value


def lbm_batch_autotune(b, trial_steps=200, check_every=100):
    v, k, ms = _I(), _I(), _D()
    _bcheck(load_library().lbm_batch_autotune(b, trial_steps, check_every, ctypes.byref(v), ctypes.byref(k),
                                              ctypes.byref(ms)), b)
    return v.value, k.value, ms.value


def lbm_lsa_growth(model, rates, flows, k, growth, eig=None, jac=None, stream=None, eq_order=4):
    """flows: device (nflows, 3) doubles; k: device (nk, 2); growth: device (nflows, nk)."""
    if isinstance(model, str):
        model = MODELS[model]
    r = rates if isinstance(rates, lbm_rates) else lbm_rates(*rates)
    nflows, nk = int(flows.shape[0]), int(k.shape[0])
    _check(load_library().lbm_lsa_growth(model, r, eq_order, _addr(flows), nflows, _addr(k), nk, _addr(growth),
                                         _addr(eig) if eig is not None else None,
                                         _addr(jac) if jac is not None else None, _stream(stream)))


def lbm_halo_pack(ctx, send_up, send_down):
    """send_up / send_down: device tensors of 3 * nx storage elements (any dtype of that size)."""
    _check(load_library().lbm_halo_pack(ctx, send_up.data_ptr(), send_down.data_ptr()), ctx)


def lbm_halo_unpack(ctx, from_below, from_above):
    _check(load_library().lbm_halo_unpack(ctx, from_below.data_ptr(), from_above.data_ptr()), ctx)


def lbm_selftest_recip(x, approx, rounded, stream=None):
    """x, approx, rounded: device float32 tensors of n elements (the library's FP32 reciprocal
    and the correctly rounded one of x)."""
    _check(load_library().lbm_selftest_recip(x.data_ptr(), approx.data_ptr(), rounded.data_ptr(), int(x.numel()),
                                             _stream(stream)))


def lbm_version():
    return load_library().lbm_version().decode()


class Lattice:
    """Owns one lbm_ctx; methods forward to the C calls of the same names."""

    def __init__(self, nx, ny, model, rates, storage=LBM_F32, eq_order=4, rho0=1.0, stream=None):
        self.nx, self.ny = nx, ny
        self.ctx = lbm_create(nx, ny, model, rates, storage, eq_order, rho0, stream)

    def close(self):
        if self.ctx:
            lbm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init_equilibrium(self, rho, ux, uy):
        lbm_init_equilibrium(self.ctx, rho, ux, uy)

    def step(self, n):
        lbm_step(self.ctx, n)

    def moments(self, *fields):
        lbm_moments(self.ctx, *fields)

    def reduce(self, out8):
        lbm_reduce(self.ctx, out8)

    def get_populations(self, f):
        lbm_get_populations(self.ctx, f)

    def set_populations(self, f):
        lbm_set_populations(self.ctx, f)

    def set_check(self, every, ke_ref=0.0, ke_factor=1.0, uref=(0.0, 0.0)):
        lbm_set_check(self.ctx, every, ke_ref, ke_factor, uref)

    def status(self):
        return lbm_status(self.ctx)

    def synchronize(self):
        lbm_synchronize(self.ctx)

    def set_rates(self, rates):
        lbm_set_rates(self.ctx, rates)

    def set_shift_velocity(self, ux_ref, uy_ref):
        lbm_set_shift_velocity(self.ctx, ux_ref, uy_ref)

    def set_kernel_path(self, path, stages=0):
        lbm_set_kernel_path(self.ctx, path, stages)

    def set_launch_shape(self, steps_per_launch=0, order=LBM_ORDER_AUTO):
        lbm_set_launch_shape(self.ctx, steps_per_launch, order)

    def set_tile_form(self, form=LBM_FORM_AUTO):
        lbm_set_tile_form(self.ctx, form)
