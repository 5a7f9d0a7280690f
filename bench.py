"""Throughput benchmark of the D2Q9 stream-and-collide kernels.

Workload (one benchmark step): the periodic double shear layer on 1024 x 1024 lattices
(tanh width L/80, Ma = 0.1, transverse perturbation 0.05, nu = 1e-5), one lattice per
collision model (BGK, RM, HM, CM, CHM, K, PR, RR; FP32 shifted storage, FP32 collision),
each initialised at equilibrium, advanced 20000 time steps with the FP64 blow-up check every
100 steps, and reduced to its moments.  The eight lattices advance together, one time step
of each in turn, so the 604 MB working set streams from HBM (larger than the 126 MB L2).

Metric: lattice updates per second (GLUPS) over all lattices; `e2e` repeats the step through
the same C calls with pinned host buffers (host->device copy of rho, u and device->host copy
of rho, u inside the timed region).  `--impl reference` times the FP64 CPU oracle on the
host cores instead.
"""

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

MODELS = ["bgk", "rm", "hm", "cm", "chm", "k", "pr", "rr"]
L = 1024
SIM_STEPS = 20000
CHECK_EVERY = 100
GRAPH_STEPS = 100
NU = 1e-5
MA = 0.1
CS = 1.0 / np.sqrt(3.0)
BYTES_PER_LU = {"f64": 144, "f32": 72, "f16": 36, "bf16": 36}


def _preset(model):
    # BGK uses omega_nu only and PR fixes omega3 = omega4 = 1; the moment-space models run
    # with equilibrated high-order moments (the paper's REG configuration)
    return "srt" if model == "bgk" else "reg"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--sim-steps", type=int, default=SIM_STEPS)
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-per-model", action="store_true",
                   help="skip the per-model x storage timing on the 16384^2 vortex")
    p.add_argument("--no-batch-key", action="store_true", help="skip the bounded batched-sweep measurement")
    p.add_argument("--no-accuracy-key", action="store_true", help="skip the storage-accuracy table")
    p.add_argument("--no-adjoint", action="store_true", help="skip the adjoint / forward time ratio")
    p.add_argument("--batch", action="store_true",
                   help="instead of the benchmark step, run the batched stability sweep (4096 lattices)")
    p.add_argument("--instances", type=int, default=4096)
    p.add_argument("--batch-steps", type=int, default=50000)
    p.add_argument("--accuracy", type=int, default=0,
                   help="instead of the benchmark step, the storage-accuracy study on an LxL vortex (L given)")
    p.add_argument("--sweep", default=None,
                   help="instead of the benchmark step, time single lattices: MODELS:STORAGES:SIZE, e.g. "
                        "all:f32,f16,bf16:16384 (one JSON line per combination)")
    p.add_argument("--stability-map", type=int, default=0,
                   help="instead of the benchmark step, the numerical stability maps of the convected vortex "
                        "on an LxL lattice (L given): maximal stable Mach number per model, rate preset and viscosity")
    p.add_argument("--map-tc", type=float, default=50.0, help="characteristic times t_c = L/u0 per map instance")
    p.add_argument("--transport", type=int, default=0,
                   help="instead of the benchmark step, the long-distance vortex transport of Sec. 5c on an LxL "
                        "lattice (L given): Ma = 0.5, nu = 1e-4, 50 t_c, SRT-RR / REG-CHM / REG-K vorticity errors")
    p.add_argument("--lsa", type=int, default=0,
                   help="instead of the benchmark step, linear stability curves (App. A) on a KxK wavenumber grid "
                        "(K given): largest linearly stable Ma per model, rate preset and viscosity")
    p.add_argument("--slab", type=int, default=0,
                   help="instead of the benchmark step, one LxL lattice (L given) split into y-slabs over the ranks "
                        "with a halo exchange every step (strong scaling)")
    p.add_argument("--slab-storage", default="f32", choices=["f64", "f32", "f16", "bf16"])
    p.add_argument("--map-storage", default="f32", choices=["f64", "f32"])
    p.add_argument("--path", default="auto", choices=["auto", "vector", "bulk"],
                   help="step-kernel family: copy-engine staged (bulk), register-staged (vector), or the "
                        "library's choice (auto: bulk where the row length allows it)")
    p.add_argument("--stages", type=int, default=0, help="shared-memory stages of the bulk-copy kernel (0 = default)")
    p.add_argument("--launch-steps", type=int, default=0,
                   help="time steps per bulk-copy launch (0 = the library's default)")
    p.add_argument("--order", default="auto", choices=["auto", "step", "wave", "block"],
                   help="work order of multi-step bulk-copy launches (auto: wavefront when the state exceeds 64 MB)")
    p.add_argument("--form", default="auto", choices=["auto", "general", "light", "wide"],
                   help="kernel form of the bulk-copy kernel (auto: the library's choice)")
    return p.parse_args()


PATHS = {"auto": 0, "vector": 1, "bulk": 2}
ORDERS = {"auto": 0, "step": 1, "wave": 2, "block": 3}
FORMS = {"auto": 0, "general": 1, "light": 2, "wide": 3}


def shape_lattice(lat, args):
    """Kernel family and launch shape of a benchmark lattice from the command line."""
    lat.set_kernel_path(PATHS[args.path], args.stages)
    lat.set_launch_shape(args.launch_steps, ORDERS[args.order])
    lat.set_tile_form(FORMS[args.form])


def dist_setup(args):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend=backend)
    if torch.cuda.is_available():
        torch.cuda.set_device(local)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=5)
        sm, smax, power = [], [], []
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
                power.append(float(parts[2]))
            except ValueError:
                continue
            for name, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)), "samples": len(sm),
                "power_w_max": float(max(power)) if power else None, "reasons": sorted(reasons)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def source_hashes(names):
    """sha256 of kernel source files of csrc/ (the ncu figures are valid only for these)."""
    import hashlib
    out = {}
    for n in names:
        with open(os.path.join(ROOT, "paper_2002_05265_gb300", "csrc", n), "rb") as fh:
            out[n] = hashlib.sha256(fh.read()).hexdigest()
    return out


def ncu_traffic(kernel_tag):
    """Per-launch DRAM bytes of the step kernel from the committed ncu summary, if it was
    taken on the current kernel sources (else None)."""
    path = os.path.join(ROOT, "profiles", "step_kernel_traffic.json")
    if not os.path.exists(path):
        return None
    e = json.load(open(path)).get(kernel_tag)
    if not e or e.get("sources") != source_hashes(sorted(e.get("sources", {}))):
        return None
    return e.get("dram_bytes_per_launch_full_size")


_ORACLE_F0 = None
CPU_SLAB = 128   # rows per oracle task (L / CPU_SLAB tasks per model and time step)


def _oracle_init():
    """Worker start-up: the FP64 oracle's initial state of the 1024 x 1024 double shear layer."""
    global _ORACLE_F0
    import oracle.lbm as olbm
    from paper_2002_05265_gb300 import flows
    _ORACLE_F0 = olbm.init_equilibrium(*flows.double_shear_layer(L, Ma=MA))


def oracle_slab_step(f, model, rates, y0, rows):
    """One oracle time step of one collision model on rows y0 .. y0 + rows - 1 of the
    population field f[9][ny][nx]: the oracle steps the slab plus one halo row on each side
    (periodic in x), which gives those rows exactly what a step of the whole lattice gives
    them (a stream-and-collide step reaches one node).  Returns the slab's own rows."""
    import oracle.lbm as olbm
    idx = np.arange(y0 - 1, y0 + rows + 1) % f.shape[1]
    return olbm.step(f[:, idx, :], model, rates)[:, 1:-1, :]


def _oracle_slab_step(task):
    """Worker task: one time step of one model on one CPU_SLAB-row slab of the benchmark
    lattice (the result is discarded); returns the lattice updates of the slab's rows."""
    import oracle.lbm as olbm
    model, y0 = task
    oracle_slab_step(_ORACLE_F0, model, olbm.rates_from_nu(NU, _preset(model)), y0, CPU_SLAB)
    return CPU_SLAB * L


def oracle_pool():
    """Worker processes for the oracle timing, one per host core; spawned (not forked), so
    a process that already holds a CUDA context can start them."""
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    procs = max(1, os.cpu_count() or 1)
    return ProcessPoolExecutor(max_workers=procs, mp_context=mp.get_context("spawn"), initializer=_oracle_init), procs


ORACLE_TASKS = [(m, y0) for m in MODELS for y0 in range(0, L, CPU_SLAB)]


def oracle_round(pool):
    """One time step of each of the 8 models on the whole lattice: every (model, row slab)
    a task, the tasks spread over the worker processes (so the slow models use many cores).
    Returns the lattice updates done."""
    return sum(pool.map(_oracle_slab_step, ORACLE_TASKS, chunksize=1))


CPU_ROUNDS = 8   # about 20 s of CPU work on a 16-core Grace host (one round: 8 models x 1024^2 updates)


def cpu_baseline():
    """FP64 oracle as it stands, CPU_ROUNDS time steps of each collision model on the
    1024 x 1024 double shear layer, spread over all host cores as (model, 128-row slab)
    tasks in single-threaded numpy processes."""
    pool, procs = oracle_pool()
    try:
        oracle_round(pool)   # start-up (imports, initial state) outside the timing
        t0 = time.perf_counter()
        lu = 0
        for _ in range(CPU_ROUNDS):
            lu += oracle_round(pool)
        dt = time.perf_counter() - t0
    finally:
        pool.shutdown()
    return {"value": lu / dt / 1e9, "unit": "GLUPS", "cores": procs, "host_cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{CPU_ROUNDS} time steps of each of the {len(MODELS)} models on the {L}x{L} double shear "
                      f"layer ({lu} lattice updates, {dt:.1f} s wall), numpy FP64, as {len(ORACLE_TASKS)} "
                      f"(model, {CPU_SLAB}-row slab + halo) tasks per step over {procs} single-threaded processes"}


def adjoint_ratio(lbm, flows, stream, path=0, stages=0):
    """Adjoint / forward time ratio on the 512 x 512 vortex, 4000 steps, FP32, REG rates,
    misfit loss to the translated vortex plus N(0, (1e-3 u0)^2) noise, sqrt(N) checkpoints:
    backward (recomputation + adjoint steps) over the plain forward run of the same 4000
    steps; then the FP32 gradient against FP64 (adjoint_gradient_check)."""
    import torch
    N, n = 512, 4000
    u0 = 0.1 / np.sqrt(3.0)
    rho, ux, uy = flows.vortex(N, Ma=0.1)
    _, tx, ty = flows.vortex(N, Ma=0.1, center=((N / 2 + u0 * n) % N, N / 2))
    tx = tx + flows.gaussian_noise(tx.shape, 1e-3 * u0, 21)
    ty = ty + flows.gaussian_noise(ty.shape, 1e-3 * u0, 22)
    dev = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (rho, ux, uy, tx, ty)]
    w = 1.0 / (3e-4 + 0.5)
    res = {}
    for m in ("chm", "k"):
        lat = lbm.Lattice(N, N, lbm.MODELS[m], (w, 1.0, 1.0), storage=lbm.LBM_F32, stream=stream)
        lat.set_kernel_path(path, stages)
        lat.init_equilibrium(*dev[:3])
        lat.step(64)
        lat.synchronize()
        lat.init_equilibrium(*dev[:3])
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        lat.step(n)
        e1.record(stream)
        stream.synchronize()
        fwd = e0.elapsed_time(e1)
        lat.init_equilibrium(*dev[:3])
        gx = torch.empty_like(dev[1])
        gy = torch.empty_like(dev[2])
        loss, gr, (f_ms, b_ms) = lbm.lbm_adjoint_run(lat.ctx, n, 0, dev[3], dev[4], gx, gy, 0)
        lat.close()
        res[m] = {"forward_ms": fwd, "forward_with_checkpoints_ms": f_ms, "backward_ms": b_ms,
                  "ratio": b_ms / fwd, "loss": loss,
                  "gradient_check": adjoint_gradient_check(lbm, flows, m, (w, 1.0, 1.0), n, dev, gx, gy, gr, stream)}
    return {"workload": "512x512 vortex, 4000 steps, FP32, REG rates, misfit loss to the translated vortex plus "
                        "N(0, (1e-3 u0)^2) noise, 64 checkpoints", "models": res}


def adjoint_gradient_check(lbm, flows, m, rates, n, dev, gx32, gy32, gr32, stream):
    """FP32 adjoint gradient of the misfit against FP64 adjoint gradients (the FP64 adjoint
    matches FP64 central differences to 1e-7 in the tests): relative errors of the
    directional derivative along two smooth random u0 directions and of dL/domega_nu,
    (a) against the FP64 model's gradient and (b) against the FP64 adjoint on the FP32 run's
    own final residual (target shifted by u^N_FP32 - u^N_FP64), which isolates the adjoint
    from the forward trajectory's rounding."""
    import torch
    N = dev[0].shape[0]

    def final_u(storage):
        lat = lbm.Lattice(N, N, lbm.MODELS[m], rates, storage=storage, stream=stream)
        lat.init_equilibrium(*dev[:3])
        lat.step(n)
        mx, my = torch.empty_like(dev[1]), torch.empty_like(dev[2])
        lat.moments(None, mx, my)
        lat.synchronize()
        lat.close()
        return mx, my

    def adj64(tx, ty):
        lat = lbm.Lattice(N, N, lbm.MODELS[m], rates, storage=lbm.LBM_F64, stream=stream)
        lat.init_equilibrium(*dev[:3])
        gx, gy = torch.empty_like(dev[1]), torch.empty_like(dev[2])
        _, gr, _ = lbm.lbm_adjoint_run(lat.ctx, n, 0, tx, ty, gx, gy, 0)
        lat.close()
        return gx, gy, gr

    u64 = final_u(lbm.LBM_F64)
    u32 = final_u(lbm.LBM_F32)
    g64 = adj64(dev[3], dev[4])
    gsr = adj64((dev[3] - (u32[0] - u64[0])).contiguous(), (dev[4] - (u32[1] - u64[1])).contiguous())
    dirs = [[torch.from_numpy(flows.smooth_random_field(N, N, 8, 31 + 2 * k + j)).cuda() for j in range(2)]
            for k in range(2)]

    def rel_errs(ref):
        out = []
        for dx, dy in dirs:
            a = float((gx32 * dx).sum() + (gy32 * dy).sum())
            b = float((ref[0] * dx).sum() + (ref[1] * dy).sum())
            out.append(abs(a - b) / abs(b))
        return {"u0_directional": out, "omega_nu": abs(gr32[0] - ref[2][0]) / abs(ref[2][0])}
    return {"tolerance": 1e-3, "fp32_vs_fp64": rel_errs(g64), "fp32_vs_fp64_same_residual": rel_errs(gsr),
            "final_u_fp32_minus_fp64_max": float(torch.max(torch.abs(u32[0] - u64[0])).item())}


BIG_L = 16384
BIG_STORAGES = ("f32", "f16", "bf16")


def vortex_on_device(n, Ma, slab=1024):
    """The n x n convected vortex as FP64 device fields, generated in row slabs (the full
    16384^2 field would need several host copies of 2 GB arrays at once)."""
    import torch
    from paper_2002_05265_gb300 import flows
    out = [torch.empty((n, n), dtype=torch.float64, device="cuda") for _ in range(3)]
    for y0 in range(0, n, slab):
        y1 = min(n, y0 + slab)
        for o, a in zip(out, flows.vortex(n, Ma=Ma, rows=(y0, y1))):
            o[y0:y1].copy_(torch.from_numpy(a))
    return out


def form_name(lbm, g):
    """Kernel family and form the library chose for a group (lbm_group_describe)."""
    d = lbm.lbm_group_describe(g)
    if d["family"] != lbm.LBM_PATH_BULK:
        return "register-staged"
    return {lbm.LBM_FORM_GENERAL: "general", lbm.LBM_FORM_LIGHT: "light", lbm.LBM_FORM_WIDE: "wide"}[d["form"]]


def per_model_big(lbm, stream, peak, n=BIG_L, warmup=16, steps=48):
    """Throughput of every collision model x storage type on one n x n lattice: the
    convected vortex at Ma = 0.2, nu = 1e-6 (BGK single-rate, the others with equilibrated
    high-order moments), one time step per launch in step order, so every step reads and
    writes both population buffers through HBM (9.7 GB for 16-bit storage, 19.3 GB for FP32:
    75-150x the L2).  Time = CUDA events around the graph replays of the step kernel on the
    launching stream; frac = algorithmic bytes (2 x 9 populations per lattice update) / time /
    measured HBM copy bandwidth."""
    import torch
    fields = vortex_on_device(n, 0.2)
    res = {}
    for s in BIG_STORAGES:
        res[s] = {}
        for m in MODELS:
            rates = lbm.lbm_rates_from_nu(1e-6, lbm.LBM_PRESET_SRT if _preset(m) == "srt" else lbm.LBM_PRESET_REG)
            lat = lbm.Lattice(n, n, lbm.MODELS[m], rates, storage=lbm.STORAGES[s], stream=stream)
            lat.set_kernel_path(lbm.LBM_PATH_AUTO, 0)
            lat.set_launch_shape(1, lbm.LBM_ORDER_STEP)
            lat.init_equilibrium(*fields)
            g = lbm.lbm_group_create([lat.ctx], graph_steps=16)
            lbm.lbm_group_step(g, warmup, lat.ctx)
            lbm.lbm_group_set_timing(g, True)
            lbm.lbm_group_step(g, steps, lat.ctx)
            rms, nl, nk = lbm.lbm_group_timing(g)
            t = rms / 1e3 / nl
            gbs = BYTES_PER_LU[s] * n * n / t / 1e9
            res[s][m] = {"glups": n * n / t / 1e9, "alg_gbs": gbs, "frac": gbs / peak,
                         "launches": nk, "status": lat.status()[0], "form": form_name(lbm, g)}
            lbm.lbm_group_destroy(g)
            lat.close()
    del fields
    torch.cuda.empty_cache()
    return {"workload": f"convected vortex {n}x{n}, Ma=0.2, nu=1e-6, {steps} timed steps after {warmup}, "
                        "one step per launch, step order, each model x storage alone",
            "peak_gbs": peak, "bytes_per_lu": {k: BYTES_PER_LU[k] for k in BIG_STORAGES},
            "l2": "inputs larger than L2: 9.7-19.3 GB of populations per step", "results": res}


ACCURACY_CASES = (("f32", False), ("f16", False), ("bf16", False), ("f32", True), ("f16", True), ("bf16", True))


def storage_accuracy(lbm, n, nus=(1e-6, 1e-4)):
    """Error of reduced-precision storage after 10 domain traversals of the convected vortex
    (Ma = 0.2, radius 0.1 L, n x n, no seed noise, so that nothing but the storage differs):
    normalised L2 velocity error of every model (BGK and RR single-rate, the others REG) with
    FP32, FP16 and BF16 storage (shift w rho0, and shift at the mean flow) against the FP64
    kernel on the same lattice (itself checked against the FP64 CPU oracle by the tests).
    Yields one record per nu x model x storage x shift."""
    import torch
    from paper_2002_05265_gb300 import flows
    Ma = 0.2
    u0 = Ma / np.sqrt(3.0)
    steps = int(round(10 * n / u0))
    fields = [torch.from_numpy(a).cuda() for a in flows.vortex(n, Ma=Ma)]

    def velocity(model, storage, shift, w):
        # RR in its single-rate form (SRT-RR, among the most stable configurations of Sec. 5b;
        # REG-RR equals PR)
        srt = _preset(model) == "srt" or model == "rr"
        rates = (w, w, w) if srt else (w, 1.0, 1.0)
        lat = lbm.Lattice(n, n, lbm.MODELS[model], rates, storage=lbm.STORAGES[storage])
        if shift:
            lat.set_shift_velocity(u0, 0.0)
        lat.init_equilibrium(*fields)
        lat.step(steps)
        ux = torch.empty((n, n), dtype=torch.float64, device="cuda")
        uy = torch.empty_like(ux)
        lat.moments(None, ux, uy)
        lat.close()
        return ux, uy

    for nu in nus:
        w = 1.0 / (3.0 * nu + 0.5)
        for m in MODELS:
            rx, ry = velocity(m, "f64", False, w)
            ok = bool(torch.isfinite(rx).all() and torch.isfinite(ry).all())
            norm = torch.sqrt((rx * rx + ry * ry).sum())
            for storage, shift in ACCURACY_CASES:
                gx, gy = velocity(m, storage, shift, w)
                err = float(torch.sqrt(((gx - rx) ** 2 + (gy - ry) ** 2).sum()) / norm) if ok else None
                yield {"nu": nu, "model": m, "storage": storage, "shift": "mean flow" if shift else "w rho0",
                       "lattice": f"{n}x{n}", "steps": steps, "traversals": 10, "fp64_reference_finite": ok,
                       "l2_rel_error_u": err, "finite": bool(torch.isfinite(gx).all())}


def accuracy_table(lbm, n=256):
    """storage_accuracy as a nested table: nu -> storage/shift -> model -> error (None where
    the FP64 reference itself blew up, 'blown up' where only the reduced storage did)."""
    table = {}
    for r in storage_accuracy(lbm, n):
        key = f'{r["storage"]}, {r["shift"]} shift'
        val = r["l2_rel_error_u"] if r["finite"] else "blown up"
        table.setdefault(f'nu={r["nu"]:g}', {}).setdefault(key, {})[r["model"]] = val
    return {"workload": f"convected vortex {n}x{n}, Ma=0.2, 10 domain traversals "
                        f"({int(round(10 * n / (0.2 / np.sqrt(3.0))))} steps), normalised L2 error of u "
                        "against the FP64 kernel on the same lattice (None: the FP64 run blew up)",
            "target": "FP16-shifted storage <= 1e-3", "errors": table}


METRIC = "D2Q9 lattice updates per second, 8 collision models (GLUPS)"


def bench_config(S, world):
    """The benchmark workload's `config` (both arms report the same one)."""
    return {"workload": f"double shear layer {L}x{L}, Ma={MA}, nu={NU}, {S} steps per lattice, "
                        f"8 collision models (BGK, RM, HM, CM, CHM, K, PR, RR), FP32 shifted storage",
            "lattices": len(MODELS), "lattice": f"{L}x{L}", "sim_steps": S,
            "check_every": CHECK_EVERY, "graph_steps": GRAPH_STEPS,
            "l2": "inputs larger than L2: 8 lattices x 75.5 MB advanced in turn each time step",
            "parallelism": f"replicas x{world}" if world > 1 else "single GPU"}


def run_reference(args, rank, world):
    if rank != 0:
        return
    pool, procs = oracle_pool()
    try:
        oracle_round(pool)   # worker start-up outside the timing
        for _ in range(args.warmup):
            oracle_round(pool)
        t0 = time.perf_counter()
        lu = 0
        for _ in range(args.steps):
            lu += oracle_round(pool)
        dt = time.perf_counter() - t0
    finally:
        pool.shutdown()
    v = lu / dt / 1e9
    # single-process figures beside it: one time step per model on the same lattice, and the
    # 128 x 128 vortex (BGK, FP64, 1000 steps) run in full
    import oracle.lbm as olbm
    from paper_2002_05265_gb300 import flows
    f0 = olbm.init_equilibrium(*flows.double_shear_layer(L, Ma=MA))
    per_model = {}
    for m in MODELS:
        t0 = time.perf_counter()
        olbm.step(f0, m, olbm.rates_from_nu(NU, _preset(m)))
        per_model[m] = L * L / (time.perf_counter() - t0) / 1e6
    vf = flows.vortex(128, Ma=0.1, noise=1e-8, seed=1)
    t0 = time.perf_counter()
    olbm.run(olbm.init_equilibrium(*vf), "bgk", olbm.rates_from_nu(1e-4, "srt"), 1000)
    vortex_s = time.perf_counter() - t0
    out = {"impl": "reference", "metric": METRIC,
           "value": v, "unit": "GLUPS", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": bench_config(args.sim_steps, world),
           "cpu_baseline": {"value": v, "unit": "GLUPS", "cores": procs, "host_cores": os.cpu_count(), "kind": "oracle",
                            "sample": "each benchmark step a bounded sample of the workload: one time step of "
                                      f"each of the 8 models on its {L}x{L} lattice (not {args.sim_steps}), "
                                      f"as {len(ORACLE_TASKS)} (model, {CPU_SLAB}-row slab + halo) tasks over "
                                      f"{procs} single-threaded numpy processes"},
           "e2e": {"value": v, "unit": "GLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
           "single_process": {"per_model_mlups_1024": per_model, "vortex_128_bgk_1000_steps_seconds": vortex_s}}
    print(json.dumps(out))


MAP_CONFIGS = ([("bgk", "srt")] + [(m, c) for m in ("rm", "hm", "cm", "chm", "k", "rr") for c in ("srt", "reg")]
               # the two alternative readings of the cumulant rebuild (pre-collision / equilibrium)
               + [(m, c) for m in ("k_pre", "k_eq") for c in ("srt", "reg")])


def run_stability_map(args):
    """Numerical stability maps of the convected vortex (Sec. 5b): for every collision model in
    both rate presets (SRT: omega_3 = omega_4 = omega_nu; REG: omega_3 = omega_4 = 1), every
    viscosity nu in 1e-6 .. 1e-1 (half decades) and Mach number Ma in 0.05 .. 0.8, an LxL
    vortex (beta = 0.5, R = L/20, centred) is advanced for M t_c = M L / u0 steps in the batched
    persistent launch; an instance is unstable when its mean kinetic energy <|u|^2> exceeds
    its initial value by more than 1% at a check (every 100 steps; the kinetic energy of this
    flow only decays, an instability grows it exponentially), or rho / u turn non-finite.  Prints one
    JSON line per (model, preset, nu) with the stable Mach numbers and the largest Ma below
    which every tested Ma is stable (the stability curve of the paper's figures)."""
    import torch
    from paper_2002_05265_gb300 import build, flows, lbm
    build.build_library()
    lbm.load_library()
    n = args.stability_map
    nus = [float(v) for v in np.logspace(-6, -1, 11)]
    mas = [round(0.05 * k, 2) for k in range(1, 17)]
    stream = torch.cuda.Stream()
    stable = {}   # (model, preset, nu) -> {Ma: bool}
    t_all, lu_all = 0.0, 0.0
    for Ma in mas:
        u0 = Ma * CS
        steps = int(np.ceil(args.map_tc * n / u0 / CHECK_EVERY)) * CHECK_EVERY
        rho, ux, uy = flows.vortex(n, Ma=Ma, radius_frac=0.05)
        ke0 = float(np.mean(ux * ux + uy * uy))
        descs = []
        for m, preset in MAP_CONFIGS:
            for nu in nus:
                w = 1.0 / (3.0 * nu + 0.5)
                rates = (w, w, w) if preset == "srt" else (w, 1.0, 1.0)
                descs.append({"nx": n, "ny": n, "model": m, "rates": rates, "ux_ref": u0, "uy_ref": 0.0,
                              "ke_ref": ke0, "ke_factor": 1.01})
        b = lbm.lbm_batch_create(descs, storage=args.map_storage, stream=stream)
        cat = [torch.from_numpy(np.ascontiguousarray(np.tile(a.ravel(), len(descs)))).cuda() for a in (rho, ux, uy)]
        lbm.lbm_batch_init_equilibrium(b, *cat)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            e0.record(stream)
            lbm.lbm_batch_run(b, steps, check_every=CHECK_EVERY, growth=1e300)
            e1.record(stream)
            stream.synchronize()
        t_all += e0.elapsed_time(e1) / 1e3
        st, bs, done, _ = lbm.lbm_batch_status(b, len(descs))
        lu_all += float(sum(int(x) for x in done)) * n * n
        lbm.lbm_batch_destroy(b)
        k = 0
        for m, preset in MAP_CONFIGS:
            for nu in nus:
                stable.setdefault((m, preset, nu), {})[Ma] = bool(st[k] == 0)
                k += 1
    for (m, preset, nu), res in stable.items():
        ma_max = 0.0
        for Ma in mas:
            if not res[Ma]:
                break
            ma_max = Ma
        print(json.dumps({"stability_map": True, "lattice": f"{n}x{n}", "tc": args.map_tc, "model": m,
                          "preset": preset, "nu": nu, "ma_max": ma_max,
                          "stable_ma": [Ma for Ma in mas if res[Ma]], "storage": args.map_storage}), flush=True)
    print(json.dumps({"stability_map_summary": True, "lattice": f"{n}x{n}", "instances": len(stable) * len(mas),
                      "lattice_updates": lu_all, "seconds": t_all, "glups": lu_all / t_all / 1e9}), flush=True)


def vorticity(ux, uy):
    """omega_z = d uy/dx - d ux/dy by periodic central differences (arrays [y][x])."""
    return 0.5 * ((np.roll(uy, -1, 1) - np.roll(uy, 1, 1)) - (np.roll(ux, -1, 0) - np.roll(ux, 1, 0)))


def run_transport(args):
    """Vortex transport over long distances (Sec. 5c): Ma = 0.5, nu = 1e-4, beta = 0.5,
    R = L/20, 50 t_c = 50 L / u0 steps (the exact solution is the initial vortex moved by 50 L,
    i.e. back at its start), FP32, for the most stable models SRT-RR, REG-CHM and REG-K.
    Reports per model: normalised L2 error of the vorticity against the initial field
    (normalised by its max - min, as in the paper's figures), the peak-vorticity ratio
    (dissipation), the shift of the vorticity-weighted centre from the start (dispersion),
    and the difference between REG-CHM and SRT-RR."""
    import torch
    from paper_2002_05265_gb300 import build, flows, lbm
    build.build_library()
    lbm.load_library()
    n = args.transport
    Ma, nu = 0.5, 1e-4
    u0 = Ma * CS
    steps = int(round(50 * n / u0))
    steps += steps % 2
    rho, ux, uy = flows.vortex(n, Ma=Ma, radius_frac=0.05)
    w0 = vorticity(ux, uy)
    span = float(w0.max() - w0.min())
    dev = [torch.from_numpy(a).cuda() for a in (rho, ux, uy)]
    w = 1.0 / (3.0 * nu + 0.5)
    y, x = np.meshgrid(np.arange(n, dtype=float), np.arange(n, dtype=float), indexing="ij")

    def centre(om):
        a = np.abs(om - np.median(om))
        # circular mean of the position (periodic domain)
        cx = np.angle(np.sum(a * np.exp(2j * np.pi * x / n))) * n / (2 * np.pi) % n
        cy = np.angle(np.sum(a * np.exp(2j * np.pi * y / n))) * n / (2 * np.pi) % n
        return cx, cy

    c0 = centre(w0)
    out = {}
    for name, m, rates in (("SRT-RR", "rr", (w, w, w)), ("REG-CHM", "chm", (w, 1.0, 1.0)), ("REG-K", "k", (w, 1.0, 1.0))):
        lat = lbm.Lattice(n, n, lbm.MODELS[m], rates, storage=lbm.LBM_F32)
        lat.set_shift_velocity(u0, 0.0)
        lat.init_equilibrium(*dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        lat.step(steps)
        e1.record()
        torch.cuda.synchronize()
        st = lat.status()[0]
        gx = torch.empty((n, n), dtype=torch.float64, device="cuda")
        gy = torch.empty_like(gx)
        lat.moments(None, gx, gy)
        lat.close()
        om = vorticity(gx.cpu().numpy(), gy.cpu().numpy())
        c = centre(om)
        dx = (c[0] - c0[0] + n / 2) % n - n / 2
        dy = (c[1] - c0[1] + n / 2) % n - n / 2
        out[name] = om
        print(json.dumps({"transport": True, "model": name, "lattice": f"{n}x{n}", "steps": steps, "status": st,
                          "l2_vorticity_error": float(np.sqrt(np.mean((om - w0) ** 2)) / span),
                          "peak_ratio": float((om.max() - om.min()) / span),
                          "centre_shift": [float(dx), float(dy)], "ms": e0.elapsed_time(e1),
                          "glups": n * n * steps / (e0.elapsed_time(e1) / 1e3) / 1e9}), flush=True)
    d = float(np.sqrt(np.mean((out["REG-CHM"] - out["SRT-RR"]) ** 2)) / span)
    print(json.dumps({"transport_summary": True, "lattice": f"{n}x{n}", "reg_chm_vs_srt_rr_l2": d}))


def run_lsa_map(args):
    """Linear stability curves of the stream-and-collide scheme (Sec. 4c, App. A): for every
    model in both rate presets (and BGK with the second-order and partial third-order
    equilibria) and nu in 1e-6 .. 1e-1, the largest Mach number (bisection to
    1e-3) for which no plane wave grows, max over a K x K wavenumber grid on [-pi, pi]^2 and 16
    mean-flow angles phi in [0, pi/4] (the D2Q9 symmetries cover the rest) of
    Im(omega) <= 1e-10 (the conserved modes at k = 0 have exactly 0).  Uses lbm_lsa_growth (the
    exact Jacobian of this library's collision, FP64 eigenvalues on the GPU)."""
    import torch
    from paper_2002_05265_gb300 import build, lbm
    build.build_library()
    lbm.load_library()
    K = args.lsa
    k1 = np.linspace(-np.pi, np.pi, K)
    ks = torch.from_numpy(np.array([(a, b) for a in k1 for b in k1])).cuda()
    phis = np.linspace(0.0, np.pi / 4.0, 16)
    nus = [float(v) for v in np.logspace(-6, -1, 11)]
    growth = torch.empty((len(phis), K * K), dtype=torch.float64, device="cuda")
    calls, t0 = 0, time.perf_counter()

    def unstable(m, rates, ma, eq_order):
        u = ma * CS
        fl = torch.from_numpy(np.stack([np.ones_like(phis), u * np.cos(phis), u * np.sin(phis)], axis=1)).cuda()
        lbm.lbm_lsa_growth(m, rates, fl, ks, growth, eq_order=eq_order)
        return float(growth.max()) > 1e-10

    # BGK with the second-order and partial third-order equilibria first (the lattice
    # counterpart of Fig. 4's three truncations), then every model with the extended one
    configs = [("bgk", "srt", 2), ("bgk", "srt", 3)] + [(m, c, 4) for m, c in MAP_CONFIGS]
    for m, preset, eq_order in configs:
        for nu in nus:
            w = 1.0 / (3.0 * nu + 0.5)
            rates = (w, w, w) if preset == "srt" else (w, 1.0, 1.0)
            if unstable(m, rates, 0.0, eq_order):
                ma_max = 0.0
            else:
                lo, hi = 0.0, 1.0
                while hi - lo > 1e-3:
                    mid = 0.5 * (lo + hi)
                    if unstable(m, rates, mid, eq_order):
                        hi = mid
                    else:
                        lo = mid
                    calls += 1
                ma_max = lo
            calls += 1
            print(json.dumps({"lsa": True, "model": m, "preset": preset, "eq_order": eq_order, "nu": nu,
                              "ma_max": round(ma_max, 4), "k_grid": K, "angles": len(phis)}), flush=True)
    dt = time.perf_counter() - t0
    print(json.dumps({"lsa_summary": True, "calls": calls, "matrices": calls * len(phis) * K * K, "seconds": dt}))
    # Fig. 7 (right): BGK at Ma = 0.1 along x, nu = 1e-5, growth-rate map over k in [0, pi]^2
    # (512 x 512), per equilibrium order: the largest growth rate and where it is
    k2 = np.linspace(0.0, np.pi, 512)
    kk = torch.from_numpy(np.array([(a, b) for a in k2 for b in k2])).cuda()
    g2 = torch.empty((1, kk.shape[0]), dtype=torch.float64, device="cuda")
    w = 1.0 / (3.0 * 1e-5 + 0.5)
    fl = torch.tensor([[1.0, 0.1 * CS, 0.0]], dtype=torch.float64, device="cuda")
    for eq_order in (2, 3, 4):
        lbm.lbm_lsa_growth("bgk", (w, w, w), fl, kk, g2, eq_order=eq_order)
        i = int(torch.argmax(g2))
        print(json.dumps({"lsa_fig7": True, "model": "bgk", "eq_order": eq_order, "Ma": 0.1, "nu": 1e-5,
                          "max_growth": float(g2.max()), "at_k": [float(kk[i, 0]), float(kk[i, 1])],
                          "unstable_fraction": float((g2 > 1e-10).double().mean())}))


def run_accuracy(args):
    """`--accuracy L`: storage_accuracy on an L x L lattice, one JSON line per record."""
    from paper_2002_05265_gb300 import build, lbm
    build.build_library()
    lbm.load_library()
    for r in storage_accuracy(lbm, args.accuracy):
        print(json.dumps(dict(accuracy=True, **r)), flush=True)


def run_sweep(args):
    """Single-lattice throughput per model x storage on the convected vortex (Ma = 0.2,
    nu = 1e-6): `--steps` timed time steps after `--warmup`, CUDA events around the graph
    replays of the step kernel only."""
    import torch
    from paper_2002_05265_gb300 import build, flows, lbm
    build.build_library()
    lbm.load_library()
    ms, st, size = args.sweep.split(":")
    models = MODELS if ms == "all" else ms.split(",")
    storages = st.split(",")
    n = int(size)
    stream = torch.cuda.Stream()
    fields = [torch.from_numpy(a).cuda() for a in flows.vortex(n, Ma=0.2, noise=1e-8, seed=3)]
    for s in storages:
        for m in models:
            rates = lbm.lbm_rates_from_nu(1e-6, lbm.LBM_PRESET_SRT if _preset(m) == "srt" else lbm.LBM_PRESET_REG)
            lat = lbm.Lattice(n, n, lbm.MODELS[m], rates, storage=lbm.STORAGES[s], stream=stream)
            shape_lattice(lat, args)
            lat.init_equilibrium(*fields)
            # graphs of 16 steps (room for multi-step launches); counts rounded to whole graphs
            g = lbm.lbm_group_create([lat.ctx], graph_steps=16)
            lbm.lbm_group_step(g, 16 * max(1, -(-args.warmup // 16)), lat.ctx)
            lbm.lbm_group_set_timing(g, True)
            lbm.lbm_group_step(g, 16 * max(1, args.steps // 16), lat.ctx)
            rms, nl, _ = lbm.lbm_group_timing(g)
            t = rms / 1e3 / nl
            print(json.dumps({"sweep": True, "model": m, "storage": s, "path": args.path, "stages": args.stages,
                              "launch_steps": args.launch_steps, "order": args.order,
                              "lattice": f"{n}x{n}", "steps": nl,
                              "glups": n * n / t / 1e9, "gbs": BYTES_PER_LU[s] * n * n / t / 1e9,
                              "ms_per_step": t * 1e3}), flush=True)
            lbm.lbm_group_destroy(g)
            lat.close()
            torch.cuda.synchronize()


def run_slab(args, rank, world):
    """One L x L lattice -- the convected vortex at Ma = 0.2, nu = 1e-6, CHM with REG rates --
    split into `world` y-slabs (one per rank, each with two ghost rows), advanced one step at a
    time with the halo exchange of the xi_y = +-1 populations after every step (NCCL point to
    point between neighbouring ranks; one rank exchanges with itself across the periodic
    boundary).  `--steps` timed steps after `--warmup`, CUDA events on every rank, max over
    ranks; value = L^2 x steps / time (strong scaling: the lattice is fixed)."""
    import torch
    from paper_2002_05265_gb300 import build, flows, lbm, slab
    if rank == 0 or world == 1:
        build.build_library()
    barrier(world)
    lbm.load_library()
    n = args.slab
    rates = lbm.lbm_rates_from_nu(1e-6, lbm.LBM_PRESET_REG)
    sl = slab.SlabLattice(n, n, lbm.LBM_CHM, rates, args.slab_storage, rank, world)
    # local rows (ghosts included) generated slab by slab of contiguous global rows
    loc = [torch.empty((len(sl.rows), n), dtype=torch.float64, device="cuda") for _ in range(3)]
    r0 = 0
    while r0 < len(sl.rows):
        r1 = r0
        while r1 + 1 < len(sl.rows) and sl.rows[r1 + 1] == sl.rows[r1] + 1 and r1 + 1 - r0 < 1024:
            r1 += 1
        for t, a in zip(loc, flows.vortex(n, Ma=0.2, rows=(int(sl.rows[r0]), int(sl.rows[r1]) + 1))):
            t[r0:r1 + 1].copy_(torch.from_numpy(a))
        r0 = r1 + 1
    sl.init_equilibrium_local(*loc)
    del loc
    sl.step(args.warmup)
    torch.cuda.synchronize()
    barrier(world)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    sl.step(args.steps)
    e1.record()
    torch.cuda.synchronize()
    ms = max_over_ranks(e0.elapsed_time(e1), world)
    st = sl.lat.status()[0]
    sl.close()
    if rank == 0:
        v = n * n * args.steps / (ms / 1e3) / 1e9
        print(json.dumps({"slab": True, "metric": "D2Q9 lattice updates per second, one lattice in y-slabs",
                          "value": v, "unit": "GLUPS", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                          "ms_per_step": ms / args.steps, "scaling": "strong", "storage": args.slab_storage,
                          "status": st, "alg_gbs": v * BYTES_PER_LU[args.slab_storage],
                          "config": {"workload": f"convected vortex {n}x{n}, Ma=0.2, nu=1e-6, CHM REG, "
                                                 f"{world} y-slab(s), halo exchange every step"}}))


def shard(items, rank, world):
    """Instances of the batched sweep owned by one rank: every world-th instance (the
    instances are independent, so ranks share nothing but the final timing reduction)."""
    return items[rank::world]


def batch_workload(n, seed=4):
    """The batched stability sweep: n lattices, nx, ny ~ U{32..256} independently, model
    uniform over the 8 models, preset uniform over SRT/REG, Ma ~ U[0, 0.6] along +x,
    nu log-uniform in [1e-7, 1e-2], rho = 1, u = (Ma c_s, 0) + U(-1e-6, 1e-6) noise."""
    from paper_2002_05265_gb300 import flows
    g = np.random.Generator(np.random.Philox(seed))
    descs, fields = [], []
    cs = 1.0 / np.sqrt(3.0)
    for k in range(n):
        nx, ny = (int(v) for v in g.integers(32, 257, 2))
        m = MODELS[int(g.integers(0, len(MODELS)))]
        preset = "srt" if g.integers(0, 2) == 0 else "reg"
        Ma = float(g.uniform(0.0, 0.6))
        nu = float(np.exp(g.uniform(np.log(1e-7), np.log(1e-2))))
        w = 1.0 / (nu * 3.0 + 0.5)
        rates = (w, w, w) if preset == "srt" else (w, 1.0, 1.0)
        descs.append(dict(nx=nx, ny=ny, model=m, preset=preset, Ma=Ma, nu=nu, rates=rates,
                          ux_ref=Ma * cs, uy_ref=0.0))
        fields.append(flows.uniform_noise(nx, ny, Ma=Ma, amp=1e-6, seed=10000 + k))
    return descs, fields


def batch_measure(lbm, instances, batch_steps, rank=0, world=1, subset=256, peak=None):
    """Batched stability sweep throughput (one persistent launch in a CUDA graph) against
    the plain per-lattice FP32 kernel on a `subset`-instance sample (1000 steps each, one
    context and graph each).  With several ranks the instances are sharded (weak scaling, no
    collective but the timing maximum)."""
    import torch
    descs, fields = batch_workload(instances)
    descs, fields = shard(descs, rank, world), shard(fields, rank, world)
    stream = torch.cuda.Stream()
    b = lbm.lbm_batch_create(descs, storage=lbm.LBM_F32, stream=stream)
    cat = [torch.from_numpy(np.ascontiguousarray(np.concatenate([f[i].ravel() for f in fields]))).cuda()
           for i in range(3)]
    nodes = lbm.lbm_batch_nodes(b)
    lbm.lbm_batch_init_equilibrium(b, *cat)
    vec, block, trial_ms = lbm.lbm_batch_autotune(b, trial_steps=200, check_every=CHECK_EVERY)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        ev0.record(stream)
        lbm.lbm_batch_run(b, batch_steps, check_every=CHECK_EVERY, growth=1e4)
        ev1.record(stream)
        stream.synchronize()
    ms = ev0.elapsed_time(ev1)
    st, bs, steps, diag = lbm.lbm_batch_status(b, len(descs))
    lu = float(sum(int(s) * d["nx"] * d["ny"] for s, d in zip(steps, descs)))
    stable = {}
    for d, s in zip(descs, st):
        key = f'{d["preset"]}-{d["model"]}'
        a = stable.setdefault(key, [0, 0])
        a[0] += int(s == 0)
        a[1] += 1
    sub = list(range(0, len(descs), max(1, len(descs) // subset)))[:subset]
    lu_sub, t_sub = 0.0, 0.0
    with torch.cuda.stream(stream):
        for k in sub:
            d = descs[k]
            lat = lbm.Lattice(d["nx"], d["ny"], lbm.MODELS[d["model"]], d["rates"], storage=lbm.LBM_F32, stream=stream)
            lat.set_shift_velocity(d["ux_ref"], 0.0)
            lat.init_equilibrium(*[torch.from_numpy(a).cuda() for a in fields[k]])
            lat.step(64)
            stream.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            lat.step(1000)
            e1.record(stream)
            stream.synchronize()
            t_sub += e0.elapsed_time(e1) / 1e3
            lu_sub += 1000.0 * d["nx"] * d["ny"]
            lat.close()
    lbm.lbm_batch_destroy(b)
    glups = lu / (ms / 1e3) / 1e9
    per_inst = lu_sub / t_sub / 1e9
    out = {"metric": "batched stability sweep, lattice updates per second", "unit": "GLUPS",
           "value": glups, "instances": len(descs), "nodes": nodes, "target_steps": batch_steps,
           "lattice_updates": lu, "ms": ms, "shape": {"vec": vec, "block": block, "trial_ms": trial_ms},
           "stable_instances": int((st == 0).sum()), "blown_up": int((st != 0).sum()),
           "stable_by_model": {k: f"{v[0]}/{v[1]}" for k, v in sorted(stable.items())},
           "per_instance_kernel_glups": per_inst, "speedup_vs_per_instance": glups / per_inst,
           "per_instance_subset": f"{len(sub)} instances x 1000 steps, one context and graph each",
           "dtype": "f32", "data": "synthetic"}
    if peak:
        # a CTA advances one instance (<= 4.7 MB for both FP32 buffers) for many steps, so the
        # instances live in the L2: this is algorithmic bytes over the HBM copy bandwidth, not
        # an HBM fraction
        out["algorithmic_gbs"] = glups * BYTES_PER_LU["f32"]
        out["algorithmic_over_hbm_peak_l2_resident"] = glups * BYTES_PER_LU["f32"] / peak
    return out


def run_batch(args, rank=0, world=1):
    """`--batch`: the full batched stability sweep (default 4096 lattices, 50000 steps)."""
    from paper_2002_05265_gb300 import build, lbm
    build.build_library()
    lbm.load_library()
    out = batch_measure(lbm, args.instances, args.batch_steps, rank, world, peak=measured_peaks()[0])
    print(json.dumps(dict(batch=True, **out)))


def main():
    args = parse()
    rank, world, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.sweep:
        run_sweep(args)
        return
    if args.batch:
        run_batch(args, rank, world)
        return
    if args.accuracy:
        run_accuracy(args)
        return
    if args.stability_map:
        run_stability_map(args)
        return
    if args.lsa:
        run_lsa_map(args)
        return
    if args.transport:
        run_transport(args)
        return
    if args.slab:
        run_slab(args, rank, world)
        return
    import torch
    from paper_2002_05265_gb300 import build, flows, lbm
    if rank == 0 or world == 1:
        build.build_library()
    barrier(world)
    lbm.load_library()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")

    stream = torch.cuda.Stream()
    fields = flows.double_shear_layer(L, Ma=MA)
    dev_fields = [torch.from_numpy(a).cuda() for a in fields]
    host_fields = [torch.from_numpy(a).pin_memory() for a in fields]
    lats = []
    for m in MODELS:
        rates = lbm.lbm_rates_from_nu(NU, lbm.LBM_PRESET_SRT if _preset(m) == "srt" else lbm.LBM_PRESET_REG)
        lat = lbm.Lattice(L, L, lbm.MODELS[m], rates, storage=lbm.LBM_F32, stream=stream)
        shape_lattice(lat, args)
        lat.set_check(CHECK_EVERY)
        lats.append(lat)
    group = lbm.lbm_group_create([x.ctx for x in lats], graph_steps=GRAPH_STEPS)
    out_dev = [[torch.empty((L, L), dtype=torch.float64, device="cuda") for _ in range(3)] for _ in MODELS]
    out_host = [[torch.empty((L, L), dtype=torch.float64).pin_memory() for _ in range(3)] for _ in MODELS]

    S = args.sim_steps

    def bench_step(fields_in, outs):
        for lat in lats:
            lat.init_equilibrium(*fields_in)
        lbm.lbm_group_step(group, S, lats[0].ctx)
        for lat, o in zip(lats, outs):
            lat.moments(o[0], o[1], o[2])

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            bench_step(dev_fields, out_dev)
        stream.synchronize()
        barrier(world)
        torch.cuda.synchronize()
        clocks = ClockSampler(local)
        clocks.start()
        lbm.lbm_group_set_timing(group, True)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(args.steps):
            bench_step(dev_fields, out_dev)
        ev1.record(stream)
        stream.synchronize()
        clock_info = clocks.stop()
        barrier(world)
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1)
        replay_ms, lattice_steps, kernel_launches = lbm.lbm_group_timing(group)
        lbm.lbm_group_set_timing(group, False)
    ms = max_over_ranks(ms, world)
    statuses = {m: lat.status()[:2] for m, lat in zip(MODELS, lats)}

    lu_per_step = len(MODELS) * L * L * S
    value = world * lu_per_step * args.steps / (ms / 1e3) / 1e9

    # dominant kernel: the multi-lattice step kernel (one launch advances the 8 lattices one
    # time step); average launch duration from the CUDA events around every graph replay of
    # the timed region (the graphs contain only step launches)
    peak, peak_kind = measured_peaks()
    avg_launch_s = replay_ms / 1e3 / kernel_launches
    bytes_per_launch = BYTES_PER_LU["f32"] * L * L * lattice_steps / kernel_launches
    achieved = bytes_per_launch / avg_launch_s / 1e9
    form = form_name(lbm, group)
    bulk = form != "register-staged"
    # the committed ncu traffic records: the wide form (the default here) and the
    # register-staged group kernel
    traffic = ncu_traffic("f32_tile_8x1024") if form == "wide" else (
        ncu_traffic("f32_group_8x1024") if not bulk else None)
    kname = (f"lbm::tile_step_kernel<float> (cp.async.bulk ring, {form} form)" if bulk
             else "lbm::group_step_kernel<float> (register-staged)")
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "peak_source": peak_kind, "launch_us": avg_launch_s * 1e6,
                "bytes_per_launch": bytes_per_launch,
                "kernel": kname + f": one launch = {lattice_steps // kernel_launches // len(MODELS)} time step(s) "
                          "of the 8 lattices, 72 B per lattice update"}

    # step-kernel launches counted by the group's replay timing, plus one reduction launch per
    # check of the eight lattices (they fall due together and share a launch; each lattice's
    # last block folds its partials), and per lattice the equilibrium init and the moments
    # gather
    launches_per_step = kernel_launches // args.steps + S // CHECK_EVERY + 2 * len(MODELS)

    e2e = None
    if not args.no_e2e:
        with torch.cuda.stream(stream):
            barrier(world)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(args.steps):
                bench_step(host_fields, out_host)
            stream.synchronize()
            dt = time.perf_counter() - t0
            barrier(world)
        dt = max_over_ranks(dt, world)
        e2e = {"value": world * lu_per_step * args.steps / dt / 1e9, "unit": "GLUPS",
               "h2d_bytes_per_step": len(MODELS) * 3 * L * L * 8,
               "d2h_bytes_per_step": len(MODELS) * 3 * L * L * 8}

    per_model = None
    if not args.no_per_model:
        per_model = per_model_big(lbm, stream, peak)

    batch = None
    if not args.no_batch_key:
        batch = batch_measure(lbm, 4096, 5000, peak=peak)

    accuracy = None
    if not args.no_accuracy_key:
        accuracy = accuracy_table(lbm, 256)

    adjoint = None
    if not args.no_adjoint:
        adjoint = adjoint_ratio(lbm, flows, stream, PATHS[args.path], args.stages)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline()

    if rank == 0:
        out = {"metric": METRIC,
               "value": value, "unit": "GLUPS", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
               "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
               "vs_baseline": None, "dtype": "f32", "data": "synthetic",
               "config": bench_config(S, world),
               "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clock_info,
               "gpu_launches": launches_per_step * args.steps,
               "blowup": {m: (s[1] if s[0] != 0 else None) for m, s in statuses.items()}}
        if per_model:
            out["per_model_16384"] = per_model
        if batch:
            out["batch"] = batch
        if accuracy:
            out["storage_accuracy"] = accuracy
        if adjoint:
            out["adjoint"] = adjoint
        print(json.dumps(out))

    lbm.lbm_group_destroy(group)
    for lat in lats:
        lat.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
