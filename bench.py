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
    p.add_argument("--per-model", action="store_true", help="also time each model alone on 4096^2")
    return p.parse_args()


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


def ncu_traffic(kernel_tag):
    """Per-launch DRAM bytes of the step kernel from the committed ncu summary, if it was
    taken on the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "step_kernel_traffic.json")
    if not os.path.exists(path):
        return None
    d = json.load(open(path))
    import hashlib
    src = os.path.join(ROOT, "paper_2002_05265_gb300", "csrc", "lbm_device.cuh")
    h = hashlib.sha256(open(src, "rb").read()).hexdigest()
    e = d.get(kernel_tag)
    if not e or d.get("kernel_source_sha256") != h:
        return None
    return e.get("dram_bytes_per_launch_full_size")


def cpu_baseline(n_models=len(MODELS)):
    """FP64 oracle as it stands, one time step of each collision model on the 1024 x 1024
    double shear layer, on this host's cores (numpy runs it single-threaded)."""
    import oracle.lbm as olbm
    from paper_2002_05265_gb300 import flows
    fields = flows.double_shear_layer(L, Ma=MA)
    f0 = olbm.init_equilibrium(*fields)
    t0 = time.perf_counter()
    for m in MODELS[:n_models]:
        olbm.step(f0, m, olbm.rates_from_nu(NU, _preset(m)))
    dt = time.perf_counter() - t0
    lu = n_models * L * L
    return {"value": lu / dt / 1e9, "unit": "GLUPS", "cores": 1, "kind": "oracle",
            "sample": f"one time step of each of {n_models} models on the {L}x{L} double shear layer "
                      f"({lu} lattice updates, {dt:.1f} s), numpy FP64 single-threaded"}


def run_reference(args, rank, world):
    if rank != 0:
        return
    import oracle.lbm as olbm
    from paper_2002_05265_gb300 import flows
    fields = flows.double_shear_layer(L, Ma=MA)
    f0 = olbm.init_equilibrium(*fields)

    def one():
        for m in MODELS:
            olbm.step(f0, m, olbm.rates_from_nu(NU, _preset(m)))
    for _ in range(args.warmup):
        one()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        one()
    dt = time.perf_counter() - t0
    lu = args.steps * len(MODELS) * L * L
    v = lu / dt / 1e9
    out = {"impl": "reference", "metric": "D2Q9 lattice updates per second, 8 collision models",
           "value": v, "unit": "GLUPS", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": f"double shear layer {L}x{L}, 8 models, one time step per model per step "
                                  f"(bounded sample of the {args.sim_steps}-step run)",
                      "lattice": f"{L}x{L}", "models": MODELS},
           "cpu_baseline": {"value": v, "unit": "GLUPS", "cores": 1, "kind": "oracle",
                            "sample": "one time step of each of the 8 models per benchmark step"},
           "e2e": {"value": v, "unit": "GLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def main():
    args = parse()
    rank, world, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, rank, world)
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
        replay_ms, step_launches = lbm.lbm_group_timing(group)
        lbm.lbm_group_set_timing(group, False)
    ms = max_over_ranks(ms, world)
    statuses = {m: lat.status()[:2] for m, lat in zip(MODELS, lats)}

    lu_per_step = len(MODELS) * L * L * S
    value = world * lu_per_step * args.steps / (ms / 1e3) / 1e9

    # dominant kernel: the fused step kernel (all models); average launch duration from the
    # CUDA events around every graph replay of the timed region
    peak, peak_kind = measured_peaks()
    avg_launch_s = replay_ms / 1e3 / step_launches
    achieved = BYTES_PER_LU["f32"] * L * L / avg_launch_s / 1e9
    traffic = ncu_traffic("f32_1024")
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "peak_source": peak_kind,
                "kernel": "lbm::step_kernel<model, 4, float> (8 models), 72 B per lattice update"}

    launches_per_step = len(MODELS) * (1 + S + 2 * (S // CHECK_EVERY) + 1)

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
    if args.per_model:
        per_model = {}
        for m in MODELS:
            rates = lbm.lbm_rates_from_nu(NU, lbm.LBM_PRESET_SRT if _preset(m) == "srt" else lbm.LBM_PRESET_REG)
            big = lbm.Lattice(4096, 4096, lbm.MODELS[m], rates, storage=lbm.LBM_F32, stream=stream)
            f4 = flows.double_shear_layer(4096, Ma=MA)
            big.init_equilibrium(*[torch.from_numpy(a).cuda() for a in f4])
            g1 = lbm.lbm_group_create([big.ctx], graph_steps=32)
            lbm.lbm_group_step(g1, 64, big.ctx)
            lbm.lbm_group_set_timing(g1, True)
            lbm.lbm_group_step(g1, 256, big.ctx)
            rms, nl = lbm.lbm_group_timing(g1)
            t = rms / 1e3 / nl
            per_model[m] = {"glups": 4096 * 4096 / t / 1e9, "gbs": 72 * 4096 * 4096 / t / 1e9}
            lbm.lbm_group_destroy(g1)
            big.close()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline()

    if rank == 0:
        out = {"metric": "D2Q9 lattice updates per second, 8 collision models (GLUPS)",
               "value": value, "unit": "GLUPS", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
               "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
               "vs_baseline": None, "dtype": "f32", "data": "synthetic",
               "config": {"workload": f"double shear layer {L}x{L}, Ma={MA}, nu={NU}, {S} steps per lattice, "
                                      f"8 collision models (BGK, RM, HM, CM, CHM, K, PR, RR), FP32 shifted storage",
                          "lattices": len(MODELS), "lattice": f"{L}x{L}", "sim_steps": S,
                          "check_every": CHECK_EVERY, "graph_steps": GRAPH_STEPS,
                          "l2": "inputs larger than L2: 8 lattices x 75.5 MB advanced in turn each time step",
                          "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
               "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clock_info,
               "gpu_launches": launches_per_step * args.steps,
               "blowup": {m: (s[1] if s[0] != 0 else None) for m, s in statuses.items()}}
        if per_model:
            out["per_model_4096_f32"] = per_model
        print(json.dumps(out))

    lbm.lbm_group_destroy(group)
    for lat in lats:
        lat.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
