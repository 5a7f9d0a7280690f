"""The JSON line of `bench.py --impl reference` (the FP64 oracle timed on the host cores), run
on the CPU: one line, the keys of the benchmark contract, the same metric, unit and config
as the GPU arm, and a cpu_baseline that describes the bounded sample it timed."""

import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [x for x in r.stdout.splitlines() if x.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    sys.path.insert(0, ROOT)
    import bench
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == "GLUPS" and d["higher_is_better"] is True
    assert d["config"] == bench.bench_config(bench.SIM_STEPS, 1)
    assert d["value"] > 0 and d["steps"] == 1 and d["warmup"] == 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "GLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_oracle_row_slabs_reproduce_a_whole_lattice_step():
    """The CPU baseline spreads each oracle time step over the host cores as row slabs with one
    halo row on each side; the slabs' rows together equal one oracle step of the whole lattice."""
    import numpy as np
    sys.path.insert(0, ROOT)
    import bench
    import oracle.lbm as olbm
    from paper_2002_05265_gb300 import flows
    f = olbm.init_equilibrium(*flows.double_shear_layer(48, 40, Ma=0.2, width_frac=0.1))
    f = f * (1 + flows.random_populations_perturbation(f.shape, 1e-3, seed=5))
    for model in ("bgk", "k", "rr"):
        rates = olbm.rates_from_nu(1e-3, "reg")
        whole = olbm.step(f, model, rates)
        slabs = np.concatenate([bench.oracle_slab_step(f, model, rates, y0, 8) for y0 in range(0, 40, 8)], axis=1)
        np.testing.assert_array_equal(slabs, whole)


def test_transport_vorticity_is_the_periodic_central_difference():
    """bench.vorticity (the Sec. 5c vorticity error metric): for u = (-sin(ky y), sin(kx x)) the
    periodic central differences give exactly omega = sin(kx) cos(kx x) + sin(ky) cos(ky y)
    (the discrete counterpart of kx cos(kx x) + ky cos(ky y))."""
    import numpy as np
    sys.path.insert(0, ROOT)
    import bench
    ny, nx = 48, 64
    kx, ky = 2 * np.pi * 3 / nx, 2 * np.pi * 2 / ny
    y, x = np.meshgrid(np.arange(ny, dtype=float), np.arange(nx, dtype=float), indexing="ij")
    om = bench.vorticity(-np.sin(ky * y), np.sin(kx * x))
    np.testing.assert_allclose(om, np.sin(kx) * np.cos(kx * x) + np.sin(ky) * np.cos(ky * y), atol=1e-13)
