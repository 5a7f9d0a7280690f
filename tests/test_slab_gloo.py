"""The y-slab decomposition's host logic (paper_2002_05265_gb300.slab: row partition, periodic
ring of neighbours, point-to-point halo exchange, step loop) with gloo ranks on the CPU.  Each
rank advances its slab with the FP64 oracle in the same form as the GPU buffers -- the
post-collision state A, one step A <- collide(stream(A)) (Eq. StreamCollide), the three
xi_y = +1 / -1 populations of its boundary rows packed after each step and unpacked into its
ghost rows -- and the slabs' rows after N steps must equal one oracle run of the whole lattice
bit for bit."""

import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

UP, DOWN = [2, 5, 6], [4, 7, 8]     # planes with xi_y = +1 and xi_y = -1


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _case():
    from paper_2002_05265_gb300 import flows
    import oracle.lbm as olbm
    nx, ny = 24, 20
    f0 = olbm.init_equilibrium(*flows.vortex(nx, ny, Ma=0.3, noise=1e-4, seed=5))
    return f0, "k", olbm.rates_from_nu(1e-3, "reg"), 30


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch
    import torch.distributed as dist
    import oracle.lbm as olbm
    from oracle.collision import collide
    from oracle.d2q9 import XI
    from paper_2002_05265_gb300 import slab

    dist.init_process_group("gloo", rank=rank, world_size=world)
    f0, model, rates, nsteps = _case()
    _, ny, nx = f0.shape
    y0, y1 = slab.slab_rows(ny, rank, world)
    rows = slab.local_rows(ny, y0, y1)
    h = len(rows)
    # post-collision form of the initial state: A_i(z) = f_i(z + xi_i), so stream(A) = f0
    fl = f0[:, rows, :]
    A = np.stack([np.roll(fl[i], shift=(-int(XI[i, 1]), -int(XI[i, 0])), axis=(0, 1)) for i in range(9)])
    state = {"A": A}

    def step_one():
        state["A"] = collide(model, olbm.stream(state["A"]), *rates)

    def pack(send_up, send_down):
        send_up.copy_(torch.from_numpy(state["A"][UP, h - 2, :].ravel()))
        send_down.copy_(torch.from_numpy(state["A"][DOWN, 1, :].ravel()))

    def unpack(from_below, from_above):
        state["A"][UP, 0, :] = from_below.numpy().reshape(3, nx)
        state["A"][DOWN, h - 1, :] = from_above.numpy().reshape(3, nx)

    msgs = [torch.zeros(3 * nx, dtype=torch.float64) for _ in range(4)]
    slab.advance(nsteps, step_one, pack, unpack, msgs, rank, world)
    out[rank] = (y0, y1, olbm.stream(state["A"])[:, 1:-1, :])
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_slab_ranks_match_one_lattice(world):
    import oracle.lbm as olbm
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    f0, model, rates, nsteps = _case()
    ref = olbm.run(f0, model, rates, nsteps)
    covered = []
    for r in range(world):
        y0, y1, f = out[r]
        np.testing.assert_array_equal(f, ref[:, y0:y1, :])
        covered += list(range(y0, y1))
    assert covered == list(range(f0.shape[1]))


def test_slab_partition_and_ring():
    from paper_2002_05265_gb300 import slab
    for ny in (3, 7, 20, 1025):
        for world in range(1, min(ny, 9) + 1):
            spans = [slab.slab_rows(ny, r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == ny
            assert all(a[1] == b[0] for a, b in zip(spans, spans[1:]))
            sizes = [b - a for a, b in spans]
            assert min(sizes) >= 1 and max(sizes) - min(sizes) <= 1
    assert slab.neighbours(0, 4) == (3, 1) and slab.neighbours(3, 4) == (2, 0)
    assert list(slab.local_rows(10, 0, 3)) == [9, 0, 1, 2, 3]
    with pytest.raises(ValueError):
        slab.slab_rows(4, 0, 5)
