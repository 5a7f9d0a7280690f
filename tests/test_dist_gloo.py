"""The multi-rank host logic of bench.py on CPU: two gloo ranks on 127.0.0.1 check the
timing maximum over ranks, the barrier and the sharding of the batched sweep's instances
(independent problems: every instance on exactly one rank)."""

import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    bench.barrier(world)
    t = bench.max_over_ranks(10.0 + rank, world)
    mine = bench.shard(list(range(37)), rank, world)
    got = [None] * world
    dist.all_gather_object(got, mine)
    out[rank] = (t, got)
    dist.destroy_process_group()


def test_two_gloo_ranks():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        t, shards = out[r]
        assert t == 11.0
        flat = sorted(x for sh in shards for x in sh)
        assert flat == list(range(37))
        assert all(set(a).isdisjoint(b) for i, a in enumerate(shards) for b in shards[i + 1:])
