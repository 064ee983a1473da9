"""The multi-rank host logic of bench.py on CPU: two gloo ranks (spawned
processes, rendezvous on 127.0.0.1), the barrier, the max-over-ranks timing
and the whole-job value of independent replicas."""

import os
import socket

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    bench.barrier(world)
    # rank r "took" 10 (r + 1) ms: every rank must see the slowest
    slowest = bench.max_over_ranks(10.0 * (rank + 1), world)
    bench.barrier(world)
    out[rank] = slowest
    dist.destroy_process_group()


def test_two_gloo_ranks():
    import torch.multiprocessing as mp
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
        got = dict(out)
    assert got == {0: 20.0, 1: 20.0}


def test_replica_value():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    # 2 replicas of 1 GB per step, 10 steps in 5 s (the slowest rank): 4 GB/s
    assert bench.replica_value(2, 1e9, 10, 5000.0) == pytest.approx(4.0)
    assert bench.replica_value(1, 1e9, 10, 5000.0) == pytest.approx(2.0)
