"""The multi-GPU path of bench.py is replicas only: every rank solves its own problem and
only the timing is reduced (max over ranks).  Exercised here with two gloo ranks on CPU."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    ms = 100.0 + 50.0 * rank                         # rank 1 is the slow one
    t = bench.max_over_ranks(ms, world)
    out[rank] = (t, bench.replica_seeds(rank), bench.aggregate_value(world, 16, 297222, t))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_replicas():
    world, port = 2, _free_port()
    out = mp.Manager().dict()
    mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
    assert out[0][0] == out[1][0] == 150.0          # max over ranks
    assert out[0][1] != out[1][1]                   # independent problems
    assert out[0][2] == pytest.approx(2 * 16 * 297222 / 0.150)


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5, 1) == 12.5
    assert bench.aggregate_value(1, 16, 10, 1000.0) == 160.0
