"""The benchmark's whole-job figures over several ranks (bench.reduce_over_ranks):
max of the times, sum of the counts, on two gloo ranks on the CPU; identity on one."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, results):
    import torch
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    maxes, sums = bench.reduce_over_ranks(torch, world, [10.0 + rank, 5.0 - rank], [100 + rank], "cpu")
    results[rank] = (maxes, sums)
    dist.barrier()
    dist.destroy_process_group()


def test_reduce_over_two_ranks():
    import torch.multiprocessing as mp

    results = mp.get_context("spawn").Manager().dict()
    mp.start_processes(_worker, args=(2, _port(), results), nprocs=2, join=True, start_method="spawn")
    for rank in (0, 1):
        maxes, sums = results[rank]
        assert maxes == [11.0, 5.0] and sums == [201.0]


def test_reduce_on_one_rank_is_the_identity():
    torch = pytest.importorskip("torch")
    sys.path.insert(0, ROOT)
    import bench

    assert bench.reduce_over_ranks(torch, 1, [3.5, 2], [7], "cpu") == ([3.5, 2.0], [7.0])
