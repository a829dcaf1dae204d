"""The multi-GPU path of bench.py is replicas only: each rank advances its own simulation and
the ranks exchange nothing but a barrier and the max of their times.  This runs that
aggregation with two gloo ranks on the CPU."""

import os
import socket
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    dist.barrier()
    ms_local = 100.0 * (rank + 1)          # rank 1 is the slower one
    value, ms_max = bench.aggregate_ranks(dist, ms_local, units_per_rank=1000, steps=5)
    out[rank] = (value, ms_max)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_as_weak_scaling():
    world = 2
    mgr = mp.get_context("spawn").Manager()  # no fork of this (threaded) test process
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    for rank in range(world):
        value, ms_max = out[rank]
        assert ms_max == 200.0
        # all ranks' units over the slowest rank's time
        assert abs(value - 2 * 1000 * 5 / 0.2) < 1e-9


def test_single_process_aggregate():
    sys.path.insert(0, ROOT)
    import bench
    value, ms_max = bench.aggregate_ranks(None, 50.0, units_per_rank=10, steps=4)
    assert ms_max == 50.0 and abs(value - 10 * 4 / 0.05) < 1e-9
