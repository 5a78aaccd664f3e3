"""The multi-GPU (replicas) aggregation of bench.py, run as two gloo ranks on
the CPU: the job value is every rank's work over the slowest rank's time."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = 100.0 * (rank + 1)  # rank 1 is the slow one
    value, ms = bench.job_value(local_ms, world, 1000, dist)
    bench.barrier(dist)
    out[rank] = (value, ms)
    dist.destroy_process_group()


def test_job_value_takes_the_slowest_rank_and_sums_the_work():
    world = 2
    port = _free_port()
    manager = mp.get_context("spawn").Manager()
    out = manager.dict()
    mp.start_processes(_rank, args=(world, port, out), nprocs=world, join=True,
                       start_method="spawn")
    for r in range(world):
        value, ms = out[r]
        assert ms == 200.0
        assert value == pytest.approx(world * 1000 / 0.2)
