"""The multi-rank host logic of bench.py on CPU (gloo, world size 2).

Replicas only: each rank advances its own problem, the job time is the slowest
rank's time and the whole-job rate counts every rank's updates.  No GPU needed.
"""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 10.0 + 5.0 * rank                 # rank 1 is the slow replica
        got = bench.max_over_ranks(ms, dist, "cpu")
        rate = bench.job_rate(1000, 20, world, got * 1e-3)
        out[rank] = (got, rate)
    finally:
        dist.destroy_process_group()


def test_job_time_is_the_slowest_replica_and_rate_counts_all_ranks():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
    assert out[0][0] == out[1][0] == 15.0
    assert out[0][1] == out[1][1] == pytest.approx(1000 * 20 * 2 / 15e-3)


def test_single_process_needs_no_group():
    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5
    assert bench.job_rate(10, 2, 1, 0.5) == 40.0
