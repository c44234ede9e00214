"""The benchmark's multi-rank bookkeeping on CPU: replicas only (one lattice per rank, no
collective on the data path), the job time is the slowest rank's, and the value counts the
sites of every rank. World size 2 over gloo on 127.0.0.1."""
import os

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 10.0 + 5.0 * rank  # rank 1 is the slow one
        t = bench.max_over_ranks(ms, dist, "cpu")
        out[rank] = (t, bench.job_value(1000, 3, 100, world, t))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_job_value_gloo():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = 29500 + (os.getpid() % 1000)
    mp.start_processes(_worker, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
    assert out[0][0] == out[1][0] == 15.0
    # 2 replicas x 1000 sites x 3 components x 100 steps in 15 ms
    assert out[0][1] == pytest.approx(2 * 1000 * 3 * 100 / 0.015 / 1e6)


def test_single_process_is_its_own_max():
    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5
