"""The multi-rank bookkeeping of bench.py on two gloo ranks (CPU): the step time
is the maximum over ranks and the whole-job throughput counts every replica."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = bench.max_over_ranks(10.0 + 5.0 * rank, dist, "cpu")
    out[rank] = (ms, bench.job_throughput(10, world, ms))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_max_and_throughput():
    world = 2
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        ms, thr = res[r]
        assert ms == 15.0
        assert thr == pytest.approx(world * 1000.0 / 15.0)


def test_single_rank_is_identity():
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.job_throughput(10, 1, 50.0) == pytest.approx(20.0)
