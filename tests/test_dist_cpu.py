"""The multi-rank host logic of bench.py on CPU: two gloo ranks on
127.0.0.1.  Under torchrun every rank evaluates its own replica of the
workload (weak scaling, no data-path collective); the job's step time is the
slowest rank's and its throughput counts the units of every rank."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = [3.0, 5.0][rank]  # the second rank is slower
        job_ms = bench.max_over_ranks(ms, dist, "cpu")
        out[rank] = (job_ms, bench.job_throughput(1000.0, world, job_ms))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_step():
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0] == res[1]
    job_ms, value = res[0]
    assert job_ms == 5.0
    assert value == pytest.approx(2 * 1000.0 / 5e-3)


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(4.0, None) == 4.0
    assert bench.job_throughput(10.0, 1, 2.0) == pytest.approx(5000.0)
