"""The bench's multi-process bookkeeping on CPU ranks (gloo, world size 2): the job's time is the
slowest rank's, the job's value counts every rank's units, and the reference arm runs on rank 0 only.
(GPU ranks use NCCL with the same functions; one GPU is available here.)"""
import io
import os
import socket
from contextlib import redirect_stdout

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 10.0 + 5.0 * rank          # rank 1 is the slow one
        job_ms = bench.max_over_ranks(ms, dist, torch.device("cpu"))
        out[rank] = (job_ms, bench.job_value(1000, world, job_ms))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_job_time_is_the_slowest_rank_and_value_counts_all_ranks():
    world = 2
    out = mp.Manager().dict()
    mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
    for rank in range(world):
        job_ms, value = out[rank]
        assert job_ms == 15.0
        assert value == pytest.approx(1000 * world / 15e-3)


def test_single_process_keeps_its_own_time():
    assert bench.max_over_ranks(12.5, None, torch.device("cpu")) == 12.5
    assert bench.job_value(100, 1, 2.0) == pytest.approx(5e4)


def test_reference_arm_prints_nothing_on_other_ranks(monkeypatch):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class Args:
        nb, steps, warmup, gpus = 1, 1, 1, 2

    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(Args())
    assert buf.getvalue() == ""
