"""The N > 1 path of bench.py, run as two gloo ranks on the CPU.

Each rank of `bench.py --gpus N` integrates its own replica of the workload;
the bench brackets the timed steps with barriers, keeps the slowest rank's time
and reports the units of all ranks over that time.  These tests run exactly
those helpers in a world of two processes, and check that the reference arm's
non-zero ranks exit without work.
"""
import os
import socket
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        secs = 1.5 + rank            # rank 1 is the slow one
        worst = bench.max_over_ranks(secs, dist)
        rate = bench.whole_job_rate(1000.0, 4, world, worst)
        out[rank] = (worst, rate)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
    assert out[0] == out[1]
    worst, rate = out[0]
    assert worst == 2.5
    assert rate == pytest.approx(1000.0 * 4 * 2 / 2.5)


def test_single_process_helpers():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.0) == 3.0
    assert bench.whole_job_rate(10.0, 5, 1, 2.0) == 25.0


def test_reference_arm_nonzero_rank_does_no_work(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class Args:
        steps, warmup = 1, 0
    assert bench.run_reference(Args()) is None
