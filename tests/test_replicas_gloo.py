"""Multi-GPU form (replicas only) on CPU: two gloo ranks reduce their timed-region
durations to the job's (the slowest rank's) and report the whole-job throughput."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = 10.0 + 5.0 * rank  # rank 1 is slower
    job = bench.job_time_ms(ms, dist, "cpu")
    out[rank] = (job, bench.job_value(1000, 4, world, job))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_report_the_slowest_rank():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    port = _free_port()
    mp.start_processes(_rank, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
    assert out[0][0] == out[1][0] == 15.0
    # 2 ranks x 4 steps x 1000 units in 15 ms
    assert out[0][1] == pytest.approx(2 * 4 * 1000 / 0.015)
    del torch


def test_single_rank_needs_no_collective():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_time_ms(12.5, None, "cpu") == 12.5
    assert bench.job_value(10, 3, 1, 12.5) == pytest.approx(30 / 0.0125)
