"""The multi-process side of bench.py (CPU, gloo, world size 2): every rank
runs its own replica, the job's time is the slowest rank's and the job's
rate counts the units of all ranks."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local = [3.0, 5.5][rank]
        ms = bench.job_time_ms(local, world, torch.device("cpu"))
        out[rank] = ms
        out[world + rank] = bench.job_rate(1 << 20, world, ms)
    finally:
        dist.destroy_process_group()


def test_job_time_is_the_max_over_two_gloo_ranks():
    world = 2
    out = mp.get_context("spawn").Array("d", 2 * world)
    mp.start_processes(_rank_main, args=(world, _free_port(), out), nprocs=world,
                       start_method="spawn", join=True)
    assert list(out[:world]) == [5.5, 5.5]
    expect = 2 * (1 << 20) / (5.5e-3) / 1e9
    assert out[world] == pytest.approx(expect) and out[world + 1] == pytest.approx(expect)


def test_single_rank_is_identity():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_time_ms(2.5, 1, torch.device("cpu")) == 2.5
    assert bench.job_rate(1000, 1, 1.0) == pytest.approx(1e-3)
