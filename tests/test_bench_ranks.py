"""The multi-rank host logic of bench.py on CPU ranks (gloo, world size 2): each rank times its
own replica of the workload; the job time is the slowest rank's, and the job value counts the
work of every rank."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, times, out):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = bench.max_over_ranks(times[rank], "cpu")
        dist.barrier()
        out[rank] = t
    finally:
        dist.destroy_process_group()


def test_job_time_is_slowest_rank_and_value_counts_all_ranks():
    sys.path.insert(0, ROOT)
    import bench

    world, times = 2, [1.25, 3.5]
    out = mp.get_context("spawn").Manager().dict()
    mp.start_processes(_rank, args=(world, _free_port(), times, out), nprocs=world, join=True, start_method="spawn")
    assert out[0] == out[1] == max(times)
    # replicas: twice the work in the slowest rank's time
    assert bench.job_value(263169, 34000, 3.5, 2) == pytest.approx(2 * 263169 * 34000 / 3.5)
    assert bench.job_value(263169, 34000, 3.5, 1) * 2 == pytest.approx(bench.job_value(263169, 34000, 3.5, 2))
