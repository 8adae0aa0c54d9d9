"""The multi-rank timing of bench.py (replicas, one per GPU) with two gloo
ranks on the CPU: every rank gets the slowest rank's time, and the job's
value counts every replica's work in that time."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 100.0 + 50.0 * rank          # rank 1 is the slowest
        dist.barrier()
        slow = bench.max_over_ranks(ms, dist)
        out[rank] = (slow, bench.job_gflops(10 ** 9, slow, world))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_max_time_and_job_value():
    world = 2
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 150.0
    # 2 replicas x 2e9 FLOP in 0.15 s
    assert res[0][1] == pytest.approx(2 * 2e9 / 0.15 / 1e9)
