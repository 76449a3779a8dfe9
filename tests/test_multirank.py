"""The N > 1 path of bench.py (replicas, one process per GPU) on CPU ranks:
two gloo processes check the host logic that turns per-rank step times into
the job's number -- the maximum over ranks of the step time, and the
whole-job throughput of every rank's units over that time."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        ms = 1.0 + 0.5 * rank                     # rank 1 is the slow one
        slowest = bench.max_over_ranks(ms, dist, torch.device("cpu"))
        dist.barrier()
        out[rank] = (slowest, bench.job_value(4_784_128, world, slowest))
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_rank_max_timing_and_job_value():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 1.5
    assert res[0][1] == res[1][1] == pytest.approx(2 * 4_784_128 / 1.5e-3)


def test_single_process_value():
    import bench
    assert bench.max_over_ranks(2.0, None, None) == 2.0
    assert bench.job_value(100, 1, 1.0) == pytest.approx(1e5)
