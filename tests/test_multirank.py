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


def _shard_rank(rank, world, port, out):
    """Rank j owns the rows of node (g, j), g = log2(world): it forms the
    partial V^T x of its own rows for every node of levels 1..g, one
    all-reduce (sum) of these zero-padded blocks gives every rank the full
    Y of all of them, and the rest of the product (levels below g and the
    leaves) uses only local rows."""
    import numpy as np
    import synth
    from oracle import compress as C
    from oracle import kernels as K
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        n, depth, R, eps = 1000, 4, 3, 1e-6
        spec = synth.KernelSpec(K.GAUSS, len2=0.01, diag=1e-2)
        h = C.adaptive_hodlr(synth.uniform_points_1d(n, 8), spec, n, depth, eps, work="fp64",
                             tiers=("fp64", "fp32", "bf16", "fp16", "e4m3"))
        X = synth.rhs_normal(n, R, 6, np.float64)
        g = world.bit_length() - 1
        s0, m0 = h.levels[g][rank]
        # Y of every node at levels 1..g, zero except this rank's own nodes
        slots, off = {}, 0
        for k in range(1, g + 1):
            for i, (s, m) in enumerate(h.levels[k]):
                slots[(k, i)] = off
                off += h.Vh[k][i].shape[1]
        Yall = np.zeros((off, R))
        for k in range(1, g + 1):
            for i, (s, m) in enumerate(h.levels[k]):
                a, b = max(s, s0), min(s + m, s0 + m0)   # this rank's rows of the node
                if a < b:
                    r = h.Vh[k][i].shape[1]
                    Yall[slots[(k, i)]:slots[(k, i)] + r] += h.Vh[k][i][a - s:b - s].T @ X[a:b]
        t = torch.from_numpy(Yall)
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        Yall = t.numpy()
        B = np.zeros((m0, R))
        for k in range(1, depth + 1):
            for i, (s, m) in enumerate(h.levels[k]):
                a, b = max(s, s0), min(s + m, s0 + m0)
                if a >= b:
                    continue
                s1, m1 = h.levels[k][i ^ 1]
                if k <= g:
                    r = h.Vh[k][i ^ 1].shape[1]
                    y = Yall[slots[(k, i ^ 1)]:slots[(k, i ^ 1)] + r]
                else:
                    y = h.Vh[k][i ^ 1].T @ X[s1:s1 + m1]   # below level g the sibling is local too
                B[a - s0:b - s0] += h.Uh[k][i][a - s:b - s] @ y
        for i, (s, m) in enumerate(h.levels[depth]):
            if s0 <= s and s + m <= s0 + m0:
                B[s - s0:s - s0 + m] += h.Dh[i] @ X[s:s + m]
        out[rank] = (s0, m0, B)
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(180)
@pytest.mark.parametrize("world", [2, 4])
def test_row_partitioned_product_with_one_all_reduce(world):
    """The sharded product (one all-reduce of the level-<=g V^T x blocks)
    equals the oracle's Algorithm 3.3 on the same stored factors."""
    import numpy as np
    import synth
    from oracle import compress as C
    from oracle import kernels as K
    from oracle import matvec as M
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_shard_rank, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    n, depth, R, eps = 1000, 4, 3, 1e-6
    spec = synth.KernelSpec(K.GAUSS, len2=0.01, diag=1e-2)
    h = C.adaptive_hodlr(synth.uniform_points_1d(n, 8), spec, n, depth, eps, work="fp64",
                         tiers=("fp64", "fp32", "bf16", "fp16", "e4m3"))
    X = synth.rhs_normal(n, R, 6, np.float64)
    ref = M.hodlr_matvec(h, X)
    B = np.zeros_like(ref)
    for s0, m0, b in res.values():
        B[s0:s0 + m0] = b
    assert sorted(s0 for s0, _m, _b in res.values()) == [s for s, _m in h.levels[world.bit_length() - 1]]
    assert np.allclose(B, ref, rtol=1e-13, atol=1e-13 * np.abs(ref).max())
