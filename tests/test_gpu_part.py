"""Partitioned products (hodlr_part_*) through the C ABI: Algorithm 3.3 split
by rows at tree level g (part j owns the rows of node (g, j)), the levels
1..g of V^T X summed over the parts between the two steps.  The parts run on
separate CUDA streams of one GPU (and, in the last test, as two gloo
processes sharing it, the sum an all-reduce between the steps); the
assembled product is compared entrywise with the oracle's exact product of
the same stored factors within the product's rounding bound (the bound
holds for any order of the sums), and with hodlr_matvec."""
import math
import os
import socket

import numpy as np
import pytest
import torch

import synth
from oracle import bounds as Bd
from oracle import compress as C
from oracle import formats as F
from oracle import kernels as K
from oracle import matvec as M
from oracle.abi_lists import oracle_to_abi

pytestmark = pytest.mark.gpu

TIERS = ("fp64", "fp32", "bf16", "fp16", "e4m3")


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2407_21637_gb300 import build as B
    B.build()
    torch.cuda.set_device(0)


def _tol(h, X, ref, work):
    u = F.unit_roundoff(work)
    return (Bd.gamma(M.max_chain(h), u) + 2 * u) * M.abs_product(h, X) + u * np.abs(ref)


def _matrix(n, depth, eps, work, seed, kind=0):
    """(oracle matrix, GPU matrix) of the uneven-size workload's kernels,
    per-block adaptive formats (mixed tiers)."""
    from paper_2407_21637_gb300 import HodlrMatrix
    pts = synth.uniform_points_1d(n, seed)
    if kind == 0:
        spec = synth.KernelSpec(K.INV_DIST, c=1e-3, diag=float(n))
    else:
        spec = synth.KernelSpec(K.GAUSS, len2=0.1 ** 2, diag=1e-2)
    h = C.adaptive_hodlr(pts, spec, n, depth, eps, work=work, tiers=TIERS, per_block=True)
    ranks, U, V, D = oracle_to_abi(h)
    g = HodlrMatrix.from_factors(n, depth, ranks, U, V, D, eps=eps, work=work, tiers=TIERS, per_block=True)
    return h, g


def _partitioned(g, level, X):
    """The product assembled from 2^level parts, each on its own stream."""
    from paper_2407_21637_gb300 import HodlrPart
    R = X.shape[1]
    parts = [HodlrPart(g, level, j, R) for j in range(1 << level)]
    streams = [torch.cuda.Stream() for _ in parts]
    xs = [X[p.row0:p.row0 + p.rows] for p in parts]
    yreds = [p.new_yred() for p in parts]
    torch.cuda.synchronize()
    for p, s, x, y in zip(parts, streams, xs, yreds):
        with torch.cuda.stream(s):
            p.partial(x, y, stream=s)
    torch.cuda.synchronize()
    ysum = yreds[0].clone()
    for y in yreds[1:]:
        ysum += y   # the exchange: a sum over the parts
    Bs = []
    for p, s, x in zip(parts, streams, xs):
        with torch.cuda.stream(s):
            Bs.append(p.finish(x, ysum, stream=s))
    torch.cuda.synchronize()
    rows = [(p.row0, p.rows) for p in parts]
    counts = [p.yred_count for p in parts]
    for p in parts:
        p.close()
    return torch.cat(Bs), rows, counts


@pytest.mark.parametrize("work", ["fp32", "fp64"])
def test_parts_on_streams_match_the_oracle(work):
    h, g = _matrix(3000, 5, 1e-7, work, 11)
    dt = torch.float32 if work == "fp32" else torch.float64
    for R in (1, 5, 16):
        X = torch.from_numpy(synth.rhs_normal(g.n, R, 40 + R, np.float64)).to(dt).cuda()
        X64 = X.cpu().numpy().astype(np.float64)
        ref = M.hodlr_matvec(h, X64)
        tol = _tol(h, X64, ref, work)
        whole = g.matvec(X).cpu().numpy().astype(np.float64)
        for level in range(0, 4):
            B, rows, counts = _partitioned(g, level, X)
            got = B.cpu().numpy().astype(np.float64)
            assert np.all(np.abs(got - ref) <= tol), (work, R, level)
            assert np.all(np.abs(got - whole) <= 2 * tol), (work, R, level)
            # the parts tile [0, n) in order; the summed buffer holds levels 1..g
            assert rows[0][0] == 0 and sum(r for _, r in rows) == g.n
            assert all(a[0] + a[1] == b[0] for a, b in zip(rows, rows[1:]))
            rb = 1 if R == 1 else 2 if R == 2 else 4 if R <= 4 else 8 if R <= 8 else 16
            ranks = [h.rank(k, i) for k in range(1, level + 1) for i in range(1 << k)]   # V ranks total the same
            assert all(c == rb * sum(ranks) for c in counts), (counts, rb, sum(ranks))
    g.close()


def test_deep_partition_and_ragged_sizes():
    """g = depth (one leaf per part) on an odd n with a Gaussian kernel."""
    h, g = _matrix(1537, 4, 1e-9, "fp32", 5, kind=1)
    X = torch.from_numpy(synth.rhs_normal(g.n, 3, 9, np.float32)).cuda()
    X64 = X.cpu().numpy().astype(np.float64)
    ref = M.hodlr_matvec(h, X64)
    B, _rows, _c = _partitioned(g, 4, X)
    assert np.all(np.abs(B.cpu().numpy().astype(np.float64) - ref) <= _tol(h, X64, ref, "fp32"))
    g.close()


def test_part_argument_errors():
    import ctypes
    from paper_2407_21637_gb300 import HodlrError, HodlrPart, _lib
    _h, g = _matrix(1024, 3, 1e-6, "fp32", 2)
    for args in ((4, 0, 1), (2, 4, 1), (2, -1, 1), (1, 0, 17), (1, 0, 0)):
        with pytest.raises(HodlrError) as ei:
            HodlrPart(g, *args)
        assert ei.value.status == 1
    p = HodlrPart(g, 2, 1, 4)
    X = torch.zeros(p.rows, 4, device="cuda")
    with pytest.raises(ValueError):
        p.partial(torch.zeros(p.rows + 1, 4, device="cuda"), p.new_yred())   # wrong rows (binding)
    lib = _lib.load()
    assert lib.hodlr_part_partial(p._p, X.data_ptr(), 4, None, None) == 1    # no buffer for the summed levels
    assert lib.hodlr_part_partial(p._p, X.data_ptr(), 3, p.new_yred().data_ptr(), None) == 1   # ldx < nrhs
    assert lib.hodlr_part_finish(p._p, X.data_ptr(), 4, p.new_yred().data_ptr(), None, 4, None) == 1   # no B
    assert lib.hodlr_part_partial(None, X.data_ptr(), 4, None, None) == 1
    info = ctypes.c_int64()
    assert lib.hodlr_part_info(None, ctypes.byref(info), None, None) == 1
    p.close()
    g.close()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _gloo_rank(rank, world, port, out):
    """One process per part on the same GPU; the summed levels go through a
    gloo all-reduce on the host between the two steps (no kernel waits on
    another process)."""
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        torch.cuda.set_device(0)
        from paper_2407_21637_gb300 import HodlrPart
        h, g = _matrix(2048, 4, 1e-6, "fp32", 21)
        X = torch.from_numpy(synth.rhs_normal(g.n, 4, 77, np.float32)).cuda()
        p = HodlrPart(g, int(math.log2(world)), rank, 4)
        x = X[p.row0:p.row0 + p.rows]
        y = p.new_yred()
        p.partial(x, y)
        yh = y.cpu()
        dist.all_reduce(yh)
        B = p.finish(x, yh.cuda()).cpu()
        parts = [None] * world
        dist.all_gather_object(parts, (p.row0, B.numpy()))
        if rank == 0:
            X64 = X.cpu().numpy().astype(np.float64)
            ref = M.hodlr_matvec(h, X64)
            got = np.concatenate([b for _, b in sorted(parts, key=lambda t: t[0])]).astype(np.float64)
            out["ok"] = bool(np.all(np.abs(got - ref) <= _tol(h, X64, ref, "fp32")))
        p.close()
        g.close()
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(300)
def test_two_gloo_processes_share_one_gpu():
    import torch.multiprocessing as mp
    with mp.get_context("spawn").Manager() as m:   # nothing forked after CUDA is up
        out = m.dict()
        mp.start_processes(_gloo_rank, args=(2, _free_port(), out), nprocs=2, join=True, start_method="spawn")
        assert out.get("ok") is True
