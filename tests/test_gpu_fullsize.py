"""Parity at the benchmark's full size, in the launch configuration bench.py
times: gauss_65536 (n = 65536 sorted U[0,1] points, exp(-r^2/0.01) + 1e-2 I,
leaf 256, depth 8, eps 1e-6, per-block rule over {fp64, fp32, bf16, fp16,
e4m3}, fp32 work) and the benchmark's mixed-format workload on the same
points (1/(|x_i - x_j| + 1e-3), eps 1e-4, per-block rule: fp32 and fp16
blocks), both built on the GPU with max_nrhs 64, products of R = 1, 8 and 64
columns (streamed CUDA-core kernel; tensor cores from 16 columns on).
The oracle's fp64 product of the same stored generators (exported exactly)
is formed on sampled rows -- both ends of every leaf, the matrix ends and
seeded random rows -- and every sampled entry must lie within the
entrywise bound of the other parity tests; the full products must be finite
and bitwise repeatable."""
import numpy as np
import pytest
import torch

import bench
import synth
from oracle import bounds as Bd
from oracle import compress as C
from oracle import formats as F
from oracle import matvec as M
from oracle.abi_lists import abi_to_levels

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", params=["headline", "mixed"])
def full(request):
    from paper_2407_21637_gb300 import build as B
    from paper_2407_21637_gb300 import HodlrMatrix
    B.build()
    torch.cuda.set_device(0)
    W = bench.WL if request.param == "headline" else bench.WL_MIXED
    n, depth = W["n"], W["depth"]
    pts = torch.from_numpy(synth.uniform_points_1d(n, W["seed"])).cuda()
    g = HodlrMatrix.build(pts, W["kind"], depth, W["eps"], c=W["c"], len2=W["len2"], diag=W["diag"],
                          work=W["work"], tiers=W["tiers"], per_block=W["per_block"], max_nrhs=64)
    if request.param == "mixed":   # the adaptive rule must really have mixed formats here
        bpt = g.info()["bytes_per_tier"]
        assert bpt["fp16"] > 0 and bpt["fp32"] > 0
    U, V, D = g.export()
    h = C.from_factors(n, depth, abi_to_levels(depth, U), abi_to_levels(depth, V), D)
    h.Uh, h.Vh, h.Dh = h.U, h.V, h.D          # the exported values are the stored ones
    rng = np.random.default_rng(12)
    ends = [s for (s, m) in h.levels[depth]] + [s + m - 1 for (s, m) in h.levels[depth]]
    rows = np.unique(np.concatenate([ends, [0, n - 1], rng.integers(0, n, 256)]))
    yield h, g, rows
    g.close()


@pytest.mark.parametrize("R", [1, 8, 64])
def test_full_size_sampled_parity(full, R):
    h, g, rows = full
    X = synth.rhs_normal(h.n, R, 500 + R, np.float32)
    Xd = torch.from_numpy(X).cuda()
    B1 = g.matvec(Xd)
    B2 = g.matvec(Xd)
    g.sync_status()
    assert torch.equal(B1, B2)
    assert bool(torch.isfinite(B1).all())
    X64 = X.astype(np.float64)
    ref = M.hodlr_matvec_rows(h, X64, rows)
    gabs = M.abs_product_rows(h, X64, rows)
    u = F.unit_roundoff("fp32")
    if R >= 16:   # tensor-core products (tf32 split of both factors)
        tol = (Bd.gamma(M.max_chain(h), 2 * u) + 14 * u) * gabs + u * np.abs(ref)
    else:
        tol = (Bd.gamma(M.max_chain(h), u) + 2 * u) * gabs + u * np.abs(ref)
    got = B1.cpu().numpy().astype(np.float64)[rows]
    err = np.abs(got - ref)
    assert np.all(err <= tol), float(np.max(err / tol))


def test_full_size_partitioned(full):
    """The row-partitioned product (hodlr_part_*, 8 parts of tree level 3 on
    separate streams, the levels 1..3 of V^T X summed on the device) at full
    size: every sampled entry within the same entrywise bound (it holds for
    any order of the sums)."""
    from paper_2407_21637_gb300 import HodlrPart
    h, g, rows = full
    R = 8
    X = synth.rhs_normal(h.n, R, 900, np.float32)
    Xd = torch.from_numpy(X).cuda()
    parts = [HodlrPart(g, 3, j, R) for j in range(8)]
    streams = [torch.cuda.Stream() for _ in parts]
    xs = [Xd[p.row0:p.row0 + p.rows] for p in parts]
    yreds = [p.new_yred() for p in parts]
    torch.cuda.synchronize()
    for p, s, x, y in zip(parts, streams, xs, yreds):
        p.partial(x, y, stream=s)
    torch.cuda.synchronize()
    ysum = torch.stack(yreds).sum(dim=0)
    Bs = [p.finish(x, ysum, stream=s) for p, s, x in zip(parts, streams, xs)]
    torch.cuda.synchronize()
    for p in parts:
        p.close()
    B = torch.cat(Bs)
    assert bool(torch.isfinite(B).all())
    X64 = X.astype(np.float64)
    ref = M.hodlr_matvec_rows(h, X64, rows)
    gabs = M.abs_product_rows(h, X64, rows)
    u = F.unit_roundoff("fp32")
    tol = (Bd.gamma(M.max_chain(h), u) + 2 * u) * gabs + u * np.abs(ref)
    err = np.abs(B.cpu().numpy().astype(np.float64)[rows] - ref)
    assert np.all(err <= tol), float(np.max(err / tol))
