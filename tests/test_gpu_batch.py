"""Batched products (hodlr_batch_*) through the C ABI: 32 matrices drawn like
the batched workload (n log-uniform, leaf 128, kernels 1/(r + 1e-3) and
exp(-r^2 / l^2) with l ~ U[0.02, 0.2], eps log-uniform in [1e-10, 1e-3],
per-block adaptive formats over {fp64, fp32, bf16, fp16, e4m3}, fp32 work,
1 to 16 right-hand sides each), every product compared entrywise with the
oracle's exact product of the same stored factors within the product's
rounding bound; one handle used by several items; the launch captured in a
CUDA graph and replayed on new X; the measured CTA-size search; argument
errors."""
import math

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


def _tol(h, X, ref):
    u = F.unit_roundoff("fp32")
    return (Bd.gamma(M.max_chain(h), u) + 2 * u) * M.abs_product(h, X) + u * np.abs(ref)


def _draw(count, seed, nlo=256, nhi=2048):
    """(oracle matrix, GPU matrix, R) triples of the batched workload's
    distribution, sizes log-uniform in [nlo, nhi]."""
    from paper_2407_21637_gb300 import HodlrMatrix
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(round(math.exp(rng.uniform(math.log(nlo), math.log(nhi)))))
        depth = max(0, math.ceil(math.log2(n / 128)))
        eps = float(math.exp(rng.uniform(math.log(1e-10), math.log(1e-3))))
        if rng.uniform() < 0.5:
            spec = synth.KernelSpec(K.INV_DIST, c=1e-3, diag=float(n))
        else:
            ell = float(rng.uniform(0.02, 0.2))
            spec = synth.KernelSpec(K.GAUSS, len2=ell * ell, diag=1e-2)
        R = int(rng.integers(1, 17))
        pts = synth.uniform_points_1d(n, 100 + i)
        h = C.adaptive_hodlr(pts, spec, n, depth, eps, work="fp32", tiers=TIERS, per_block=True)
        ranks, U, V, D = oracle_to_abi(h)
        g = HodlrMatrix.from_factors(n, depth, ranks, U, V, D, eps=eps, work="fp32", tiers=TIERS, per_block=True)
        out.append((h, g, R))
    return out


def test_batch_of_32_matches_the_oracle():
    from paper_2407_21637_gb300 import HodlrBatch
    mats = _draw(32, 31)
    Xs = [torch.from_numpy(synth.rhs_normal(g.n, R, 200 + i, np.float32)).cuda() for i, (_h, g, R) in enumerate(mats)]
    Bs = [torch.full_like(X, float("nan")) for X in Xs]
    bt = HodlrBatch([g for _h, g, _R in mats], Xs, Bs)
    for _ in range(2):   # twice in a row: the scratch holds nothing that must start at zero
        bt.run()
        torch.cuda.synchronize()
        for (h, g, R), X, B in zip(mats, Xs, Bs):
            X64 = X.cpu().numpy().astype(np.float64)
            ref = M.hodlr_matvec(h, X64)
            got = B.cpu().numpy().astype(np.float64)
            assert np.all(np.abs(got - ref) <= _tol(h, X64, ref)), (g.n, g.depth, R)
    bt.close()
    for _h, g, _R in mats:
        g.close()


def test_one_handle_in_several_items_and_larger_sizes():
    """The same handle with different X (items share the stored matrix,
    not the scratch), sizes up to 8192 (several units per node), against
    hodlr_matvec of each item within twice the product bound."""
    from paper_2407_21637_gb300 import HodlrBatch
    mats = _draw(3, 77, nlo=4096, nhi=8192)
    items = [mats[0], mats[0], mats[1], mats[2], mats[1]]
    Xs = [torch.from_numpy(synth.rhs_normal(g.n, R, 300 + i, np.float32)).cuda() for i, (_h, g, R) in enumerate(items)]
    Bs = [torch.empty_like(X) for X in Xs]
    bt = HodlrBatch([g for _h, g, _R in items], Xs, Bs)
    bt.run()
    torch.cuda.synchronize()
    for (h, g, R), X, B in zip(items, Xs, Bs):
        X64 = X.cpu().numpy().astype(np.float64)
        ref = M.hodlr_matvec(h, X64)
        assert np.all(np.abs(B.cpu().numpy().astype(np.float64) - ref) <= _tol(h, X64, ref))
        single = g.matvec(X).cpu().numpy().astype(np.float64)
        assert np.all(np.abs(B.cpu().numpy().astype(np.float64) - single) <= 2 * _tol(h, X64, ref))
    bt.close()
    for _h, g, _R in mats:
        g.close()


def test_graph_capture_and_tune():
    """hodlr_batch_run allocates nothing and copies nothing from the host:
    captured in a CUDA graph, the replay on new contents of X gives the new
    products; hodlr_batch_tune keeps one of the three CTA sizes."""
    from paper_2407_21637_gb300 import HodlrBatch
    mats = _draw(8, 5)
    Xs = [torch.from_numpy(synth.rhs_normal(g.n, R, 400 + i, np.float32)).cuda() for i, (_h, g, R) in enumerate(mats)]
    Bs = [torch.empty_like(X) for X in Xs]
    bt = HodlrBatch([g for _h, g, _R in mats], Xs, Bs)
    th, ms = bt.tune()
    assert th in (128, 256, 512) and ms > 0
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        bt.run(stream=s)   # warm-up on the capture stream
    torch.cuda.current_stream().wait_stream(s)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        bt.run()
    for i, X in enumerate(Xs):
        X.copy_(torch.from_numpy(synth.rhs_normal(X.shape[0], X.shape[1], 500 + i, np.float32)))
    graph.replay()
    torch.cuda.synchronize()
    for (h, g, R), X, B in zip(mats, Xs, Bs):
        X64 = X.cpu().numpy().astype(np.float64)
        ref = M.hodlr_matvec(h, X64)
        assert np.all(np.abs(B.cpu().numpy().astype(np.float64) - ref) <= _tol(h, X64, ref))
    bt.close()
    for _h, g, _R in mats:
        g.close()


def test_batch_argument_errors():
    import ctypes
    from paper_2407_21637_gb300 import HodlrBatch, HodlrError, _lib
    (h, g, R), = _draw(1, 9)
    X = torch.zeros(g.n, 17, device="cuda")
    with pytest.raises(HodlrError) as ei:
        HodlrBatch([g], [X], [torch.zeros_like(X)])   # 17 right-hand sides
    assert ei.value.status == 1
    X64 = torch.zeros(g.n, 2, device="cuda", dtype=torch.float64)
    with pytest.raises(ValueError):
        HodlrBatch([g], [X64], [torch.zeros_like(X64)])   # fp64 X for an fp32 matrix (caught by the binding)
    # working precisions mixed in one batch: rejected by the library
    from paper_2407_21637_gb300 import HodlrMatrix
    ranks, U, V, D = oracle_to_abi(h)
    g64 = HodlrMatrix.from_factors(g.n, g.depth, ranks, U, V, D, eps=1e-6, work="fp64", tiers=TIERS)
    hs = (ctypes.c_void_p * 2)(g._h, g64._h)
    nr = (ctypes.c_int32 * 2)(1, 1)
    Xa = torch.zeros(g.n, 1, device="cuda")
    ptrs = (ctypes.c_void_p * 2)(Xa.data_ptr(), Xa.data_ptr())
    lds = (ctypes.c_int64 * 2)(1, 1)
    out = ctypes.c_void_p()
    assert _lib.load().hodlr_batch_create(2, hs, nr, ptrs, lds, ptrs, lds, 1, ctypes.byref(out)) == 1
    g64.close()
    assert _lib.load().hodlr_batch_run(None, 0, None) == 1
    g.close()
