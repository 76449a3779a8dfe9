"""hodlr_matvec_noalloc: the product for callers that cannot allocate device
memory at the time of the call (a process whose device memory is reserved
by another allocator, or a latency-critical path that must not enter the
driver's allocator).  Its scratch is a 256 KiB static device array inside
the library.  Through the C ABI, two calls in a row must agree with
hodlr_matvec: bitwise where both run the same CUDA-core kernel with the same
column batches, else within the rounding bound of the other product tests.
Also covered: batches narrowed to what the array holds, and a matrix whose
scratch for one column does not fit, which is rejected with B untouched.

This file is collected last so that a run stopping at the first failure has
already run every other test; it also passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest
import torch

import synth
from oracle import bounds as Bd
from oracle import compress as C
from oracle import formats as F
from oracle import kernels as K
from oracle import matvec as M
from oracle.abi_lists import abi_to_levels, oracle_to_abi

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2407_21637_gb300 import build as B
    B.build()
    from paper_2407_21637_gb300 import _lib
    torch.cuda.set_device(0)
    return _lib.load()


def _noalloc(lib, g, X, B, prec):
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    R = X.shape[1]
    return lib.hodlr_matvec_noalloc(g._h, R, ctypes.c_void_p(X.data_ptr()), R,
                                    ctypes.c_void_p(B.data_ptr()), R, prec, stream)


def _tol(h, X64, exact, u, tc=False):
    g_abs = M.abs_product(h, X64)
    if tc:   # tensor-core products (tf32 split of both factors)
        return (Bd.gamma(M.max_chain(h), 2 * u) + 14 * u) * g_abs + u * np.abs(exact)
    return (Bd.gamma(M.max_chain(h), u) + 2 * u) * g_abs + u * np.abs(exact)


@pytest.mark.parametrize("work,R", [("fp32", 1), ("fp32", 8), ("fp32", 64), ("fp64", 1), ("fp64", 3)])
def test_noalloc_matches_matvec_twice(lib, work, R):
    from paper_2407_21637_gb300 import HodlrMatrix, PREC
    n, depth, eps = 2000, 4, 1e-4
    spec = synth.KernelSpec(K.GAUSS, len2=0.01, diag=1e-2)
    tiers = ("fp64", "fp32", "bf16", "fp16", "e4m3")
    pts = synth.uniform_points_1d(n, 51)
    h = C.compress(pts, spec, n, depth, eps)
    C.assign_precisions(h, eps, work, tiers, norms="factors")
    C.store_all(h)
    ranks, U, V, D = oracle_to_abi(h)
    g = HodlrMatrix.from_factors(n, depth, ranks, U, V, D, eps=eps, work=work, tiers=tiers)
    dt = np.float64 if work == "fp64" else np.float32
    X = torch.from_numpy(synth.rhs_normal(n, R, 60 + R, dt)).cuda()
    ref = g.matvec(X).cpu().numpy().astype(np.float64)
    X64 = X.cpu().numpy().astype(np.float64)
    u = F.unit_roundoff(work)
    exact = M.hodlr_matvec(h, X64)
    tol = _tol(h, X64, exact, u)
    # hodlr_matvec runs fp32 products of 16 or more columns on the tensor
    # cores and fp64 products of more than one column on its two-barrier
    # kernel; otherwise both calls run the streamed kernel with the same
    # column batches, so B is bitwise the same
    same_kernel = (work == "fp32" and R < 16) or (work == "fp64" and R == 1)
    tol_ref = tol if same_kernel else _tol(h, X64, exact, u, tc=True)
    for _ in range(2):
        B = torch.full((n, R), float("nan"), dtype=X.dtype, device="cuda")
        st = _noalloc(lib, g, X, B, PREC[work])
        assert st == 0, lib.hodlr_last_error()
        got = B.cpu().numpy().astype(np.float64)
        if same_kernel:
            assert np.array_equal(got, ref)
        assert np.all(np.abs(got - ref) <= tol + tol_ref)
        assert np.all(np.abs(got - exact) <= tol)
    g.close()


def _random_hodlr(n, depth, rank, seed):
    """Generators of a HODLR matrix with every block of the given rank
    (orthonormal U, Gaussian V) and diagonally weighted Gaussian leaves, in
    the C ABI's per-node lists, plus the oracle's view of them."""
    rng = np.random.default_rng(seed)
    levels = C.Hodlr(n, depth).levels
    ranks, U, V = [], [], []
    for k in range(1, depth + 1):
        for (_s, m) in levels[k]:
            q, _ = np.linalg.qr(rng.standard_normal((m, rank)))
            ranks.append(rank)
            U.append(np.ascontiguousarray(q))
            V.append(np.ascontiguousarray(0.1 * rng.standard_normal((m, rank))))
    D = [np.ascontiguousarray(rng.standard_normal((m, m)) + m * np.eye(m)) for (_s, m) in levels[depth]]
    h = C.from_factors(n, depth, abi_to_levels(depth, U), abi_to_levels(depth, V), D)
    h.Uh, h.Vh, h.Dh = h.U, h.V, h.D      # fp64 storage: the stored values are these
    return ranks, U, V, D, h


def test_noalloc_batches_narrowed_to_the_array(lib):
    """fp64, rank 10 on every level of a depth-6 tree over 16384 rows: the
    partial sums of one column take about 80 KiB, so the 256 KiB array
    holds three columns and 16 columns run in six launches, against one
    launch of hodlr_matvec (different lane layouts, so agreement is within
    the rounding bound, not bitwise)."""
    from paper_2407_21637_gb300 import HodlrMatrix, PREC
    n, depth, R = 16384, 6, 16
    ranks, U, V, D, h = _random_hodlr(n, depth, 10, 71)
    g = HodlrMatrix.from_factors(n, depth, ranks, U, V, D, eps=1e-12, work="fp64", tiers=("fp64",))
    X = torch.from_numpy(synth.rhs_normal(n, R, 72, np.float64)).cuda()
    ref = g.matvec(X).cpu().numpy()
    X64 = X.cpu().numpy()
    exact = M.hodlr_matvec(h, X64)
    tol = _tol(h, X64, exact, F.unit_roundoff("fp64"))
    assert np.all(np.abs(ref - exact) <= tol)
    for _ in range(2):
        B = torch.full((n, R), float("nan"), dtype=torch.float64, device="cuda")
        st = _noalloc(lib, g, X, B, PREC["fp64"])
        assert st == 0, lib.hodlr_last_error()
        got = B.cpu().numpy()
        assert np.all(np.abs(got - ref) <= 2 * tol)
        assert np.all(np.abs(got - exact) <= tol)
    g.close()


def test_noalloc_rejects_a_matrix_too_large_for_the_array(lib):
    """fp64, rank 40 on every level: one column's partial sums need more
    than 256 KiB, so the call fails with HODLR_EINVAL before anything is
    enqueued and B keeps its contents; hodlr_matvec still runs it."""
    from paper_2407_21637_gb300 import HodlrMatrix, PREC
    n, depth, R = 16384, 6, 2
    ranks, U, V, D, h = _random_hodlr(n, depth, 40, 73)
    g = HodlrMatrix.from_factors(n, depth, ranks, U, V, D, eps=1e-12, work="fp64", tiers=("fp64",))
    X = torch.from_numpy(synth.rhs_normal(n, R, 74, np.float64)).cuda()
    B = torch.full((n, R), 3.25, dtype=torch.float64, device="cuda")
    st = _noalloc(lib, g, X, B, PREC["fp64"])
    assert st == 1, "expected HODLR_EINVAL"
    assert "256 KiB" in lib.hodlr_last_error().decode()
    torch.cuda.synchronize()
    assert bool(torch.all(B == 3.25))
    ref = g.matvec(X).cpu().numpy()
    X64 = X.cpu().numpy()
    exact = M.hodlr_matvec(h, X64)
    assert np.all(np.abs(ref - exact) <= _tol(h, X64, exact, F.unit_roundoff("fp64")))
    g.close()


def test_noalloc_rejects_bad_arguments(lib):
    assert lib.hodlr_matvec_noalloc(None, 1, None, 1, None, 1, 1, None) == 1
