"""hodlr_matvec_noalloc: the product for callers that cannot allocate device
memory at the time of the call (its scratch is a static device array inside
the library).  Through the C ABI, two calls in a row must agree with
hodlr_matvec within the parity tolerance of the other product tests.

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
from oracle.abi_lists import oracle_to_abi

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2407_21637_gb300 import build as B
    B.build()
    from paper_2407_21637_gb300 import _lib
    torch.cuda.set_device(0)
    return _lib.load()


@pytest.mark.parametrize("work,R", [("fp32", 1), ("fp32", 8), ("fp32", 64), ("fp64", 3)])
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
    g_abs = M.abs_product(h, X64)
    tol = (Bd.gamma(M.max_chain(h), u) + 2 * u) * g_abs + u * np.abs(exact)
    # the reference product (hodlr_matvec) runs its leaf products and the
    # fp32 V^T X on the tensor cores from 16 fp32 columns on (tf32 products
    # of the hi/lo split of both factors)
    tol_ref = tol if (work != "fp32" or R < 16) else \
        (Bd.gamma(M.max_chain(h), 2 * u) + 14 * u) * g_abs + u * np.abs(exact)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for _ in range(2):
        B = torch.full((n, R), float("nan"), dtype=X.dtype, device="cuda")
        st = lib.hodlr_matvec_noalloc(g._h, R, ctypes.c_void_p(X.data_ptr()), R,
                                      ctypes.c_void_p(B.data_ptr()), R, PREC[work], stream)
        assert st == 0, lib.hodlr_last_error()
        got = B.cpu().numpy().astype(np.float64)
        assert np.all(np.abs(got - ref) <= tol + tol_ref)
        assert np.all(np.abs(got - exact) <= tol)
    g.close()


def test_noalloc_rejects_bad_arguments(lib):
    assert lib.hodlr_matvec_noalloc(None, 1, None, 1, None, 1, 1, None) == 1
