"""Leaf products on the tensor cores (fp32 work, 16 or more right-hand sides):
parity of the whole product against the oracle (Algorithm 3.3 on the stored
factors, fp64), for ragged leaves (row counts that are not multiples of 32,
128 or of the 32-column K-chunks), column counts that are not multiples of
16 or 4, strided X and B, batches of columns, and bitwise repeatability.

The bound: the tensor-core products are sums of tf32 products of the split
fp32 values (hi + lo, both parts of both factors), so each product carries
up to about 2 * 2^-22 = 8u relative error from the rounding of the lo
parts; 14u is allowed, and the tensor core's fp32 accumulation 2u per
addition: |b_gpu - b| <= (gamma_N(2u) + 14u) g + u|b| with
g = |U|(|V|^T|x|) + |D||x| and N the longest accumulation chain.
"""
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


def _setup(n, depth, eps, spec, seed, tiers=TIERS):
    from paper_2407_21637_gb300 import HodlrMatrix
    pts = synth.uniform_points_1d(n, seed)
    h = C.compress(pts, spec, n, depth, eps)
    C.assign_precisions(h, eps, "fp32", tiers, norms="factors")
    C.store_all(h)
    ranks, U, V, D = oracle_to_abi(h)
    g = HodlrMatrix.from_factors(n, depth, ranks, U, V, D, eps=eps, work="fp32", tiers=tiers, max_nrhs=256)
    return h, g


def _tol_tc(h, X64, ref):
    u = F.unit_roundoff("fp32")
    return (Bd.gamma(M.max_chain(h), 2 * u) + 14 * u) * M.abs_product(h, X64) + u * np.abs(ref)


@pytest.mark.parametrize("n,depth", [(1024, 2), (1000, 3), (1500, 2), (700, 1)])
@pytest.mark.parametrize("R", [16, 17, 40, 64])
def test_tc_parity(n, depth, R):
    spec = synth.KernelSpec(K.GAUSS, len2=0.01, diag=1e-2)
    h, g = _setup(n, depth, 1e-6, spec, 7)
    X = synth.rhs_normal(n, R, 300 + R, np.float32)
    B = g.matvec(torch.from_numpy(X).cuda()).cpu().numpy().astype(np.float64)
    X64 = X.astype(np.float64)
    ref = M.hodlr_matvec(h, X64)
    err = np.abs(B - ref)
    tol = _tol_tc(h, X64, ref)
    assert np.all(err <= tol), float(np.max(err / tol))
    assert np.linalg.norm(B - ref) <= 1e-5 * np.linalg.norm(ref)
    g.close()


@pytest.mark.parametrize("n,depth", [(4096, 4), (2000, 3), (1500, 2)])
@pytest.mark.parametrize("R", [16, 64])
def test_tc_fp32_generators(n, depth, R):
    """Every generator stored in fp32, so every V chunk that covers one run
    of rows goes to the tensor cores in a V group: all of them for n = 4096
    and 2000 (256-row padded leaves), and for n = 1500 (375-row leaves) the
    256- and 119-row pieces of the leaves, while the chunks that span two
    leaves stay on the CUDA cores."""
    spec = synth.KernelSpec(K.GAUSS, len2=0.01, diag=1e-2)
    h, g = _setup(n, depth, 1e-6, spec, 5, tiers=("fp32",))
    X = synth.rhs_normal(n, R, 900 + R, np.float32)
    B = g.matvec(torch.from_numpy(X).cuda()).cpu().numpy().astype(np.float64)
    X64 = X.astype(np.float64)
    ref = M.hodlr_matvec(h, X64)
    tol = _tol_tc(h, X64, ref)
    assert np.all(np.abs(B - ref) <= tol), float(np.max(np.abs(B - ref) / tol))
    g.close()


def test_tc_wide_strided_and_repeatable():
    """256 columns in one launch, 300 in two; X and B strided inside wider
    buffers; repeated products are bitwise identical."""
    n, depth = 2048, 3
    spec = synth.KernelSpec(K.INV_DIST, c=1e-3, diag=float(n))
    h, g = _setup(n, depth, 1e-4, spec, 11)
    for R in (256, 300):
        Xw = torch.from_numpy(synth.rhs_normal(n, R + 12, 5, np.float32)).cuda()
        X = Xw[:, 4:4 + R]
        Bw = torch.full((n, R + 8), 3.0, device="cuda")
        Bv = Bw[:, 4:4 + R]
        g.matvec(X, out=Bv)
        b1 = Bv.cpu().numpy().astype(np.float64)
        X64 = X.cpu().numpy().astype(np.float64)
        ref = M.hodlr_matvec(h, X64)
        assert np.all(np.abs(b1 - ref) <= _tol_tc(h, X64, ref))
        assert torch.all(Bw[:, :4] == 3.0) and torch.all(Bw[:, 4 + R:] == 3.0)
        g.matvec(X, out=Bv)
        assert np.array_equal(Bv.cpu().numpy(), b1.astype(np.float32))
    g.close()


def test_tc_matches_cuda_core_path_closely():
    """The tensor-core product (16 columns) and the CUDA-core product (the
    same columns one at a time) agree to within both bounds."""
    n, depth = 1024, 2
    spec = synth.KernelSpec(K.GAUSS, len2=0.01, diag=1e-2)
    h, g = _setup(n, depth, 1e-6, spec, 3)
    X = torch.from_numpy(synth.rhs_normal(n, 16, 77, np.float32)).cuda()
    B16 = g.matvec(X).cpu().numpy().astype(np.float64)
    B1 = np.stack([g.matvec(X[:, j].contiguous()).cpu().numpy() for j in range(16)], axis=1).astype(np.float64)
    X64 = X.cpu().numpy().astype(np.float64)
    ref = M.hodlr_matvec(h, X64)
    u = F.unit_roundoff("fp32")
    tol1 = (Bd.gamma(M.max_chain(h), u) + 2 * u) * M.abs_product(h, X64) + u * np.abs(ref)
    assert np.all(np.abs(B16 - B1) <= _tol_tc(h, X64, ref) + tol1)
    g.close()
