"""GPU parity of the adaptive-precision HODLR product (Algorithm 3.3) against
the CPU oracle, through the C ABI.

* precision rule: the block formats chosen on the device equal the oracle's
  (Algorithm 3.2 on the factor norms);
* storage: hodlr_export returns exactly the oracle's rounded generators (bit
  for bit, every format, with the per-block scales);
* product: fp64 working precision within 1e-12 relative (and the entrywise
  bound); fp32 within the entrywise a-priori bound
      |b^_i - b_i| <= (gamma_N(u) + 2u) g_i + u |b_i|,
  g = sum |U|(|V|^T|x|) + |D||x|, N = the longest accumulation chain,
  where b is the oracle's fp64 product on the same stored generators.
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

ALL = ("fp64", "fp32", "bf16", "fp16", "e4m3", "e5m2")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2407_21637_gb300 import build as B
    B.build()
    torch.cuda.set_device(0)


_CACHE = {}


def _oracle(n, depth, eps, spec, work, tiers, per_block=False, seed=31):
    key = (n, depth, eps, spec.kind, spec.c, spec.len2, spec.diag, work, tuple(tiers), per_block, seed)
    if key not in _CACHE:
        _CACHE[key] = _oracle_build(n, depth, eps, spec, work, tiers, per_block, seed)
    return _CACHE[key]


def _oracle_build(n, depth, eps, spec, work, tiers, per_block, seed):
    pts = synth.uniform_points_1d(n, seed)
    h = C.compress(pts, spec, n, depth, eps)
    C.assign_precisions(h, eps, work, tiers, per_block=per_block, norms="factors")
    C.store_all(h)
    return h


def _gpu(h, eps, work, tiers, per_block=False, max_nrhs=64):
    from paper_2407_21637_gb300 import HodlrMatrix
    ranks, U, V, D = oracle_to_abi(h)
    return HodlrMatrix.from_factors(h.n, h.depth, ranks, U, V, D, eps=eps, work=work, tiers=tiers,
                                    per_block=per_block, max_nrhs=max_nrhs)


TC_MIN_COLS = 16   # fp32 products with this many columns use the tensor-core leaf kernel


def _tol(h, X, ref, work):
    """Per-entry bound of the GPU product against the exact product of the
    stored factors: Higham's standard model for the longest accumulation
    chain N (gamma_N(u) g + 2u g for the format decode and scaling, u |b| for
    the final rounding), g = |U|(|V|^T |x|) + |D||x|.  With TC_MIN_COLS or more
    fp32 columns the leaf products and V^T X of the fp32 chunks run on the
    tensor cores on the tf32 hi/lo split of both factors; each product then
    carries up to about 2 * 2^-22 = 8u relative error (14u allowed) and the
    fp32 accumulation of the tensor core is allowed 2u per addition:
    (gamma_N(2u) + 14u) g + u |b|."""
    u = F.unit_roundoff(work)
    g = M.abs_product(h, X)
    if work == "fp32" and X.shape[1] >= TC_MIN_COLS:
        return (Bd.gamma(M.max_chain(h), 2 * u) + 14 * u) * g + u * np.abs(ref)
    return (Bd.gamma(M.max_chain(h), u) + 2 * u) * g + u * np.abs(ref)


SPEC_GAUSS = synth.KernelSpec(K.GAUSS, len2=0.01, diag=1e-2)
SPEC_INV = synth.KernelSpec(K.INV_DIST, c=1e-3, diag=1024.0)
SPEC_LOG = synth.KernelSpec(K.LOG, c=1e-4, diag=1024.0)


@pytest.mark.parametrize("spec", [SPEC_GAUSS, SPEC_INV, SPEC_LOG])
@pytest.mark.parametrize("eps", [1e-1, 1e-3, 1e-6])
@pytest.mark.parametrize("per_block", [False, True])
def test_tiers_match_oracle(spec, eps, per_block):
    tiers = ("fp64", "fp32", "bf16", "fp16", "e4m3")
    h = _oracle(1024, 4, eps, spec, "fp32", tiers, per_block=per_block)
    g = _gpu(h, eps, "fp32", tiers, per_block=per_block)
    got, ranks = g.block_tiers()
    want = [t for k in range(1, h.depth + 1) for t in h.tier[k]]
    assert ranks == oracle_to_abi(h)[0]
    assert got == want
    info = g.info()
    for k in range(1, h.depth + 1):
        up = h.u_prime[k] if not per_block else eps / (2 ** (k / 2) * max(h.xi[k]))
        assert info["u_prime"][k] == pytest.approx(up, rel=1e-12)
    g.close()


@pytest.mark.parametrize("fmt", ALL)
@pytest.mark.parametrize("work", ["fp32", "fp64"])
def test_export_is_bitwise_oracle_storage(fmt, work):
    """Large eps and a two-format set force every block into ``fmt``."""
    n, depth, eps = 768, 3, 0.5
    tiers = (fmt,)
    h = _oracle(n, depth, eps, SPEC_INV, work, tiers)
    for k in range(1, depth + 1):
        assert set(h.tier[k]) == {fmt if F.unit_roundoff(fmt) >= F.unit_roundoff(work) else work}
    g = _gpu(h, eps, work, tiers)
    U, V, D = g.export()
    q = 0
    for k in range(1, depth + 1):
        for i in range(1 << k):
            assert np.array_equal(U[q].view(np.int64), h.Uh[k][i].view(np.int64)), (k, i, "U")
            assert np.array_equal(V[q].view(np.int64), h.Vh[k][i].view(np.int64)), (k, i, "V")
            q += 1
    for i, d in enumerate(D):
        assert np.array_equal(d, h.Dh[i])
    g.close()


CASES = [
    # n, depth, eps, spec, work, tiers
    (1024, 4, 1e-8, SPEC_INV, "fp64", ("fp64",)),                      # the all-fp64 case
    (4096, 4, 1e-6, SPEC_GAUSS, "fp32", ("fp64", "fp32", "bf16", "fp16", "e4m3")),
    (1000, 3, 1e-2, SPEC_LOG, "fp32", ("fp64", "fp32", "bf16", "fp16", "e4m3")),  # ragged
    (777, 5, 1e-1, SPEC_INV, "fp32", ALL),                              # ragged, low tiers
    (2048, 5, 1e-3, SPEC_GAUSS, "fp64", ALL),
    (300, 0, 1e-3, SPEC_GAUSS, "fp32", ("fp32",)),                      # a single leaf
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"n{c[0]}_d{c[1]}_{c[4]}")
@pytest.mark.parametrize("R", [1, 3, 8, 64])
def test_matvec_parity(case, R):
    n, depth, eps, spec, work, tiers = case
    h = _oracle(n, depth, eps, spec, work, tiers)
    g = _gpu(h, eps, work, tiers)
    dt = np.float64 if work == "fp64" else np.float32
    X = synth.rhs_normal(n, R, 100 + R, dt)
    B = g.matvec(torch.from_numpy(X).cuda()).cpu().numpy().astype(np.float64)
    X64 = X.astype(np.float64)
    ref = M.hodlr_matvec(h, X64)
    assert np.all(np.abs(B - ref) <= _tol(h, X64, ref, work))
    if work == "fp64":
        assert np.linalg.norm(B - ref) <= 1e-12 * np.linalg.norm(ref)
    else:
        assert np.linalg.norm(B - ref) <= 1e-5 * np.linalg.norm(ref)
    g.close()


def test_batches_and_strides_and_determinism():
    """nrhs beyond max_nrhs is split into batches; strided X/B; repeated calls
    are bitwise identical."""
    n, depth, eps, work = 2000, 4, 1e-4, "fp32"
    tiers = ("fp64", "fp32", "bf16", "fp16", "e4m3")
    h = _oracle(n, depth, eps, SPEC_GAUSS, work, tiers)
    g = _gpu(h, eps, work, tiers, max_nrhs=16)
    R = 37
    Xfull = torch.from_numpy(synth.rhs_normal(n, 50, 7)).cuda()
    X = Xfull[:, 5:5 + R]                                 # ldx = 50
    Bfull = torch.full((n, 45), 7.0, device="cuda")
    Bv = Bfull[:, 3:3 + R]                                # ldb = 45
    g.matvec(X, out=Bv)
    b1 = Bv.cpu().numpy().astype(np.float64)
    X64 = X.cpu().numpy().astype(np.float64)
    ref = M.hodlr_matvec(h, X64)
    assert np.all(np.abs(b1 - ref) <= _tol(h, X64, ref, work))
    assert torch.all(Bfull[:, :3] == 7.0) and torch.all(Bfull[:, 3 + R:] == 7.0)
    for _ in range(3):
        g.matvec(X, out=Bv)
        assert np.array_equal(Bv.cpu().numpy(), b1.astype(np.float32))
    g.close()


@pytest.mark.parametrize("ld,off", [(8, 0), (12, 4), (10, 1)])
def test_eight_columns_lane_layouts(ld, off):
    """Eight fp32 columns: four per lane when rows start on 16-byte
    boundaries (contiguous X staged in shared memory, or strided X read
    directly), one per lane otherwise (ldx = 10, odd offset)."""
    n, depth, eps, work = 1500, 3, 1e-6, "fp32"
    tiers = ("fp64", "fp32", "bf16", "fp16", "e4m3")
    h = _oracle(n, depth, eps, SPEC_GAUSS, work, tiers)
    g = _gpu(h, eps, work, tiers)
    R = 8
    Xfull = torch.from_numpy(synth.rhs_normal(n, ld, 21, np.float32)).cuda()
    X = Xfull[:, off:off + R] if ld > R else Xfull
    Bfull = torch.full((n, ld), 5.0, device="cuda")
    Bv = Bfull[:, off:off + R] if ld > R else Bfull
    g.matvec(X, out=Bv)
    b = Bv.cpu().numpy().astype(np.float64)
    X64 = X.cpu().numpy().astype(np.float64)
    ref = M.hodlr_matvec(h, X64)
    assert np.all(np.abs(b - ref) <= _tol(h, X64, ref, work))
    if ld > R:
        assert torch.all(Bfull[:, :off] == 5.0) and torch.all(Bfull[:, off + R:] == 5.0)
    g.close()


def test_single_generator_pair_on_gpu():
    """D = 0 and one generator pair: the GPU writes exactly U (V^T x_sib) on the
    rows of node i and zero elsewhere (level/sibling indexing)."""
    from paper_2407_21637_gb300 import HodlrMatrix
    n, depth = 512, 3
    rng = np.random.default_rng(3)
    lv = C.cluster_tree(n, depth)
    for (k, i) in [(1, 0), (2, 3), (3, 5)]:
        h = C.Hodlr(n, depth)
        for kk in range(1, depth + 1):
            h.U[kk] = [np.zeros((m, 0)) for (_s, m) in lv[kk]]
            h.V[kk] = [np.zeros((m, 0)) for (_s, m) in lv[kk]]
        (s, m), (s1, m1) = lv[k][i], lv[k][i ^ 1]
        h.U[k][i] = rng.standard_normal((m, 2))
        h.V[k][i ^ 1] = rng.standard_normal((m1, 2))
        h.D = [np.zeros((mm, mm)) for (_s, mm) in lv[depth]]
        ranks, U, V, D = oracle_to_abi(h)
        g = HodlrMatrix.from_factors(n, depth, ranks, U, V, D, eps=1e-12, work="fp64", tiers=("fp64",))
        x = rng.standard_normal(n)
        b = g.matvec(torch.from_numpy(x).cuda()).cpu().numpy()
        expect = np.zeros(n)
        expect[s:s + m] = h.U[k][i] @ (h.V[k][i ^ 1].T @ x[s1:s1 + m1])
        assert np.array_equal(b != 0, expect != 0)
        assert np.allclose(b, expect, rtol=1e-13, atol=0)
        g.close()


def test_dense_kernel_matvec_matches_oracle():
    from paper_2407_21637_gb300 import dense_kernel_matvec
    n = 1500
    for kind, spec, pts in [
        (K.GAUSS, SPEC_GAUSS, synth.uniform_points_1d(n, 1)),
        (K.INV_DIST, synth.KernelSpec(K.INV_DIST, c=1e-3, diag=float(n)), synth.uniform_points_1d(n, 2)),
        (K.LOG, synth.KernelSpec(K.LOG, c=0.0), synth.grid_s2(n)),
        (K.INV_X_MINUS_Y, synth.KernelSpec(K.INV_X_MINUS_Y, diag=1.0), synth.grid_s1(n)),
    ]:
        A = K.kernel_matrix(pts, spec)
        X = synth.rhs_normal(n, 3, 5, np.float64)
        ref = A @ X
        rows = np.array([0, 7, 1499, 3, 800], dtype=np.int32)
        tp = torch.from_numpy(pts).cuda()
        B = dense_kernel_matvec(tp, kind, torch.from_numpy(X).cuda(), c=spec.c, len2=spec.len2,
                                diag=spec.diag).cpu().numpy()
        assert np.linalg.norm(B - ref) <= 1e-13 * np.linalg.norm(ref)
        Bs = dense_kernel_matvec(tp, kind, torch.from_numpy(X).cuda(), c=spec.c, len2=spec.len2,
                                 diag=spec.diag, rows=torch.from_numpy(rows).cuda()).cpu().numpy()
        assert np.allclose(Bs, ref[rows], rtol=1e-12, atol=1e-12 * np.abs(ref).max())


def test_matvec_rejects_wrong_dtype_and_overlap():
    from paper_2407_21637_gb300 import HodlrError
    h = _oracle(256, 2, 1e-3, SPEC_GAUSS, "fp32", ("fp32",))
    g = _gpu(h, 1e-3, "fp32", ("fp32",))
    with pytest.raises(ValueError):
        g.matvec(torch.zeros(256, dtype=torch.float64, device="cuda"))
    X = torch.zeros((256, 4), device="cuda")
    with pytest.raises(HodlrError):
        g.matvec(X, out=X)
    g.close()
