"""Pins for oracle.matvec (Algorithm 3.3): dense assembly, brute-force dense
products, Thm 3.5, level/sibling indexing, linearity, and the qualitative
behaviour of Fig. 4.2 (parity unpinned: the figure prints no numbers)."""
import numpy as np
import pytest

import synth
from oracle import bounds as Bd
from oracle import compress as C
from oracle import formats as F
from oracle import kernels as K
from oracle import matvec as M

TIERS = ("fp64", "fp32", "bf16", "fp16", "e4m3")


def _build(n, depth, eps, spec, seed=21, work="fp64", tiers=TIERS):
    pts = synth.uniform_points_1d(n, seed)
    A = K.kernel_matrix(pts, spec)
    h = C.adaptive_hodlr(pts, spec, n, depth, eps, work=work, tiers=tiers, A=A)
    return h, A


@pytest.mark.parametrize("n,depth,R", [(512, 3, 1), (1000, 4, 3), (777, 5, 8), (64, 0, 2)])
def test_matvec_equals_dense_assembly(n, depth, R):
    spec = synth.KernelSpec(K.INV_DIST, c=1e-3, diag=float(n))
    h, _A = _build(n, depth, 1e-4, spec)
    X = synth.rhs_normal(n, R, 3, np.float64)
    b = M.hodlr_matvec(h, X)
    ref = M.assemble(h) @ X
    assert np.linalg.norm(b - ref) <= 1e-14 * np.linalg.norm(ref)


@pytest.mark.parametrize("eps", [1e-3, 1e-6, 1e-9])
def test_theorem_3_5_backward_error(eps):
    """u(fp64) <= eps/n holds here, so ||b^ - A x|| / (||A||_F ||x||) obeys Thm 3.5."""
    n, depth = 1024, 4
    spec = synth.KernelSpec(K.INV_DIST, c=1e-3, diag=float(n))
    h, A = _build(n, depth, eps, spec)
    assert F.unit_roundoff("fp64") <= eps / n
    x = synth.rhs_normal(n, 1, 4, np.float64)[:, 0]
    b = M.hodlr_matvec(h, x)
    be = np.linalg.norm(b - A @ x) / (np.linalg.norm(A) * np.linalg.norm(x))
    assert be <= Bd.matvec_backward_bound(eps, depth)


def test_single_generator_pair_indexing():
    """D = 0 and one non-zero generator pair at level k: b is non-zero exactly
    on the rows of node i and equals U (V^T x[sibling rows])."""
    n, depth = 96, 3
    rng = np.random.default_rng(2)
    lv = C.cluster_tree(n, depth)
    for k in range(1, depth + 1):
        for i in range(1 << k):
            U = [[np.zeros((m, 1)) for (_s, m) in lv[kk]] for kk in range(depth + 1)]
            V = [[np.zeros((m, 1)) for (_s, m) in lv[kk]] for kk in range(depth + 1)]
            (s, m), (s1, m1) = lv[k][i], lv[k][i ^ 1]
            U[k][i] = rng.standard_normal((m, 1))
            V[k][i ^ 1] = rng.standard_normal((m1, 1))
            D = [np.zeros((mm, mm)) for (_s, mm) in lv[depth]]
            h = C.from_factors(n, depth, U, V, D)
            h.tier = [[]] + [["fp64"] * (1 << kk) for kk in range(1, depth + 1)]
            C.store_all(h)
            x = rng.standard_normal(n)
            b = M.hodlr_matvec(h, x)
            expect = np.zeros(n)
            expect[s:s + m] = U[k][i][:, 0] * float(V[k][i ^ 1][:, 0] @ x[s1:s1 + m1])
            assert np.array_equal(b != 0, expect != 0)
            assert np.allclose(b, expect, rtol=1e-15, atol=0)


def test_linearity():
    n, depth = 700, 4
    spec = synth.KernelSpec(K.GAUSS, len2=0.01, diag=1e-2)
    h, _A = _build(n, depth, 1e-3, spec)
    rng = np.random.default_rng(8)
    X, Y = rng.standard_normal((n, 2)), rng.standard_normal((n, 2))
    a, b = 0.7, -2.5
    lhs = M.hodlr_matvec(h, a * X + b * Y)
    rhs = a * M.hodlr_matvec(h, X) + b * M.hodlr_matvec(h, Y)
    assert np.linalg.norm(lhs - rhs) <= 1e-14 * np.linalg.norm(rhs)


def test_abs_product_bounds_fp32_simulation():
    """The entrywise bound gamma_N(u) g used for GPU parity holds for the
    simulated fp32 evaluation of Algorithm 3.3."""
    n, depth = 512, 3
    spec = synth.KernelSpec(K.GAUSS, len2=0.01, diag=1e-2)
    h, _A = _build(n, depth, 1e-6, spec, work="fp32")
    x = synth.rhs_normal(n, 1, 5, np.float32).astype(np.float64)
    b64 = M.hodlr_matvec(h, x)
    b32 = M.hodlr_matvec(h, x, work="fp32")
    g = M.abs_product(h, x)
    tol = Bd.gamma(M.max_chain(h), F.unit_roundoff("fp32")) * g
    assert np.all(np.abs(b32 - b64) <= tol)
    assert np.max(np.abs(b32 - b64)) > 0       # the simulation really rounds


def test_planted_dropped_level_is_caught():
    """Skipping one level in Algorithm 3.3 (a plausible indexing slip) breaks
    agreement with the dense assembly."""
    n, depth = 512, 3
    spec = synth.KernelSpec(K.INV_DIST, c=1e-3, diag=float(n))
    h, _A = _build(n, depth, 1e-6, spec)
    x = synth.rhs_normal(n, 1, 3, np.float64)
    saved = h.Uh[2]
    h.Uh[2] = [u * 0 for u in saved]
    b = M.hodlr_matvec(h, x)
    h.Uh[2] = saved
    ref = M.assemble(h) @ x
    assert np.linalg.norm(b - ref) > 1e-6 * np.linalg.norm(ref)


PAPER_MATS = {
    # Sect. 4.2, eq. (4.1): n = 2000, depth 8
    "mat-1": (lambda n: synth.grid_s1(n), synth.KernelSpec(K.INV_X_MINUS_Y, diag=1.0)),
    "mat-3": (lambda n: synth.grid_s2(n), synth.KernelSpec(K.GAUSS, len2=2.0 * 1.0 ** 2)),
}


@pytest.mark.slow
@pytest.mark.parametrize("name", list(PAPER_MATS))
def test_fig_4_2_qualitative(name):
    """Fig. 4.2 behaviour (parity unpinned, qualitative): with fp64 working
    precision the backward error follows eps and stays under Thm 3.5; with
    fp32 working precision it floors near u(fp32) once eps < u(fp32)."""
    n, depth = 2000, 8
    ptsf, spec = PAPER_MATS[name]
    pts = ptsf(n)
    A = K.kernel_matrix(pts, spec)
    x = synth.rhs_uniform(n, 1, 10)[:, 0]
    nA, nx = np.linalg.norm(A), np.linalg.norm(x)
    errs = {}
    for eps in (1e-4, 1e-10):
        h = C.adaptive_hodlr(pts, spec, n, depth, eps, work="fp64",
                             tiers=("fp64", "fp32", "fp16", "bf16", "e5m2"), A=A)
        b64 = M.hodlr_matvec(h, x)
        errs[("fp64", eps)] = np.linalg.norm(b64 - A @ x) / (nA * nx)
        b32 = M.hodlr_matvec(h, x, work="fp32")
        errs[("fp32", eps)] = np.linalg.norm(b32 - A @ x) / (nA * nx)
        assert errs[("fp64", eps)] <= Bd.matvec_backward_bound(eps, depth)
    # fp64 follows eps: shrinking eps by 1e6 shrinks the error by >= 1e3
    assert errs[("fp64", 1e-10)] < 1e-3 * errs[("fp64", 1e-4)]
    # fp32 floors near u(fp32): at eps = 1e-10 < u it is far above the fp64 error
    assert errs[("fp32", 1e-10)] > 10 * errs[("fp64", 1e-10)]
    assert errs[("fp32", 1e-10)] < 1e3 * F.unit_roundoff("fp32")


@pytest.mark.parametrize("n,depth,R", [(1000, 4, 3), (777, 5, 1), (512, 3, 8)])
def test_sampled_rows_equal_the_dense_product(n, depth, R):
    """The sampled-row product (used where the full product is too large for
    the host) equals the dense assembly's rows times x, and its |.| twin the
    rows of abs_product; rows include both ends of leaves and of the matrix."""
    spec = synth.KernelSpec(K.GAUSS, len2=0.01, diag=1e-2)
    h, _A = _build(n, depth, 1e-6, spec)
    X = synth.rhs_normal(n, R, 9, np.float64)
    rng = np.random.default_rng(4)
    ends = [s for (s, m) in h.levels[h.depth]] + [s + m - 1 for (s, m) in h.levels[h.depth]]
    rows = np.unique(np.concatenate([rng.integers(0, n, 40), ends, [0, n - 1]]))
    ref = M.assemble(h)[rows] @ X
    got = M.hodlr_matvec_rows(h, X, rows)
    assert np.allclose(got, ref, rtol=1e-13, atol=1e-13 * np.abs(ref).max())
    assert np.allclose(M.abs_product_rows(h, X, rows), M.abs_product(h, X)[rows], rtol=1e-13, atol=0)
