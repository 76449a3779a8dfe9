"""GPU construction (hodlr_build, Algorithm 3.2 with a randomized range
finder) against the CPU oracle's truncated-SVD construction.

Construction is an approximation, so parity is checked through what the
paper fixes: every block satisfies Def. 2.3 (relative Frobenius error <= eps,
hence Lemma 2.4 at every level), U has orthonormal columns (eq. (3.1)), the
global error obeys Thm 3.1, the block formats follow Algorithm 3.2 on the
exact block norms, and the ranks are close to the truncated SVD's (the
randomized rank can exceed the optimal one by a few).
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
from oracle.abi_lists import abi_to_levels

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2407_21637_gb300 import build as B
    B.build()
    torch.cuda.set_device(0)


def _gpu_build(pts, spec, depth, eps, work, tiers, **kw):
    from paper_2407_21637_gb300 import HodlrMatrix
    return HodlrMatrix.build(torch.from_numpy(pts).cuda(), spec.kind, depth, eps, c=spec.c,
                             len2=spec.len2, diag=spec.diag, work=work, tiers=tiers, **kw)


def _as_oracle(g, n, depth):
    """The GPU's stored generators (exported, decoded) as an oracle object."""
    U, V, D = g.export()
    h = C.from_factors(n, depth, abi_to_levels(depth, U), abi_to_levels(depth, V), D)
    return h


CASES = [
    ("gauss", synth.KernelSpec(K.GAUSS, len2=0.01, diag=1e-2), 2048, 3, 1e-6),
    ("inv", synth.KernelSpec(K.INV_DIST, c=1e-3, diag=1024.0), 1024, 4, 1e-8),
    ("log", synth.KernelSpec(K.LOG, c=1e-4, diag=1024.0), 1500, 4, 1e-4),
    ("invxy", synth.KernelSpec(K.INV_X_MINUS_Y, diag=1.0), 1000, 3, 1e-3),
]


@pytest.mark.parametrize("name,spec,n,depth,eps", CASES, ids=[c[0] for c in CASES])
def test_build_fp64_blocks_meet_def_2_3(name, spec, n, depth, eps):
    pts = synth.grid_s1(n) if spec.kind == K.INV_X_MINUS_Y else synth.uniform_points_1d(n, 41)
    A = K.kernel_matrix(pts, spec)
    g = _gpu_build(pts, spec, depth, eps, "fp64", ("fp64",))
    h = _as_oracle(g, n, depth)
    ref = C.compress(pts, spec, n, depth, eps, A=A)
    for k in range(1, depth + 1):
        for i, (s, m) in enumerate(h.levels[k]):
            (s1, m1) = h.levels[k][i ^ 1]
            blk = A[s:s + m, s1:s1 + m1]
            U, Vs = h.U[k][i], h.V[k][i ^ 1]
            err = np.linalg.norm(blk - U @ Vs.T)
            assert err <= eps * np.linalg.norm(blk) * (1 + 1e-6) + 1e-300, (k, i)
            r = U.shape[1]
            assert np.linalg.norm(U.T @ U - np.eye(r)) <= 1e-12
            r_opt = ref.rank(k, i)
            assert r_opt <= r <= r_opt + 3, (k, i, r, r_opt)
    At = M.assemble(h, stored=False)
    for k in range(depth + 1):                     # Lemma 2.4 at every level
        for (s, m) in h.levels[k]:
            sl = slice(s, s + m)
            assert np.linalg.norm(At[sl, sl] - A[sl, sl]) <= eps * np.linalg.norm(A[sl, sl]) * (1 + 1e-6)
    # leaves are the kernel entries evaluated on the GPU (exp/log/sqrt of CUDA's
    # math library vs the host's: a few ulps, amplified by r^2/len2 <= 100)
    assert np.allclose(np.concatenate([d.ravel() for d in h.D]),
                       np.concatenate([A[s:s + m, s:s + m].ravel() for (s, m) in h.levels[depth]]),
                       rtol=1e-13, atol=0)
    g.close()


@pytest.mark.parametrize("eps", [1e-1, 1e-3, 1e-6])
@pytest.mark.parametrize("per_block", [False, True])
def test_build_adaptive_tiers_and_theorem_3_1(eps, per_block):
    n, depth = 2048, 4
    spec = synth.KernelSpec(K.INV_DIST, c=1e-3, diag=float(n))
    tiers = ("fp64", "fp32", "bf16", "fp16", "e4m3")
    pts = synth.uniform_points_1d(n, 42)
    A = K.kernel_matrix(pts, spec)
    g = _gpu_build(pts, spec, depth, eps, "fp32", tiers, per_block=per_block)
    got, _ = g.block_tiers()
    # Algorithm 3.2 with the exact block norms of H applied to the GPU's blocks
    h = _as_oracle(g, n, depth)
    h.block_norm2 = [[]] + [[float(np.sum(A[s:s + m, s1:s1 + m1] ** 2))
                             for (s, m), (s1, m1) in zip(h.levels[k], [h.levels[k][i ^ 1] for i in range(1 << k)])]
                            for k in range(1, depth + 1)]
    h.norm2_all = float(np.sum(A * A))
    C.assign_precisions(h, eps, "fp32", tiers, per_block=per_block, norms="original")
    want = [t for k in range(1, depth + 1) for t in h.tier[k]]
    info = g.info()
    for k in range(1, depth + 1):
        up = h.u_prime[k] if not per_block else eps / (2 ** (k / 2) * max(h.xi[k]))
        assert info["u_prime"][k] == pytest.approx(up, rel=1e-10)
    assert got == want
    # the stored matrix (export = decoded stored values) obeys Thm 3.1
    err = np.linalg.norm(M.assemble(h, stored=False) - A)
    assert err <= Bd.global_bound_rule(eps, depth) * np.linalg.norm(A)
    g.close()


def test_build_then_matvec_backward_error():
    """Full path on the GPU: build, then the product, against the dense
    kernel matrix (Thm 3.5 for fp64 work, u <= eps/n)."""
    n, depth, eps = 2048, 4, 1e-9
    spec = synth.KernelSpec(K.GAUSS, len2=0.01, diag=1e-2)
    pts = synth.uniform_points_1d(n, 43)
    A = K.kernel_matrix(pts, spec)
    g = _gpu_build(pts, spec, depth, eps, "fp64", ("fp64", "fp32", "bf16", "fp16", "e4m3"))
    x = synth.rhs_normal(n, 1, 9, np.float64)[:, 0]
    b = g.matvec(torch.from_numpy(x).cuda()).cpu().numpy()
    be = np.linalg.norm(b - A @ x) / (np.linalg.norm(A) * np.linalg.norm(x))
    assert F.unit_roundoff("fp64") <= eps / n
    assert be <= Bd.matvec_backward_bound(eps, depth)
    g.close()


def test_build_is_deterministic():
    n, depth, eps = 1024, 3, 1e-5
    spec = synth.KernelSpec(K.GAUSS, len2=0.01, diag=1e-2)
    pts = synth.uniform_points_1d(n, 44)
    g1 = _gpu_build(pts, spec, depth, eps, "fp32", ("fp32", "bf16"), seed=5)
    g2 = _gpu_build(pts, spec, depth, eps, "fp32", ("fp32", "bf16"), seed=5)
    U1, V1, _ = g1.export()
    U2, V2, _ = g2.export()
    for a, b in zip(U1 + V1, U2 + V2):
        assert np.array_equal(a, b)
    g1.close()
    g2.close()


@pytest.mark.parametrize("sketch", [16, 32, 64])
def test_build_oversized_sketch_is_exact(sketch):
    """A sketch far wider than the numerical rank (ranks 2-7 here) leaves
    columns that lie in the span of the others to working accuracy; the
    orthonormalisation must drop them, not amplify rounding noise."""
    n, depth, eps = 4096, 4, 1e-6
    spec = synth.KernelSpec(K.GAUSS, len2=0.01, diag=1e-2)
    pts = synth.uniform_points_1d(n, 45)
    A = K.kernel_matrix(pts, spec)
    g = _gpu_build(pts, spec, depth, eps, "fp64", ("fp64",), sketch=sketch, max_sketch=64)
    h = _as_oracle(g, n, depth)
    for k in range(1, depth + 1):
        for i, (s, m) in enumerate(h.levels[k]):
            (s1, m1) = h.levels[k][i ^ 1]
            blk = A[s:s + m, s1:s1 + m1]
            U, Vs = h.U[k][i], h.V[k][i ^ 1]
            assert np.linalg.norm(blk - U @ Vs.T) <= eps * np.linalg.norm(blk) * (1 + 1e-6)
            assert U.shape[1] <= 10
            assert np.linalg.norm(U.T @ U - np.eye(U.shape[1])) <= 1e-12
    g.close()


def test_build_2d_points_in_kd_order():
    """The LU workload's kernel, log(r + 1e-4) + n I, on 2D points U[0,1]^2
    put in kd order by hodlr_tree_order (eps 1e-4, fp64 work): every block
    meets Def. 2.3 with a rank within +5 of the truncated SVD's, and the
    product's backward error obeys Thm 3.5."""
    from paper_2407_21637_gb300 import tree_order
    n, depth, eps = 1024, 3, 1e-4
    spec = synth.KernelSpec(K.LOG, c=1e-4, diag=float(n))
    raw = synth.uniform_points_2d(n, 47)
    pts = np.ascontiguousarray(raw[tree_order(raw, depth)])
    A = K.kernel_matrix(pts, spec)
    g = _gpu_build(pts, spec, depth, eps, "fp64", ("fp64",))
    h = _as_oracle(g, n, depth)
    ref = C.compress(pts, spec, n, depth, eps, A=A)
    for k in range(1, depth + 1):
        for i, (s, m) in enumerate(h.levels[k]):
            (s1, m1) = h.levels[k][i ^ 1]
            blk = A[s:s + m, s1:s1 + m1]
            err = np.linalg.norm(blk - h.U[k][i] @ h.V[k][i ^ 1].T)
            assert err <= eps * np.linalg.norm(blk) * (1 + 1e-6), (k, i)
            r, r_opt = h.U[k][i].shape[1], ref.rank(k, i)
            assert r_opt <= r <= r_opt + 5, (k, i, r, r_opt)
    x = synth.rhs_normal(n, 1, 11, np.float64)[:, 0]
    b = g.matvec(torch.from_numpy(x).cuda()).cpu().numpy()
    assert F.unit_roundoff("fp64") <= eps / n
    assert np.linalg.norm(b - A @ x) / (np.linalg.norm(A) * np.linalg.norm(x)) <= Bd.matvec_backward_bound(eps, depth)
    g.close()
