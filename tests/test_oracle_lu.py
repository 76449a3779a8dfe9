"""Pins for oracle.lu (Algorithm 3.4, HODLR_LU; Cor. 3.11): the leaf LU on a
textbook example, the block LU without truncation equal to the dense LU,
Assumption 3.6 for the Schur-complement truncation, Cor. 3.11's backward
error bound with truncation, the triangular solves and fp64-residual
iterative refinement to a 1e-12 backward error, GMRES (exact after n steps)
and GMRES-IR with a coarse LU, and a planted mistake (the Schur update
dropped) that the pins catch."""
import numpy as np
import pytest

import synth
from oracle import compress as C
from oracle import kernels as K
from oracle import lu as LU
from oracle import matvec as M

TIERS = ("fp64", "fp32", "bf16", "fp16", "e4m3")


def test_doolittle_textbook_example():
    A = np.array([[4.0, 3.0], [6.0, 3.0]])
    L, U = LU.doolittle(A)
    assert np.array_equal(L, [[1.0, 0.0], [1.5, 1.0]])
    assert np.array_equal(U, [[4.0, 3.0], [0.0, -1.5]])


def test_doolittle_random_dominant():
    rng = np.random.default_rng(0)
    A = rng.standard_normal((40, 40)) + 40 * np.eye(40)
    L, U = LU.doolittle(A)
    assert np.allclose(L @ U, A, rtol=0, atol=1e-12 * np.abs(A).max())
    assert np.array_equal(np.diag(L), np.ones(40))
    assert np.all(np.triu(L, 1) == 0) and np.all(np.tril(U, -1) == 0)


def _hodlr(n, depth, eps, seed=3):
    spec = synth.KernelSpec(K.INV_DIST, c=1e-3, diag=float(n))
    pts = synth.uniform_points_1d(n, seed)
    A = K.kernel_matrix(pts, spec)
    h = C.adaptive_hodlr(pts, spec, n, depth, eps, work="fp64", tiers=TIERS, A=A)
    return h, A


@pytest.mark.parametrize("n,depth", [(500, 3), (333, 2), (256, 0)])
def test_block_lu_without_truncation_is_the_dense_lu(n, depth):
    """eps_lu = 0: Algorithm 3.4 is an exact block LU, and the LU without
    pivoting is unique, so it equals the dense Doolittle LU of H-hat."""
    h, _A = _hodlr(n, depth, 1e-6)
    Hh = M.assemble(h)
    L, U = LU.hodlr_lu(Hh, h.levels, 0.0)
    Ld, Ud = LU.doolittle(Hh)
    assert np.allclose(L @ U, Hh, rtol=0, atol=1e-13 * np.abs(Hh).max())
    assert np.allclose(L, Ld, rtol=0, atol=1e-10) and np.allclose(U, Ud, rtol=0, atol=1e-10 * np.abs(Ud).max())


@pytest.mark.parametrize("eps", [1e-3, 1e-6])
def test_schur_truncation_obeys_assumption_3_6(eps):
    n, depth = 512, 4
    h, _A = _hodlr(n, depth, 1e-10)
    Hh = M.assemble(h)
    lv = h.levels
    (sa, ma), (sb, mb) = lv[1]
    L11, U11 = LU.hodlr_lu(Hh[:ma, :ma], lv, 0.0, 1, 0)
    U12 = np.linalg.solve(L11, Hh[:ma, ma:])
    L21 = np.linalg.solve(U11.T, Hh[ma:, :ma].T).T
    S = Hh[ma:, ma:] - L21 @ U12
    St = LU.truncate_subtree(S, lv, 1, 1, eps)
    assert np.linalg.norm(St - S) <= eps * np.linalg.norm(S)
    assert np.linalg.norm(St - S) > 0.0          # something was truncated
    for (s, m) in lv[depth][len(lv[depth]) // 2:]:   # the leaves are kept as computed
        assert np.array_equal(St[s - sb:s - sb + m, s - sb:s - sb + m], S[s - sb:s - sb + m, s - sb:s - sb + m])


@pytest.mark.parametrize("eps", [1e-4, 1e-8])
def test_corollary_3_11_backward_error(eps):
    """||L^ U^ - A||_F <= 2 (2^l - 1) eps ||A||_F + 11 (2^l - 1) eps ||L^||_F ||U^||_F
    (u = 2^-53 <= eps / n)."""
    n, depth = 512, 4
    h, A = _hodlr(n, depth, eps)
    L, U = LU.hodlr_lu(M.assemble(h), h.levels, eps)
    lhs = np.linalg.norm(L @ U - A)
    c = (1 << depth) - 1
    rhs = 2 * c * eps * np.linalg.norm(A) + 11 * c * eps * np.linalg.norm(L) * np.linalg.norm(U)
    assert lhs <= rhs
    assert lhs > 0.0


def test_solve_and_refinement_reach_1e_12():
    """Four right-hand sides; the truncated HODLR LU (eps 1e-4) as the solver
    and the fp64 residual with the dense A: the backward error falls below
    1e-12 within a few refinement steps."""
    n, depth, eps = 512, 4, 1e-4
    h, A = _hodlr(n, depth, eps)
    L, U = LU.hodlr_lu(M.assemble(h), h.levels, eps)
    B = synth.rhs_normal(n, 4, 5, np.float64)
    X, hist = LU.refine(A, L, U, B, tol=1e-12)
    assert hist[-1] <= 1e-12 and len(hist) <= 8
    assert hist[0] > hist[-1]
    assert np.linalg.norm(A @ X - B) <= 1e-11 * np.linalg.norm(A) * np.linalg.norm(X)


def test_planted_dropped_schur_update_is_caught(monkeypatch):
    """Planting the mistake S = H22 (the L21 U12 update dropped) breaks the
    exact block LU pin."""
    n, depth = 500, 3
    h, _A = _hodlr(n, depth, 1e-6)
    Hh = M.assemble(h)
    real = LU.solve_triangular

    def no_u12(a, b, lower=False, unit_diagonal=False, **kw):
        x = real(a, b, lower=lower, unit_diagonal=unit_diagonal, **kw)
        return np.zeros_like(x) if (lower and unit_diagonal) else x

    monkeypatch.setattr(LU, "solve_triangular", no_u12)
    L, U = LU.hodlr_lu(Hh, h.levels, 0.0)
    assert not np.allclose(L @ U, Hh, rtol=0, atol=1e-13 * np.abs(Hh).max())


def test_gmres_is_exact_after_n_steps_without_preconditioner():
    """Unpreconditioned GMRES on an n x n system reaches the solution in at
    most n Arnoldi steps (Krylov space = R^n)."""
    rng = np.random.default_rng(1)
    n = 30
    A = rng.standard_normal((n, n)) + 5 * np.eye(n)
    b = rng.standard_normal(n)
    x, steps = LU.gmres(lambda v: A @ v, b, tol=1e-13, restart=n)
    assert steps <= n
    assert np.allclose(x, np.linalg.solve(A, b), rtol=1e-10, atol=1e-10)


def test_gmres_ir_with_a_coarse_lu_reaches_1e_12():
    """NEXT-2's target on four right-hand sides: the HODLR LU truncated at
    eps = 1e-2 as GMRES preconditioner, fp64 residuals: backward error
    <= 1e-12 within a few refinement steps, few GMRES steps each."""
    n, depth = 512, 4
    h, A = _hodlr(n, depth, 1e-2)
    L, U = LU.hodlr_lu(M.assemble(h), h.levels, 1e-2)
    B = synth.rhs_normal(n, 4, 7, np.float64)
    X, hist, inner = LU.gmres_ir(A, L, U, B, tol=1e-12)
    assert hist[-1] <= 1e-12 and len(hist) <= 5
    assert max(inner) <= 30
