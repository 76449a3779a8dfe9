"""HODLR_LU (Algorithm 3.4), its triangular solves, iterative refinement and
GMRES-based iterative refinement with the LU factors as preconditioner (the
use Sect. 3.4 names for a HODLR LU inside an iterative solver).

Test infrastructure (see ``oracle/__init__``).

Algorithm 3.4 on a matrix with the HODLR partition of the cluster tree, in
fp64, with every block held densely so that each step can be read off the
algorithm:

* at a leaf (k = l): the LU factorization of the dense diagonal block;
* above it: split the node into its children 1, 2 (eq. (2.1)); L11, U11 =
  HODLR_LU(H11); U12 solves L11 U12 = H12; L21 solves L21 U11 = H21; the
  Schur complement H22 - L21 U12 is truncated back to the HODLR format of
  the second child; L22, U22 = HODLR_LU(truncated Schur complement);
* L = [[L11, 0], [L21, L22]], U = [[U11, U12], [0, U22]].

Readings of points the paper leaves open:

* Pivoting: none.  The algorithm is a block LU that needs the leading
  blocks to be nonsingular; the leaf factorization is the Doolittle LU
  (unit lower L) written out below, which exists for the diagonally
  dominant workloads used here.
* Truncation of the Schur complement (line "rank truncation",
  Assumption 3.6): every off-diagonal block of every level inside the
  second child is replaced by its truncated SVD with the per-block relative
  Frobenius criterion of the construction (``compress.truncated_svd``);
  since the blocks partition the matrix, the whole truncation error obeys
  ||S^ - S~||_F <= eps ||S~||_F, the assumption's bound.  The leaves of the
  Schur complement are kept as computed.  eps_lu = 0 keeps every block
  exact (no truncation).
* Working precision: fp64 (u = 2^-53), so Cor. 3.11's hypothesis u <~ eps/n
  holds for the tolerances tested.

Parity: pinned (exact block LU when nothing is truncated: L U = H, unit
lower L and upper U, equal to the dense Doolittle LU; Cor. 3.11's backward
error bound with truncation; solves and refinement against the dense
system; GMRES exact after n steps without a preconditioner).
"""
from __future__ import annotations

import numpy as np
from scipy.linalg import solve_triangular

from .compress import truncated_svd


def doolittle(A: np.ndarray):
    """Dense LU without pivoting: A = L U, L unit lower, U upper (the leaf
    step of Algorithm 3.4)."""
    A = np.array(A, dtype=np.float64)
    m = A.shape[0]
    L = np.eye(m)
    U = np.zeros_like(A)
    for j in range(m):
        U[j, j:] = A[j, j:] - L[j, :j] @ U[:j, j:]
        if U[j, j] == 0.0:
            raise ZeroDivisionError("zero pivot")
        L[j + 1:, j] = (A[j + 1:, j] - L[j + 1:, :j] @ U[:j, j]) / U[j, j]
    return L, U


def truncate_subtree(S: np.ndarray, levels, k: int, i: int, eps: float) -> np.ndarray:
    """The block S (rows and columns of node (k, i)) with every off-diagonal
    block of the levels below node (k, i) replaced by its truncated SVD
    (relative Frobenius eps).  ``levels`` is the cluster tree."""
    S = np.array(S, dtype=np.float64)
    if eps <= 0.0:
        return S
    s0 = levels[k][i][0]
    depth = len(levels) - 1
    for kk in range(k + 1, depth + 1):
        span = 1 << (kk - k)
        for j in range(i * span, (i + 1) * span):
            (s, m), (s1, m1) = levels[kk][j], levels[kk][j ^ 1]
            blk = S[s - s0:s - s0 + m, s1 - s0:s1 - s0 + m1]
            Uu, V = truncated_svd(blk, eps)[:2]
            S[s - s0:s - s0 + m, s1 - s0:s1 - s0 + m1] = Uu @ V.T
    return S


def hodlr_lu(H: np.ndarray, levels, eps_lu: float = 0.0, k: int = 0, i: int = 0):
    """L, U of Algorithm 3.4 for the block of node (k, i) of H (dense,
    n x n for the root), with the Schur complements truncated to eps_lu."""
    depth = len(levels) - 1
    if k == depth:
        return doolittle(H)
    (s_a, m_a), (s_b, m_b) = levels[k + 1][2 * i], levels[k + 1][2 * i + 1]
    s0 = levels[k][i][0]
    a = slice(s_a - s0, s_a - s0 + m_a)
    b = slice(s_b - s0, s_b - s0 + m_b)
    H11, H12, H21, H22 = H[a, a], H[a, b], H[b, a], H[b, b]
    L11, U11 = hodlr_lu(H11, levels, eps_lu, k + 1, 2 * i)
    U12 = solve_triangular(L11, H12, lower=True, unit_diagonal=True)      # L11 U12 = H12
    L21 = solve_triangular(U11.T, H21.T, lower=True).T                    # L21 U11 = H21
    S = truncate_subtree(H22 - L21 @ U12, levels, k + 1, 2 * i + 1, eps_lu)
    L22, U22 = hodlr_lu(S, levels, eps_lu, k + 1, 2 * i + 1)
    n = m_a + m_b
    L = np.zeros((n, n))
    U = np.zeros((n, n))
    L[a, a], L[b, a], L[b, b] = L11, L21, L22
    U[a, a], U[a, b], U[b, b] = U11, U12, U22
    return L, U


def lu_solve(L: np.ndarray, U: np.ndarray, B: np.ndarray) -> np.ndarray:
    """X with L U X = B: forward substitution with the unit lower L, then
    back substitution with U."""
    Y = solve_triangular(L, B, lower=True, unit_diagonal=True)
    return solve_triangular(U, Y, lower=False)


def refine(A: np.ndarray, L: np.ndarray, U: np.ndarray, B: np.ndarray, tol: float = 1e-12,
           max_it: int = 20):
    """Iterative refinement with the LU factors as the solver and the
    residual B - A X in fp64: X_{j+1} = X_j + (LU)^{-1} (B - A X_j), until
    the normwise backward error ||B - A X||_F / (||A||_F ||X||_F) <= tol.
    Returns X and the backward errors of every iterate."""
    X = lu_solve(L, U, B)
    nA = np.linalg.norm(A)
    hist = []
    for _ in range(max_it + 1):
        R = B - A @ X
        be = np.linalg.norm(R) / (nA * np.linalg.norm(X))
        hist.append(be)
        if be <= tol:
            break
        X = X + lu_solve(L, U, R)
    return X, hist


def gmres(apply_A, b: np.ndarray, apply_M=None, tol: float = 1e-12, restart: int = 60, max_it: int = 600):
    """Left-preconditioned restarted GMRES for one right-hand side: x with
    M^{-1} A x ~ M^{-1} b (M^{-1} = apply_M, identity if None), Arnoldi with
    modified Gram-Schmidt and Givens rotations, stopped when the
    preconditioned residual falls to tol times its initial norm.  Returns x
    and the number of Arnoldi steps."""
    Minv = apply_M if apply_M is not None else (lambda v: v)
    n = b.shape[0]
    x = np.zeros(n)
    r = Minv(b - apply_A(x))
    beta0 = np.linalg.norm(r)
    if beta0 == 0.0:
        return x, 0
    steps = 0
    while steps < max_it:
        beta = np.linalg.norm(r)
        Q = np.zeros((n, restart + 1))
        Hh = np.zeros((restart + 1, restart))
        cs, sn = np.zeros(restart), np.zeros(restart)
        g = np.zeros(restart + 1)
        g[0] = beta
        Q[:, 0] = r / beta
        j = 0
        for j in range(restart):
            w = Minv(apply_A(Q[:, j]))
            for i in range(j + 1):
                Hh[i, j] = Q[:, i] @ w
                w = w - Hh[i, j] * Q[:, i]
            Hh[j + 1, j] = np.linalg.norm(w)
            if Hh[j + 1, j] > 0.0:
                Q[:, j + 1] = w / Hh[j + 1, j]
            for i in range(j):   # earlier rotations on the new column
                t = cs[i] * Hh[i, j] + sn[i] * Hh[i + 1, j]
                Hh[i + 1, j] = -sn[i] * Hh[i, j] + cs[i] * Hh[i + 1, j]
                Hh[i, j] = t
            den = np.hypot(Hh[j, j], Hh[j + 1, j])
            cs[j], sn[j] = Hh[j, j] / den, Hh[j + 1, j] / den
            Hh[j, j] = den
            Hh[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            steps += 1
            if abs(g[j + 1]) <= tol * beta0 or steps >= max_it:
                break
        k = j + 1
        y = solve_triangular(Hh[:k, :k], g[:k], lower=False)
        x = x + Q[:, :k] @ y
        r = Minv(b - apply_A(x))
        if np.linalg.norm(r) <= tol * beta0:
            break
    return x, steps


def gmres_ir(A: np.ndarray, L: np.ndarray, U: np.ndarray, B: np.ndarray, tol: float = 1e-12,
             inner_tol: float = 1e-4, max_it: int = 10):
    """GMRES-based iterative refinement: X_0 = (LU)^{-1} B; each step solves
    A D = R (R = B - A X_j in fp64) by GMRES preconditioned with the LU
    factors to inner_tol and adds D, until the normwise backward error
    ||B - A X||_F / (||A||_F ||X||_F) <= tol.  Returns X, the backward
    errors of the iterates and the GMRES steps of every refinement step."""
    X = lu_solve(L, U, B)
    nA = np.linalg.norm(A)
    hist, inner = [], []
    for _ in range(max_it + 1):
        R = B - A @ X
        be = np.linalg.norm(R) / (nA * np.linalg.norm(X))
        hist.append(be)
        if be <= tol:
            break
        D = np.zeros_like(X)
        its = 0
        for c in range(B.shape[1]):
            D[:, c], k = gmres(lambda v: A @ v, R[:, c], lambda v: lu_solve(L, U, v), tol=inner_tol)
            its = max(its, k)
        inner.append(its)
        X = X + D
    return X, hist, inner
