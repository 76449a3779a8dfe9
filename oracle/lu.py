"""HODLR_LU (Algorithm 3.4), its triangular solves, and iterative refinement.

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
system).
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
