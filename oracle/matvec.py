"""HODLR_MATVEC (Algorithm 3.3) and the dense assembly of H-hat.

Test infrastructure (see ``oracle/__init__``).

Algorithm 3.3: b = 0; for k = 1..l, for every sibling pair (2i-1, 2i):
b_{2i-1} += U_{2i-1} (V_{2i}^T x_{2i}),  b_{2i} += U_{2i} (V_{2i-1}^T x_{2i-1});
then b_i += D_i x_i for every leaf.  Low-precision generators are used at their
stored values, cast to the working precision (Sect. 3.3).

``work="fp64"`` computes in fp64 (the plain definition, used as the parity
reference).  ``work="fp32"`` and ``work="bf16"`` simulate the working precision
of Sect. 4.2 by rounding every product and every partial sum (the paper
simulates with a rounding function as well); they are used only for the
qualitative reproduction of Fig. 4.2.

``abs_product`` returns g = sum_blocks |U| (|V|^T |x|) + |D| |x|, the quantity
that bounds the rounding error of the two-stage product U (V^T x) entrywise
(standard model, Higham sect. 3.5, cited in the proof of Lemma 3.3).

Parity: pinned (dense assembly times x and brute-force dense A x within the
paper's bounds; the dense assembly is an independent path through the same
stored factors).
"""
from __future__ import annotations

import numpy as np

from . import formats as F


def _factors(h, stored: bool):
    if stored:
        return h.Uh, h.Vh, h.Dh
    return h.U, h.V, h.D


def _mm(A: np.ndarray, B: np.ndarray, work: str) -> np.ndarray:
    """A @ B in the working precision (fp64 exact library product, or every
    product and partial sum rounded to ``work``)."""
    if work == "fp64":
        return A @ B
    if work == "fp32":
        A32, B32 = A.astype(np.float32), B.astype(np.float32)
        acc = np.zeros((A.shape[0], B.shape[1]), dtype=np.float32)
        for j in range(A.shape[1]):
            acc = acc + A32[:, j:j + 1] * B32[j:j + 1, :]
        return acc.astype(np.float64)
    Ar, Br = F.round_to(A, work), F.round_to(B, work)
    acc = np.zeros((A.shape[0], B.shape[1]))
    for j in range(A.shape[1]):
        acc = F.round_to(acc + F.round_to(Ar[:, j:j + 1] * Br[j:j + 1, :], work), work)
    return acc


def hodlr_matvec(h, X, work: str = "fp64", stored: bool = True) -> np.ndarray:
    """b = H-hat X by Algorithm 3.3.  X has shape (n,) or (n, R)."""
    X = np.asarray(X, dtype=np.float64)
    vec = X.ndim == 1
    if vec:
        X = X.reshape(-1, 1)
    U, V, D = _factors(h, stored)
    B = np.zeros_like(X)
    for k in range(1, h.depth + 1):
        nodes = h.levels[k]
        for i in range(0, len(nodes), 2):
            a, b = i, i + 1                      # the pair (2i-1, 2i) in 1-based terms
            (sa, ma), (sb, mb) = nodes[a], nodes[b]
            ya = _mm(V[k][b].T, X[sb:sb + mb], work)     # V_{2i}^T x_{2i}
            B[sa:sa + ma] = _add(B[sa:sa + ma], _mm(U[k][a], ya, work), work)
            yb = _mm(V[k][a].T, X[sa:sa + ma], work)     # V_{2i-1}^T x_{2i-1}
            B[sb:sb + mb] = _add(B[sb:sb + mb], _mm(U[k][b], yb, work), work)
    for i, (s, m) in enumerate(h.levels[h.depth]):
        B[s:s + m] = _add(B[s:s + m], _mm(D[i], X[s:s + m], work), work)
    return B[:, 0] if vec else B


def _rows_product(h, X, rows, stored, absval):
    """Rows ``rows`` of the two-stage product of Algorithm 3.3 in fp64 (or of
    its absolute-value twin g): for an output row r in node i of level k,
    U_i[r] (V_{i^1}^T x_{i^1}) summed over the levels, plus D_leaf[r] x_leaf.
    Each V^T x is formed only for nodes that hold a requested row."""
    X = np.asarray(X, dtype=np.float64)
    vec = X.ndim == 1
    if vec:
        X = X.reshape(-1, 1)
    if absval:
        X = np.abs(X)
    f = np.abs if absval else (lambda a: a)
    U, V, D = _factors(h, stored)
    rows = np.asarray(rows, dtype=np.int64)
    out = np.zeros((len(rows), X.shape[1]))
    for k in range(1, h.depth + 1):
        for i, (s, m) in enumerate(h.levels[k]):
            sel = np.nonzero((rows >= s) & (rows < s + m))[0]
            if len(sel) == 0:
                continue
            s1, m1 = h.levels[k][i ^ 1]
            y = f(V[k][i ^ 1]).T @ X[s1:s1 + m1]
            out[sel] += f(U[k][i])[rows[sel] - s] @ y
    for i, (s, m) in enumerate(h.levels[h.depth]):
        sel = np.nonzero((rows >= s) & (rows < s + m))[0]
        if len(sel):
            out[sel] += f(D[i])[rows[sel] - s] @ X[s:s + m]
    return out[:, 0] if vec else out


def hodlr_matvec_rows(h, X, rows, stored: bool = True) -> np.ndarray:
    """Rows ``rows`` of H-hat X (fp64), for products too large to form in
    full on the host; equals ``hodlr_matvec(h, X)[rows]`` up to the order of
    the fp64 sums."""
    return _rows_product(h, X, rows, stored, absval=False)


def abs_product_rows(h, X, rows, stored: bool = True) -> np.ndarray:
    """Rows ``rows`` of ``abs_product(h, X)``."""
    return _rows_product(h, X, rows, stored, absval=True)


def _add(a, b, work):
    if work == "fp64":
        return a + b
    if work == "fp32":
        return (a.astype(np.float32) + b.astype(np.float32)).astype(np.float64)
    return F.round_to(a + b, work)


def abs_product(h, X, stored: bool = True) -> np.ndarray:
    """g = sum over blocks of |U|(|V|^T|X|) plus |D||X| (fp64)."""
    X = np.abs(np.asarray(X, dtype=np.float64))
    vec = X.ndim == 1
    if vec:
        X = X.reshape(-1, 1)
    U, V, D = _factors(h, stored)
    G = np.zeros_like(X)
    for k in range(1, h.depth + 1):
        nodes = h.levels[k]
        for i in range(len(nodes)):
            (s, m), (s1, m1) = nodes[i], nodes[i ^ 1]
            G[s:s + m] += np.abs(U[k][i]) @ (np.abs(V[k][i ^ 1]).T @ X[s1:s1 + m1])
    for i, (s, m) in enumerate(h.levels[h.depth]):
        G[s:s + m] += np.abs(D[i]) @ X[s:s + m]
    return G[:, 0] if vec else G


def assemble(h, stored: bool = True) -> np.ndarray:
    """Dense n x n matrix represented by the HODLR factors (eq. (2.1))."""
    U, V, D = _factors(h, stored)
    A = np.zeros((h.n, h.n))
    for k in range(1, h.depth + 1):
        nodes = h.levels[k]
        for i in range(len(nodes)):
            (s, m), (s1, m1) = nodes[i], nodes[i ^ 1]
            A[s:s + m, s1:s1 + m1] = U[k][i] @ V[k][i ^ 1].T
    for i, (s, m) in enumerate(h.levels[h.depth]):
        A[s:s + m, s:s + m] = D[i]
    return A


def max_chain(h) -> int:
    """Longest chain of floating-point additions behind one output entry of
    Algorithm 3.3: the longest V^T x inner product (a node size), plus the
    longest U y inner product (a rank) per level, plus a leaf row, plus the
    l+1 accumulations into b."""
    longest_v = max((m for k in range(1, h.depth + 1) for (_s, m) in h.levels[k]), default=0)
    sum_r = sum(max((h.U[k][i].shape[1] for i in range(len(h.levels[k]))), default=0)
                for k in range(1, h.depth + 1))
    leaf = max((m for (_s, m) in h.levels[h.depth]), default=0)
    return longest_v + sum_r + leaf + h.depth + 1
