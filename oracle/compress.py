"""Compression of the off-diagonal blocks and the adaptive precision rule.

Test infrastructure (see ``oracle/__init__``).

Follows Algorithm 3.2 (adaptive-precision HODLR format) step by step:

 1. nrmAll = ||H||_F^2.
 2. For k = 1..l: partition every level-(k-1) diagonal block by eq. (2.1);
    nrm = max over the level-k off-diagonal blocks of ||H_ij||_F^2;
    xi_k = sqrt(nrm / nrmAll); u'_k = eps / (2^{k/2} xi_k);
    u_k = max{ u* <= u'_k : u* in {u} U calU }.
 3. Compress each pair of sibling blocks, H_{i,i^1} ~ U_i V_{i^1}^T, and store
    both generators in u_k (eq. (3.1): U has orthonormal columns).
 4. Store the leaves H_ii^(l) in the working precision u.

Readings of points the paper leaves open:

* Truncation (Sect. 3.1, Sect. 4: "SVD with parameter eps"): per-block
  relative Frobenius, the smallest r with (sum_{j>r} s_j^2)^{1/2} <= eps (sum_j
  s_j^2)^{1/2}; this is exactly the condition of Def. 2.3 in the Frobenius
  norm used by Lemma 2.4.  ``trunc="2"`` gives s_{r+1} <= eps s_1 instead.
* Which factor carries Sigma: U = U_r (orthonormal, eq. (3.1)), V = V_r S_r, so
  ||U V^T||_F = ||V||_F.
* Norms for xi: ``norms="original"`` uses H itself (Algorithm 3.2 as printed);
  ``norms="factors"`` uses the compressed fp64 HODLR, ||H||_F^2 ~ sum ||D_i||^2
  + sum ||V||^2 (the O(eps) estimate allowed in Sect. 3.2).
* Empty admissible set: take the most precise available format.
* Tie: u* = u'_k is admissible (the rule uses <=).
* ``per_block=True``: xi_ij = ||H_ij||_F / ||H||_F per block instead of the
  level maximum (the proof of Thm 3.1 sums per-block terms, so the bound is
  unchanged).
* Narrow formats (fp16, e4m3, e5m2) store s*U and s*V with a per-block
  power-of-two s (see ``formats.store``).

Parity: pinned (known-rank kernels, exact reconstruction as eps -> 0, Lemma
2.4, eq. (3.5) per block, Thm 3.1 globally, hand-built tier boundaries).
"""
from __future__ import annotations

import math

import numpy as np

from . import formats as F
from .kernels import kernel_block
from .tree import cluster_tree


def truncated_svd(A: np.ndarray, eps: float, trunc: str = "fro"):
    """Best low-rank factors U (orthonormal columns) and V = V_r S_r of A with
    the truncation criterion above.  Returns (U, V, singular values)."""
    A = np.asarray(A, dtype=np.float64)
    m, p = A.shape
    if m == 0 or p == 0:
        return np.zeros((m, 0)), np.zeros((p, 0)), np.zeros(0)
    W, s, Zt = np.linalg.svd(A, full_matrices=False)
    total2 = float(np.sum(s * s))
    if total2 == 0.0:
        return np.zeros((m, 0)), np.zeros((p, 0)), s
    if trunc == "fro":
        # tail2[r] = sum_{j >= r} s_j^2 (0-based), r = 0..len(s)
        tail2 = np.concatenate([np.cumsum((s * s)[::-1])[::-1], [0.0]])
        r = int(np.argmax(np.sqrt(tail2) <= eps * math.sqrt(total2)))
    elif trunc == "2":
        r = int(np.sum(s > eps * s[0]))
    else:
        raise ValueError(trunc)
    U = W[:, :r].copy()
    V = (Zt[:r, :].T * s[:r]).copy()
    return U, V, s


class Hodlr:
    """A HODLR matrix in the oracle: exact fp64 factors plus their stored
    (rounded, decoded) values.

    Indexing (0-based): ``U[k][i]`` is the left generator of the level-k block
    H(I_i, I_{i^1}) and ``V[k][i]`` is the right generator of the block
    H(I_{i^1}, I_i), so H(I_i, I_{i^1}) ~ U[k][i] @ V[k][i^1].T.  ``tier[k][i]``
    is the storage format of block (i, i^1), i.e. of U[k][i] and V[k][i^1].
    ``U[0]``/``V[0]``/``tier[0]`` are unused placeholders.
    """

    def __init__(self, n: int, depth: int):
        self.n, self.depth = n, depth
        self.levels = cluster_tree(n, depth)
        self.U = [[] for _ in range(depth + 1)]
        self.V = [[] for _ in range(depth + 1)]
        self.D = []
        self.block_norm2 = [[] for _ in range(depth + 1)]   # ||H(I_i, I_{i^1})||_F^2
        self.sing = [[] for _ in range(depth + 1)]
        self.norm2_all = None
        # filled by assign_precisions / store_all
        self.tier = [[] for _ in range(depth + 1)]
        self.xi = [None] * (depth + 1)
        self.u_prime = [None] * (depth + 1)
        self.work = "fp64"
        self.Uh = self.Vh = self.Dh = None
        self.sU = self.sV = None

    # ---- sizes -----------------------------------------------------------
    def rank(self, k: int, i: int) -> int:
        """Rank of block (i, i^1) at level k."""
        return self.U[k][i].shape[1]

    def nodes(self, k: int):
        return self.levels[k]


def compress(points, spec, n: int, depth: int, eps: float, trunc: str = "fro", A=None) -> Hodlr:
    """Partition and compress (steps 2-3 of Algorithm 3.2 without the
    precision choice).  The dense matrix is formed block by block from the
    kernel unless ``A`` is given."""
    h = Hodlr(n, depth)

    def block(rs, cs):
        if A is not None:
            return A[np.ix_(rs, cs)]
        return kernel_block(points, rs, cs, spec)

    total = 0.0
    for k in range(1, depth + 1):
        nodes = h.levels[k]
        h.V[k] = [None] * len(nodes)
        for i in range(len(nodes)):
            (s0, m0) = nodes[i]
            (s1, m1) = nodes[i ^ 1]
            Hij = block(np.arange(s0, s0 + m0), np.arange(s1, s1 + m1))
            nrm2 = float(np.sum(Hij * Hij))
            h.block_norm2[k].append(nrm2)
            total += nrm2
            U, Vsib, s = truncated_svd(Hij, eps, trunc)
            h.U[k].append(U)          # left generator of block (i, i^1)
            h.V[k][i ^ 1] = Vsib      # right generator of block (i, i^1)
            h.sing[k].append(s)
    for (s0, m0) in h.levels[depth]:
        idx = np.arange(s0, s0 + m0)
        Dii = block(idx, idx)
        h.D.append(Dii)
        total += float(np.sum(Dii * Dii))
    h.norm2_all = total          # ||H||_F^2: the blocks partition H
    return h


def from_factors(n: int, depth: int, U, V, D) -> Hodlr:
    """Wrap externally produced fp64 factors (same indexing as ``Hodlr``)."""
    h = Hodlr(n, depth)
    for k in range(1, depth + 1):
        h.U[k] = [np.asarray(u, dtype=np.float64) for u in U[k]]
        h.V[k] = [np.asarray(v, dtype=np.float64) for v in V[k]]
        h.block_norm2[k] = [float(np.sum(v * v)) for v in h.V[k]]
        # block_norm2 is indexed by block (i, i^1) whose V is V[k][i^1]
        h.block_norm2[k] = [h.block_norm2[k][i ^ 1] for i in range(len(h.V[k]))]
    h.D = [np.asarray(d, dtype=np.float64) for d in D]
    h.norm2_all = None
    return h


def factor_norms(h: Hodlr):
    """Norm estimates from the fp64 factors: ||U_i V_{i^1}^T||_F^2 = ||V_{i^1}||_F^2
    (U orthonormal) and ||H||_F^2 ~ sum of those plus sum ||D_i||_F^2."""
    bn = [[] for _ in range(h.depth + 1)]
    total = 0.0
    for k in range(1, h.depth + 1):
        for i in range(len(h.levels[k])):
            v = h.V[k][i ^ 1]
            b = float(np.sum(v * v))
            bn[k].append(b)
            total += b
    for d in h.D:
        total += float(np.sum(d * d))
    return bn, total


def choose_format(u_prime: float, avail) -> str:
    """u_k = max{u* <= u'_k : u* in avail}; the most precise format when the
    admissible set is empty (reading of Algorithm 3.2)."""
    ok = [f for f in avail if F.unit_roundoff(f) <= u_prime]
    if not ok:
        return min(avail, key=F.unit_roundoff)
    return max(ok, key=F.unit_roundoff)


def assign_precisions(h: Hodlr, eps: float, work: str, tiers, per_block: bool = False,
                      norms: str = "original") -> Hodlr:
    """Steps 1-2 of Algorithm 3.2: xi_k, u'_k and u_k for every level (or
    block).  ``avail`` = {u} U calU."""
    if norms == "original":
        bn, total = h.block_norm2, h.norm2_all
    elif norms == "factors":
        bn, total = factor_norms(h)
    else:
        raise ValueError(norms)
    avail = list(dict.fromkeys([work] + list(tiers)))
    h.work = work
    for k in range(1, h.depth + 1):
        nb = len(h.levels[k])
        scale = 2.0 ** (k / 2.0)
        if per_block:
            xis = [math.sqrt(bn[k][i] / total) if total > 0 else 0.0 for i in range(nb)]
            ups = [eps / (scale * x) if x > 0 else math.inf for x in xis]
            h.xi[k] = xis
            h.u_prime[k] = ups
            h.tier[k] = [choose_format(up, avail) for up in ups]
        else:
            nrm = max(bn[k]) if nb else 0.0
            xi = math.sqrt(nrm / total) if total > 0 else 0.0
            up = eps / (scale * xi) if xi > 0 else math.inf
            h.xi[k] = xi
            h.u_prime[k] = up
            h.tier[k] = [choose_format(up, avail)] * nb
    return h


def store_all(h: Hodlr) -> Hodlr:
    """Step 3-4 storage: generators in their block's format, leaves in u."""
    h.Uh = [[] for _ in range(h.depth + 1)]
    h.Vh = [[None] * len(h.levels[k]) for k in range(h.depth + 1)]
    h.sU = [[] for _ in range(h.depth + 1)]
    h.sV = [[None] * len(h.levels[k]) for k in range(h.depth + 1)]
    for k in range(1, h.depth + 1):
        for i in range(len(h.levels[k])):
            fmt = h.tier[k][i]
            uh, su = F.store(h.U[k][i], fmt)
            vh, sv = F.store(h.V[k][i ^ 1], fmt)
            h.Uh[k].append(uh)
            h.sU[k].append(su)
            h.Vh[k][i ^ 1] = vh
            h.sV[k][i ^ 1] = sv
    h.Dh = [F.round_to(d, h.work) for d in h.D]
    return h


def adaptive_hodlr(points, spec, n: int, depth: int, eps: float, work: str = "fp64",
                   tiers=("fp64", "fp32", "fp16", "bf16", "e5m2"), per_block: bool = False,
                   norms: str = "original", trunc: str = "fro", A=None) -> Hodlr:
    """Algorithm 3.2 end to end (the paper's default set of formats is
    {q52, bf16, fp16, fp32, fp64}, Sect. 4)."""
    h = compress(points, spec, n, depth, eps, trunc=trunc, A=A)
    assign_precisions(h, eps, work, tiers, per_block=per_block, norms=norms)
    return store_all(h)


def storage_bits(h: Hodlr, stored: bool = True) -> int:
    """Storage cost S of Sect. 4.4: bits of U, V and D (``stored=False``
    counts everything as fp64)."""
    bits = 0
    for k in range(1, h.depth + 1):
        for i in range(len(h.levels[k])):
            b = 8 * (F.BYTES[h.tier[k][i]] if stored else 8)
            bits += b * (h.U[k][i].size + h.V[k][i ^ 1].size)
    bd = 8 * (F.BYTES[h.work] if stored else 8)
    bits += bd * sum(d.size for d in h.D)
    return bits
