"""Cluster tree of Def. 2.1 with the practical split of Sect. 4.

Test infrastructure (see ``oracle/__init__``).

Level k has 2^k nodes I_1^k .. I_{2^k}^k that partition {0..n-1} into
consecutive ranges; node i at level k has children 2i-1 and 2i at level k+1
(1-based, Def. 2.1(c)).  Sect. 4 sets the size of a left child to the ceiling
of half its parent's size, so leaf sizes are floor(n/2^l) or ceil(n/2^l).  For
n = 2^l n_min this is the perfectly balanced tree used in the analysis.

Nodes are returned 0-based: ``levels[k][i] = (start, size)`` for
i = 0..2^k-1; the sibling of node i is i ^ 1 and its parent is i // 2.

``kd_order`` puts points in 2 or 3 dimensions into an order in which the
cluster tree's consecutive ranges are spatial clusters (a kd-tree with the
tree's node sizes; the LU workload's 2D points are ordered so).

Parity: pinned (closed form for power-of-two n; partition and ceil-split
properties checked by brute force in the tests; ``kd_order`` by brute-force
separation and widest-coordinate checks at every node, its 1D case against
a stable sort, and the lower ranks it gives a 2D kernel matrix).
"""
from __future__ import annotations

import numpy as np


def cluster_tree(n: int, depth: int):
    """Return ``levels`` with levels[0] = [(0, n)] and levels[depth] the leaves."""
    if n < 0 or depth < 0:
        raise ValueError("n and depth must be non-negative")
    levels = [[(0, n)]]
    for _k in range(depth):
        nxt = []
        for (s, m) in levels[-1]:
            left = (m + 1) // 2          # ceil(m / 2), Sect. 4
            nxt.append((s, left))
            nxt.append((s + left, m - left))
        levels.append(nxt)
    return levels


def depth_for_leaf(n: int, leaf: int) -> int:
    """Smallest depth whose ceil-split leaves have size <= leaf."""
    depth = 0
    while (n + (1 << depth) - 1) >> depth > leaf:
        depth += 1
    return depth


def kd_order(points, depth: int) -> np.ndarray:
    """Permutation ``perm`` (perm[t] = original index of the point at tree
    position t) that makes the nodes of ``cluster_tree(n, depth)`` spatial
    clusters: going down the tree, the points of each node (start, m) are
    ordered by the coordinate along which they spread most (max - min; the
    lowest such coordinate on a tie), ties by original index, so that its
    left child (the first ceil(m/2) positions) holds the ones with the
    smallest values of that coordinate."""
    P = np.asarray(points, dtype=np.float64)
    n = P.shape[0]
    P = P.reshape(n, -1)
    perm = np.arange(n)
    levels = cluster_tree(n, depth)
    for k in range(depth):
        for (s, m) in levels[k]:
            if m < 2:
                continue
            idx = perm[s:s + m]
            pts = P[idx]
            spread = pts.max(axis=0) - pts.min(axis=0)
            d = int(np.argmax(spread))                      # first maximum
            perm[s:s + m] = idx[np.lexsort((idx, pts[:, d]))]   # by coordinate, then index
    return perm
