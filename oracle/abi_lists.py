"""Per-node list layout of the C ABI for an oracle HODLR object.

Test infrastructure (see ``oracle/__init__``).  The C ABI passes generators as
per-node lists in level order: node (k, i) is entry 2^k - 2 + i.  ``U[q]`` is
the left generator of block (i, i^1); ``V[q]`` is the right generator of block
(i^1, i).  This module only rearranges lists; it does no arithmetic.
"""
import numpy as np


def oracle_to_abi(h):
    ranks, U, V = [], [], []
    for k in range(1, h.depth + 1):
        for i in range(len(h.levels[k])):
            ranks.append(h.U[k][i].shape[1])
            U.append(np.ascontiguousarray(h.U[k][i]))
            V.append(np.ascontiguousarray(h.V[k][i]))
    D = [np.ascontiguousarray(d) for d in h.D]
    return ranks, U, V, D


def abi_to_levels(depth, per_node):
    out = [[]]
    q = 0
    for k in range(1, depth + 1):
        out.append(list(per_node[q:q + (1 << k)]))
        q += 1 << k
    return out
