"""Pins for oracle.tree: closed form for n = 2^l n_min and the ceil-half split
of Sect. 4 for ragged n (Def. 2.1 partition properties by brute force); the
kd ordering by brute-force separation at every node, its 1D case against a
stable sort, and the rank drop it gives the 2D log kernel."""
import numpy as np
import pytest

import synth
from oracle import kernels as K
from oracle.tree import cluster_tree, depth_for_leaf, kd_order


@pytest.mark.parametrize("nmin,depth", [(1, 0), (4, 3), (64, 4), (256, 8)])
def test_balanced_closed_form(nmin, depth):
    n = nmin << depth
    lv = cluster_tree(n, depth)
    for k in range(depth + 1):
        m = n >> k
        assert lv[k] == [(i * m, m) for i in range(1 << k)]


@pytest.mark.parametrize("n,depth", [(1000, 3), (2000, 8), (1023, 5), (7, 3), (65537, 8)])
def test_ragged_partition_and_ceil_split(n, depth):
    lv = cluster_tree(n, depth)
    for k in range(depth + 1):
        assert len(lv[k]) == 1 << k
        covered = []
        for (s, m) in lv[k]:
            covered.extend(range(s, s + m))
        assert covered == list(range(n))          # consecutive partition, Def 2.1(b)
    for k in range(depth):
        for i, (s, m) in enumerate(lv[k]):
            (s1, m1), (s2, m2) = lv[k + 1][2 * i], lv[k + 1][2 * i + 1]
            assert s1 == s and m1 == (m + 1) // 2 and s2 == s + m1 and m1 + m2 == m
    leaves = [m for (_s, m) in lv[depth]]
    assert set(leaves) <= {n >> depth, -(-n // (1 << depth))}


def test_depth_for_leaf():
    assert depth_for_leaf(65536, 256) == 8
    assert depth_for_leaf(1024, 64) == 4
    assert depth_for_leaf(1000, 128) == 3
    assert depth_for_leaf(100, 128) == 0


def _check_kd(P, depth, perm):
    """Every node above the leaves: its points are split along a coordinate
    of largest spread (the lowest on a tie) and every point of the left
    child precedes every point of the right one in (coordinate, index)."""
    n = P.shape[0]
    assert sorted(perm.tolist()) == list(range(n))
    lv = cluster_tree(n, depth)
    for k in range(depth):
        for i, (s, m) in enumerate(lv[k]):
            if m < 2:
                continue
            idx = perm[s:s + m]
            spread = P[idx].max(axis=0) - P[idx].min(axis=0)
            (s1, m1), (s2, m2) = lv[k + 1][2 * i], lv[k + 1][2 * i + 1]
            left, right = perm[s1:s1 + m1], perm[s2:s2 + m2]
            ok_dims = [d for d in range(P.shape[1])
                       if spread[d] == spread.max() and all(spread[e] < spread[d] for e in range(d))]
            assert len(ok_dims) == 1
            d = ok_dims[0]
            for a in left:          # brute force over all pairs
                for b in right:
                    assert (P[a, d], a) < (P[b, d], b)


@pytest.mark.parametrize("n,depth,dim", [(1, 0, 2), (2, 1, 2), (7, 2, 2), (100, 4, 2), (129, 5, 3), (64, 3, 1)])
def test_kd_order_separates_every_node(n, depth, dim):
    rng = np.random.default_rng(n + depth)
    P = rng.random((n, dim))
    _check_kd(P, depth, kd_order(P, depth))


def test_kd_order_grid_ties_and_depth_zero():
    P = synth.grid_s2(64)                    # many equal coordinates
    _check_kd(P, 3, kd_order(P, 3))
    assert kd_order(P, 0).tolist() == list(range(64))


def test_kd_order_1d_is_a_stable_sort():
    x = np.random.default_rng(0).permutation(np.repeat(np.linspace(0, 1, 25), 4))
    assert kd_order(x.reshape(-1, 1), 3).tolist() == np.argsort(x, kind="stable").tolist()


def test_kd_order_lowers_the_rank_of_a_2d_kernel_block():
    """The top off-diagonal block of the 2D log kernel (LU workload form)
    on 512 random points: numerical rank at 1e-4 in random order against kd
    order (207 against 28 here)."""
    pts = synth.uniform_points_2d(512, 3)
    spec = synth.KernelSpec(K.LOG, c=1e-4, diag=512.0)
    ranks = []
    for P in (pts, pts[kd_order(pts, 2)]):
        A = K.kernel_block(P, np.arange(256), np.arange(256, 512), spec)
        sv = np.linalg.svd(A, compute_uv=False)
        ranks.append(int(np.sum(sv > 1e-4 * sv[0])))
    assert ranks[1] < ranks[0] / 4, ranks
