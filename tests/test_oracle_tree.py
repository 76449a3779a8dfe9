"""Pins for oracle.tree: closed form for n = 2^l n_min and the ceil-half split
of Sect. 4 for ragged n (Def. 2.1 partition properties by brute force)."""
import pytest

from oracle.tree import cluster_tree, depth_for_leaf


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
