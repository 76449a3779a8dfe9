"""hodlr_tree_order (host function of the library, no device work) against
the oracle's kd ordering (oracle/tree.py): the same permutation, index for
index, for 1D, 2D and 3D points, grids with equal coordinates, ragged sizes
and every depth; argument errors."""
import numpy as np
import pytest

import synth
from oracle.tree import kd_order


@pytest.fixture(scope="module")
def tree_order():
    from paper_2407_21637_gb300 import build as B
    B.build()
    from paper_2407_21637_gb300 import tree_order as T
    return T


@pytest.mark.parametrize("n,dim", [(1, 2), (2, 2), (7, 2), (100, 2), (1000, 2), (4097, 2), (129, 3), (300, 1)])
def test_same_permutation_as_the_oracle(tree_order, n, dim):
    P = np.random.default_rng(n * 7 + dim).random((n, dim))
    for depth in range(0, int(np.log2(n)) + 1):
        got = tree_order(P, depth)
        assert got.dtype == np.int32
        assert np.array_equal(got, kd_order(P, depth)), depth


def test_grids_with_ties_and_the_workload_points(tree_order):
    for P, depth in ((synth.grid_s2(2000), 6), (synth.grid_s2(64), 6), (synth.uniform_points_2d(65536, 4), 8)):
        assert np.array_equal(tree_order(P, depth), kd_order(P, depth))
    x = synth.grid_s1(50)
    assert np.array_equal(tree_order(x, 3), np.arange(50))   # sorted 1D points stay put


def test_argument_errors(tree_order):
    from paper_2407_21637_gb300 import HodlrError
    P = np.zeros((8, 2))
    for bad in ((np.zeros((8, 4)), 1), (P, 4), (P, -1), (np.full((8, 2), np.nan), 1)):
        with pytest.raises(HodlrError) as ei:
            tree_order(*bad)
        assert ei.value.status == 1
