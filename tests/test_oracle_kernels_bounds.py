"""Pins of ``oracle.kernels`` and ``oracle.bounds`` against values evaluated
by hand from their definitions.

Every expected number below is a decimal literal worked out from the stated
formula at the stated points (the arithmetic is in the comment beside it);
none is produced by the oracle's own code.  A planted mistake in the oracle
(a wrong length scale, a dropped diagonal term, a swapped sign, a changed
constant in a printed bound) must fail these pins, and the tests at the end
check that it does.

Kernels: eq. (4.1) of Sect. 4.2 and the synthetic workloads (1/(r+c),
exp(-r^2/len2), log(r+c), 1/(x_i - x_j)), diagonal f(0) + diag where f(0) is
finite, else diag.  Bounds: gamma_n (standard model, Sect. 1), eq. (3.5),
Thm 3.1 (both forms), Thm 3.5, Cor. 3.11.
"""
import math

import numpy as np
import pytest

import synth
from oracle import bounds as Bd
from oracle import kernels as K

P1 = np.array([[0.0], [0.25], [1.0]])          # 1D points: |dx| = 0.25, 1.0, 0.75
P2 = np.array([[0.0, 0.0], [0.3, 0.4], [1.0, 0.0]])   # 2D: r01 = 0.5, r02 = 1, r12 = sqrt(0.65)


def _block(points, spec):
    idx = np.arange(len(points))
    return K.kernel_block(points, idx, idx, spec)


def test_inv_dist_1d_hand_values():
    A = _block(P1, synth.KernelSpec(K.INV_DIST, c=1e-3, diag=5.0))
    want = np.array([
        [1005.0, 3.9840637450199203, 0.9990009990009991],      # 1/c + 5; 1/0.251; 1/1.001
        [3.9840637450199203, 1005.0, 1.3315579227696406],      # 1/0.751
        [0.9990009990009991, 1.3315579227696406, 1005.0]])
    np.testing.assert_allclose(A, want, rtol=1e-15, atol=0)


def test_gauss_1d_hand_values():
    pts = np.array([[0.0], [0.1], [0.3]])                     # r = 0.1, 0.3, 0.2
    A = _block(pts, synth.KernelSpec(K.GAUSS, len2=0.01, diag=1e-2))
    want = np.array([
        [1.01, 0.36787944117144233, 0.00012340980408667956],   # 1 + 1e-2; e^-1; e^-9
        [0.36787944117144233, 1.01, 0.01831563888873418],      # e^-4
        [0.00012340980408667956, 0.01831563888873418, 1.01]])
    np.testing.assert_allclose(A, want, rtol=1e-13, atol=0)


def test_log_1d_singular_and_shifted():
    pts = np.array([[0.0], [0.5], [1.25]])                    # r = 0.5, 1.25, 0.75
    A0 = _block(pts, synth.KernelSpec(K.LOG, c=0.0, diag=0.0))
    want0 = np.array([
        [0.0, -0.6931471805599453, 0.22314355131420976],       # diag 0 (log 0 not finite); log 0.5; log 1.25
        [-0.6931471805599453, 0.0, -0.2876820724517809],       # log 0.75
        [0.22314355131420976, -0.2876820724517809, 0.0]])
    np.testing.assert_allclose(A0, want0, rtol=1e-15, atol=0)
    A1 = _block(pts, synth.KernelSpec(K.LOG, c=1e-4, diag=3.0))
    assert A1[0, 0] == pytest.approx(-6.210340371976182, rel=1e-15)     # log(1e-4) + 3
    assert A1[0, 1] == pytest.approx(-0.6929472005572791, rel=1e-15)    # log(0.5001)
    assert A1[1, 2] == pytest.approx(-0.28754874800654645, rel=1e-15)   # log(0.7501)


def test_inv_x_minus_y_antisymmetric_with_unit_diagonal():
    A = _block(P1, synth.KernelSpec(K.INV_X_MINUS_Y, diag=1.0))
    want = np.array([
        [1.0, -4.0, -1.0],                                     # 1/(0 - 0.25); 1/(0 - 1)
        [4.0, 1.0, -1.3333333333333333],                       # 1/(0.25 - 1)
        [1.0, 1.3333333333333333, 1.0]])
    np.testing.assert_allclose(A, want, rtol=1e-15, atol=0)


def test_two_dimensional_points():
    Ai = _block(P2, synth.KernelSpec(K.INV_DIST, c=0.5))
    want_i = np.array([
        [2.0, 1.0, 0.6666666666666666],                        # 1/0.5; 1/(0.5+0.5); 1/(1+0.5)
        [1.0, 2.0, 0.7655644370746374],                        # 1/(sqrt(0.65) + 0.5)
        [0.6666666666666666, 0.7655644370746374, 2.0]])
    np.testing.assert_allclose(Ai, want_i, rtol=1e-15, atol=0)
    Ag = _block(P2, synth.KernelSpec(K.GAUSS, len2=0.25))
    want_g = np.array([
        [1.0, 0.36787944117144233, 0.01831563888873418],       # e^-(0.25/0.25); e^-(1/0.25)
        [0.36787944117144233, 1.0, 0.07427357821433388],       # e^-(0.65/0.25)
        [0.01831563888873418, 0.07427357821433388, 1.0]])
    np.testing.assert_allclose(Ag, want_g, rtol=1e-13, atol=0)


def test_sub_blocks_index_the_same_entries():
    # rows and columns are global indices: the diagonal rule follows the
    # index, not the position inside the block
    spec = synth.KernelSpec(K.INV_DIST, c=1e-3, diag=5.0)
    B = K.kernel_block(P1, [2, 0], [1, 0], spec)
    np.testing.assert_allclose(B, [[1.3315579227696406, 0.9990009990009991],
                                   [3.9840637450199203, 1005.0]], rtol=1e-15)


# ---- bounds ------------------------------------------------------------------
def test_gamma_hand_value():
    # 10 u / (1 - 10 u), u = 2^-24
    assert Bd.gamma(10, 2.0 ** -24) == pytest.approx(5.960468030254859e-07, rel=1e-15)
    assert Bd.gamma(2 ** 24, 2.0 ** -24) == math.inf


def test_block_storage_bound_hand_value():
    # eq. (3.5): (2 + sqrt(4) 2^-8) 2^-8 = 2.0078125 * 0.00390625
    assert Bd.block_storage_bound(4, 2.0 ** -8) == 0.007843017578125


def test_global_bound_rule_hand_values():
    # Thm 3.1 under the rule: (2 sqrt(2 l) + 1) eps; l = 8 -> 9 eps, l = 2 -> 5 eps
    assert Bd.global_bound_rule(1e-6, 8) == pytest.approx(9e-6, rel=1e-15)
    assert Bd.global_bound_rule(1e-3, 2) == pytest.approx(5e-3, rel=1e-15)


def test_global_bound_general_hand_value():
    # Thm 3.1: 2 sqrt(2) (2^1 0.5^2 2^-16 + 2^2 0.25^2 2^-22)^(1/2) + 1e-3
    xi = [None, 0.5, 0.25]
    u = [None, 2.0 ** -8, 2.0 ** -11]
    assert Bd.global_bound_general(1e-3, xi, u) == pytest.approx(0.00884295820518018, rel=1e-14)


def test_matvec_backward_bound_hand_value():
    # Thm 3.5 at l = 2: 2 (sqrt(2) + 1) sqrt(2^3 + 2^1) eps
    assert Bd.matvec_backward_bound(1e-6, 2) == pytest.approx(1.5268827230335918e-05, rel=1e-14)


def test_lu_backward_bound_hand_value():
    # Cor. 3.11 at l = 3, eps 1e-4, ||H|| = 2, ||L|| = 3, ||U|| = 5:
    # 2 (2^3 - 1) 1e-4 2 + 11 (2^3 - 1) 1e-4 15 = 0.0028 + 0.1155
    assert Bd.lu_backward_bound(1e-4, 3, 2.0, 3.0, 5.0) == pytest.approx(0.1183, rel=1e-14)


# ---- planted mistakes: the pins above must catch them -------------------------
def test_planted_length_scale_is_caught():
    pts = np.array([[0.0], [0.1]])
    wrong = _block(pts, synth.KernelSpec(K.GAUSS, len2=2 * 0.01))   # exp(-r^2/(2 len2))
    assert not np.isclose(wrong[0, 1], 0.36787944117144233, rtol=1e-6)


def test_planted_missing_diagonal_is_caught():
    A = _block(P1, synth.KernelSpec(K.INV_DIST, c=1e-3, diag=0.0))   # diag dropped
    assert not np.isclose(A[0, 0], 1005.0)


def test_planted_bound_constants_are_caught(monkeypatch):
    def loose_rule(eps, depth):          # 2 sqrt(2 l) + 2 instead of + 1
        return (2.0 * math.sqrt(2.0 * depth) + 2.0) * eps

    def loose_matvec(eps, depth):        # 2^(l+2) instead of 2^(l+1)
        return 2.0 * (math.sqrt(2.0) + 1.0) * math.sqrt(2.0 ** (depth + 2) + 2.0 ** (depth - 1)) * eps

    monkeypatch.setattr(Bd, "global_bound_rule", loose_rule)
    monkeypatch.setattr(Bd, "matvec_backward_bound", loose_matvec)
    with pytest.raises(AssertionError):
        test_global_bound_rule_hand_values()
    with pytest.raises(AssertionError):
        test_matvec_backward_bound_hand_value()
