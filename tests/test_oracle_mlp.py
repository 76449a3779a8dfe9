"""Pins for oracle.mlp (the rank predictor that sizes the construction's
first sketch): the chain-rule gradient against central finite differences
of the loss, a one-sample case computed by hand, Adam's first step against
its closed form, fp16 rounding of the parameters, and a planted mistake in
the relu derivative that the finite-difference pin catches."""
import numpy as np
import pytest

from oracle import mlp as P


def _data(seed, S=7):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((S, P.N_IN))
    t = rng.standard_normal(S)
    return X, t


def _fd_check(p, X, t, idx, h=1e-6, rtol=1e-6):
    g = P.backward(p, X, t, rounded=False)
    for i in idx:
        e = np.zeros_like(p)
        e[i] = h
        fd = (P.loss(p + e, X, t, rounded=False) - P.loss(p - e, X, t, rounded=False)) / (2 * h)
        assert abs(fd - g[i]) <= rtol * max(1.0, abs(fd)), (i, fd, g[i])


def test_parameter_count_and_layout():
    assert P.N_PARAMS == 64 * 11 + 64 + 2 * (64 * 64 + 64) + 64 + 1 == 9153
    p = np.arange(P.N_PARAMS, dtype=np.float64)
    parts = P.unpack(p)
    assert parts[0].shape == (64, 11) and parts[0][1, 0] == 11 and parts[1][0] == 704
    assert parts[-1][0] == P.N_PARAMS - 1


def test_gradient_matches_finite_differences():
    p = P.init_params(1) * 0.5
    X, t = _data(2)
    rng = np.random.default_rng(3)
    # a sample of every layer's weights and biases
    idx = np.concatenate([rng.choice(P.N_PARAMS, 40, replace=False), [0, 703, 704, 767, 9151, 9152]])
    _fd_check(p, X, t, idx)


def test_one_sample_by_hand():
    """One path through the network: x_0 = 3, W1[0,0] = W2[0,0] = W3[0,0] = 1,
    W4[0,0] = 2, b4 = 0.5, everything else 0: h = 3 on every layer,
    y = 6.5; with t = 1: L = 30.25, dL/db4 = 2 (y - t) = 11,
    dL/dW4[0,0] = 33, dL/dW1[0,0] = 11 * 2 * 3 = 66, and 0 for a unit that
    never activates."""
    p = np.zeros(P.N_PARAMS)
    W1, b1, W2, b2, W3, b3, W4, b4 = P.unpack(p)
    W1[0, 0] = W2[0, 0] = W3[0, 0] = 1.0
    W4[0, 0] = 2.0
    b4[0] = 0.5
    X = np.zeros((1, P.N_IN))
    X[0, 0] = 3.0
    y, _ = P.forward(p, X)
    assert y[0] == 6.5
    assert P.loss(p, X, np.array([1.0])) == 30.25
    g = P.unpack(P.backward(p, X, np.array([1.0])))
    assert g[7][0] == 11.0 and g[6][0, 0] == 33.0 and g[0][0, 0] == 66.0
    assert g[0][1, 0] == 0.0 and g[2][1, 1] == 0.0


def test_adam_first_step_is_lr_times_sign():
    """At step 1 the bias-corrected moments are g and g^2, so the update is
    lr * g / (|g| + eps): lr * sign(g) up to eps / |g|."""
    rng = np.random.default_rng(4)
    w = rng.standard_normal(50)
    g = rng.standard_normal(50)
    w1, m, v = P.adam_step(w, np.zeros(50), np.zeros(50), g, 1, 1e-3)
    assert np.allclose(w - w1, 1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=0)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_parameters_are_rounded_to_fp16():
    p = np.full(P.N_PARAMS, 1.0 + 2.0 ** -12)          # halfway between two fp16 values: ties to even
    assert np.all(P.round_params(p) == 1.0)
    p = np.full(P.N_PARAMS, 1.0 + 3 * 2.0 ** -12)
    assert np.all(P.round_params(p) == 1.0 + 2.0 ** -10)


def test_sketch_from_prediction():
    y = np.log2(np.array([0.0, 7.0, 15.0, 20.0, 100.0]) + 1.0)
    assert P.sketch_from_prediction(y).tolist() == [16, 16, 24, 32, 64]
    assert P.sketch_from_prediction(y, smin=8).tolist() == [8, 16, 24, 32, 64]


def test_planted_wrong_relu_derivative_is_caught(monkeypatch):
    monkeypatch.setattr(P, "_relu_grad", lambda z: np.ones_like(z))
    p = P.init_params(1) * 0.5
    X, t = _data(2)
    with pytest.raises(AssertionError):
        _fd_check(p, X, t, np.arange(0, 704, 7))
