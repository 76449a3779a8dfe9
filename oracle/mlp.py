"""A small multilayer perceptron that predicts the rank of an off-diagonal
block from cheap features, used to size the first sketch of the randomized
construction (the adaptive rule of Algorithm 3.2 still decides every rank;
the paper itself has no learned component).  Test infrastructure (see
``oracle/__init__``).

The plain definitions, in fp64:

* layers: h_1 = relu(W_1 x + b_1), h_2 = relu(W_2 h_1 + b_2),
  h_3 = relu(W_3 h_2 + b_3), y = W_4 h_3 + b_4 (x in R^11, hidden 64,
  y scalar); relu(t) = max(t, 0);
* the weights the model holds are fp16 (``round_params`` rounds them to
  the nearest fp16, ties to even); every product and sum is fp64 here;
* loss over a batch of S samples: L = (1/S) sum_s (y_s - t_s)^2;
* gradients by the chain rule (``backward``), derivative of relu taken as 0
  at t = 0;
* Adam (Kingma and Ba, 2015) with beta1 = 0.9, beta2 = 0.999, eps = 1e-8
  on fp32 master weights: m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2,
  w -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).

Parameter vector layout (P = 9153 values): W_1 (64 x 11, row-major), b_1
(64), W_2 (64 x 64), b_2, W_3 (64 x 64), b_3, W_4 (1 x 64), b_4 (1).

Parity: pinned (central finite differences of the loss against
``backward``; a hand-computed one-sample case; Adam's first step
against its closed form |step| = lr; a planted wrong relu derivative
caught).
"""
from __future__ import annotations

import numpy as np

N_IN, N_HID = 11, 64
SHAPES = [(N_HID, N_IN), (N_HID,), (N_HID, N_HID), (N_HID,), (N_HID, N_HID), (N_HID,), (1, N_HID), (1,)]
N_PARAMS = int(sum(np.prod(s) for s in SHAPES))


def unpack(p: np.ndarray):
    """The eight arrays of the parameter vector (views)."""
    out, o = [], 0
    for s in SHAPES:
        k = int(np.prod(s))
        out.append(p[o:o + k].reshape(s))
        o += k
    return out


def round_params(p: np.ndarray) -> np.ndarray:
    """The values the model holds: every parameter rounded to fp16 (RNE)."""
    return np.asarray(p, dtype=np.float64).astype(np.float16).astype(np.float64)


def _relu_grad(z: np.ndarray) -> np.ndarray:
    """d relu / dz (0 at z = 0)."""
    return (z > 0).astype(np.float64)


def forward(p: np.ndarray, X: np.ndarray, rounded: bool = True):
    """y (S,) and the activations (h_1, h_2, h_3, and their pre-activations)
    for X (S x 11), with the fp16-rounded parameters (rounded=False: the
    parameters as given, for finite-difference checks)."""
    W1, b1, W2, b2, W3, b3, W4, b4 = unpack(round_params(p) if rounded else np.asarray(p, dtype=np.float64))
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ W1.T + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2.T + b2
    h2 = np.maximum(z2, 0.0)
    z3 = h2 @ W3.T + b3
    h3 = np.maximum(z3, 0.0)
    y = (h3 @ W4.T + b4)[:, 0]
    return y, (X, z1, h1, z2, h2, z3, h3)


def loss(p: np.ndarray, X: np.ndarray, t: np.ndarray, rounded: bool = True) -> float:
    y, _ = forward(p, X, rounded)
    return float(np.mean((y - np.asarray(t, dtype=np.float64)) ** 2))


def backward(p: np.ndarray, X: np.ndarray, t: np.ndarray, rounded: bool = True) -> np.ndarray:
    """dL/dp (P,) of the mean squared error, by the chain rule through the
    fp16-rounded parameters (the rounding itself is treated as identity)."""
    W1, b1, W2, b2, W3, b3, W4, b4 = unpack(round_params(p) if rounded else np.asarray(p, dtype=np.float64))
    y, (X, z1, h1, z2, h2, z3, h3) = forward(p, X, rounded)
    S = X.shape[0]
    dy = 2.0 * (y - np.asarray(t, dtype=np.float64)) / S          # (S,)
    gW4 = dy[None, :] @ h3                                          # (1, 64)
    gb4 = np.array([dy.sum()])
    d3 = (dy[:, None] @ W4) * _relu_grad(z3)                        # (S, 64)
    gW3 = d3.T @ h2
    gb3 = d3.sum(axis=0)
    d2 = (d3 @ W3) * _relu_grad(z2)
    gW2 = d2.T @ h1
    gb2 = d2.sum(axis=0)
    d1 = (d2 @ W2) * _relu_grad(z1)
    gW1 = d1.T @ X
    gb1 = d1.sum(axis=0)
    return np.concatenate([a.ravel() for a in (gW1, gb1, gW2, gb2, gW3, gb3, gW4, gb4)])


def adam_step(w: np.ndarray, m: np.ndarray, v: np.ndarray, g: np.ndarray, step: int, lr: float,
              b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
    """One Adam update (step counts from 1); returns new (w, m, v)."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** step)
    vh = v / (1.0 - b2 ** step)
    return w - lr * mh / (np.sqrt(vh) + eps), m, v


def init_params(seed: int) -> np.ndarray:
    """He-style initialization: weights ~ N(0, 2 / fan_in), biases 0."""
    rng = np.random.default_rng(seed)
    parts = []
    for s in SHAPES:
        if len(s) == 2:
            parts.append(rng.standard_normal(s).ravel() * np.sqrt(2.0 / s[1]))
        else:
            parts.append(np.zeros(s))
    return np.concatenate(parts)


def sketch_from_prediction(y: np.ndarray, smin: int = 16, smax: int = 64, over: int = 8) -> np.ndarray:
    """First sketch size per block from the predicted log2(rank + 1): the
    predicted rank plus `over` columns, rounded up to a multiple of 8, in
    [smin, smax] (smin = the construction's default first sketch: the
    prediction only ever raises it)."""
    r = np.maximum(np.exp2(np.asarray(y, dtype=np.float64)) - 1.0, 0.0)
    s = np.ceil((r + over) / 8.0) * 8.0
    return np.clip(s, smin, smax).astype(np.int32)
