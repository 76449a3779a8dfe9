"""Dense kernel-matrix entries, fp64.

Test infrastructure (see ``oracle/__init__``).

Kernels of eq. (4.1) and of the synthetic workloads, A_ij = f(r_ij) + diag*delta_ij
with r_ij = ||x_i - x_j||_2:

  INV_DIST      f = 1/(r + c)
  GAUSS         f = exp(-r^2 / len2)          (paper (iii): len2 = 2 h^2)
  LOG           f = log(r + c)                (paper (ii): c = 0)
  INV_X_MINUS_Y f = 1/(x_i - x_j), 1D only    (paper (i), read as x = x_i, y = x_j)

At i == j (the same index) f is f(0) where that is finite and 0 otherwise;
paper kernels (i) and (ii) then get their stated diagonals 1 and 0 through
``diag``.  Off the diagonal, coincident points of a singular kernel would give
inf; the workloads never produce them.

Parity: pinned.  Every kind is compared with entries evaluated by hand at
fixed 1D and 2D points (diagonal rules included) in
``tests/test_oracle_kernels_bounds.py``; planted mistakes (a doubled length
scale, a dropped diagonal term) fail those pins.
"""
from __future__ import annotations

import numpy as np

INV_DIST, GAUSS, LOG, INV_X_MINUS_Y = 0, 1, 2, 3


def _singular_at_zero(spec) -> bool:
    if spec.kind == INV_X_MINUS_Y:
        return True
    if spec.kind in (INV_DIST, LOG):
        return spec.c == 0.0
    return False


def kernel_block(points: np.ndarray, rows, cols, spec) -> np.ndarray:
    """Dense block A[rows, cols] (rows/cols are index arrays or ranges)."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    P = np.asarray(points, dtype=np.float64)
    if P.ndim == 1:
        P = P.reshape(-1, 1)
    pr, pc = P[rows], P[cols]
    same = rows[:, None] == cols[None, :]
    if spec.kind == INV_X_MINUS_Y:
        d = pr[:, 0][:, None] - pc[:, 0][None, :]
        with np.errstate(divide="ignore"):
            f = np.where(same, 0.0, 1.0 / np.where(same, 1.0, d))
    else:
        diff = pr[:, None, :] - pc[None, :, :]
        r2 = np.sum(diff * diff, axis=2)
        r = np.sqrt(r2)
        if spec.kind == INV_DIST:
            base = np.where(same, 1.0, r + spec.c)
            f = 1.0 / base
        elif spec.kind == GAUSS:
            f = np.exp(-r2 / spec.len2)
        elif spec.kind == LOG:
            base = np.where(same, 1.0, r + spec.c)
            f = np.log(base)
        else:
            raise ValueError(f"unknown kernel kind {spec.kind}")
        if _singular_at_zero(spec):
            f = np.where(same, 0.0, f)
        elif spec.kind in (INV_DIST, LOG):
            # finite f(0): 1/c or log(c)
            f0 = 1.0 / spec.c if spec.kind == INV_DIST else np.log(spec.c)
            f = np.where(same, f0, f)
    return f + np.where(same, spec.diag, 0.0)


def kernel_matrix(points: np.ndarray, spec) -> np.ndarray:
    n = len(points)
    idx = np.arange(n)
    return kernel_block(points, idx, idx, spec)
