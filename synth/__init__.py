"""Seeded synthetic inputs shared by the CPU oracle and the GPU library.

This module draws point sets and right-hand sides only.  It holds none of the
HODLR method's arithmetic: no kernel evaluation, no compression, no matvec.
Both sides (``oracle/`` and ``paper_2407_21637_gb300/``) take their inputs from
here so that a parity test compares two independent computations on the same
numbers.

Workloads (Sect. 4.2 uses kernel matrices on 1D/2D point sets; the sizes below
are the synthetic stand-ins for the paper's SuiteSparse/P64 matrices, which are
not available):

``inv_dist_1024``   x ~ U[0,1] sorted, n = 1024, seed 1
``gauss_65536``     x ~ U[0,1] sorted, n = 65536, seed 2
``log2d_262144``    x ~ U[0,1]^2, n = 262144, seed 4 (kd ordering is done by
                    the caller; this module only draws the points)
``inv_dist_1m``     x ~ U[0,1] sorted, n = 1048576, seed 5

The paper's own point sets s1 (uniform grid on [0,1]) and s2 (uniform grid on
[-1,1]^2), Sect. 4.2, are provided by :func:`grid_s1` and :func:`grid_s2`.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "KernelSpec",
    "WORKLOADS",
    "uniform_points_1d",
    "uniform_points_2d",
    "grid_s1",
    "grid_s2",
    "rhs_normal",
    "rhs_uniform",
    "workload",
]

# Kernel kind codes.  The numeric values are part of the C ABI (hodlr.h).
INV_DIST = 0        # 1/(r + c)
GAUSS = 1           # exp(-r^2 / len2)
LOG = 2             # log(r + c)
INV_X_MINUS_Y = 3   # 1/(x_i - x_j)  (1D, antisymmetric; paper kernel (i))


class KernelSpec:
    """Parameters of a kernel matrix A_ij = f(x_i, x_j) + diag * delta_ij.

    The value of f at i == j is f(0) when it is finite (c > 0 or GAUSS) and 0
    otherwise (paper kernels (i) and (ii) define the diagonal separately).
    This is a plain record: the evaluation lives on each side separately.
    """

    __slots__ = ("kind", "c", "len2", "diag")

    def __init__(self, kind: int, c: float = 0.0, len2: float = 1.0, diag: float = 0.0):
        self.kind = int(kind)
        self.c = float(c)
        self.len2 = float(len2)
        self.diag = float(diag)

    def __repr__(self) -> str:  # pragma: no cover - debugging aid
        return f"KernelSpec(kind={self.kind}, c={self.c}, len2={self.len2}, diag={self.diag})"


def uniform_points_1d(n: int, seed: int) -> np.ndarray:
    """n points x_i ~ U[0,1], sorted ascending, shape (n, 1), float64."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.sort(rng.random(n)).reshape(n, 1)


def uniform_points_2d(n: int, seed: int) -> np.ndarray:
    """n points ~ U[0,1]^2, shape (n, 2), float64 (unordered)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.random((n, 2))


def grid_s1(n: int) -> np.ndarray:
    """Point set s1 of Sect. 4.2: n uniform grid points in [0, 1], shape (n, 1)."""
    return np.linspace(0.0, 1.0, n).reshape(n, 1)


def grid_s2(n: int) -> np.ndarray:
    """Point set s2 of Sect. 4.2: uniform grid in [-1,1]^2.

    The paper does not state the grid for n = 2000.  Reading used here: the
    smallest square grid g x g with g^2 >= n, row-major, first n points.
    """
    g = int(np.ceil(np.sqrt(n)))
    t = np.linspace(-1.0, 1.0, g)
    yy, xx = np.meshgrid(t, t, indexing="ij")
    pts = np.stack([xx.ravel(), yy.ravel()], axis=1)
    return np.ascontiguousarray(pts[:n])


def rhs_normal(n: int, nrhs: int, seed: int, dtype=np.float32) -> np.ndarray:
    """X ~ N(0,1), shape (n, nrhs), row-major (RHS fastest)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.ascontiguousarray(rng.standard_normal((n, nrhs)).astype(dtype))


def rhs_uniform(n: int, nrhs: int, seed: int, dtype=np.float64) -> np.ndarray:
    """X ~ U(-1,1), shape (n, nrhs) (the distribution of Sect. 4.2)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.ascontiguousarray((2.0 * rng.random((n, nrhs)) - 1.0).astype(dtype))


WORKLOADS = {
    # name: (n, leaf, depth, eps, kernel, seed, work precision, tiers)
    "inv_dist_1024": dict(n=1024, leaf=64, depth=4, eps=1e-8,
                          kernel=KernelSpec(INV_DIST, c=1e-3, diag=1024.0),
                          seed=1, work="fp64", tiers=("fp64",)),
    "gauss_65536": dict(n=65536, leaf=256, depth=8, eps=1e-6,
                        kernel=KernelSpec(GAUSS, len2=0.01, diag=1e-2),
                        seed=2, work="fp32", tiers=("fp64", "fp32", "bf16", "fp16", "e4m3")),
    "inv_dist_1m": dict(n=1048576, leaf=256, depth=12, eps=1e-6,
                        kernel=KernelSpec(INV_DIST, c=1e-4, diag=0.0),
                        seed=5, work="fp32", tiers=("fp64", "fp32", "bf16", "fp16", "e4m3")),
}


def workload(name: str, n: int | None = None):
    """Return (points, params) for a named workload; ``n`` overrides the size
    (the leaf size is kept, the depth follows n) for small parity cases."""
    p = dict(WORKLOADS[name])
    if n is not None and n != p["n"]:
        leaf = p["leaf"]
        depth = 0
        while (n + (1 << depth) - 1) >> depth > leaf:
            depth += 1
        p["n"], p["depth"] = n, depth
        if p["kernel"].kind == INV_DIST and p["kernel"].diag > 0:
            p["kernel"] = KernelSpec(INV_DIST, c=p["kernel"].c, diag=float(n))
    pts = uniform_points_1d(p["n"], p["seed"])
    return pts, p
