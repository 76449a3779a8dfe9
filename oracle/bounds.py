"""Rounding constants and the paper's error bounds.

Test infrastructure (see ``oracle/__init__``).

* gamma_n = n u / (1 - n u)                       (Sect. 1, standard model)
* per-block storage error (eq. (3.5)):
      ||H~_ij - H^_ij||_F <= (2 + sqrt(p) u_k) u_k ||H~_ij||_F
* global representation error (Thm 3.1 with the rule u_k <= eps/(2^{k/2} xi_k)):
      ||H - H^||_F <~ (2 sqrt(2 l) + 1) eps ||H||_F
  and the general form 2 sqrt(2) (sum_k 2^k xi_k^2 u_k^2)^{1/2} + eps.
* matvec backward error (Thm 3.5, when u <= eps/n):
      ||Delta H||_F <= 2 (sqrt(2) + 1) sqrt(2^{l+1} + 2^{l-1}) eps ||H||_F
* HODLR LU backward error (Cor. 3.11, when u <~ eps/n):
      ||Delta H||_F <~ 2 (2^l - 1) eps ||H||_F + 11 (2^l - 1) eps ||L^||_F ||U^||_F

Parity: pinned.  Each function is compared with its value worked out by hand
at fixed arguments (``tests/test_oracle_kernels_bounds.py``), so a changed
constant fails; the oracle's own computations are also checked to satisfy
the bounds (tests of compress, matvec and lu).
"""
from __future__ import annotations

import math


def gamma(n: int, u: float) -> float:
    nu = n * u
    if nu >= 1.0:
        return math.inf
    return nu / (1.0 - nu)


def block_storage_bound(p: int, u: float) -> float:
    """eq. (3.5) relative factor (2 + sqrt(p) u) u."""
    return (2.0 + math.sqrt(p) * u) * u


def global_bound_rule(eps: float, depth: int) -> float:
    """Thm 3.1 relative bound (2 sqrt(2 l) + 1) eps under the precision rule."""
    return (2.0 * math.sqrt(2.0 * depth) + 1.0) * eps


def global_bound_general(eps: float, xi, u) -> float:
    """Thm 3.1 general relative bound 2 sqrt(2) (sum_k 2^k xi_k^2 u_k^2)^{1/2} + eps
    (xi, u indexed by level k = 1..l; index 0 unused)."""
    s = sum((2.0 ** k) * xi[k] ** 2 * u[k] ** 2 for k in range(1, len(xi)))
    return 2.0 * math.sqrt(2.0) * math.sqrt(s) + eps


def matvec_backward_bound(eps: float, depth: int) -> float:
    """Thm 3.5 relative bound on ||Delta H||_F / ||H||_F."""
    return 2.0 * (math.sqrt(2.0) + 1.0) * math.sqrt(2.0 ** (depth + 1) + 2.0 ** (depth - 1)) * eps


def lu_backward_bound(eps: float, depth: int, normH: float, normL: float, normU: float) -> float:
    """Cor. 3.11 absolute bound on ||L^U^ - H||_F."""
    c = (2.0 ** depth) - 1.0
    return 2.0 * c * eps * normH + 11.0 * c * eps * normL * normU
