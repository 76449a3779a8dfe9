"""Floating-point formats of Table 1.1 and round-to-nearest-even emulators.

Test infrastructure (see ``oracle/__init__``).

Table 1.1 lists, per format, the unit roundoff u, the smallest positive normal
x_min, the largest finite x_max and the significand length t.  The paper
simulates low precisions with a rounding function and does not state the mode;
the reading used here is IEEE round-to-nearest-ties-to-even with gradual
underflow, which is also what a GPU ``cvt.rn`` does.  The emulators below are
written from the format definitions (significand length and exponent range),
not from any library:

    value = (-1)^s * 2^E * (1.f)   for E >= e_min     (normal)
    value = (-1)^s * 2^e_min * (0.f)                  (subnormal)

so the spacing (ulp) at |x| in [2^E, 2^(E+1)) is 2^(max(E, e_min) - t + 1), and
rounding is "scale by the ulp, round to the nearest integer with ties to even,
scale back".  Overflow goes to +/-inf for the IEEE formats; the OCP FP8 E4M3
("fn") variant has no infinity and saturates to +/-448, as ``cvt.satfinite``
does.

Garbled entry: Table 1.1 prints t = -16 for q52.  q52 is the 8-bit format with
5 exponent bits and 2 stored fraction bits (OCP E5M2), so t = 3; the printed
u = 1.25e-1 = 2^-3 and x_max = 5.73e4 = 57344 agree with t = 3.

Parity: pinned (tests compare these emulators bit for bit with
``torch.Tensor.to(dtype)`` on random values including subnormals and ties, and
the unit roundoffs with the printed Table 1.1 values).
"""
from __future__ import annotations

import numpy as np

# name -> (t, e_min, e_max, x_max, has_inf)
FORMATS = {
    "fp64": (53, -1022, 1023, np.finfo(np.float64).max, True),
    "fp32": (24, -126, 127, float((2 - 2.0 ** -23) * 2.0 ** 127), True),
    "bf16": (8, -126, 127, float((2 - 2.0 ** -7) * 2.0 ** 127), True),
    "fp16": (11, -14, 15, 65504.0, True),
    "e4m3": (4, -6, 8, 448.0, False),
    "e5m2": (3, -14, 15, 57344.0, True),
}

# Storage widths in bytes (used for the storage-cost metric of Sect. 4.4).
BYTES = {"fp64": 8, "fp32": 4, "bf16": 2, "fp16": 2, "e4m3": 1, "e5m2": 1}

# Formats whose exponent range is narrower than fp32: these get a per-block
# power-of-two scale before rounding (reading of Sect. 3.1 for formats whose
# x_max is far below the generator entries; bf16 shares fp32's range).
SCALED = ("fp16", "e4m3", "e5m2")


def unit_roundoff(fmt: str) -> float:
    """u = 2^-t (Table 1.1)."""
    return 2.0 ** (-FORMATS[fmt][0])


def x_min(fmt: str) -> float:
    """Smallest positive normal number 2^e_min (Table 1.1)."""
    return 2.0 ** FORMATS[fmt][1]


def x_max(fmt: str) -> float:
    return FORMATS[fmt][3]


def round_to(x, fmt: str) -> np.ndarray:
    """Round float64 values to the nearest value of ``fmt`` (ties to even),
    returned as float64.  Exact for every finite float64 input."""
    x = np.asarray(x, dtype=np.float64)
    if fmt == "fp64":
        return x.copy()
    t, emin, _emax, xmax, has_inf = FORMATS[fmt]
    out = x.copy()
    fin = np.isfinite(x) & (x != 0.0)
    ax = np.abs(x[fin])
    _, e = np.frexp(ax)              # ax = m * 2^e with m in [0.5, 1)
    E = np.maximum(e - 1, emin)      # exponent of the leading bit, clamped
    ulp = np.ldexp(1.0, E - t + 1)
    r = np.rint(x[fin] / ulp) * ulp  # np.rint rounds half to even
    big = np.abs(r) > xmax
    if has_inf:
        r[big] = np.copysign(np.inf, r[big])
    else:
        r[big] = np.copysign(xmax, r[big])
    out[fin] = r
    return out


def pow2_scale(amax: float, fmt: str) -> float:
    """Per-block power-of-two scale s = 2^floor(log2(x_max / (2 amax))) for the
    narrow formats (SCALED), 1 otherwise and for an all-zero block.

    floor(log2(y)) is taken exactly from the binary exponent of y."""
    if fmt not in SCALED or amax == 0.0:
        return 1.0
    y = x_max(fmt) / (2.0 * amax)
    _, e = np.frexp(y)               # y = m 2^e, m in [0.5,1) -> floor(log2 y) = e-1
    return float(np.ldexp(1.0, int(e) - 1))


def store(M: np.ndarray, fmt: str):
    """Store a generator in ``fmt``: returns (decoded float64 values, scale).

    The stored entries are round_to(M * s, fmt); the decoded value used by the
    matvec is stored / s.  s is a power of two, so the scaling is exact."""
    M = np.asarray(M, dtype=np.float64)
    s = pow2_scale(float(np.max(np.abs(M))) if M.size else 0.0, fmt)
    q = round_to(M * s, fmt)
    return q / s, s
