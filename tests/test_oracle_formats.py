"""Pins for oracle.formats: Table 1.1 values and bit-exact agreement of the
round-to-nearest-even emulators with torch's dtype conversions."""
import os

import numpy as np
import pytest
import torch

from oracle import formats as F

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table_1_1.txt")


def _table():
    rows = {}
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        name, u, xmin, xmax, t = line.split()
        rows[name] = (float(u), float(xmin), float(xmax), int(t))
    return rows


def test_table_1_1_values():
    """Unit roundoff, x_min, x_max and t as printed in Table 1.1 (3 s.f.)."""
    for name, (u, xmin, xmax, t) in _table().items():
        assert F.FORMATS[name][0] == t
        assert abs(F.unit_roundoff(name) - u) <= 0.005 * u
        assert abs(F.x_min(name) - xmin) <= 0.005 * xmin
        assert abs(F.x_max(name) - xmax) <= 0.005 * xmax


TORCH = {
    "fp32": torch.float32,
    "bf16": torch.bfloat16,
    "fp16": torch.float16,
    "e4m3": torch.float8_e4m3fn,
    "e5m2": torch.float8_e5m2,
}


def _samples(fmt, n=200_000, seed=0):
    """Random magnitudes across the whole range incl. subnormals, plus exact
    midpoints between neighbouring representable values (the ties)."""
    rng = np.random.default_rng(seed)
    t, emin, emax, xmax, _ = F.FORMATS[fmt]
    lo = emin - t - 2
    e = rng.uniform(lo, emax + 0.99, n)
    x = np.ldexp(rng.uniform(1.0, 2.0, n), np.floor(e).astype(int)) * rng.choice([-1.0, 1.0], n)
    # ties: representable value +/- half an ulp
    r = F.round_to(x[: n // 4], fmt)
    fin = np.isfinite(r) & (r != 0)
    r = r[fin]
    _, ee = np.frexp(np.abs(r))
    ulp = np.ldexp(1.0, np.maximum(ee - 1, emin) - t + 1)
    ties = np.concatenate([r + ulp / 2, r - ulp / 2])
    x = np.concatenate([x, ties, [0.0, -0.0, xmax, -xmax]])
    # keep the finite range of every format (overflow semantics differ for e4m3)
    return x[np.abs(x) <= xmax]


@pytest.mark.parametrize("fmt", list(TORCH))
def test_round_to_matches_torch_bitwise(fmt):
    """torch converts float64 to the narrow formats through float32, so the
    comparison uses float32-representable inputs (then that step is exact)."""
    x = _samples(fmt)
    if fmt != "fp32":
        x = x.astype(np.float32).astype(np.float64)
    ours = F.round_to(x, fmt)
    ref = torch.from_numpy(x).to(TORCH[fmt]).to(torch.float64).numpy()
    assert np.array_equal(ours.view(np.int64), ref.view(np.int64))


BITS = {"bf16": (torch.int16, torch.bfloat16), "fp16": (torch.int16, torch.float16),
        "e4m3": (torch.int8, torch.float8_e4m3fn), "e5m2": (torch.int8, torch.float8_e5m2)}


@pytest.mark.parametrize("fmt", list(BITS))
def test_round_to_brute_force_nearest_even(fmt):
    """Brute force on float64 inputs: enumerate every finite value of the
    format, take the nearest, and break ties towards the even encoding."""
    itype, ftype = BITS[fmt]
    nb = 16 if itype == torch.int16 else 8
    codes = torch.arange(-(1 << (nb - 1)), 1 << (nb - 1), dtype=torch.int32).to(itype)
    vals = codes.view(ftype).to(torch.float64).numpy()
    ok = np.isfinite(vals)
    vals, codes = vals[ok], codes.numpy()[ok].astype(np.int64)
    order = np.lexsort((codes, vals))
    vals, codes = vals[order], codes[order]
    keep = np.concatenate([[True], np.diff(vals) > 0])      # drop -0 duplicate of +0
    vals, codes = vals[keep], codes[keep]
    x = _samples(fmt, n=50_000, seed=7)
    x = x[(x > vals[0]) & (x < vals[-1])]
    j = np.searchsorted(vals, x)
    lo, hi = vals[j - 1], vals[j]
    exact = vals[np.minimum(j, len(vals) - 1)] == x
    dlo, dhi = x - lo, hi - x
    pick_hi = (dhi < dlo) | ((dhi == dlo) & ((codes[j] & 1) == 0))
    ref = np.where(exact, x, np.where(pick_hi, hi, lo))
    ours = F.round_to(x, fmt)
    assert np.array_equal(ours, ref)


def test_overflow_to_inf_fp16():
    x = np.array([65504.0, 65519.99, 65520.0, 1e6, -1e6])
    r = F.round_to(x, "fp16")
    ref = torch.from_numpy(x).to(torch.float16).to(torch.float64).numpy()
    assert np.array_equal(r, ref)
    assert np.isinf(r[2:]).all()


def test_e4m3_saturates():
    r = F.round_to(np.array([500.0, -1e9, 448.0]), "e4m3")
    assert list(r) == [448.0, -448.0, 448.0]


@pytest.mark.parametrize("fmt", ["fp16", "e4m3", "e5m2"])
def test_pow2_scale_range(fmt):
    rng = np.random.default_rng(3)
    for amax in np.exp(rng.uniform(-40, 40, 500)):
        s = F.pow2_scale(amax, fmt)
        assert np.log2(s) == np.round(np.log2(s))
        assert F.x_max(fmt) / 4 < amax * s <= F.x_max(fmt) / 2


def test_store_relative_error_bound():
    """Every normal stored entry is within u relative (scaled formats)."""
    rng = np.random.default_rng(4)
    M = rng.standard_normal((300, 7)) * 1e3
    for fmt in ("fp32", "bf16", "fp16", "e4m3", "e5m2"):
        d, s = F.store(M, fmt)
        rel = np.abs(d - M) / np.abs(M)
        big = np.abs(M * s) >= F.x_min(fmt)
        assert np.all(rel[big] <= F.unit_roundoff(fmt) * (1 + 1e-15))


def test_planted_mistake_is_caught():
    """A ties-away-from-zero rounding planted in the oracle fails the torch
    comparison: the pin is sensitive to the tie rule."""
    x = _samples("bf16", n=20_000, seed=9)

    def ties_away(v, fmt):
        t, emin = F.FORMATS[fmt][0], F.FORMATS[fmt][1]
        out = v.copy()
        nz = v != 0
        _, e = np.frexp(np.abs(v[nz]))
        ulp = np.ldexp(1.0, np.maximum(e - 1, emin) - t + 1)
        out[nz] = np.sign(v[nz]) * np.floor(np.abs(v[nz]) / ulp + 0.5) * ulp
        return out

    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert not np.array_equal(ties_away(x, "bf16"), ref)
