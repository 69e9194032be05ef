"""Host checks of two exactness claims the tensor-pipe Galerkin kernel relies on (CPU only).

1. The raw-input prefetch divides a piece index q by the pieces per site, pps = 24 k + 9, as a
   multiply-high with m = floor((2^32 - 1) / pps) + 1: floor(q m / 2^32) = floor(q / pps) for
   every q < NB pps, NB = 4 or 8, k = 1 .. 24 (checked exhaustively).
2. The base-256 digit split of a double-float value v = hi + lo (|v| < 2, normalised) into
   7 digits, d = rint(hi), then (hi - d, lo) renormalised by one fast two-sum and scaled by
   256, is exact at every step: (hi + lo) after a step equals 256 (hi + lo - d) before it, as
   rationals; every digit has |d| <= 129 (exact in bfloat16), and the value minus its digit
   expansion sum_i d_i 2^(-6-8i) is at most 2^-55 (1 + 2^-16): the last step leaves
   |hi - d + lo| <= 1/2 + 2^-17 of weight 2^-54 (2^-55 itself occurs).  The FP32 operations
   are emulated with numpy float32 scalars (IEEE round to nearest even, like the kernel's _rn
   intrinsics and rintf).
"""
from fractions import Fraction

import numpy as np

F = np.float32


def test_prefetch_index_multiply_high_is_exact():
    for k in range(1, 25):
        pps = 2 * (2 * k) * 6 + 9
        m = (0xFFFFFFFF // pps + 1) & 0xFFFFFFFF
        for nb in (4, 8):
            q = np.arange(nb * pps, dtype=np.uint64)
            h = (q * np.uint64(m)) >> np.uint64(32)
            assert np.array_equal(h, q // np.uint64(pps)), (k, nb)


def _digits(hi, lo):
    """The kernel's digit loop on float32 scalars; returns digits and the (hi, lo) trail."""
    hi, lo = F(hi) * F(64.0), F(lo) * F(64.0)
    ds, trail = [], [(hi, lo)]
    for _ in range(7):
        d = F(np.rint(hi))
        r = F(hi - d)
        h2 = F(r + lo)
        l2 = F(lo - F(h2 - r))
        hi, lo = F(h2 * F(256.0)), F(l2 * F(256.0))
        ds.append(d)
        trail.append((hi, lo))
    return ds, trail


def _values():
    rng = np.random.default_rng(12)
    x = list(rng.uniform(-2.0, 2.0, 3000))
    x += list(rng.uniform(-1.0, 1.0, 1000) * 10.0 ** rng.uniform(-12, 0, 1000))
    x += [0.0, 1.0, -1.0, 1.9999999999, -1.9999999999, 2.0 ** -40, 0.5 + 2.0 ** -30]
    return x


def test_digit_split_is_exact():
    for x in _values():
        hi = F(x)
        lo = F(x - float(hi))          # normalised double-float pair of x
        ds, trail = _digits(hi, lo)
        for i, d in enumerate(ds):
            assert abs(float(d)) <= 129 and float(d) == int(d)
            before = Fraction(float(trail[i][0])) + Fraction(float(trail[i][1]))
            after = Fraction(float(trail[i + 1][0])) + Fraction(float(trail[i + 1][1]))
            assert after == 256 * (before - Fraction(float(d))), (x, i)
        v = Fraction(float(hi)) + Fraction(float(lo))
        expansion = sum(Fraction(int(d)) * Fraction(1, 2 ** (6 + 8 * i)) for i, d in enumerate(ds))
        assert abs(v - expansion) <= Fraction(1, 2 ** 55) * (1 + Fraction(1, 2 ** 16)), x


def test_digit_products_accumulate_exactly_in_fp32():
    """One staging batch's FP32 accumulator of weight d sums at most 7 digit pairs (i + j = d)
    over the 12 NB stacked rows, each product at most 129^2 in magnitude: below 2^24, so every
    partial sum of integers is exact in FP32 (NB = 8 and 4)."""
    for nb in (8, 4):
        assert 7 * (12 * nb) * 129 ** 2 < 2 ** 24
    # the fold's weights 2^(-12-8d), d < 7, are FP32 numbers (normal, exact powers of two)
    for d in range(7):
        w = F(2.0) ** F(-12 - 8 * d)
        assert float(w) == 2.0 ** (-12 - 8 * d) and np.isfinite(w) and w > np.finfo(F).tiny
