"""CPU pins of two FP32 arithmetic facts the batch kernel relies on.

1. A correctly rounded FP32 quotient c / a equals the FP64 quotient rounded to
   FP32 (double rounding through binary64 is innocuous for binary32 division,
   Figueroa 1995), so FP32 jobs may form multipliers without FP64 division.
2. A butterfly of Knuth TwoSum steps on (hi, lo) FP32 pairs sums 32 lane
   partials to far better than FP32 accuracy (the error term of TwoSum is exact).
"""
from fractions import Fraction

import numpy as np


def _special_f32(rng, n):
    mant = rng.integers(0, 2**23, n, dtype=np.uint64)
    exp = rng.integers(0, 255, n, dtype=np.uint64)   # includes subnormals (0), excludes inf/nan (255)
    sign = rng.integers(0, 2, n, dtype=np.uint64)
    bits = (sign << 31) | (exp << 23) | mant
    return bits.astype(np.uint32).view(np.float32)


def test_fp32_division_equals_rounded_fp64_division():
    rng = np.random.default_rng(0)
    c = np.concatenate([_special_f32(rng, 400000), rng.standard_normal(200000).astype(np.float32)])
    a = np.concatenate([_special_f32(rng, 400000), rng.standard_normal(200000).astype(np.float32)])
    a[a == 0] = np.float32(1.0)
    with np.errstate(over="ignore", under="ignore", divide="ignore", invalid="ignore"):
        q32 = c / a                                         # IEEE binary32 division, round to nearest
        q64 = (c.astype(np.float64) / a.astype(np.float64)).astype(np.float32)
    same = (q32 == q64) | (np.isnan(q32) & np.isnan(q64))
    assert same.all(), np.nonzero(~same)[0][:5]


def test_fp32_reciprocal_of_difference_is_reproducible():
    rng = np.random.default_rng(1)
    x = rng.uniform(-1, 1, 100000).astype(np.float32)
    y = rng.uniform(2, 4, 100000).astype(np.float32)
    d = x - y
    r = np.float32(1.0) / d
    r64 = (1.0 / d.astype(np.float64)).astype(np.float32)
    assert np.array_equal(r, r64)


def _two_sum_butterfly(v):
    hi = v.astype(np.float32).copy()
    lo = np.zeros_like(hi)
    lanes = np.arange(32)
    o = 16
    while o:
        h2, l2 = hi[lanes ^ o], lo[lanes ^ o]
        s = hi + h2
        bb = s - hi
        e = (hi - (s - bb)) + (h2 - bb)
        hi, lo = s, (lo + l2) + e
        o >>= 1
    return hi, lo


def test_two_sum_butterfly_is_accurate_and_lane_symmetric():
    rng = np.random.default_rng(2)
    worst = 0.0
    for trial in range(300):
        scale = 10.0 ** rng.uniform(-20, 20, 32)
        v = (rng.random(32) * scale).astype(np.float32)
        hi, lo = _two_sum_butterfly(v)
        assert np.all(hi == hi[0]) and np.all(lo == lo[0])
        exact = sum(Fraction(float(t)) for t in v)
        got = Fraction(float(hi[0])) + Fraction(float(lo[0]))
        worst = max(worst, abs(float((got - exact) / exact)))
    assert worst < 2.0**-40
