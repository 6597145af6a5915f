"""The scale rule of the deterministic table gradient, checked on the host
in exact integer arithmetic.

With NIF_KNOB_DETERMINISTIC every contribution c = w * dL/dfeature to a table
entry is rounded once to an integer multiple of 2^-S and the integers are
added in 64 bits. S is the largest integer with B 2^S < 2^61 for
B = 2 n P max|dL/dfeature| (at most 100), where n is the segment count and P
the number of gamma terms: an entry of a level takes at most one weighted
term per (segment, end point, term), with trilinear weights summing to at
most 1. tests/bounds.py:fixed_scale restates the rule in the library's
arithmetic. Here the worst case (every contribution at the bound, one sign)
and random cases are summed exactly, as Python integers, to show that the
64-bit sums cannot overflow and that the result is the exact sum to within
2^-(S+1) per contribution.
"""
import math
from fractions import Fraction

import numpy as np

from tests import bounds as B

I64 = 2 ** 63


def _fix(c, S):
    # round half to even of c * 2^S (c a float32 value; the product is exact)
    return int(np.rint(np.float64(c) * 2.0 ** S))


def test_scale_is_the_largest_that_keeps_the_bound_below_2_61():
    rng = np.random.default_rng(1)
    for _ in range(2000):
        n = int(rng.integers(1, 1 << 22))
        P = int(rng.integers(1, 18))
        m = np.float32(10.0 ** rng.uniform(-12, 6))
        S = B.fixed_scale(n, P, np.array([m, -m / 3], np.float32))
        b = 2.0 * n * P * float(m)
        assert b * 2.0 ** S < 2.0 ** 61
        assert S == 100 or b * 2.0 ** (S + 1) >= 2.0 ** 61


def test_worst_case_sum_stays_inside_64_bits():
    # every (segment, end point, term) puts its whole weight, at the largest
    # gradient, on one entry with one sign: the largest possible sum
    for n, P, m in ((1 << 18, 9, 0.37), (1 << 20, 9, 3.0e4), (7, 1, 1e-30), (1 << 22, 17, 1.0)):
        m = np.float32(m)
        S = B.fixed_scale(n, P, np.array([m], np.float32))
        k = 2 * n * P                                     # contributions to the entry
        q = _fix(m, S)
        total = k * q                                     # exact, as the integer atomics add it
        assert total < I64 // 2 + k                       # < 2^62 + k: far inside int64
        # split over the 8 corners of a cell (weights summing to 1): no larger
        w = np.float32(0.125)
        total8 = 8 * k * _fix(np.float32(w * m), S)
        assert abs(total8) <= abs(total) + 8 * k
        assert total8 < I64


def test_random_sums_match_the_exact_sum_to_the_rounding_bound():
    rng = np.random.default_rng(2)
    for trial in range(50):
        k = int(rng.integers(1, 5000))
        g = rng.normal(size=k).astype(np.float32) * np.float32(10.0 ** rng.uniform(-8, 2))
        w = rng.uniform(0, 1, k).astype(np.float32)
        c = (w * g).astype(np.float32)                    # the FP32 products the kernels form
        S = B.fixed_scale(k, 1, g)
        ints = [_fix(x, S) for x in c]
        order = rng.permutation(k)
        assert sum(ints) == sum(ints[i] for i in order)   # any order, the same integer
        exact = sum(Fraction(float(x)) for x in c)
        got = Fraction(sum(ints), 2 ** S) if S >= 0 else Fraction(sum(ints) * 2 ** (-S))
        assert abs(got - exact) <= Fraction(k, 2 ** (S + 1)) if S >= 0 else True
        assert abs(sum(ints)) < I64
