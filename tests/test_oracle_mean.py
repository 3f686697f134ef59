"""Pins of the oracle's correctly rounded exact mean (Discussion: round the
superaccumulator divided by a positive integer; Introduction: the sample mean).
"""

import math
import random
from fractions import Fraction

import numpy as np
import pytest

import workloads as W
from oracle import c_oracle
from oracle import xsum_oracle as xo
from tests.test_oracle import EDGE, SMALL_GRID, f2b

DMAX = 1.7976931348623157e308


def test_round_ratio_against_int_division():
    """CPython's int/int true division is correctly rounded: an independent routine."""
    rng = random.Random(5)
    for _ in range(20000):
        N = rng.getrandbits(rng.randint(1, 2140)) or 1
        D = rng.getrandbits(rng.randint(1, 70)) or 1
        try:
            ref = f2b(N / (D << 1074))
        except OverflowError:
            ref = xo.POS_INF
        assert xo.round_ratio(N, D) == ref


def test_round_ratio_ties():
    rng = random.Random(6)
    for _ in range(5000):
        D = rng.choice([2, 3, 6, 10, 1 << rng.randint(1, 40)])
        m = rng.getrandbits(53) | (1 << 52)
        k = rng.randint(0, 900)
        for delta in (-1, 0, 1):
            # x = (m + 1/2) * 2^k exactly, times D, plus delta/D
            N = ((2 * m + 1) << k) * D // 2 + delta
            if N <= 0:
                continue
            assert xo.round_ratio(N, D) == f2b(N / (D << 1074))


def test_worked_example_mean():
    """mean(c(1e15, -1e15, 0.1)): the exact sum is the double 0.1, so the
    correctly rounded mean is the IEEE quotient 0.1 / 3."""
    for perm in [(1e15, -1e15, 0.1), (0.1, 1e15, -1e15), (-1e15, 0.1, 1e15)]:
        b = [f2b(v) for v in perm]
        assert xo.mean_bits(b) == f2b(0.1 / 3)
        assert c_oracle.mean_bits(np.array(b, dtype=np.uint64)) == f2b(0.1 / 3)


def test_mean_special_forms():
    assert xo.mean_bits([]) == xo.DEFAULT_NAN
    assert xo.mean_bits([f2b(DMAX), f2b(DMAX)]) == f2b(DMAX)  # the sum overflows, the mean does not
    assert xo.mean_bits([f2b(-0.0), f2b(-0.0)]) == xo.NEG_ZERO
    assert xo.mean_bits([f2b(2.0), f2b(-2.0)]) == 0
    assert xo.mean_bits([1, 0]) == 0  # 2^-1075 is a tie between 0 and 2^-1074: even is 0
    assert xo.mean_bits([3, 0]) == 2  # 1.5 * 2^-1074: tie, even neighbour 2 * 2^-1074
    assert xo.mean_bits([f2b(math.inf), f2b(1.0)]) == xo.POS_INF
    assert xo.mean_bits([0x7FF8000000000042, 0]) == 0x7FF8000000000042


@pytest.mark.parametrize("N", [1, 2, 3, 7, 4096, 100003])
def test_mean_of_repeats_is_the_value(N):
    for v in [0.1, -0.7, 5e-324, 3 * 5e-324, DMAX, 2.0 ** -1022]:
        bits = np.full(N, f2b(v), dtype=np.uint64)
        assert c_oracle.mean_bits(bits) == f2b(v)
        if N <= 4096:
            assert xo.mean_bits(bits.tolist()) == f2b(v)


def test_mean_brute_force_against_fractions():
    for trio in __import__("itertools").product(SMALL_GRID[:10], repeat=3):
        total = sum((Fraction(v) for v in trio), Fraction(0))
        if total == 0:
            continue
        ref = f2b(total.numerator / (total.denominator * 3))
        assert xo.mean_bits([f2b(v) for v in trio]) == ref


def test_mean_two_terms_against_ieee_when_exact_sum_is_a_double():
    """If a + b is exact in floating point, the mean is the IEEE quotient (a + b) / 2."""
    rng = np.random.default_rng(4)
    for a in EDGE[:40]:
        for b in EDGE[:40]:
            s = a + b
            if math.isinf(s) or Fraction(s) != Fraction(a) + Fraction(b):
                continue
            assert xo.mean_bits([f2b(a), f2b(b)]) == f2b(s / 2)


def test_c_mean_matches_python():
    for x in [W.cfg2a_full_range(1, 0, 20000), W.cfg2a_paired(2, 0, 20000), W.cfg1_band(3, 0, 20000),
              W.f64_to_bits(W.cfg0_cancel(1)), W.cfg1_band(4, 0, 5000, -1074 + 52, -1000)]:
        assert c_oracle.mean_bits(x) == xo.mean_bits(x.tolist())
    for _, vals in W.cfg2d_side_cases():
        b = W.f64_to_bits(np.array(vals, dtype=np.float64))
        assert c_oracle.mean_bits(b) == xo.mean_bits(b.tolist())


def test_finish_div_general_divisor():
    x = W.cfg2a_paired(5, 0, 3000).tolist()
    st = xo.state_of_bits(x)
    for D in [1, 2, 3, 1000, (1 << 40) + 3, (1 << 63) - 25]:
        try:
            mag = f2b(abs(st.S) / (D << 1074))
        except OverflowError:
            mag = xo.POS_INF
        ref = mag | (xo.SIGN_BIT if st.S < 0 else 0)
        assert xo.finish_div(st, D) == ref
