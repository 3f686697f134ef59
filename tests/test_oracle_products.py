"""Pins of the dot-product / squared-norm oracle."""

import itertools
import math
import struct
from fractions import Fraction

import numpy as np

import workloads as W
from oracle import c_oracle, products
from oracle import xsum_oracle as xo
from tests.test_oracle import EDGE, SMALL_GRID, f2b


def test_numpy_products_match_python_multiply():
    """Two independent IEEE multiplies agree bit for bit (NaNs aside)."""
    rng = np.random.default_rng(1)
    pool = np.concatenate([W.cfg2a_full_range(1, 0, 4000), W.cfg1_band(1, 0, 4000),
                           W.f64_to_bits(np.array(EDGE))])
    a = pool[rng.integers(0, pool.size, 20000)]
    b = pool[rng.integers(0, pool.size, 20000)]
    got = products.product_bits(a, b)
    for x, y, p in zip(a.tolist(), b.tolist(), got.tolist()):
        fx, fy = struct.unpack("<d", struct.pack("<Q", x))[0], struct.unpack("<d", struct.pack("<Q", y))[0]
        r = fx * fy
        assert p == (products.DEFAULT_NAN if math.isnan(r) else f2b(r))


def test_dot_with_ones_is_the_sum():
    x = W.cfg2a_paired(3, 0, 50000)
    ones = np.full(x.size, f2b(1.0), dtype=np.uint64)
    assert products.dot_bits(x, ones) == c_oracle.sum_bits(x)


def test_one_product():
    for a in EDGE[:30]:
        for b in EDGE[::3]:
            assert products.dot_bits(np.array([f2b(a)], dtype=np.uint64),
                                     np.array([f2b(b)], dtype=np.uint64)) == f2b(a * b)


def test_brute_force_against_fractions():
    grid = SMALL_GRID[:8] + [-v for v in SMALL_GRID[1:5]]
    for xs in itertools.product(grid, repeat=2):
        for ys in [(1.5, -3.0), (1e-200, 1e200), (0.1, 0.1)]:
            prods = [x * y for x, y in zip(xs, ys)]
            if any(math.isinf(p) or math.isnan(p) for p in prods):
                continue
            total = sum((Fraction(p) for p in prods), Fraction(0))
            got = products.dot_bits(W.f64_to_bits(np.array(xs)), W.f64_to_bits(np.array(ys)))
            if total == 0:
                continue
            assert got == f2b(total.numerator / total.denominator)


def test_norm2_is_dot_with_itself_and_specials():
    x = W.cfg1_band(7, 0, 30000)
    assert products.norm2_bits(x) == products.dot_bits(x, x)
    big = W.f64_to_bits(np.array([1e300, -1e300]))
    one = W.f64_to_bits(np.array([1e300, 1e300]))
    assert products.dot_bits(big, one) == xo.DEFAULT_NAN  # +Inf + -Inf products
    assert products.dot_bits(big[:1], one[:1]) == xo.POS_INF
    nan = np.array([0x7FF8000000000123], dtype=np.uint64)
    assert products.dot_bits(nan, W.f64_to_bits(np.array([1.0]))) == products.DEFAULT_NAN
    inf0 = products.dot_bits(W.f64_to_bits(np.array([math.inf])), W.f64_to_bits(np.array([0.0])))
    assert inf0 == products.DEFAULT_NAN
