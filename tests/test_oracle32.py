"""Pins of the binary32 exact-sum oracle (no GPU)."""

import itertools

import numpy as np
import pytest

from oracle import c_oracle
from oracle import xsum_oracle32 as xo32

FMAX = float(np.finfo(np.float32).max)


def f32b(x) -> int:
    return int(np.array([x], dtype=np.float32).view(np.uint32)[0])


def rand32(seed, n, lo=-126, hi=128, specials=False):
    """float32 bit patterns: random sign and mantissa, exponent e in [lo+127, hi+127)."""
    rng = np.random.default_rng(seed)
    e = rng.integers(lo + 127, hi + 127, n).astype(np.uint32)
    e = np.clip(e, 0, 254)
    m = rng.integers(0, 1 << 23, n).astype(np.uint32)
    s = rng.integers(0, 2, n).astype(np.uint32)
    b = (s << np.uint32(31)) | (e << np.uint32(23)) | m
    if specials:
        sel = rng.integers(0, n, max(1, n // 300))
        b[sel] = np.array([0x7F800000, 0xFF800000, 0x7FC00123, 0x80000000, 0],
                          dtype=np.uint32)[rng.integers(0, 5, sel.size)]
    return b


GOLDEN32 = [
    # (inputs, expected, derivation)
    ([f32b(1.0), f32b(2.0 ** -24)], f32b(1.0), "midpoint of 1 and 1+2^-23: even is 1"),
    ([f32b(1.0), f32b(2.0 ** -24), 1], f32b(1.0 + 2.0 ** -23), "just above the midpoint"),
    ([f32b(1.0 + 2.0 ** -23), f32b(2.0 ** -24)], f32b(1.0 + 2.0 ** -22), "midpoint, even is up"),
    ([f32b(FMAX), f32b(2.0 ** 103)], 0x7F800000, "FLT_MAX + half ulp rounds to 2^128: +Inf"),
    ([f32b(FMAX), f32b(2.0 ** 102)], f32b(FMAX), "below the midpoint"),
    ([f32b(FMAX), f32b(FMAX), f32b(-FMAX)], f32b(FMAX), "no intermediate overflow"),
    ([0x00800000, 0x80000001], 0x007FFFFF, "largest subnormal"),
    ([0x80000000, 0x80000000], 0x80000000, "-0 + -0"),
    ([0x80000000, 0], 0, "+0"),
    ([0x7F800000, 0xFF800000], 0x7FC00000, "Inf - Inf: default NaN"),
    ([0x7FC00001, 0xFF800ABC, 0x7FA00ABC], 0x7FE00ABC, "largest 22-bit payload, quieted"),
]


@pytest.mark.parametrize("bits,expected,why", GOLDEN32)
def test_golden32(bits, expected, why):
    assert xo32.sum_f32_bits(bits) == expected
    assert c_oracle.sum_f32_bits(np.array(bits, dtype=np.uint32)) == expected


def test_two_term_identity_float32():
    """Two float32 terms: the exact sum rounded once is the IEEE single addition."""
    rng = np.random.default_rng(1)
    pool = np.concatenate([rand32(1, 3000), rand32(2, 3000, -20, 20), rand32(3, 3000, -150, -100)])
    pool = pool[((pool >> np.uint32(23)) & np.uint32(0xFF)) != np.uint32(0xFF)]
    a = pool[rng.integers(0, pool.size, 30000)]
    b = pool[rng.integers(0, pool.size, 30000)]
    with np.errstate(over="ignore"):
        ref = (a.view(np.float32) + b.view(np.float32)).view(np.uint32)
    for x, y, r in zip(a.tolist(), b.tolist(), ref.tolist()):
        assert xo32.sum_f32_bits([x, y]) == r


def test_sums_exact_in_float64_round_once():
    """When the float64 sum of float32 terms is exact, casting it to float32
    is the correctly rounded result (a single rounding)."""
    for seed in range(40):
        x = rand32(seed, 50, -10, 15)  # exponent span far below 29 bits
        f = x.view(np.float32).astype(np.float64)
        s = float(np.sum(f))  # exact: every partial sum fits in 53 bits
        ref = f32b(np.float32(s)) if s != 0 else 0
        assert xo32.sum_f32_bits(x.tolist()) == ref or s == 0


def test_brute_force_small_grid():
    grid = [0.0, 1.0, 2.0 ** -24, 1.0 + 2.0 ** -23, 3.0, 2.0 ** -149, 2.0 ** -126, FMAX, 0.1]
    grid = grid + [-g for g in grid]
    for trio in itertools.product(grid, repeat=3):
        f = [np.float32(v) for v in trio]
        s = sum(float(v) for v in f)  # float64 exact for these spans? check with a wider sum
        from fractions import Fraction
        ex = sum((Fraction(float(v)) for v in f), Fraction(0))
        if ex != Fraction(s) or ex == 0:
            continue
        with np.errstate(over="ignore"):
            ref = f32b(np.float32(s))
        assert xo32.sum_f32_bits([f32b(v) for v in f]) == ref, trio


def test_c_matches_python_and_invariants():
    for seed in range(6):
        x = rand32(seed, 20000, specials=seed % 2 == 0)
        assert c_oracle.sum_f32_bits(x) == xo32.sum_f32_bits(x.tolist())
    x = rand32(9, 5000)
    both = np.concatenate([x, x ^ np.uint32(1 << 31)])
    assert c_oracle.sum_f32_bits(both) == 0
    rng = np.random.default_rng(0)
    assert c_oracle.sum_f32_bits(x[rng.permutation(x.size)]) == c_oracle.sum_f32_bits(x)
    for N in (255, 256, 257, 4097):
        v = np.float32(0.1)
        ref = f32b(np.float32(float(v) * N))  # N * v exact in float64, rounded once
        assert c_oracle.sum_f32_bits(np.full(N, f32b(v), dtype=np.uint32)) == ref
