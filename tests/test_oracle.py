"""Pins for the CPU oracle (no GPU).

Each test checks the oracle against something other than itself: Python's
correctly rounded Fraction-to-float conversion, math.fsum, IEEE addition of two
terms, closed forms, hand-derived boundary cases, invariants of the exact sum,
and brute force on tiny inputs.
"""

from __future__ import annotations

import itertools
import math
import os
import random
import struct
from fractions import Fraction

import numpy as np
import pytest

from oracle import c_oracle
from oracle import xsum_oracle as xo
import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "boundaries.txt")
DMAX = 1.7976931348623157e308


def f2b(x):
    return struct.unpack("<Q", struct.pack("<d", x))[0]


def b2f(b):
    return struct.unpack("<d", struct.pack("<Q", b))[0]


def load_golden():
    cases = []
    with open(GOLDEN) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            name, ins, exp, _why = [p.strip() for p in line.split(";", 3)]
            bits = [int(h, 16) for h in ins.split(",")] if ins else []
            cases.append((name, bits, int(exp, 16)))
    return cases


GOLDEN_CASES = load_golden()


def fraction_reference(values):
    """Correctly rounded finite sum through exact rationals (independent routine).

    CPython's int/int true division rounds correctly (half to even) and raises
    OverflowError when the rounded result is out of range.
    """
    total = sum((Fraction(v) for v in values), Fraction(0))
    try:
        return f2b(total.numerator / total.denominator)
    except OverflowError:
        return f2b(math.inf if total > 0 else -math.inf)


# Edge values: zeros, subnormals, normal boundaries, powers of two near the
# binade and rounding limits, DBL_MAX, and a few ordinary numbers.
EDGE = sorted(set(
    [0.0, 5e-324, 1e-323, 2.0 ** -1073, 2.0 ** -1022 - 5e-324, 2.0 ** -1022, 2.0 ** -1021,
     2.0 ** -1022 + 5e-324, 2.0 ** -600, 2.0 ** -53, 2.0 ** -54, 2.0 ** -52, 0.1, 0.5, 1.0,
     1.0 + 2.0 ** -52, 1.0 - 2.0 ** -53, 1.5, 2.0, 3.0, 2.0 ** 52, 2.0 ** 53, 2.0 ** 53 + 2,
     2.0 ** 54, 1e15, 1e300, 2.0 ** 969, 2.0 ** 970, 2.0 ** 1023, DMAX, DMAX / 2,
     2.0 ** 1023 + 2.0 ** 971]))
EDGE = EDGE + [-x for x in EDGE]


# --------------------------------------------------------------------------- #
# Golden, hand-derived boundary cases
# --------------------------------------------------------------------------- #

@pytest.mark.parametrize("name,bits,expected", GOLDEN_CASES, ids=[c[0] for c in GOLDEN_CASES])
def test_golden_python(name, bits, expected):
    assert xo.sum_bits(bits) == expected


@pytest.mark.parametrize("name,bits,expected", GOLDEN_CASES, ids=[c[0] for c in GOLDEN_CASES])
def test_golden_c(name, bits, expected):
    assert c_oracle.sum_bits(np.array(bits, dtype=np.uint64)) == expected


def test_golden_file_is_nontrivial():
    assert len(GOLDEN_CASES) >= 20


# --------------------------------------------------------------------------- #
# Rounding step against Fraction -> float
# --------------------------------------------------------------------------- #

def _random_S(rng):
    bl = rng.choice([1, 2, 30, 52, 53, 54, 55, 64, 100, 500, 1000, 1074, 1075, 1076, 2000,
                     2097, 2098, 2099, 2100, 2120]) if rng.random() < 0.5 else rng.randint(1, 2130)
    S = rng.getrandbits(bl) | (1 << (bl - 1))
    return -S if rng.random() < 0.5 else S


def test_round_matches_fraction_random():
    rng = random.Random(1234)
    for _ in range(20000):
        S = _random_S(rng)
        try:
            ref = f2b(S / (1 << 1074))  # int/int true division rounds correctly
        except OverflowError:
            ref = f2b(math.inf if S > 0 else -math.inf)
        assert xo.round_rne(S) == ref, S


def test_round_matches_fraction_midpoints():
    """Exact midpoints and their neighbours, where ties-to-even decides."""
    rng = random.Random(99)
    for _ in range(5000):
        sh = rng.randint(1, 1100)
        q = rng.getrandbits(53) | (1 << 52)
        for delta in (-1, 0, 1):
            S = (q << sh) + (1 << (sh - 1)) + delta
            for sgn in (1, -1):
                try:
                    ref = f2b((sgn * S) / (1 << 1074))
                except OverflowError:
                    ref = f2b(math.inf * sgn)
                assert xo.round_rne(sgn * S) == ref


# --------------------------------------------------------------------------- #
# math.fsum (Shewchuk, correctly rounded) on finite inputs without overflow
# --------------------------------------------------------------------------- #

def _finite_arrays():
    yield W.cfg0_cancel(0)
    yield W.bits_to_f64(W.cfg1_band(0, 0, 20000))
    yield W.bits_to_f64(W.cfg1_band(1, 0, 5000, -1074 + 60, -900))
    yield W.zero_sum_mirror(0, 4000)
    yield W.bits_to_f64(W.cfg3_values(2, 1000, 3000))
    x = W.bits_to_f64(W.cfg2a_full_range(0, 0, 3000)).copy()
    x[np.abs(x) > 1e300] = 1.0  # fsum overflows on intermediate values near DBL_MAX
    yield x


@pytest.mark.parametrize("k", range(6))
def test_fsum_agrees(k):
    x = list(_finite_arrays())[k]
    got = xo.sum_floats(x.tolist())
    ref = math.fsum(x.tolist())
    assert got == ref
    if ref != 0:
        assert f2b(got) == f2b(ref)


# --------------------------------------------------------------------------- #
# Two-term identity: sums of two terms are exactly rounded by IEEE addition
# (Discussion) -- so oracle([a, b]) must equal a + b bit for bit.
# --------------------------------------------------------------------------- #

def test_two_term_identity_random():
    rng = np.random.default_rng(5)
    cls = [W.cfg2a_full_range(3, 0, 40000), W.cfg1_band(4, 0, 40000),
           W.cfg1_band(5, 0, 40000, -1022, -1000), W.cfg1_band(6, 0, 40000, 1000, 1024)]
    pool = np.concatenate(cls)
    a = pool[rng.integers(0, pool.size, 60000)]
    b = pool[rng.integers(0, pool.size, 60000)]
    # make some pairs close in magnitude (massive cancellation)
    b[:10000] = (a[:10000] ^ np.uint64(1 << 63)) + np.uint64(rng.integers(0, 4))
    for x, y in zip(a.tolist(), b.tolist()):
        fx, fy = b2f(x), b2f(y)
        if math.isnan(fx) or math.isnan(fy) or math.isinf(fx) or math.isinf(fy):
            continue
        assert xo.sum_bits([x, y]) == f2b(fx + fy)


def test_two_term_identity_edges():
    for a, b in itertools.product(EDGE, EDGE):
        assert xo.sum_bits([f2b(a), f2b(b)]) == f2b(a + b), (a, b)


def test_one_term_identity():
    vals = EDGE + [b2f(int(v)) for v in W.cfg2a_full_range(9, 0, 2000)] + [-0.0]
    for v in vals:
        assert xo.sum_bits([f2b(v)]) == f2b(v)
    assert xo.sum_bits([xo.POS_INF]) == xo.POS_INF
    assert xo.sum_bits([0x7FF0000000000123]) == 0x7FF8000000000123  # quietened


# --------------------------------------------------------------------------- #
# Worked example of the Introduction
# --------------------------------------------------------------------------- #

def test_worked_example_all_orders():
    base = [1e15, -1e15, 0.1]
    assert (1e15 + 0.1) - 1e15 == 0.125  # naive summation really fails here
    for perm in itertools.permutations(base):
        assert xo.sum_bits([f2b(v) for v in perm]) == f2b(0.1)
        assert c_oracle.sum_bits(W.f64_to_bits(list(perm))) == f2b(0.1)
    assert xo.sum_floats(base) / 3 == 0.1 / 3


# --------------------------------------------------------------------------- #
# Closed form for repeats: N copies of v sum to fl(N * v) (one IEEE multiply,
# exact product rounded once, N < 2^53)
# --------------------------------------------------------------------------- #

REPEAT_V = [0.1, 1.0 - 2.0 ** -53, 3 * 5e-324, DMAX / 2 ** 30, -0.7, 2.0 ** -1030]


@pytest.mark.parametrize("v", REPEAT_V)
@pytest.mark.parametrize("N", [1, 2, 3, 2047, 2048, 4095, 4096, 4097, 8192, 100003])
def test_repeat_closed_form(v, N):
    bits = np.full(N, f2b(v), dtype=np.uint64)
    expect = f2b(v * N)
    assert c_oracle.sum_bits(bits) == expect
    if N <= 8192:
        assert xo.sum_bits(bits.tolist()) == expect


@pytest.mark.slow
@pytest.mark.parametrize("v", [0.1, 1.0 - 2.0 ** -53, 3 * 5e-324, DMAX / 2 ** 30])
def test_repeat_closed_form_1e8(v):
    N = 10 ** 8
    assert c_oracle.sum_bits(np.full(N, f2b(v), dtype=np.uint64)) == f2b(v * N)


# --------------------------------------------------------------------------- #
# Invariants of the exact sum
# --------------------------------------------------------------------------- #

def test_exact_cancellation():
    x = W.cfg2a_full_range(11, 0, 3000)
    both = np.concatenate([x, x ^ np.uint64(1 << 63)])
    nan_inf = ((both >> np.uint64(52)) & np.uint64(0x7FF)) == np.uint64(0x7FF)
    both = both[~nan_inf]
    assert xo.sum_bits(both.tolist()) == 0
    assert c_oracle.sum_bits(both) == 0


def test_mirror_workload_sums_to_zero():
    x = W.zero_sum_mirror(3, 10000)
    assert c_oracle.sum_bits(W.f64_to_bits(x)) == 0
    perm = np.random.default_rng(0).permutation(x.size)
    assert xo.sum_bits(W.f64_to_bits(x[perm]).tolist()) == 0


def test_permutation_invariance():
    x = W.cfg2a_paired(0, 0, 5000, n_log2=28)
    ref = xo.sum_bits(x.tolist())
    rng = np.random.default_rng(1)
    for _ in range(3):
        assert xo.sum_bits(x[rng.permutation(x.size)].tolist()) == ref
        assert c_oracle.sum_bits(x[rng.permutation(x.size)]) == ref


def test_split_merge_invariance():
    x = W.cfg0_cancel(2)
    bits = W.f64_to_bits(x).tolist()
    ref = xo.sum_bits(bits)
    rng = random.Random(3)
    for _ in range(20):
        cuts = sorted(rng.sample(range(1, len(bits)), rng.randint(1, 8)))
        parts = [bits[i:j] for i, j in zip([0] + cuts, cuts + [len(bits)])]
        st = xo.ExactState()
        for p in parts:
            st = st.merge(xo.state_of_bits(p))
        assert xo.finish(st) == ref


def test_canonical_chunks_represent_value():
    x = W.cfg2a_paired(1, 0, 2000, n_log2=28)
    st = xo.state_of_bits(x.tolist())
    ch = xo.canonical_chunks(st)
    assert len(ch) == 67
    assert all(0 <= c < 2 ** 32 for c in ch[:66])
    assert -(2 ** 32) <= ch[66] < 2 ** 32
    assert sum(c << (32 * i) for i, c in enumerate(ch)) == 2 * st.S


# --------------------------------------------------------------------------- #
# Brute force on tiny inputs against exact rationals
# --------------------------------------------------------------------------- #

SMALL_GRID = [0.0, 5e-324, 2.0 ** -1022, 2.0 ** -1022 - 5e-324, 2.0 ** -53, 1.0,
              1.0 + 2.0 ** -52, 1.5, 2.0 ** 53, 1e15, 2.0 ** 970, DMAX, 0.1]
SMALL_GRID = SMALL_GRID + [-v for v in SMALL_GRID]


def test_brute_force_three_terms():
    for trio in itertools.product(SMALL_GRID, repeat=3):
        bits = [f2b(v) for v in trio]
        got = xo.sum_bits(bits)
        ref = fraction_reference(trio)
        if Fraction(0) == sum((Fraction(v) for v in trio), Fraction(0)):
            ref = 0x8000000000000000 if all(b == 0x8000000000000000 for b in bits) else 0
        assert got == ref, trio


def test_brute_force_random_short():
    rng = np.random.default_rng(7)
    pool = np.concatenate([W.cfg2a_full_range(5, 0, 5000), W.cfg1_band(5, 0, 5000)])
    pool = pool[((pool >> np.uint64(52)) & np.uint64(0x7FF)) != np.uint64(0x7FF)]
    for _ in range(2000):
        n = int(rng.integers(1, 50))
        bits = pool[rng.integers(0, pool.size, n)].tolist()
        vals = [b2f(b) for b in bits]
        ref = fraction_reference(vals)
        if sum((Fraction(v) for v in vals), Fraction(0)) == 0:
            ref = 0x8000000000000000 if all(b == 0x8000000000000000 for b in bits) else 0
        assert xo.sum_bits(bits) == ref
        assert c_oracle.sum_bits(np.array(bits, dtype=np.uint64)) == ref


# --------------------------------------------------------------------------- #
# C oracle against the Python oracle, bit for bit
# --------------------------------------------------------------------------- #

def _arrays_for_c_check():
    yield W.cfg2a_full_range(0, 0, 30000)
    yield W.cfg2a_paired(0, 0, 30000, n_log2=28)
    yield W.cfg2b_cancel_1e300(0, 0, 30000, n_log2=28)
    yield W.cfg1_band(0, 0, 30000)
    yield W.f64_to_bits(W.cfg0_cancel(0))
    for _, vals in W.cfg2d_side_cases():
        yield W.f64_to_bits(np.array(vals, dtype=np.float64))


@pytest.mark.parametrize("k", range(5 + len(W.cfg2d_side_cases())))
def test_c_oracle_matches_python(k):
    a = list(_arrays_for_c_check())[k]
    assert c_oracle.sum_bits(a) == xo.sum_bits(a.tolist())


def test_c_oracle_segments():
    lengths = np.array([0, 1, 2, 5, 100, 3000, 1, 7], dtype=np.int64)
    off = W.cfg3_offsets(lengths)
    vals = W.cfg2a_full_range(2, 0, int(off[-1]))
    got = c_oracle.segment_sums_bits(vals, off)
    ref = xo.segment_sums_bits(vals.tolist(), off.tolist())
    assert got.tolist() == ref


# --------------------------------------------------------------------------- #
# The pins bite: plausible mistakes planted in a copy of the oracle fail them
# --------------------------------------------------------------------------- #

def _mutant_round_ties_away(S):
    if S == 0:
        return 0
    neg = S < 0
    A = abs(S)
    if A < (1 << 53):
        return A | (neg << 63)
    sh = A.bit_length() - 53
    q = A >> sh
    if (A >> (sh - 1)) & 1:
        q += 1  # ties away from zero: wrong
    if q == 1 << 53:
        q >>= 1
        sh += 1
    e = sh + 1
    bits = 0x7FF0000000000000 if e >= 2047 else ((e - 1) << 52) + q
    return bits | (neg << 63)


def _mutant_scaled_no_implicit(e, m):
    return m << max(e - 1, 0)  # dropped implicit bit


def _mutant_scaled_off_by_one(e, m):
    return m if e == 0 else ((1 << 52) + m) << e  # wrong exponent offset


@pytest.mark.parametrize("mutant", ["ties_away", "no_implicit", "off_by_one"])
def test_pins_detect_planted_mistakes(monkeypatch, mutant):
    if mutant == "ties_away":
        monkeypatch.setattr(xo, "round_rne", _mutant_round_ties_away)
    elif mutant == "no_implicit":
        monkeypatch.setattr(xo, "scaled_integer", _mutant_scaled_no_implicit)
    else:
        monkeypatch.setattr(xo, "scaled_integer", _mutant_scaled_off_by_one)
    failures = sum(xo.sum_bits(bits) != exp for _, bits, exp in GOLDEN_CASES)
    assert failures > 0
