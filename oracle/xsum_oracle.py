"""CPU oracle for the correctly rounded exact sum of binary64 values.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module. The library under
``paper_1505_05571_gb300`` never imports it and has no CPU fallback.

Neal, "Fast Exact Summation Using Small and Large Superaccumulators" (2015)
computes the exact sum of a set of doubles and rounds it once to the nearest
double, ties to even (abstract; Introduction; small-superaccumulator section on
rounding). The method reaches exactly that result, so this oracle is the plain
definition of it, not the superaccumulator algorithm:

1. Decode each value into sign s, biased exponent e and 52-bit field m
   (section "Floating-point and integer formats", Fig. 1).
2. e == 2047: infinity (m == 0) or NaN (m != 0), kept aside.
3. Finite values scale exactly to an integer in units of 2^-1074:
   K = m when e == 0 (value m * 2^-1074), else K = (2^52 + m) << (e - 1)
   (value (1 + m 2^-52) 2^(e-1023)).
4. S = sum of (-1)^s K with Python's arbitrary-precision integers.
5. Round S * 2^-1074 to nearest, ties to even, overflowing to +-Inf.

Readings where the paper is silent (each also listed in the design notes):

* An exact zero is -0 only when there is at least one term and every term is
  -0; otherwise +0 (IEEE sum semantics; an empty sum is +0).
* With several NaNs, the result is the NaN with the largest 51-bit payload
  (bits & 0x0007FFFFFFFFFFFF), positive sign preferred on ties, with the quiet
  bit set. This makes the choice independent of order.
* +Inf together with -Inf (no NaN input) gives the default quiet NaN
  0x7FF8000000000000.
* Infinite inputs decide the result regardless of the finite part, so
  [+Inf, -DBL_MAX, -DBL_MAX] is +Inf, never NaN.

Pins (tests/test_oracle.py): rounding against ``fractions.Fraction`` to float
conversion, ``math.fsum``, the two-term identity with IEEE addition, the worked
example of the Introduction, closed forms for repeated values, exact
cancellation, permutation and split invariance, hand-derived boundary cases in
``tests/golden/boundaries.txt``, and brute force over a grid of edge values.
"""

from __future__ import annotations

import struct
from dataclasses import dataclass, field

SIGN_BIT = 1 << 63
EXP_MASK = 0x7FF
MANT_BITS = 52
MANT_MASK = (1 << 52) - 1
PAYLOAD_MASK = 0x0007FFFFFFFFFFFF
QUIET_BIT = 1 << 51
POS_INF = 0x7FF0000000000000
NEG_INF = 0xFFF0000000000000
DEFAULT_NAN = 0x7FF8000000000000
NEG_ZERO = 0x8000000000000000


def f2b(x: float) -> int:
    """Bit pattern of a Python float."""
    return struct.unpack("<Q", struct.pack("<d", x))[0]


def b2f(b: int) -> float:
    return struct.unpack("<d", struct.pack("<Q", b & ((1 << 64) - 1)))[0]


def decode(b: int) -> tuple[int, int, int]:
    """Step 1: sign, biased exponent, mantissa field (Fig. 1)."""
    return (b >> 63) & 1, (b >> MANT_BITS) & EXP_MASK, b & MANT_MASK


def scaled_integer(e: int, m: int) -> int:
    """Step 3: the finite value as an exact integer multiple of 2^-1074."""
    if e == 0:
        return m
    return ((1 << MANT_BITS) + m) << (e - 1)


@dataclass
class ExactState:
    """Exact sum of the terms seen so far plus the special-value record."""

    S: int = 0
    n: int = 0
    pos_inf: bool = False
    neg_inf: bool = False
    nans: list = field(default_factory=list)
    all_neg_zero: bool = True

    def add_bits(self, b: int) -> None:
        s, e, m = decode(b)
        self.n += 1
        if b != NEG_ZERO:
            self.all_neg_zero = False
        if e == EXP_MASK:
            if m == 0:
                if s:
                    self.neg_inf = True
                else:
                    self.pos_inf = True
            else:
                self.nans.append(b)
            return
        K = scaled_integer(e, m)
        self.S += -K if s else K

    def merge(self, other: "ExactState") -> "ExactState":
        out = ExactState(self.S + other.S, self.n + other.n,
                         self.pos_inf or other.pos_inf, self.neg_inf or other.neg_inf,
                         self.nans + other.nans, self.all_neg_zero and other.all_neg_zero)
        return out


def choose_nan(nans: list[int]) -> int:
    """Largest payload; on ties the smaller raw pattern (positive first); quiet."""
    best = min(nans, key=lambda b: (-(b & PAYLOAD_MASK), b))
    return best | QUIET_BIT


def round_rne(S: int) -> int:
    """Step 5: bits of the double nearest to S * 2^-1074, ties to even.

    For |S| < 2^53 the value is exactly representable and its bit pattern equals
    |S| (subnormals and the lowest normal binade share that encoding). Otherwise
    keep the top 53 bits, round on the remainder, and overflow to Inf when the
    biased exponent reaches 2047.
    """
    if S == 0:
        return 0
    neg = S < 0
    A = -S if neg else S
    if A < (1 << 53):
        bits = A
    else:
        sh = A.bit_length() - 53
        q = A >> sh
        r = A & ((1 << sh) - 1)
        half = 1 << (sh - 1)
        if r > half or (r == half and (q & 1)):
            q += 1
        if q == (1 << 53):
            q >>= 1
            sh += 1
        e = sh + 1
        if e >= EXP_MASK:
            bits = POS_INF
        else:
            bits = ((e - 1) << MANT_BITS) + q
    return bits | (SIGN_BIT if neg else 0)


def finish(st: ExactState) -> int:
    """Apply the special-value rules, then round."""
    if st.nans:
        return choose_nan(st.nans)
    if st.pos_inf and st.neg_inf:
        return DEFAULT_NAN
    if st.pos_inf:
        return POS_INF
    if st.neg_inf:
        return NEG_INF
    if st.S == 0:
        return NEG_ZERO if (st.n > 0 and st.all_neg_zero) else 0
    return round_rne(st.S)


def round_ratio(N: int, D: int) -> int:
    """Bits (sign excluded) of the double nearest to (N / D) * 2^-1074, ties to even.

    N >= 0, D >= 1. The double grid spacing at x = N/D (in units of 2^-1074) is
    2^k with k = max(0, bitlen(floor(x)) - 53): spacing 1 covers the subnormals
    and the lowest normal binade. m = floor(x / 2^k) is rounded on the exact
    remainder; a carry to 2^53 moves to the next binade.
    """
    if N == 0:
        return 0
    q = N // D
    k = max(0, q.bit_length() - 53)
    den = D << k
    m, r = divmod(N, den)
    if 2 * r > den or (2 * r == den and (m & 1)):
        m += 1
    if m == (1 << 53):
        m >>= 1
        k += 1
    bits = (k << MANT_BITS) + m
    return POS_INF if bits >= POS_INF else bits


def finish_div(st: ExactState, D: int) -> int:
    """(exact sum) / D rounded once, D >= 1; specials and signed zeros as for the sum."""
    if st.nans or st.pos_inf or st.neg_inf or st.S == 0:
        return finish(st)
    sign = SIGN_BIT if st.S < 0 else 0
    return round_ratio(abs(st.S), D) | sign


def finish_mean(st: ExactState) -> int:
    """Correctly rounded exact mean: (exact sum) / n rounded once (Discussion).

    n = 0 gives the default quiet NaN (0/0).
    """
    if st.n == 0:
        return DEFAULT_NAN
    return finish_div(st, st.n)


def mean_bits(bits) -> int:
    return finish_mean(state_of_bits(bits))


def state_of_bits(bits) -> ExactState:
    st = ExactState()
    for b in bits:
        st.add_bits(int(b))
    return st


def sum_bits(bits) -> int:
    """Bits of the correctly rounded exact sum of an iterable of bit patterns."""
    return finish(state_of_bits(bits))


def sum_floats(values) -> float:
    return b2f(sum_bits(f2b(float(v)) for v in values))


def segment_sums_bits(bits, offsets) -> list[int]:
    """Per-segment sums of a CSR layout: segment k is bits[offsets[k]:offsets[k+1]]."""
    return [sum_bits(bits[int(offsets[k]):int(offsets[k + 1])]) for k in range(len(offsets) - 1)]


def canonical_chunks(st: ExactState) -> list[int]:
    """The value as the paper's 67 normalised chunks (small-superaccumulator form).

    The value S * 2^-1074 equals sum_i c_i 2^(32 i - 1075) with c_0..c_65 in
    [0, 2^32) and c_66 in [-2^32, 2^32) (small-superaccumulator section: after
    carry propagation all chunks but the top are non-negative). This is the
    base-2^32 expansion of 2S taken as a two's complement number.
    """
    T = 2 * st.S
    chunks = []
    for _ in range(66):
        chunks.append(T & 0xFFFFFFFF)
        T >>= 32  # floor shift: two's complement digits
    chunks.append(T)
    return chunks
