"""Counter-based generators for the synthetic exact-summation workloads.

All arithmetic is on unsigned 64-bit integers that wrap modulo 2**64; numpy
uint64 arrays wrap silently, and scalar key derivation is done with Python ints
masked to 64 bits. The CUDA twin (``workloads/csrc/xsgen.cu``) implements the
same formulas for the device-generated configurations; a test checks the two
bit for bit on index ranges.

Recipes (each value is built from its bits, so host and device agree exactly):

* ``mix64`` is the SplitMix64 output function; ``draw(key, i)`` is
  ``mix64(key + (i + 1) * GAMMA)``.
* ``pow2_band_bits(u, v, lo, hi)``: uniform sign and 52-bit mantissa from ``u``,
  unbiased exponent ``E = lo + floor((v >> 32) * (hi - lo) / 2**32)`` in
  ``[lo, hi - 1]``. This stands in for "magnitude 2^U(lo, hi)".
* ``full_range_bits(u, v)``: biased exponent uniform over 0..2046 (zeros and
  subnormals included), uniform sign and mantissa.
"""

from __future__ import annotations

import math

import numpy as np

MASK64 = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15
_M1 = 0xBF58476D1CE4E5B9
_M2 = 0x94D049BB133111EB
_KEY_MUL_STREAM = 0xD1B54A32D192ED03
_KEY_ADD = 0x632BE59BD9B4E019

# Named sub-streams, so different uses of one seed never share draws.
STREAMS = {
    "sm": 1,      # sign + mantissa bits
    "exp": 2,     # exponent selector
    "sm2": 3,
    "exp2": 4,
    "pick": 5,    # choice without replacement
    "shuf": 6,    # full shuffle
    "len": 7,     # segment lengths
    "unif": 8,    # U(-1,1) values
    "perm": 9,    # affine permutation constants
    "arrive": 10,  # serving arrivals
    "size": 11,   # serving request sizes
    "kind": 12,   # serving request kinds / distributions
}

SIGN_BIT = 1 << 63
MANT_MASK = (1 << 52) - 1


def mix64_int(z: int) -> int:
    """SplitMix64 output function on a Python int (mod 2**64)."""
    z &= MASK64
    z = ((z ^ (z >> 30)) * _M1) & MASK64
    z = ((z ^ (z >> 27)) * _M2) & MASK64
    return z ^ (z >> 31)


def _mix64_np(z: np.ndarray) -> np.ndarray:
    z = z.astype(np.uint64, copy=True)
    z ^= z >> np.uint64(30)
    z *= np.uint64(_M1)
    z ^= z >> np.uint64(27)
    z *= np.uint64(_M2)
    z ^= z >> np.uint64(31)
    return z


def stream_key(seed: int, stream: int | str) -> int:
    """Key of one named sub-stream of a seed."""
    if isinstance(stream, str):
        stream = STREAMS[stream]
    return mix64_int(seed * GAMMA + stream * _KEY_MUL_STREAM + _KEY_ADD)


def draws(key: int, start: int, count: int) -> np.ndarray:
    """uint64 draws ``mix64(key + (i + 1) * GAMMA)`` for i in [start, start + count)."""
    idx = np.arange(start, start + count, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(key & MASK64) + (idx + np.uint64(1)) * np.uint64(GAMMA)
    return _mix64_np(z)


def draws_at(key: int, idx: np.ndarray) -> np.ndarray:
    """uint64 draws at arbitrary indices."""
    idx = np.asarray(idx, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(key & MASK64) + (idx + np.uint64(1)) * np.uint64(GAMMA)
    return _mix64_np(z)


def bits_to_f64(bits: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(bits, dtype=np.uint64).view(np.float64)


def f64_to_bits(x) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x, dtype=np.float64)).view(np.uint64)


def _expsel(v: np.ndarray, span: int) -> np.ndarray:
    """floor((v >> 32) * span / 2**32): uniform integer in [0, span)."""
    return ((v >> np.uint64(32)) * np.uint64(span)) >> np.uint64(32)


def pow2_band_bits(u: np.ndarray, v: np.ndarray, lo: int, hi: int) -> np.ndarray:
    """Random sign, uniform 52-bit mantissa, unbiased exponent in [lo, hi - 1]."""
    e = _expsel(v, hi - lo) + np.uint64(lo + 1023)
    return (u & np.uint64(SIGN_BIT)) | (e << np.uint64(52)) | (u & np.uint64(MANT_MASK))


def full_range_bits(u: np.ndarray, v: np.ndarray, emax_excl: int = 2047) -> np.ndarray:
    """Random sign and mantissa; biased exponent uniform over [0, emax_excl)."""
    e = _expsel(v, emax_excl)
    return (u & np.uint64(SIGN_BIT)) | (e << np.uint64(52)) | (u & np.uint64(MANT_MASK))


def affine_constants(seed: int, n_log2: int) -> tuple[int, int]:
    """(A^{-1} mod 2**n_log2, B) of the bijection pi(k) = (A*k + B) mod 2**n_log2, A odd."""
    n = 1 << n_log2
    a = (mix64_int(stream_key(seed, "perm")) | 1) & (n - 1)
    b = mix64_int(stream_key(seed, "perm") + 1) & (n - 1)
    return pow(a, -1, n), b


def affine_perm_inverse(seed: int, n_log2: int, i: np.ndarray) -> np.ndarray:
    """Inverse of the bijection pi(k) = (A*k + B) mod 2**n_log2 (A odd).

    Used to shuffle the device-sized adversarial arrays without materialising a
    permutation: X[i] = base[pi^{-1}(i)].
    """
    n = 1 << n_log2
    a_inv, b = affine_constants(seed, n_log2)
    i = np.asarray(i, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return ((i - np.uint64(b)) * np.uint64(a_inv)) & np.uint64(n - 1)


# --------------------------------------------------------------------------- #
# Configurations
# --------------------------------------------------------------------------- #

def cfg0_cancel(seed: int = 0) -> np.ndarray:
    """n = 10,000 with heavy cancellation.

    5,000 values U(-1,1) (53-bit grid), 2,500 values of magnitude 2^U(-40,40)
    with random sign, 2,500 exact negations of values chosen without
    replacement from those first 7,500, then a seeded full shuffle.
    """
    u = draws(stream_key(seed, "unif"), 0, 5000)
    a = (u >> np.uint64(11)).astype(np.float64) * (2.0 ** -52) - 1.0
    b = bits_to_f64(pow2_band_bits(draws(stream_key(seed, "sm"), 0, 2500),
                                   draws(stream_key(seed, "exp"), 0, 2500), -40, 40))
    first = np.concatenate([a, b])
    pick = np.argsort(draws(stream_key(seed, "pick"), 0, 7500), kind="stable")[:2500]
    allv = np.concatenate([first, -first[pick]])
    perm = np.argsort(draws(stream_key(seed, "shuf"), 0, allv.size), kind="stable")
    return np.ascontiguousarray(allv[perm])


def cfg1_band(seed: int = 0, start: int = 0, count: int = 10 ** 8,
              lo: int = -60, hi: int = 60) -> np.ndarray:
    """Elements [start, start+count) of the 2^U(-60,60) band array (bits)."""
    u = draws(stream_key(seed, "sm"), start, count)
    v = draws(stream_key(seed, "exp"), start, count)
    return pow2_band_bits(u, v, lo, hi)


def cfg2a_full_range(seed: int = 0, start: int = 0, count: int = 1 << 28) -> np.ndarray:
    """Elements of the full-exponent-range array (bits): e uniform over 0..2046."""
    u = draws(stream_key(seed, "sm"), start, count)
    v = draws(stream_key(seed, "exp"), start, count)
    return full_range_bits(u, v)


def _paired_base(seed: int, k: np.ndarray) -> np.ndarray:
    j = k >> np.uint64(1)
    ks, ke = stream_key(seed, "sm"), stream_key(seed, "exp")
    vj = full_range_bits(draws_at(ks, j), draws_at(ke, j))
    big = ((vj >> np.uint64(52)) & np.uint64(0x7FF)) >= np.uint64(1000)
    fresh = full_range_bits(draws_at(stream_key(seed, "sm2"), j),
                            draws_at(stream_key(seed, "exp2"), j), emax_excl=1000)
    odd = (k & np.uint64(1)) == np.uint64(1)
    partner = np.where(big, vj ^ np.uint64(SIGN_BIT), fresh)
    return np.where(odd, partner, vj)


def cfg2a_paired(seed: int = 0, start: int = 0, count: int = 1 << 28,
                 n_log2: int = 28) -> np.ndarray:
    """Full range, but every term with biased exponent >= 1000 has its negation.

    base[2j] is a full-range draw; base[2j+1] is its negation when that draw has
    e >= 1000, else a fresh draw with e < 1000. The array is base shuffled by an
    affine bijection, so the exact sum is finite and rounding-heavy.
    """
    i = np.arange(start, start + count, dtype=np.uint64)
    return _paired_base(seed, affine_perm_inverse(seed, n_log2, i))


def _cancel_base(seed: int, k: np.ndarray, n: int) -> np.ndarray:
    half = np.uint64(n // 2)
    j = k >> np.uint64(1)
    pair = pow2_band_bits(draws_at(stream_key(seed, "sm"), j),
                          draws_at(stream_key(seed, "exp"), j), 990, 1000)
    pair = np.where((k & np.uint64(1)) == np.uint64(1), pair ^ np.uint64(SIGN_BIT), pair)
    rest = pow2_band_bits(draws_at(stream_key(seed, "sm2"), k),
                          draws_at(stream_key(seed, "exp2"), k), -60, 60)
    return np.where(k < half, pair, rest)


def cfg2b_cancel_1e300(seed: int = 0, start: int = 0, count: int = 1 << 28,
                       n_log2: int = 28) -> np.ndarray:
    """n/4 pairs of +-2^U(990,1000) that cancel exactly, n/2 values +-2^U(-60,60).

    base[k] for k < n/2 is pair k>>1 (odd k negated); for k >= n/2 a band value.
    Shuffled by an affine bijection.
    """
    n = 1 << n_log2
    i = np.arange(start, start + count, dtype=np.uint64)
    return _cancel_base(seed, affine_perm_inverse(seed, n_log2, i), n)


def cfg2c_repeat(v: float, n: int = 10 ** 8) -> np.ndarray:
    """n copies of one value (carry and transfer stress)."""
    return np.full(n, v, dtype=np.float64)


def cfg2d_side_cases() -> list[tuple[str, list[float]]]:
    """Small hand-picked arrays: signed zeros, overflow, Inf/NaN mixes, boundaries."""
    f = float
    dmax = np.finfo(np.float64).max
    tiny = 5e-324
    nan_a = bits_to_f64(np.array([0x7FF8000000000001], dtype=np.uint64))[0]
    nan_b = bits_to_f64(np.array([0xFFF0000000000ABC], dtype=np.uint64))[0]
    nan_c = bits_to_f64(np.array([0x7FF4000000000ABC], dtype=np.uint64))[0]
    return [
        ("all_pos_zero", [0.0] * 7),
        ("all_neg_zero", [-0.0] * 7),
        ("mixed_zero", [-0.0, 0.0, -0.0]),
        ("one_neg_zero", [-0.0]),
        ("overflow_pos", [dmax, dmax, dmax]),
        ("overflow_neg", [-dmax] * 4),
        ("overflow_then_back", [dmax, dmax, -dmax]),
        ("inf_minus_inf", [f("inf"), f("-inf"), 1.0]),
        ("pos_inf_finite_overflow", [f("inf"), -dmax, -dmax]),
        ("neg_inf", [1.0, f("-inf"), 2.0]),
        ("nan_payloads", [1.0, nan_a, nan_b, nan_c, 2.0]),
        ("nan_with_inf", [f("inf"), nan_a, f("-inf")]),
        ("tie_even", [1.0, 2.0 ** -53]),
        ("tie_sticky", [1.0, 2.0 ** -53, tiny]),
        ("tie_odd", [1.0 + 2.0 ** -52, 2.0 ** -53]),
        ("max_plus_half_ulp", [dmax, 2.0 ** 970]),
        ("max_plus_under_half", [dmax, 2.0 ** 969]),
        ("max_half_ulp_minus_tiny", [dmax, 2.0 ** 970, -tiny]),
        ("subnormal_edge", [2.0 ** -1022, -tiny]),
        ("subnormal_sum", [tiny] * 1000),
        ("worked_example", [1e15, -1e15, 0.1]),
    ]


def cfg3_lengths(seed: int = 0, nseg: int = 100_000, lmax: int = 10 ** 6) -> np.ndarray:
    """Segment lengths floor(2^U(0, log2(lmax + 1))) clipped to [1, lmax]."""
    u = (draws(stream_key(seed, "len"), 0, nseg) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    lengths = np.floor(np.exp2(u * math.log2(lmax + 1))).astype(np.int64)
    return np.clip(lengths, 1, lmax)


def cfg3_offsets(lengths: np.ndarray) -> np.ndarray:
    off = np.zeros(lengths.size + 1, dtype=np.int64)
    np.cumsum(lengths, out=off[1:])
    return off


def cfg3_values(seed: int = 0, start: int = 0, count: int = 0) -> np.ndarray:
    """Values (bits) of the segmented workload at global indices [start, start+count)."""
    return cfg1_band(seed, start, count, -30, 30)


def zero_sum_mirror(seed: int, n: int) -> np.ndarray:
    """The paper's timing workload shape: U1*exp(30*U2) then negated mirror.

    Element n-1-i is the negation of element i, so the exact sum is zero. The
    paper's own congruential generator constants are not given, so the uniforms
    come from SplitMix64 instead.
    """
    h = n // 2
    u1 = ((draws(stream_key(seed, "unif"), 0, h) >> np.uint64(11)).astype(np.float64) + 0.5) * (2.0 ** -53)
    u2 = ((draws(stream_key(seed, "sm"), 0, h) >> np.uint64(11)).astype(np.float64) + 0.5) * (2.0 ** -53)
    first = u1 * np.exp(30.0 * u2)
    out = np.zeros(n, dtype=np.float64)
    out[:h] = first
    out[n - h:] = -first[::-1]
    return out
