"""CPU oracle of the exact sum of binary32 values (test infrastructure only).

Same definition as the double oracle with single-precision constants: a finite
float (-1)^s (2^23 + m) 2^(e-150) (or m 2^-149 for e == 0) is the integer
K = M << (e_eff - 1) in units of 2^-149; the exact integer sum is rounded once
to the nearest float, ties to even, overflowing to +-Inf when the biased
exponent reaches 255. NaN rule: largest 22-bit payload, positive sign on ties,
quiet bit set; +Inf with -Inf gives 0x7FC00000; -0 only if every term is -0.
"""

from __future__ import annotations

SIGN = 1 << 31
POS_INF = 0x7F800000
NEG_INF = 0xFF800000
DEFAULT_NAN = 0x7FC00000
NEG_ZERO = 0x80000000


def round_rne32(S: int) -> int:
    if S == 0:
        return 0
    neg = S < 0
    A = -S if neg else S
    if A < (1 << 24):
        bits = A
    else:
        sh = A.bit_length() - 24
        q = A >> sh
        r = A & ((1 << sh) - 1)
        half = 1 << (sh - 1)
        if r > half or (r == half and (q & 1)):
            q += 1
        if q == (1 << 24):
            q >>= 1
            sh += 1
        e = sh + 1
        bits = POS_INF if e >= 255 else ((e - 1) << 23) + q
    return bits | (SIGN if neg else 0)


def sum_f32_bits(bits) -> int:
    S, n, pinf, ninf, nans, allneg = 0, 0, False, False, [], True
    for b in bits:
        b = int(b) & 0xFFFFFFFF
        n += 1
        if b != NEG_ZERO:
            allneg = False
        s, e, m = b >> 31, (b >> 23) & 0xFF, b & 0x7FFFFF
        if e == 0xFF:
            if m == 0:
                ninf, pinf = (True, pinf) if s else (ninf, True)
            else:
                nans.append(b)
            continue
        K = m if e == 0 else (m | (1 << 23)) << (e - 1)
        S += -K if s else K
    if nans:
        return min(nans, key=lambda b: (-(b & 0x3FFFFF), b)) | 0x400000
    if pinf and ninf:
        return DEFAULT_NAN
    if pinf:
        return POS_INF
    if ninf:
        return NEG_INF
    if S == 0:
        return NEG_ZERO if (n > 0 and allneg) else 0
    return round_rne32(S)
