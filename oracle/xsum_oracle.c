/*
 * CPU oracle for the correctly rounded exact sum of binary64 values (plain C).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by tests/, by __graft_entry__.smoke() and by
 * the CPU-baseline leg of bench.py. The CUDA library shares no code with it.
 *
 * It computes the same definition as oracle/xsum_oracle.py (Neal 2015: exact
 * sum, rounded once to nearest with ties to even; abstract and the
 * small-superaccumulator section on rounding), for arrays too large for Python
 * integers:
 *
 *   - each finite value (-1)^s (2^52 + m) 2^(e-1075) (or m 2^-1074 when e == 0,
 *     section "Floating-point and integer formats", Fig. 1) is the integer
 *     K = M << (e_eff - 1) in units of 2^-1074, with M the 53-bit significand
 *     and e_eff = max(e, 1);
 *   - positive terms are added into one unsigned big integer P and negative
 *     terms into another one, N, each with full carry propagation after every
 *     add (base 2^32 limbs);
 *   - S = P - N, then round S * 2^-1074 to nearest, ties to even, with the same
 *     special-value rules as the Python oracle (NaN payload choice, Inf, -0).
 *
 * One sum runs on one thread. xo_sum_segments_bits runs independent segments
 * on OpenMP threads; the integer sum inside a segment is never split.
 */
#include <stdint.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* 72 limbs of 32 bits: 2304 bits, above the 2098 bits of the largest K plus the
 * 45 bits of headroom for 2^45 terms. */
#define XO_LIMBS 72

typedef struct {
  uint32_t pos[XO_LIMBS];
  uint32_t neg[XO_LIMBS];
  int64_t n;
  int pos_inf, neg_inf, has_nan, all_neg_zero;
  uint64_t nan_bits; /* current choice among the NaNs seen */
} xo_state;

static void xo_init(xo_state *st) {
  memset(st, 0, sizeof(*st));
  st->all_neg_zero = 1;
}

/* a += v * 2^(32*idx), rippling the carry upward. */
static void add_limb(uint32_t *a, int idx, uint32_t v) {
  uint64_t carry = v;
  while (carry != 0 && idx < XO_LIMBS) {
    uint64_t s = (uint64_t)a[idx] + carry;
    a[idx] = (uint32_t)s;
    carry = s >> 32;
    idx++;
  }
}

/* a += M << shift, M < 2^53, shift >= 0. */
static void add_shifted(uint32_t *a, uint64_t M, int shift) {
  int q = shift / 32, r = shift % 32;
  uint64_t t0 = (M & 0xFFFFFFFFu) << r; /* < 2^63 */
  uint64_t t1 = ((M >> 32) << r) + (t0 >> 32); /* < 2^53 + 2^31 */
  add_limb(a, q, (uint32_t)t0);
  add_limb(a, q + 1, (uint32_t)t1);
  add_limb(a, q + 2, (uint32_t)(t1 >> 32));
}

/* NaN choice: larger payload wins; equal payloads prefer the smaller raw
 * pattern (positive sign). Returns nonzero if b is preferred over cur. */
static int nan_better(uint64_t b, uint64_t cur) {
  const uint64_t P = 0x0007FFFFFFFFFFFFull;
  if ((b & P) != (cur & P)) return (b & P) > (cur & P);
  return b < cur;
}

static void xo_add(xo_state *st, uint64_t b) {
  uint32_t s = (uint32_t)(b >> 63);
  uint32_t e = (uint32_t)((b >> 52) & 0x7FF);
  uint64_t m = b & 0x000FFFFFFFFFFFFFull;
  st->n++;
  if (b != 0x8000000000000000ull) st->all_neg_zero = 0;
  if (e == 0x7FF) {
    if (m == 0) {
      if (s) st->neg_inf = 1; else st->pos_inf = 1;
    } else if (!st->has_nan || nan_better(b, st->nan_bits)) {
      st->has_nan = 1;
      st->nan_bits = b;
    }
    return;
  }
  if (e == 0 && m == 0) return;
  uint64_t M = (e == 0) ? m : (m | (1ull << 52));
  int shift = (e == 0) ? 0 : (int)e - 1;
  add_shifted(s ? st->neg : st->pos, M, shift);
}

static int cmp_mag(const uint32_t *a, const uint32_t *b) {
  for (int i = XO_LIMBS - 1; i >= 0; --i) {
    if (a[i] != b[i]) return a[i] > b[i] ? 1 : -1;
  }
  return 0;
}

/* out = a - b, a >= b */
static void sub_mag(const uint32_t *a, const uint32_t *b, uint32_t *out) {
  int64_t borrow = 0;
  for (int i = 0; i < XO_LIMBS; ++i) {
    int64_t d = (int64_t)a[i] - (int64_t)b[i] - borrow;
    borrow = d < 0;
    out[i] = (uint32_t)(d + (borrow ? ((int64_t)1 << 32) : 0));
  }
}

static int get_bit(const uint32_t *a, int pos) {
  if (pos < 0) return 0;
  return (a[pos / 32] >> (pos % 32)) & 1;
}

static int any_bit_below(const uint32_t *a, int pos) { /* any bit < pos set */
  for (int p = 0; p < pos; ++p) {
    if (get_bit(a, p)) return 1;
  }
  return 0;
}

/* Round the magnitude A * 2^-1074 to nearest, ties to even; returns bits
 * without the sign. */
static uint64_t round_mag(const uint32_t *A) {
  int top = -1;
  for (int i = XO_LIMBS - 1; i >= 0; --i) {
    if (A[i]) { top = i; break; }
  }
  if (top < 0) return 0;
  int bitlen = 32 * top + (32 - __builtin_clz(A[top]));
  if (bitlen <= 53) { /* exactly representable: the pattern is the integer */
    uint64_t v = A[0];
    if (top >= 1) v |= (uint64_t)A[1] << 32;
    return v;
  }
  int sh = bitlen - 53;
  uint64_t q = 0;
  for (int k = 0; k < 53; ++k) q |= (uint64_t)get_bit(A, sh + k) << k;
  int round = get_bit(A, sh - 1);
  int sticky = any_bit_below(A, sh - 1);
  if (round && (sticky || (q & 1))) q += 1;
  if (q == (1ull << 53)) { q >>= 1; sh += 1; }
  uint64_t e = (uint64_t)sh + 1;
  if (e >= 0x7FF) return 0x7FF0000000000000ull;
  return ((e - 1) << 52) + q;
}

static uint64_t xo_finish(const xo_state *st) {
  if (st->has_nan) return st->nan_bits | 0x0008000000000000ull;
  if (st->pos_inf && st->neg_inf) return 0x7FF8000000000000ull;
  if (st->pos_inf) return 0x7FF0000000000000ull;
  if (st->neg_inf) return 0xFFF0000000000000ull;
  int c = cmp_mag(st->pos, st->neg);
  if (c == 0) return (st->n > 0 && st->all_neg_zero) ? 0x8000000000000000ull : 0;
  uint32_t A[XO_LIMBS];
  if (c > 0) {
    sub_mag(st->pos, st->neg, A);
    return round_mag(A);
  }
  sub_mag(st->neg, st->pos, A);
  return round_mag(A) | 0x8000000000000000ull;
}

/* Exact mean: round (P - N) / n once. The magnitude, doubled (units of
 * 2^-1075), is divided by n from the top limb down; the quotient is rounded at
 * the double grid with the nonzero remainder as sticky information. */
static uint64_t round_quotient(const uint32_t *Q, int sticky_in) {
  int top = -1;
  for (int i = XO_LIMBS - 1; i >= 0; --i) {
    if (Q[i]) { top = i; break; }
  }
  if (top < 0) return 0; /* below half of 2^-1074 */
  int bitlen = 32 * top + (32 - __builtin_clz(Q[top]));
  if (bitlen <= 54) { /* spacing 2^-1074 = 2 units */
    uint64_t v = Q[0];
    if (top >= 1) v |= (uint64_t)Q[1] << 32;
    uint64_t m = v >> 1;
    if ((v & 1) && (sticky_in || (m & 1))) m += 1;
    return m;
  }
  int sh = bitlen - 53;
  uint64_t m = 0;
  for (int k = 0; k < 53; ++k) m |= (uint64_t)get_bit(Q, sh + k) << k;
  int round = get_bit(Q, sh - 1);
  int sticky = sticky_in || any_bit_below(Q, sh - 1);
  if (round && (sticky || (m & 1))) m += 1;
  if (m == (1ull << 53)) { m >>= 1; sh += 1; }
  uint64_t e = (uint64_t)sh; /* biased exponent in units of 2^-1075 */
  if (e >= 0x7FF) return 0x7FF0000000000000ull;
  return ((e - 1) << 52) + m;
}

uint64_t xo_mean_bits(const uint64_t *bits, int64_t n) {
  if (n <= 0) return 0x7FF8000000000000ull;
  xo_state st;
  xo_init(&st);
  for (int64_t i = 0; i < n; ++i) xo_add(&st, bits[i]);
  if (st.has_nan || st.pos_inf || st.neg_inf) return xo_finish(&st);
  int c = cmp_mag(st.pos, st.neg);
  if (c == 0) return xo_finish(&st);
  uint32_t A[XO_LIMBS], D2[XO_LIMBS], Q[XO_LIMBS];
  if (c > 0) sub_mag(st.pos, st.neg, A); else sub_mag(st.neg, st.pos, A);
  /* D2 = 2 A */
  uint32_t carry = 0;
  for (int i = 0; i < XO_LIMBS; ++i) {
    D2[i] = (A[i] << 1) | carry;
    carry = A[i] >> 31;
  }
  unsigned __int128 rem = 0;
  for (int i = XO_LIMBS - 1; i >= 0; --i) {
    unsigned __int128 cur = (rem << 32) | D2[i];
    Q[i] = (uint32_t)(cur / (uint64_t)n);
    rem = cur % (uint64_t)n;
  }
  return round_quotient(Q, rem != 0) | (c < 0 ? 0x8000000000000000ull : 0);
}

/* Single precision: terms K = M << (e_eff - 1) in units of 2^-149, same
 * two-magnitude sum, rounded to a 24-bit significand. */
static uint32_t round_mag32(const uint32_t *A) {
  int top = -1;
  for (int i = XO_LIMBS - 1; i >= 0; --i) {
    if (A[i]) { top = i; break; }
  }
  if (top < 0) return 0;
  int bitlen = 32 * top + (32 - __builtin_clz(A[top]));
  if (bitlen <= 24) return A[0];
  int sh = bitlen - 24;
  uint32_t q = 0;
  for (int k = 0; k < 24; ++k) q |= (uint32_t)get_bit(A, sh + k) << k;
  int round = get_bit(A, sh - 1);
  int sticky = any_bit_below(A, sh - 1);
  if (round && (sticky || (q & 1))) q += 1;
  if (q == (1u << 24)) { q >>= 1; sh += 1; }
  uint32_t e = (uint32_t)sh + 1;
  if (e >= 0xFF) return 0x7F800000u;
  return ((e - 1) << 23) + q;
}

uint32_t xo_sum_f32_bits(const uint32_t *bits, int64_t n) {
  uint32_t P[XO_LIMBS], N[XO_LIMBS];
  memset(P, 0, sizeof P);
  memset(N, 0, sizeof N);
  int pinf = 0, ninf = 0, has_nan = 0, allneg = 1;
  uint32_t nanb = 0;
  for (int64_t i = 0; i < n; ++i) {
    uint32_t b = bits[i];
    if (b != 0x80000000u) allneg = 0;
    uint32_t s = b >> 31, e = (b >> 23) & 0xFF, m = b & 0x7FFFFF;
    if (e == 0xFF) {
      if (m == 0) {
        if (s) ninf = 1; else pinf = 1;
      } else {
        const uint32_t pl = b & 0x3FFFFF, cur = nanb & 0x3FFFFF;
        if (!has_nan || pl > cur || (pl == cur && b < nanb)) nanb = b;
        has_nan = 1;
      }
      continue;
    }
    if (e == 0 && m == 0) continue;
    uint64_t M = e == 0 ? m : (m | (1u << 23));
    add_shifted(s ? N : P, M, e == 0 ? 0 : (int)e - 1);
  }
  if (has_nan) return nanb | 0x400000u;
  if (pinf && ninf) return 0x7FC00000u;
  if (pinf) return 0x7F800000u;
  if (ninf) return 0xFF800000u;
  int c = cmp_mag(P, N);
  if (c == 0) return (n > 0 && allneg) ? 0x80000000u : 0u;
  uint32_t A[XO_LIMBS];
  if (c > 0) {
    sub_mag(P, N, A);
    return round_mag32(A);
  }
  sub_mag(N, P, A);
  return round_mag32(A) | 0x80000000u;
}

uint64_t xo_sum_bits(const uint64_t *bits, int64_t n) {
  xo_state st;
  xo_init(&st);
  for (int64_t i = 0; i < n; ++i) xo_add(&st, bits[i]);
  return xo_finish(&st);
}

/* Sums of selected CSR segments: out[j] = sum of bits[offsets[s] .. offsets[s+1])
 * for s = seg_ids[j]. Independent segments run on separate OpenMP threads. */
void xo_sum_segments_bits(const uint64_t *bits, const int64_t *offsets,
                          const int64_t *seg_ids, int64_t nsel, uint64_t *out) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t j = 0; j < nsel; ++j) {
    int64_t s = seg_ids[j];
    out[j] = xo_sum_bits(bits + offsets[s], offsets[s + 1] - offsets[s]);
  }
}

/* Several independent arrays (each given by a pointer and a length). */
void xo_sum_many_bits(const uint64_t *const *arrays, const int64_t *lengths,
                      int64_t count, uint64_t *out) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t j = 0; j < count; ++j) out[j] = xo_sum_bits(arrays[j], lengths[j]);
}

int xo_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
