// Device-side building blocks of the exact FP64 summation library.
//
// Method: R. M. Neal, "Fast Exact Summation Using Small and Large
// Superaccumulators" (2015).
//   * small superaccumulator: 67 signed 64-bit chunks, chunk i weighing
//     2^(32 i - 1075), 32-bit overlap (section "Exact summation using a small
//     superaccumulator", Fig. 2 and Fig. 3);
//   * carry propagation at most every 2^11 - 1 adds (same section);
//   * large superaccumulator: one chunk per sign+exponent, transferred into
//     the small one (section "Faster exact summation of many terms with a
//     large superaccumulator", Fig. 4);
//   * merge of partial accumulators and one final rounding (Discussion).
//
// GPU layout: every thread owns a private small superaccumulator in shared
// memory, laid out [chunk][thread] so a warp's 64-bit accesses never conflict;
// a block owns one large superaccumulator in shared memory, updated with 32-bit
// shared atomics; block partials meet in one global accumulator through 64-bit integer
// atomics (exact and order-free), and the last block to finish rounds.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace xs {

constexpr int kSChunks = 67;        // small superaccumulator chunks
constexpr int kLowExpBits = 5;      // low exponent bits: position inside a chunk
constexpr int kCarryInterval = 2047;  // adds of <= 2^52-1 between propagations
constexpr int kLChunks = 4096;      // large superaccumulator: one per sign+exponent
constexpr unsigned kFull = 0xFFFFFFFFu;

constexpr unsigned long long kPosInf = 0x7FF0000000000000ull;
constexpr unsigned long long kNegInf = 0xFFF0000000000000ull;
constexpr unsigned long long kDefaultNaN = 0x7FF8000000000000ull;
constexpr unsigned long long kNegZero = 0x8000000000000000ull;
constexpr unsigned long long kPayloadMask = 0x0007FFFFFFFFFFFFull;
constexpr unsigned long long kMantMask = 0x000FFFFFFFFFFFFFull;

// Debug build (-DXS_DEBUG): checks of the chunk indices and of the add bound
// between carry propagations. A failed check ORs its code into this
// translation unit's debug word and the access it guards is skipped, so a
// broken invariant reaches the host (xs_debug_status) instead of touching
// shared or global memory out of range. Without XS_DEBUG every check is the
// constant true and compiles to nothing.
enum : unsigned {
  kDbgSmallIndex = 1u,     // small-accumulator chunk index past chunk 65 (an add writes i, i + 1)
  kDbgCarryInterval = 2u,  // more adds between two propagations than the bound allows
  kDbgChunkBound = 4u,     // a chunk outside what that bound lets it reach
  kDbgLargeIndex = 8u,     // large-accumulator index past 4095
  kDbgFlushIndex = 16u,    // a flushed chunk's pieces past the small accumulator's top
  kDbgTableIndex = 32u,    // a segmented tile or slot index out of its table
};
#ifdef XS_DEBUG
static __device__ unsigned long long d_xs_debug_word;
__device__ __forceinline__ bool xs_dcheck(bool ok, unsigned code) {
  if (!ok) atomicOr(&d_xs_debug_word, (unsigned long long)code);
  return ok;
}
#define XS_DCHECK(cond, code) ::xs::xs_dcheck((cond), (code))
// Reads and clears this translation unit's debug word (host).
static inline cudaError_t debug_word_take(unsigned long long* v) {
  cudaError_t e = cudaMemcpyFromSymbol(v, d_xs_debug_word, sizeof *v);
  const unsigned long long zero = 0ull;
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(d_xs_debug_word, &zero, sizeof zero);
  return e;
}
#else
#define XS_DCHECK(cond, code) true
static inline cudaError_t debug_word_take(unsigned long long* v) {
  *v = 0ull;
  return cudaSuccess;
}
#endif
// A bound on a small-accumulator chunk between propagations: below 2^32 after
// one, then at most kCarryInterval adds of a low part (< 2^32) or a high part
// (< 2^52), each possibly negated.
constexpr long long kChunkBound = (1ll << 32) + (long long)kCarryInterval * ((1ll << 52) + (1ll << 32));

// Record of the terms that do not enter the chunks (Inf and NaN fields of the
// small superaccumulator, Fig. 3) plus what decides the sign of a zero.
enum : unsigned {
  kFlagPosInf = 1u,
  kFlagNegInf = 2u,
  kFlagNotNegZero = 4u,  // some term is not -0
  kFlagAny = 8u,         // at least one term
};

// Device-resident accumulator: the canonical small superaccumulator plus the
// special-value record. 560 bytes; also the export format of a handle.
struct __align__(16) AccState {
  long long chunk[kSChunks];
  unsigned flags;
  unsigned ticket;  // completion counter of the kernel writing into it; 0 at rest
  unsigned long long nan_key;  // 0 = no NaN seen
  // chunk window of a sum being rounded (kernels that track it, mode 0 only):
  // max over blocks of 0x7FF - (lowest positional exponent) and of the
  // highest; 0 and 0 = no finite nonzero term yet. 0 at rest.
  unsigned win_lo_inv;
  unsigned win_hi;
};
static_assert(sizeof(AccState) == 560, "AccState layout");

// NaN choice (order-independent): largest 51-bit payload, positive sign on
// ties; the key is maximised with atomicMax.
__device__ __forceinline__ unsigned long long nan_key_of(unsigned long long b) {
  return ((((b & kPayloadMask) << 1) | ((b >> 63) ^ 1ull)) + 1ull);
}
__device__ __forceinline__ unsigned long long nan_from_key(unsigned long long k) {
  k -= 1ull;
  return ((k & 1ull) ? 0ull : kNegZero) | 0x7FF8000000000000ull | (k >> 1);
}

// Streaming 16-byte load that does not allocate in L1.
__device__ __forceinline__ ulonglong2 ld_stream(const ulonglong2* p) {
  ulonglong2 v;
  asm("ld.global.nc.L1::no_allocate.L2::256B.v2.u64 {%0, %1}, [%2];"
      : "=l"(v.x), "=l"(v.y)
      : "l"(p));
  return v;
}
__device__ __forceinline__ unsigned long long ld_stream1(const unsigned long long* p) {
  unsigned long long v;
  asm("ld.global.nc.L1::no_allocate.u64 %0, [%1];" : "=l"(v) : "l"(p));
  return v;
}

// Bulk prefetch of [p, p + bytes) into L2 (TMA engine, no completion to wait
// for). p must be 16-byte aligned and bytes a multiple of 16; callers clamp the
// range to their input. Keeps HBM busy beyond what the threads' own loads put
// in flight.
__device__ __forceinline__ void prefetch_l2(const void* p, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// Programmatic dependent launch (the single-array kernels are launched with
// programmatic stream serialization): a grid may start while the previous
// grid on its stream finishes. wait: block until that grid has completed and
// its writes are visible (a no-op for an ordinary launch); everything before
// it may only touch shared memory or prefetch into L2 (which is coherent).
// launch_dependents: this block no longer holds the next grid back.
__device__ __forceinline__ void grid_dependency_wait() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
}
__device__ __forceinline__ void grid_launch_dependents() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// --------------------------------------------------------------------------
// Small superaccumulator, one per thread, chunks strided by `stride` longs.
// --------------------------------------------------------------------------

// Add one finite double (given as its two 32-bit halves) to the thread's
// small superaccumulator (Fig. 3, branch-free sign as the Discussion
// suggests). Zeros add nothing; the caller handles e == 2047.
// 53-bit significand M, e_eff = max(e, 1), i = e_eff >> 5, l = e_eff & 31;
// the low 32 bits of M << l go to chunk i, the rest (< 2^52) to chunk i+1.
__device__ __forceinline__ void sacc_add(long long* __restrict__ a, int stride,
                                         unsigned lo, unsigned hi) {
  const unsigned e = (hi >> 20) & 0x7FFu;
  const unsigned mh = (hi & 0xFFFFFu) | (e != 0u ? 0x100000u : 0u);
  const unsigned ee = e + (e == 0u ? 1u : 0u);
  const unsigned i = ee >> kLowExpBits;
  const unsigned l = ee & 31u;
  const unsigned p0 = lo << l;                    // bits 0..31 of M << l
  const unsigned q0 = __funnelshift_l(lo, mh, l);  // bits 32..63
  const unsigned q1 = __funnelshift_l(mh, 0u, l);  // bits 64..95
  const long long s = (long long)((int)hi >> 31);  // 0 or -1
  const long long vlo = (long long)(unsigned long long)p0;
  const long long vhi = (long long)(((unsigned long long)q1 << 32) | q0);
  if (!XS_DCHECK(i + 1u < (unsigned)kSChunks, kDbgSmallIndex)) return;
  long long* c = a + (int)i * stride;
  c[0] += (vlo ^ s) - s;
  c[stride] += (vhi ^ s) - s;
}

// Add one NORMAL finite term (1 <= e <= 2046, e = its biased exponent) -- the
// common case, kept short because the small-superaccumulator kernel is bound
// by instruction issue:
//   2^l from a wrap-mode funnel shift of e (l = e & 31),
//   M << l as two 32x32->64 multiplies by 2^l (FMA pipe instead of shifts),
//   conditional negation as XOR with the sign mask plus the sign bit, which
//   fuses into the three-input adds of the two chunk updates.
template <int STRIDE>
__device__ __forceinline__ void sacc_add_normal(long long* __restrict__ a, unsigned lo,
                                                unsigned hi, unsigned e) {
  const unsigned pw = __funnelshift_l(0u, 1u, e);     // 2^(e & 31)
  const unsigned mh = (hi & 0xFFFFFu) | 0x100000u;    // high 21 bits of M
  const unsigned long long P = (unsigned long long)lo * pw;              // lo << l
  const unsigned long long Q = (unsigned long long)mh * pw + (P >> 32);  // (M << l) >> 32
  const unsigned s = (unsigned)((int)hi >> 31);       // 0 or 0xFFFFFFFF
  const unsigned s1 = hi >> 31;                       // 0 or 1
  if (!XS_DCHECK((e >> kLowExpBits) + 1u < (unsigned)kSChunks, kDbgSmallIndex)) return;
  long long* c = a + (int)(e >> kLowExpBits) * STRIDE;
  const unsigned long long x0 = ((unsigned long long)s << 32) | ((unsigned)P ^ s);
  const unsigned long long x1 = Q ^ (((unsigned long long)s << 32) | s);
  c[0] = (long long)((unsigned long long)c[0] + x0 + s1);
  c[STRIDE] = (long long)((unsigned long long)c[STRIDE] + x1 + s1);
}

// A zero, subnormal, Inf or NaN term b that went through sacc_add_normal as if
// it were normal: cancel that add exactly (same term, sign bit flipped), then
// add a zero or subnormal through the general path (Inf and NaN add nothing).
// Out of line: it runs only for such rare terms.
template <int STRIDE>
__device__ __noinline__ static void take_back(long long* __restrict__ a, unsigned long long b) {
  const unsigned lo = (unsigned)b, hi = (unsigned)(b >> 32), e = (hi >> 20) & 0x7FFu;
  sacc_add_normal<STRIDE>(a, lo, hi ^ 0x80000000u, e);
  if (e == 0u) sacc_add(a, STRIDE, lo, hi);
}

// Per-thread state of the small-superaccumulator path: the chunks plus the
// Inf/NaN record and what decides the sign of an exact zero. With TRACK, the
// range of positional exponents max(e, 1) of the finite nonzero terms seen
// ([emin, emax], empty while emax < emin) is kept as well, so a merge can
// read, and clear, only the chunks those terms touched (Discussion: low
// fixed cost when few chunks are in use).
// A positional exponent past 2046 whose window, (e >> 5) + 1, is the top chunk:
// set as emax once a carry propagation may have filled the chunks above.
constexpr unsigned kWindowTop = (kSChunks - 2) << kLowExpBits;

struct SmallThread {
  long long* acc;  // this thread's chunks, stride BLOCK
  unsigned notnegz = 0u;  // saw a term other than -0
  unsigned sflags = 0u;
  unsigned long long nkey = 0ull;
  unsigned emin = 0x7FFu, emax = 0u;

  __device__ __forceinline__ void reset() {
    notnegz = 0u;
    sflags = 0u;
    nkey = 0ull;
    emin = 0x7FFu;
    emax = 0u;
  }
  __device__ __forceinline__ void special(unsigned long long b) {
    if (b & kMantMask) {
      const unsigned long long k = nan_key_of(b);
      nkey = k > nkey ? k : nkey;
    } else {
      sflags |= (b >> 63) ? kFlagNegInf : kFlagPosInf;
    }
  }
  __device__ __forceinline__ void track(unsigned long long b) {
    const unsigned e = (unsigned)(b >> 52) & 0x7FFu;
    if (e != 0x7FFu && (b << 1) != 0ull) {  // finite and nonzero
      const unsigned ee = e ? e : 1u;
      emin = min(emin, ee);
      emax = max(emax, ee);
    }
  }
  // Any term: zeros, subnormals and Inf/NaN included.
  template <int BLOCK, bool TRACK = false>
  __device__ __forceinline__ void one(unsigned long long b) {
    const unsigned lo = (unsigned)b, hi = (unsigned)(b >> 32);
    notnegz |= (b != kNegZero) ? 1u : 0u;
    if (TRACK) track(b);
    if (((hi >> 20) & 0x7FFu) == 0x7FFu) {
      special(b);
    } else {
      sacc_add(acc, BLOCK, lo, hi);
    }
  }
  // A group of U 16-byte vectors (2U terms): one test decides whether every
  // term is normal (then the short path), else each term takes the general one.
  template <int BLOCK, int U, bool TRACK = false>
  __device__ __forceinline__ void group(const ulonglong2* v) {
    unsigned e[2 * U];
    unsigned mx = 0u, mn = 0x7FFu;
#pragma unroll
    for (int k = 0; k < U; ++k) {
      e[2 * k] = ((unsigned)(v[k].x >> 32) >> 20) & 0x7FFu;
      e[2 * k + 1] = ((unsigned)(v[k].y >> 32) >> 20) & 0x7FFu;
      mx = max(mx, e[2 * k] - 1u);  // e == 0 wraps to the top: not normal
      mx = max(mx, e[2 * k + 1] - 1u);
      if (TRACK) mn = min(mn, min(e[2 * k], e[2 * k + 1]));
    }
    if (__builtin_expect(mx < 0x7FEu, 1)) {
      notnegz = 1u;
      if (TRACK) {
        emin = min(emin, mn);
        emax = max(emax, mx + 1u);
      }
#pragma unroll
      for (int k = 0; k < U; ++k) {
        sacc_add_normal<BLOCK>(acc, (unsigned)v[k].x, (unsigned)(v[k].x >> 32), e[2 * k]);
        sacc_add_normal<BLOCK>(acc, (unsigned)v[k].y, (unsigned)(v[k].y >> 32), e[2 * k + 1]);
      }
    } else {
#pragma unroll
      for (int k = 0; k < U; ++k) {
        one<BLOCK, TRACK>(v[k].x);
        one<BLOCK, TRACK>(v[k].y);
      }
    }
  }
  // The same group, speculatively. Every term goes through the
  // short path for normal terms straight away; whether all of them were
  // normal is only looked at after the last add, so no add waits for the
  // test. A zero, subnormal, Inf or NaN term (rare) is then taken back
  // exactly -- the short path on the same term with the sign bit flipped adds
  // the two's complement of what it added before -- and given to the general
  // path. Between two carry propagations a chunk so holds at most the adds of
  // the terms seen, as without the detour. Groups padded with -0 (the ragged
  // end of a range) take the test-first form above instead.
  // ZEROS: a zero is taken back in place (below) rather than by the general
  // path. Both are exact; the segmented kernel's compiled loop was 0.9 %
  // faster without it on its usual data (no zeros), so accumulate_range keeps
  // the general path.
  template <int BLOCK, int U, bool TRACK = false, bool ZEROS = true>
  __device__ __forceinline__ void group_spec(const ulonglong2* v) {
    unsigned mx = 0u, mn = 0x7FFu;
#pragma unroll
    for (int k = 0; k < U; ++k) {
      const unsigned h0 = (unsigned)(v[k].x >> 32), h1 = (unsigned)(v[k].y >> 32);
      const unsigned e0 = (h0 >> 20) & 0x7FFu, e1 = (h1 >> 20) & 0x7FFu;
      mx = max(mx, e0 - 1u);  // e == 0 wraps to the top: not normal
      mx = max(mx, e1 - 1u);
      if (TRACK) mn = min(mn, min(e0, e1));
      sacc_add_normal<BLOCK>(acc, (unsigned)v[k].x, h0, e0);
      sacc_add_normal<BLOCK>(acc, (unsigned)v[k].y, h1, e1);
    }
    if (__builtin_expect(mx < 0x7FEu, 1)) {
      notnegz = 1u;
      if (TRACK) {
        emin = min(emin, mn);
        emax = max(emax, mx + 1u);
      }
      return;
    }
#pragma unroll
    for (int k = 0; k < 2 * U; ++k) {
      const unsigned long long b = (k & 1) ? v[k >> 1].y : v[k >> 1].x;
      const unsigned e = ((unsigned)(b >> 32) >> 20) & 0x7FFu;
      if (TRACK) track(b);
      if (e - 1u < 0x7FEu) {
        notnegz = 1u;
        continue;
      }
      notnegz |= (b != kNegZero) ? 1u : 0u;
      if (ZEROS && (b << 1) == 0ull) {
        // a zero: the short path added 2^20 (+0) or -2^20 (-0) to chunk 1;
        // take exactly that back, with no call to the general path
        acc[BLOCK] -= (b >> 63) ? -(1ll << 20) : (1ll << 20);
        continue;
      }
      take_back<BLOCK>(acc, b);
      if (e == 0x7FFu) special(b);
    }
  }
  __device__ __forceinline__ unsigned flags() const {
    return sflags | (notnegz ? kFlagNotNegZero : 0u);
  }
};

// Carry propagation (small-superaccumulator section): from chunk 0 upward,
// move the signed high 32 bits of each chunk into the next; the top chunk
// keeps its own. Afterwards chunks 0..65 lie in [0, 2^32).
__device__ __forceinline__ void sacc_propagate(long long* __restrict__ a, int stride) {
  long long carry = 0;
#pragma unroll 6
  for (int c = 0; c < kSChunks - 1; ++c) {
    (void)XS_DCHECK(a[c * stride] <= kChunkBound && a[c * stride] >= -kChunkBound, kDbgChunkBound);
    const long long v = a[c * stride] + carry;
    a[c * stride] = v & 0xFFFFFFFFll;
    carry = v >> 32;
  }
  a[(kSChunks - 1) * stride] += carry;
}

// Adds x[lo, hi) to the per-thread accumulators of `nthr` cooperating threads
// (rank r among them). The body streams as groups of UNROLL 16-byte vectors
// per thread: full groups load without bounds checks into two register buffers
// used in turn (the next group's loads are in flight while the current one is
// added), the ragged last group is padded with -0. The head before the first
// 256-byte boundary (up to 31 elements, one per rank from rank 0: the body
// then streams from that boundary, which the loads' 256-byte L2 granules and
// the bulk prefetch need for full speed) and one odd tail element (rank
// nthr-1) go apart; nthr >= 32. With PREFETCH, rank 0 prefetches the range
// into L2 a few groups ahead.
template <int BLOCK, int UNROLL, bool PREFETCH, bool TRACK = false>
__device__ __forceinline__ void accumulate_range(SmallThread& T, const double* x, long long lo,
                                                 long long hi, int r, int nthr,
                                                 int carry_groups = 0) {
  const unsigned long long* xb = reinterpret_cast<const unsigned long long*>(x);
  long long p = lo;
  {
    const long long h = min((long long)((256u - ((uintptr_t)(x + p) & 255u)) & 255u) / 8, hi - p);
    if (r < h) T.one<BLOCK, TRACK>(xb[p + r]);
    p += h;
  }
  if (((hi - p) & 1) != 0 && p < hi) {
    if (r == nthr - 1) T.one<BLOCK, TRACK>(xb[hi - 1]);
    --hi;
  }
  const long long npairs = (hi - p) >> 1;
  const ulonglong2* xv = reinterpret_cast<const ulonglong2*>(x + p);
  const long long gsz = (long long)UNROLL * nthr;  // pairs per group
  const long long nfull = npairs / gsz;
  constexpr int kAhead = UNROLL >= 24 ? 1 : 24 / UNROLL;  // groups prefetched ahead (~24 loads per thread)
  auto prefetch = [&](long long g) {
    if (PREFETCH && r == 0 && g < nfull + 1) {
      const long long first = g * gsz;
      if (first < npairs) prefetch_l2(xv + first, (unsigned)(min(gsz, npairs - first) * 16));
    }
  };
  auto load_full = [&](long long g, ulonglong2* buf) {
    const ulonglong2* q = xv + g * gsz + r;
#pragma unroll
    for (int u = 0; u < UNROLL; ++u) buf[u] = ld_stream(q + (long long)u * nthr);
  };
  if (PREFETCH)
    for (int k = 1; k <= kAhead; ++k) prefetch(k);
  // carry_groups > 0: propagate carries after that many groups (ranges longer
  // than 2047 adds per thread); afterwards chunks up to the top may be nonzero,
  // which the window records as kWindowTop
  int since = 0;
  auto tick = [&]() {
    if (carry_groups > 0 && ++since >= carry_groups) {
      sacc_propagate(T.acc, BLOCK);
      if (TRACK) T.emax = kWindowTop;
      since = 0;
    }
  };
  ulonglong2 A[UNROLL], B[UNROLL];
  long long g = 0;
  if (nfull > 0) load_full(0, A);
  while (g < nfull) {
    prefetch(g + kAhead + 1);
    if (g + 1 < nfull) load_full(g + 1, B);
    T.group_spec<BLOCK, UNROLL, TRACK, false>(A);
    tick();
    if (++g >= nfull) break;
    prefetch(g + kAhead + 1);
    if (g + 1 < nfull) load_full(g + 1, A);
    T.group_spec<BLOCK, UNROLL, TRACK, false>(B);
    tick();
    ++g;
  }
  if (nfull * gsz < npairs) {
#pragma unroll
    for (int u = 0; u < UNROLL; ++u) {
      const long long k = nfull * gsz + (long long)u * nthr + r;
      A[u] = k < npairs ? ld_stream(xv + k) : make_ulonglong2(kNegZero, kNegZero);
    }
    T.group<BLOCK, UNROLL, TRACK>(A);  // the -0 padding is not normal: test first
  }
}

__device__ __forceinline__ long long warp_sum_ll(long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}
__device__ __forceinline__ unsigned long long warp_max_ull(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long w = __shfl_xor_sync(kFull, v, o);
    v = w > v ? w : v;
  }
  return v;
}

// Block reduction of the per-thread chunks without a final per-thread carry
// propagation: chunk c of every thread (|c| < 2^63) splits into its low 32 bits
// and its signed high part, and the high part is owed to chunk c+1. Warp w
// handles chunks w, w + BLOCK/32, ..., a batch of up to 6 at a time so their
// shared-memory reads overlap. Each lane first sums its BLOCK/32 threads'
// parts (low < 2^36, high of magnitude < 2^35 for BLOCK <= 512); the warp sums
// then come from 32-bit warp reductions of 16-bit digits of those partials
// (each digit sum stays below 2^25 in magnitude, so the reductions are exact).
// Lane 0 hands the two sums to `emit(chunk, value)`, which adds them into the
// target accumulator (global or shared). Sums stay below 2^41 in magnitude.
// Only chunks c_lo..c_hi are read (the others must be zero in every thread).
// The group form sums the NT consecutive threads whose chunk 0 starts at sm
// (accumulators strided by STRIDE); gwarp is the warp's index in the group.
template <int STRIDE, int NT, typename Emit>
__device__ __forceinline__ void group_chunk_sums(const long long* sm, int gwarp, Emit emit,
                                                 int c_lo = 0, int c_hi = kSChunks - 1) {
  static_assert(NT % 32 == 0 && NT <= 512, "digit sums sized for up to 16 warps");
  const int lane = threadIdx.x & 31, warp = gwarp;
  constexpr int NW = NT / 32;
  constexpr int BLOCK = STRIDE;
  constexpr int BATCH = 6;
  for (int c0 = c_lo + warp; c0 <= c_hi; c0 += BATCH * NW) {
    unsigned long long lo[BATCH];
    long long hi[BATCH];
#pragma unroll
    for (int j = 0; j < BATCH; ++j) {
      const int c = c0 + j * NW;
      lo[j] = 0ull;
      hi[j] = 0;
      if (c <= c_hi) {
#pragma unroll
        for (int k = 0; k < NW; ++k) {
          const long long v = sm[c * BLOCK + k * 32 + lane];
          lo[j] += (unsigned long long)(unsigned)v;
          hi[j] += v >> 32;
        }
      }
    }
#pragma unroll
    for (int j = 0; j < BATCH; ++j) {
      const int c = c0 + j * NW;
      if (c > c_hi) break;
      const unsigned l0 = __reduce_add_sync(kFull, (unsigned)lo[j] & 0xFFFFu);
      const unsigned l1 = __reduce_add_sync(kFull, (unsigned)(lo[j] >> 16));
      const unsigned h0 = __reduce_add_sync(kFull, (unsigned)hi[j] & 0xFFFFu);
      const int h1 = __reduce_add_sync(kFull, (int)(hi[j] >> 16));
      if (lane == 0) {
        const long long L = (long long)l0 + (long long)l1 * 65536ll;
        const long long H = (long long)h0 + (long long)h1 * 65536ll;
        if (c == kSChunks - 1) {
          emit(c, L + H * 4294967296ll);
        } else {
          emit(c, L);
          emit(c + 1, H);
        }
      }
    }
  }
}

template <int BLOCK, typename Emit>
__device__ __forceinline__ void block_chunk_sums(const long long* sm, Emit emit, int c_lo = 0,
                                                 int c_hi = kSChunks - 1) {
  group_chunk_sums<BLOCK, BLOCK>(sm, (int)(threadIdx.x >> 5), emit, c_lo, c_hi);
}

// --------------------------------------------------------------------------
// Warp-level normalisation and rounding of a 67-chunk accumulator.
// Lane L holds chunks L (v0), L+32 (v1) and L+64 (v2, lanes 0..2 only).
// --------------------------------------------------------------------------

// Carry propagation of a warp-spread accumulator. Two parallel rounds move
// every chunk's signed high part one chunk up; after them the remaining
// carries are -1, 0 or +1 and can only ripple through chunks equal to 0 or
// 2^32 - 1 (the typical case is a negative value, whose canonical chunks are
// 2^32 - 1 all the way up). If any carry is left, one lane finishes the
// propagation sequentially through the warp's scratch: chunk k lives at
// sc[(k >> 5) * ss + (k & 31)] (ss = 32: 67 consecutive long longs), so the
// lanes' stores and loads never conflict.
__device__ __noinline__ static void warp_normalize(long long& v0, long long& v1, long long& v2,
                                                   long long* sc, int ss) {
  const int lane = threadIdx.x & 31;
  for (int it = 0; it < 2; ++it) {
    const long long c0 = v0 >> 32;
    const long long c1 = v1 >> 32;
    const long long c2 = (lane < 2) ? (v2 >> 32) : 0;  // chunk 66 keeps its high part
    if (!__any_sync(kFull, (c0 | c1 | c2) != 0)) return;
    v0 &= 0xFFFFFFFFll;
    v1 &= 0xFFFFFFFFll;
    if (lane < 2) v2 &= 0xFFFFFFFFll;
    long long u0 = __shfl_up_sync(kFull, c0, 1);
    long long u1 = __shfl_up_sync(kFull, c1, 1);
    long long u2 = __shfl_up_sync(kFull, c2, 1);
    const long long w0 = __shfl_sync(kFull, c0, 31);
    const long long w1 = __shfl_sync(kFull, c1, 31);
    if (lane == 0) {
      u0 = 0;
      u1 = w0;
      u2 = w1;
    }
    v0 += u0;
    v1 += u1;
    v2 += u2;
  }
  const bool left = ((v0 >> 32) | (v1 >> 32) | ((lane < 2) ? (v2 >> 32) : 0)) != 0;
  if (!__any_sync(kFull, left)) return;
  sc[lane] = v0;
  sc[ss + lane] = v1;
  if (lane < 3) sc[2 * ss + lane] = v2;
  __syncwarp();
  if (lane == 0) {
    long long carry = 0;
    for (int k = 0; k < kSChunks - 1; ++k) {
      long long* p = sc + (k >> 5) * ss + (k & 31);
      const long long x = *p + carry;
      *p = x & 0xFFFFFFFFll;
      carry = x >> 32;
    }
    sc[2 * ss + 2] += carry;
  }
  __syncwarp();
  v0 = sc[lane];
  v1 = sc[ss + lane];
  v2 = lane < 3 ? sc[2 * ss + lane] : 0;
  __syncwarp();
}

__device__ __forceinline__ unsigned lanes_below(int x) {
  return x <= 0 ? 0u : (x >= 32 ? kFull : ((1u << x) - 1u));
}

// Normalise and take the magnitude; returns whether the value is negative.
// The negation of a canonical value is canonical at once: with j its lowest
// nonzero chunk below the top, chunks under j stay 0, chunk j becomes
// 2^32 - c_j, higher chunks 2^32 - 1 - c_k, and the top -c_66 - 1 (or -c_66
// when every lower chunk is 0).
__device__ __forceinline__ bool warp_abs(long long& v0, long long& v1, long long& v2,
                                         long long* sc, int ss) {
  const int lane = threadIdx.x & 31;
  warp_normalize(v0, v1, v2, sc, ss);
  if (__shfl_sync(kFull, v2, 2) >= 0) return false;
  const unsigned b0 = __ballot_sync(kFull, v0 != 0);
  const unsigned b1 = __ballot_sync(kFull, v1 != 0);
  const unsigned b2 = __ballot_sync(kFull, lane < 2 && v2 != 0);
  const int j = b0 ? __ffs(b0) - 1 : (b1 ? 32 + __ffs(b1) - 1 : (b2 ? 64 + __ffs(b2) - 1 : 66));
  auto neg = [&](long long c, int k) -> long long {
    if (k == kSChunks - 1) return j < kSChunks - 1 ? -c - 1 : -c;
    if (k < j) return 0;
    if (k == j) return 4294967296ll - c;
    return 4294967295ll - c;
  };
  v0 = neg(v0, lane);
  v1 = neg(v1, lane + 32);
  if (lane < 3) v2 = neg(v2, lane + 64);
  return true;
}

// Round to nearest, ties to even, the magnitude A * 2^-1075 + (something in
// (0, 2^-1075) when sticky_in), A given as normalised non-negative chunks
// (small section on rounding; overflow as in the Discussion). All 32 lanes
// call it; the result (without sign) is valid in every lane.
__device__ __noinline__ static unsigned long long warp_round_mag(long long v0, long long v1,
                                                                 long long v2, bool sticky_in) {
  const unsigned b0 = __ballot_sync(kFull, v0 != 0);
  const unsigned b1 = __ballot_sync(kFull, v1 != 0);
  const unsigned b2 = __ballot_sync(kFull, v2 != 0);
  if ((b0 | b1 | b2) == 0u) return 0ull;  // below half of 2^-1074: rounds to zero
  const int h = b2 ? 64 + 31 - __clz(b2) : (b1 ? 32 + 31 - __clz(b1) : 31 - __clz(b0));
  auto chunk_at = [&](int k) -> unsigned long long {
    const int slot = k < 0 ? 0 : (k >> 5);
    const long long sv = slot == 0 ? v0 : (slot == 1 ? v1 : v2);
    const long long r = __shfl_sync(kFull, sv, k < 0 ? 0 : (k & 31));
    return k < 0 ? 0ull : (unsigned long long)r;
  };
  const unsigned long long dh = chunk_at(h);
  const unsigned long long dm = chunk_at(h - 1);
  const unsigned long long dl = chunk_at(h - 2);
  const int below = h - 2;
  const bool sticky_low = ((b0 & lanes_below(below)) | (b1 & lanes_below(below - 32)) |
                           (b2 & lanes_below(below - 64))) != 0u;
  const int tb = 63 - __clzll((long long)dh);  // top bit of chunk h
  const int P = 32 * h + tb;                   // top bit of A
  unsigned long long bits;
  if (P < 54) {
    // below 2^-1021: the last kept bit is 2^-1074 (bit 1 of A); the pattern of
    // a subnormal or lowest-binade double is its integer multiple of 2^-1074
    const unsigned long long A = (h >= 1 ? (chunk_at(1) << 32) : 0ull) + chunk_at(0);
    bits = A >> 1;
    if ((A & 1ull) && (sticky_in || (bits & 1ull))) bits += 1ull;
  } else {
    const unsigned __int128 W = ((unsigned __int128)dh << 64) | ((unsigned __int128)dm << 32) |
                                (unsigned __int128)dl;
    unsigned long long q = (unsigned long long)(W >> (tb + 12));  // 53 bits
    const bool rbit = (unsigned)(W >> (tb + 11)) & 1u;
    const unsigned __int128 rest_mask = (((unsigned __int128)1) << (tb + 11)) - 1;
    const bool sticky = sticky_in || sticky_low || ((W & rest_mask) != 0);
    if (rbit && (sticky || (q & 1ull))) q += 1ull;
    const unsigned long long e = (unsigned long long)(P - 52);  // biased exponent
    bits = ((e - 1ull) << 52) + q;  // a carry out of q bumps the exponent
    if (bits >= kPosInf) bits = kPosInf;
  }
  return bits;
}

// Special values first (Inf/NaN record of Fig. 3, readings of the method).
__device__ __forceinline__ bool special_result(unsigned flags, unsigned long long nan_key,
                                               unsigned long long* out) {
  if (nan_key != 0ull) { *out = nan_from_key(nan_key); return true; }
  if ((flags & (kFlagPosInf | kFlagNegInf)) == (kFlagPosInf | kFlagNegInf)) {
    *out = kDefaultNaN;
    return true;
  }
  if (flags & kFlagPosInf) { *out = kPosInf; return true; }
  if (flags & kFlagNegInf) { *out = kNegInf; return true; }
  return false;
}

__device__ __forceinline__ bool warp_is_zero(long long v0, long long v1, long long v2) {
  return !__any_sync(kFull, (v0 | v1 | v2) != 0);
}

__device__ __forceinline__ unsigned long long signed_zero(unsigned flags) {
  return ((flags & kFlagAny) && !(flags & kFlagNotNegZero)) ? kNegZero : 0ull;
}

// Correctly rounded exact sum of a value known on a window of chunks only:
// chunk c0 + k holds w[k] (any signed 64-bit value of magnitude below 2^62),
// k < nw <= NW, every other chunk is zero; the same rounding as warp_round,
// done by one thread (every lane may call it; no shared memory).
//   1. Carry propagation gives 32-bit digits d[0..nw) and a signed top carry.
//   2. A negative value is negated as a digit string (two's complement).
//   3. The top three digits T (96 bits) and an OR of the digits below give the
//      53-bit significand, the round bit and the sticky bit of the magnitude A
//      (in units of 2^-1075; its bit 0 is always zero for sums of doubles, so
//      A / 2 is the value in units of 2^-1074), then ties to even, a carry into
//      the next binade and overflow to Inf as in the small section.
template <int NW>
__device__ __forceinline__ unsigned long long round_window(const long long (&w)[NW], int nw, int c0,
                                                           unsigned flags,
                                                           unsigned long long nan_key) {
  unsigned long long sp;
  if (special_result(flags, nan_key, &sp)) return sp;
  unsigned d[NW + 1];
  long long carry = 0;
#pragma unroll
  for (int k = 0; k < NW; ++k) {
    const long long x = (k < nw ? w[k] : 0) + carry;
    d[k] = (unsigned)x;
    carry = x >> 32;  // arithmetic: floor division by 2^32
  }
  const bool neg = carry < 0;
  if (neg) {  // -(D + carry 2^(32 NW)) = ~D + 1 + (-carry - 1) 2^(32 NW)
    unsigned long long c = 1;
#pragma unroll
    for (int k = 0; k < NW; ++k) {
      const unsigned long long x = (unsigned long long)(unsigned)~d[k] + c;
      d[k] = (unsigned)x;
      c = x >> 32;
    }
    carry = -carry - 1 + (long long)c;
  }
  d[NW] = (unsigned)carry;  // 0 <= carry < 2^32 for sums of finite doubles
  int m = -1;  // the top nonzero digit
#pragma unroll
  for (int k = 0; k <= NW; ++k)
    if (d[k] != 0u) m = k;
  if (m < 0) return signed_zero(flags);
  const unsigned long long sign = neg ? kNegZero : 0ull;
  const unsigned t2 = d[m];
  unsigned t1 = 0u, t0 = 0u;
  bool low = false;
#pragma unroll
  for (int k = 0; k <= NW; ++k) {
    if (k == m - 1) t1 = d[k];
    if (k == m - 2) t0 = d[k];
    if (k < m - 2 && d[k] != 0u) low = true;
  }
  // A = T 2^(32 (c0 + m - 2)) + (lower digits), T = t2:t1:t0
  const int top = 95 - __clz((int)t2);  // index of the top bit within T (t2 != 0)
  const int base = 32 * (c0 + m - 2);   // weight exponent of T's bit 0 (may be negative)
  const int P = base + top - 1;         // top bit of A / 2
  if (P < 53) {
    // A / 2 < 2^53: exactly representable, its bits are the value (subnormals
    // and the lowest normal binade). With t2 != 0, T >= 2^64, so this needs
    // base <= -32: the top digit is chunk 1 (A = t2:t1) or chunk 0 (A = t2).
    const unsigned long long A = base == -32 ? (((unsigned long long)t2 << 32) | t1)
                                             : (unsigned long long)t2;
    return (A >> 1) | sign;
  }
  // 53 bits from A's top bit down: bits [top - 52, top] of T (top >= 64 since t2 != 0)
  const int lsb = top - 52;  // >= 12
  const unsigned long long hi64 = ((unsigned long long)t2 << 32) | t1;
  // T = hi64 * 2^32 + t0; q = T >> lsb; rest = T mod 2^lsb; half = 2^(lsb - 1)
  const unsigned long long q0 = lsb >= 32 ? hi64 >> (lsb - 32)
                                          : (hi64 << (32 - lsb)) | ((unsigned long long)t0 >> lsb);
  unsigned long long q = q0 & ((1ull << 53) - 1ull);
  // rest and half, compared as (rest > half) / (rest == half); rest < 2^lsb <= 2^43
  unsigned long long rest;
  if (lsb >= 32) {
    rest = ((hi64 & ((1ull << (lsb - 32)) - 1ull)) << 32) | t0;
  } else {
    rest = (unsigned long long)t0 & ((1ull << lsb) - 1ull);
  }
  const unsigned long long half = 1ull << (lsb - 1);
  const bool up = rest > half || (rest == half && (low || (q & 1ull)));
  int sh = P - 52;  // bits of A / 2 below q
  q += up ? 1ull : 0ull;
  if (q == (1ull << 53)) {
    q >>= 1;
    ++sh;
  }
  const int e = sh + 1;
  if (e >= 2047) return kPosInf | sign;
  return ((unsigned long long)(e - 1) << 52) + q + sign;
}

// Correctly rounded exact sum (ties to even) of an accumulator whose chunks
// are spread over the warp as above.
__device__ __noinline__ static unsigned long long warp_round(long long v0, long long v1,
                                                             long long v2, unsigned flags,
                                                             unsigned long long nan_key,
                                                             long long* sc, int ss) {
  unsigned long long sp;
  if (special_result(flags, nan_key, &sp)) return sp;
  const bool neg = warp_abs(v0, v1, v2, sc, ss);
  if (warp_is_zero(v0, v1, v2)) return signed_zero(flags);
  return warp_round_mag(v0, v1, v2, false) | (neg ? kNegZero : 0ull);
}

// Long division of the normalised magnitude by d >= 1, from its top nonzero
// chunk down; every lane runs the same recurrence. Each step divides
// cur = rem * 2^32 + chunk (rem < d) by d: a double-precision estimate of the
// quotient is within one of the truth, and exact integer corrections fix it.
// Returns whether the remainder is nonzero.
__device__ __noinline__ static bool warp_divide(long long& v0, long long& v1, long long& v2,
                                                unsigned long long d) {
  const int lane = threadIdx.x & 31;
  const unsigned b0 = __ballot_sync(kFull, v0 != 0);
  const unsigned b1 = __ballot_sync(kFull, v1 != 0);
  const unsigned b2 = __ballot_sync(kFull, v2 != 0);
  if ((b0 | b1 | b2) == 0u) return false;
  const int h = b2 ? 64 + 31 - __clz(b2) : (b1 ? 32 + 31 - __clz(b1) : 31 - __clz(b0));
  unsigned long long rem = 0ull;
  if (d <= 0xFFFFFFFFull) {
    // Only the top four chunks T are divided: with A = T * 2^K + L (L < 2^K)
    // and T = Q d + R, A / d = Q 2^K + F where 0 <= F < 2^K and F > 0 exactly
    // when R or L is nonzero; T >= 2^96 and d < 2^32 give Q more than 64
    // bits, so Q and that sticky bit decide the rounding. (Below four chunks
    // every chunk is divided and nothing is dropped.)
    const int kmin = h >= 3 ? h - 3 : 0;
    const bool low_nonzero =
        ((b0 & lanes_below(kmin)) | (b1 & lanes_below(kmin - 32)) | (b2 & lanes_below(kmin - 64))) != 0u;
    // cur = rem * 2^32 + chunk < 2^64 (for the top chunk, chunk < 2^34 and
    // rem = 0); q from the integer reciprocal m = floor((2^64 - 1) / d) is at
    // most two below the truth
    const unsigned long long m = 0xFFFFFFFFFFFFFFFFull / d;
    for (int k = h; k >= kmin; --k) {
      const int slot = k >> 5;
      const long long sv = slot == 0 ? v0 : (slot == 1 ? v1 : v2);
      const unsigned long long limb = (unsigned long long)__shfl_sync(kFull, sv, k & 31);
      const unsigned long long cur = (rem << 32) + limb;
      unsigned long long q = __umul64hi(cur, m);
      unsigned long long r = cur - q * d;
      for (int fix = 0; fix < 4 && r >= d; ++fix) { ++q; r -= d; }
      rem = r;
      if ((k & 31) == lane) {
        if (slot == 0) v0 = (long long)q;
        else if (slot == 1) v1 = (long long)q;
        else v2 = (long long)q;
      }
    }
    if (lane < kmin) v0 = 0;
    if (lane + 32 < kmin) v1 = 0;
    if (lane + 64 < kmin) v2 = 0;
    return rem != 0ull || low_nonzero;
  }
  const double inv = 1.0 / (double)d;
  for (int k = h; k >= 0; --k) {
    const int slot = k >> 5;
    const long long sv = slot == 0 ? v0 : (slot == 1 ? v1 : v2);
    const unsigned long long limb = (unsigned long long)__shfl_sync(kFull, sv, k & 31);
    const double est = __fma_rn((double)rem, 4294967296.0, (double)limb) * inv;
    unsigned long long q = est > 0.0 ? (unsigned long long)est : 0ull;
    __int128 r = (((__int128)rem) << 32) + (__int128)limb - (__int128)q * (__int128)d;
    for (int fix = 0; fix < 4 && r < 0; ++fix) { --q; r += d; }
    for (int fix = 0; fix < 4 && r >= (__int128)d; ++fix) { ++q; r -= d; }
    rem = (unsigned long long)r;
    if ((k & 31) == lane) {
      if (slot == 0) v0 = (long long)q;
      else if (slot == 1) v1 = (long long)q;
      else v2 = (long long)q;
    }
  }
  return rem != 0ull;
}

// Correctly rounded quotient (exact sum) / d, ties to even -- the exact mean
// when d is the number of terms (Discussion: rounding the superaccumulator
// divided by a positive integer directly). The quotient of a finite sum never
// exceeds the largest term in magnitude, so it cannot overflow.
__device__ __noinline__ static unsigned long long warp_round_div(long long v0, long long v1,
                                                                 long long v2, unsigned flags,
                                                                 unsigned long long nan_key,
                                                                 unsigned long long d,
                                                                 long long* sc, int ss) {
  unsigned long long sp;
  if (special_result(flags, nan_key, &sp)) return sp;
  const bool neg = warp_abs(v0, v1, v2, sc, ss);
  if (warp_is_zero(v0, v1, v2)) return signed_zero(flags);
  const bool sticky = warp_divide(v0, v1, v2, d);
  return warp_round_mag(v0, v1, v2, sticky) | (neg ? kNegZero : 0ull);
}

// --------------------------------------------------------------------------
// Large superaccumulator in shared memory, one per block (Fig. 4), in the
// form that suits the GPU's shared-memory atomics.
//
// As in the paper there is one chunk per sign+exponent index ix = bits >> 52
// (4096 of them), every term costs one indexed add into its chunk, and the
// chunks are transferred into the small superaccumulator at the end. What
// differs: a chunk is a 96-bit unsigned integer held in three planes of 32-bit
// words (lo, hi, top), and a term adds its 53-bit significand M -- the
// implicit bit included -- instead of its raw bits. The low word is added with
// an atomic that returns the old value, so the carry out of it is known and
// goes into the high word with the rest of M; a carry out of the high word
// (after at least 2^11 adds to one chunk) adds one to the top word. Nothing
// ever needs a transfer before the end, so the paper's per-chunk count of the
// adds left (which bounded a 64-bit chunk to 4096 raw-bit adds) and its
// special path for the 4096th add are not needed. (A 64-bit shared atomic
// add costs about three times two 32-bit ones on this GPU, measured.)
//
// Terms with e == 0 (zeros and subnormals) also add the implicit bit 2^52;
// each thread counts them by sign and the flush subtracts the count from
// chunks 0x000 and 0x800. Inf and NaN terms (e == 2047) land in chunks 0x7FF
// and 0xFFF, which the flush ignores; their record (Fig. 3's Inf and NaN
// fields) is kept in registers like the small kernel's.
// --------------------------------------------------------------------------

// Shared-memory layout: R copies of the lo and hi planes (lane L adds into
// copy L mod R, so R times fewer lanes of a warp meet on one address when few
// distinct exponents occur; copy r starts r * kCopyWords words in, which puts
// the copies of one chunk in different banks: shifts of 8 banks for up to 4
// copies, of 5 for up to 6), one top plane for all copies, and the per-warp
// transfer targets of the flush. A chunk's value is the sum over the copies
// of hi:lo, plus top * 2^64.
template <int NWARPS, int R>
struct LargePlanes {
  static_assert(R >= 1 && R <= 6, "copies of the planes");
  static constexpr int kCopyWords = 2 * kLChunks + (R <= 4 ? 8 : 5);
  static constexpr int kCopiesPadded = (R * kCopyWords + 3) / 4 * 4;  // keeps `top` 16-byte aligned
  unsigned copies[kCopiesPadded];
  unsigned top[kLChunks];
  long long part[NWARPS][kSChunks];
  unsigned zeros[2];  // zero/subnormal terms of the block, by sign
};

// 32-bit shared-memory atomics on 32-bit shared addresses (volatile: they are
// neither dropped nor reordered among themselves; the planes are read with
// plain loads only after a barrier).
__device__ __forceinline__ unsigned atom_add_shared(unsigned saddr, unsigned v) {
  unsigned old;
  asm volatile("atom.shared.add.u32 %0, [%1], %2;" : "=r"(old) : "r"(saddr), "r"(v));
  return old;
}
__device__ __forceinline__ void red_add_shared(unsigned saddr, unsigned v) {
  asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(saddr), "r"(v));
}

// Shared addresses of one lane's view of the planes.
struct LargeLane {
  unsigned lo;   // lo plane of the lane's copy (hi follows at + 4 kLChunks bytes)
  unsigned top;  // the common top plane
};

// Adds S < 2^64 to chunk ix: the low word with an atomic that returns the old
// value, the high word with the carry out of it, and a carry out of the high
// word into the top plane.
__device__ __forceinline__ void large_add64(const LargeLane& L, unsigned ix, unsigned long long S) {
  if (!XS_DCHECK(ix < (unsigned)kLChunks, kDbgLargeIndex)) return;
  const unsigned l = (unsigned)S;
  const unsigned old = atom_add_shared(L.lo + (ix << 2), l);
  unsigned sum, hi;
  asm("add.cc.u32 %0, %2, %3;\n\taddc.u32 %1, %4, 0;"
      : "=r"(sum), "=r"(hi)
      : "r"(old), "r"(l), "r"((unsigned)(S >> 32)));
  (void)sum;
  const unsigned old2 = atom_add_shared(L.lo + (ix << 2) + 4u * kLChunks, hi);
  if (old2 + hi < hi) red_add_shared(L.top + (ix << 2), 1u);
}

// Adds of one group of 2U terms (U 16-byte vectors). The low words of all
// terms go first, so their atomics' returns are in flight together; then the
// high words with the carries. When all 2U terms of every lane of the warp
// are normal and share one exponent (a constant array, or values of one
// binade with either sign), each lane instead adds the net of its terms'
// signed significands, |S| < 2U 2^53, once: into the positive chunk of that
// exponent if S > 0, into the negative one if S < 0. Both chunks carry the
// same weight with opposite signs and only their difference is ever used, so
// the net leaves the sum unchanged, and lanes that meet on one word meet 2U
// times less often; when every lane has the same exponent, the warp adds the
// sum of the nets once. The test costs one logic op per term. Returns the maximum
// over the terms of ((e - 1) mod 2048) << 20, which reaches 0x7FE00000
// exactly when some term has e == 0 or e == 2047 (the rare path).
template <int U>
__device__ __forceinline__ unsigned large_group_add(const LargeLane& L, const ulonglong2* v) {
  unsigned ix[2 * U];
  unsigned mx = 0u, dx = 0u;
  const unsigned h0 = (unsigned)(v[0].x >> 32);
#pragma unroll
  for (int k = 0; k < 2 * U; ++k) {
    const unsigned h = (unsigned)(((k & 1) ? v[k >> 1].y : v[k >> 1].x) >> 32);
    ix[k] = h >> 20;
    if (!XS_DCHECK(ix[k] < (unsigned)kLChunks, kDbgLargeIndex)) ix[k] &= kLChunks - 1;
    mx = max(mx, (h - 0x00100000u) & 0x7FF00000u);
    dx |= h ^ h0;
  }
  if (__all_sync(kFull, ((dx & 0x7FF00000u) | (mx >= 0x7FE00000u ? 1u : 0u)) == 0u)) {
    long long S = 0;
#pragma unroll
    for (int k = 0; k < 2 * U; ++k) {
      const unsigned long long b = (k & 1) ? v[k >> 1].y : v[k >> 1].x;
      const long long M = (long long)((b & kMantMask) | (1ull << 52));
      const long long sg = (long long)b >> 63;  // 0 or -1
      S += (M ^ sg) - sg;
    }
    const unsigned e0 = ix[0] & 0x7FFu;
    if (__all_sync(kFull, __shfl_sync(kFull, e0, 0) == e0)) {
      // the whole warp on one exponent (a constant array): one add per warp,
      // |sum| < 32 2U 2^53 <= 2^61
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) S += __shfl_xor_sync(kFull, S, o);
      if ((threadIdx.x & 31) == 0 && S != 0)
        large_add64(L, e0 | (S < 0 ? 0x800u : 0u), (unsigned long long)(S < 0 ? -S : S));
      return mx;
    }
    if (S != 0) large_add64(L, e0 | (S < 0 ? 0x800u : 0u), (unsigned long long)(S < 0 ? -S : S));
    return mx;
  }
  unsigned v2[2 * U];
#pragma unroll
  for (int k = 0; k < 2 * U; ++k) {
    const unsigned long long b = (k & 1) ? v[k >> 1].y : v[k >> 1].x;
    const unsigned h = (unsigned)(b >> 32), l = (unsigned)b;
    const unsigned old = atom_add_shared(L.lo + (ix[k] << 2), l);
    unsigned sum, hi;
    asm("add.cc.u32 %0, %2, %3;\n\taddc.u32 %1, %4, 0;"
        : "=r"(sum), "=r"(hi)
        : "r"(old), "r"(l), "r"((h & 0xFFFFFu) | 0x100000u));
    v2[k] = hi;  // (M >> 32) + the carry out of the low word
  }
#pragma unroll
  for (int k = 0; k < 2 * U; ++k) {
    const unsigned old = atom_add_shared(L.lo + (ix[k] << 2) + 4u * kLChunks, v2[k]);
    if (old + v2[k] < v2[k]) red_add_shared(L.top + (ix[k] << 2), 1u);
  }
  return mx;
}

// One term (the unaligned head, the odd tail, the ragged last tile).
__device__ __forceinline__ void large_one_add(const LargeLane& L, unsigned long long b) {
  large_add64(L, (unsigned)(b >> 52), (b & kMantMask) | (1ull << 52));
}

// Adds x[lo, hi) into the block's large superaccumulator, all BLOCK threads
// of the block together (rank tid): the elements before the first 256-byte
// boundary by threads 0..30 (one each), an odd last one by thread BLOCK - 1,
// the body, from that boundary, as groups of UNROLL 16-byte
// vectors per thread in two register buffers used in turn (the next group's
// loads are in flight while the current one is added, and the groups after it
// stream into L2), the ragged end term by term. Every thread of the block
// must call it with the same range.
template <int BLOCK, int UNROLL, class Thread>
__device__ __forceinline__ void large_range(const LargeLane& L, Thread& T, const double* x,
                                            long long lo, long long hi, int tid) {
  const unsigned long long* xb = reinterpret_cast<const unsigned long long*>(x);
  long long p = lo;
  {
    const long long h = min((long long)((256u - ((uintptr_t)(xb + p) & 255u)) & 255u) / 8, hi - p);
    if (tid < h) {
      large_one_add(L, xb[p + tid]);
      T.term(xb[p + tid]);
    }
    p += h;
  }
  if (((hi - p) & 1) != 0 && tid == BLOCK - 1) {
    large_one_add(L, xb[hi - 1]);
    T.term(xb[hi - 1]);
  }
  const long long npairs = (hi - p) >> 1;
  const ulonglong2* xv = reinterpret_cast<const ulonglong2*>(xb + p);
  constexpr long long GP = (long long)BLOCK * UNROLL;  // pairs per group
  const long long ng = npairs / GP;
  ulonglong2 A[UNROLL], B[UNROLL];
  auto load = [&](ulonglong2* buf, long long g) {
    const ulonglong2* q = xv + g * GP + tid;
#pragma unroll
    for (int u = 0; u < UNROLL; ++u) buf[u] = ld_stream(q + u * BLOCK);
  };
  // one thread keeps the L2 bulk prefetch kPF groups ahead of the loads (the
  // first groups are the caller's to prefetch)
  constexpr long long kPF = 3;
  auto prefetch = [&](long long gp) {
    if (tid == 0 && gp < ng) prefetch_l2(xv + gp * GP, (unsigned)(GP * 16));
  };
  long long g = 0;
  if (ng > 0) load(A, 0);
  while (g < ng) {
    prefetch(g + kPF);
    if (g + 1 < ng) load(B, g + 1);
    T.template group_record<UNROLL>(large_group_add<UNROLL>(L, A), A);
    ++g;
    if (g >= ng) break;
    prefetch(g + kPF);
    if (g + 1 < ng) load(A, g + 1);
    T.template group_record<UNROLL>(large_group_add<UNROLL>(L, B), B);
    ++g;
  }
  for (long long q = ng * GP + tid; q < npairs; q += BLOCK) {
    const ulonglong2 v = ld_stream(xv + q);
    large_one_add(L, v.x);
    large_one_add(L, v.y);
    T.term(v.x);
    T.term(v.y);
  }
}

// Per-thread record of the large method: Inf/NaN and the sign of a zero as in
// SmallThread, plus the zero/subnormal counts by sign.
struct LargeThread {
  unsigned notnegz = 0u;
  unsigned sflags = 0u;
  unsigned long long nkey = 0ull;
  unsigned zpos = 0u, zneg = 0u;

  __device__ __forceinline__ void term(unsigned long long b) {
    const unsigned e = (unsigned)(b >> 52) & 0x7FFu;
    if (e == 0u) {
      if (b >> 63) ++zneg; else ++zpos;
      notnegz |= (b != kNegZero) ? 1u : 0u;
    } else if (e == 0x7FFu) {
      notnegz = 1u;
      if (b & kMantMask) {
        const unsigned long long k = nan_key_of(b);
        nkey = k > nkey ? k : nkey;
      } else {
        sflags |= (b >> 63) ? kFlagNegInf : kFlagPosInf;
      }
    } else {
      notnegz = 1u;
    }
  }
  // after large_group_add: the common case is one compare
  template <int U>
  __device__ __forceinline__ void group_record(unsigned mx, const ulonglong2* v) {
    if (__builtin_expect(mx < 0x7FE00000u, 1)) {
      notnegz = 1u;
      return;
    }
#pragma unroll
    for (int k = 0; k < 2 * U; ++k) term((k & 1) ? v[k >> 1].y : v[k >> 1].x);
  }
  __device__ __forceinline__ unsigned flags() const {
    return sflags | (notnegz ? kFlagNotNegZero : 0u);
  }
};

template <int NWARPS, int R>
__device__ __forceinline__ void large_init(LargePlanes<NWARPS, R>& P, int tid, int nthreads) {
  // copies (padded to whole 16-byte vectors) and top are contiguous and 16-byte aligned
  constexpr int W4 = (LargePlanes<NWARPS, R>::kCopiesPadded + kLChunks) / 4;
  using Planes = LargePlanes<NWARPS, R>;
  static_assert(offsetof(Planes, top) == 4 * Planes::kCopiesPadded, "planes are contiguous");
  uint4* w = reinterpret_cast<uint4*>(P.copies);
  for (int k = tid; k < W4; k += nthreads) w[k] = make_uint4(0u, 0u, 0u, 0u);
  long long* pp = &P.part[0][0];
  for (int k = tid; k < NWARPS * kSChunks; k += nthreads) pp[k] = 0;
  if (tid < 2) P.zeros[tid] = 0u;
}

template <int NWARPS, int R>
__device__ __forceinline__ LargeLane large_lane(LargePlanes<NWARPS, R>& P) {
  const unsigned b = (unsigned)__cvta_generic_to_shared(P.copies);
  LargeLane L;
  L.lo = b + 4u * (unsigned)(((threadIdx.x & 31) % R) * LargePlanes<NWARPS, R>::kCopyWords);
  L.top = (unsigned)__cvta_generic_to_shared(P.top);
  return L;
}

// Final transfer of every chunk into the small superaccumulator (large
// section; the paper walks the used chunks, here each warp checks 32 chunks at
// once and skips them when all are zero). Warp w takes the aligned runs of 32
// indices k = w, w + NWARPS, ...: the 32 chunks of a run share the sign and
// the small chunk i = max(e, 1) >> 5, so their values (the sum of M over the
// chunk's terms, shifted left by max(e, 1) & 31: below 2^127) split into four
// 32-bit pieces for small chunks i..i+3 whose warp sums are formed with 32-bit
// reductions of 16-bit digits (below 2^21 each, exact) and added, signed, into
// the warp's own row of `part`. Needs a barrier before (all adds done, zero
// counts in P.zeros). With CLEAR, the words of every run that held anything
// are zeroed as they are read, so the planes are ready for the next sum
// (the part rows and the zero counts are the caller's to clear).
template <int NWARPS, int R, bool CLEAR = false>
__device__ __forceinline__ void large_flush(LargePlanes<NWARPS, R>& P) {
  constexpr int CW = LargePlanes<NWARPS, R>::kCopyWords;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int run = warp; run < kLChunks / 32; run += NWARPS) {
    const unsigned ix = (unsigned)run * 32u + (unsigned)lane;
    const unsigned e = ix & 0x7FFu;
    unsigned __int128 V = (unsigned __int128)P.top[ix] << 64;
#pragma unroll
    for (int r = 0; r < R; ++r)
      V += ((unsigned __int128)P.copies[r * CW + kLChunks + ix] << 32) | P.copies[r * CW + ix];
    if (CLEAR && __any_sync(kFull, V != 0)) {  // raw words: a run no term reached is all zero
      P.top[ix] = 0u;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        P.copies[r * CW + ix] = 0u;
        P.copies[r * CW + kLChunks + ix] = 0u;
      }
    }
    if (e == 0x7FFu) V = 0;  // Inf / NaN record only
    if (e == 0u) V -= (unsigned __int128)P.zeros[ix >> 11] << 52;  // their implicit bits
    if (!__any_sync(kFull, V != 0)) continue;
    const unsigned ee = e ? e : 1u;
    V <<= (ee & 31u);
    const int i = (int)(ee >> kLowExpBits);  // the same for the whole run
    if (!XS_DCHECK(i + 3 < kSChunks, kDbgFlushIndex)) continue;  // uniform over the warp
    const bool neg = (ix >> 11) != 0u;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const unsigned p = (unsigned)(V >> (32 * j));
      const unsigned s0 = __reduce_add_sync(kFull, p & 0xFFFFu);
      const unsigned s1 = __reduce_add_sync(kFull, p >> 16);
      if (lane == 0) {
        const long long S = (long long)s0 + ((long long)s1 << 16);
        P.part[warp][i + j] += neg ? -S : S;
      }
    }
  }
}

}  // namespace xs
