// Exact sum of binary32 (float) values, rounded once to the nearest float,
// ties to even. The paper notes that single-precision values can be summed
// exactly even more easily, with smaller superaccumulators (Introduction);
// this is that variant of the small superaccumulator.
//
// A finite float is M * 2^(e_eff - 150) (M = 24-bit significand, e_eff =
// max(e, 1)). Chunk i (i = e_eff >> 5, 0..7) weighs 2^(32 i - 150); a term
// adds the single value M << (e_eff & 31) < 2^55 to its chunk, so each term is
// one 64-bit read-modify-write and 255 adds fit between carry propagations.
// Positive and negative terms go to separate unsigned chunk sets: the slot
// index bits >> 28 is exactly (sign, i), so the hot path needs no negation.
// Carries out of chunk 7 collect in two per-thread registers (weight 2^106).
// The grid accumulator has eleven signed chunks, enough for any sum of up to
// 2^39 floats (the entry point's limit).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "xs_host.hpp"
#include "xs_kernels.cuh"

namespace xs {

constexpr int kF32Chunks = 11;
constexpr int kF32CarryInterval = 255;  // adds of < 2^55 between propagations
constexpr unsigned kF32PosInf = 0x7F800000u;
constexpr unsigned kF32NegInf = 0xFF800000u;
constexpr unsigned kF32DefaultNaN = 0x7FC00000u;
constexpr unsigned kF32NegZero = 0x80000000u;

struct __align__(16) AccState32 {
  long long chunk[kF32Chunks + 1];  // one spare to keep 16-byte size multiples
  unsigned flags;
  unsigned ticket;
  unsigned long long nan_key;
};

// NaN choice as for doubles: largest 22-bit payload, positive sign on ties.
__device__ __forceinline__ unsigned long long nan32_key(unsigned b) {
  return ((((unsigned long long)(b & 0x3FFFFFu)) << 1) | ((b >> 31) ^ 1u)) + 1ull;
}
__device__ __forceinline__ unsigned nan32_from_key(unsigned long long k) {
  k -= 1ull;
  return ((k & 1ull) ? 0u : kF32NegZero) | 0x7FC00000u | (unsigned)(k >> 1);
}

struct SmallThread32 {
  long long* acc;  // 16 slots (positive chunks 0..7, negative chunks 0..7), stride BLOCK
  unsigned long long top_pos = 0ull, top_neg = 0ull;  // carries out of chunk 7
  unsigned notnegz = 0u, sflags = 0u;
  unsigned long long nkey = 0ull;

  template <int BLOCK>
  __device__ __forceinline__ void add_finite(unsigned b) {
    const unsigned e = (b >> 23) & 0xFFu;
    const unsigned ee = e ? e : 1u;
    const unsigned M = (b & 0x7FFFFFu) | (e ? 0x800000u : 0u);
    const unsigned long long v = (unsigned long long)M << (ee & 31u);
    unsigned long long* c = reinterpret_cast<unsigned long long*>(acc) +
                            (int)(((b >> 31) << 3) | (ee >> 5)) * BLOCK;
    *c += v;
  }
  template <int BLOCK>
  __device__ __forceinline__ void one(unsigned b) {
    notnegz |= (b != kF32NegZero) ? 1u : 0u;
    if (((b >> 23) & 0xFFu) == 0xFFu) {
      if (b & 0x7FFFFFu) {
        const unsigned long long k = nan32_key(b);
        nkey = k > nkey ? k : nkey;
      } else {
        sflags |= (b >> 31) ? kFlagNegInf : kFlagPosInf;
      }
    } else {
      add_finite<BLOCK>(b);
    }
  }
  // Normal terms only (1 <= e <= 254): slot = bits >> 28, 2^l from a
  // wrap-mode funnel shift of bits >> 23.
  template <int BLOCK>
  __device__ __forceinline__ void add_normal(unsigned b) {
    const unsigned pw = __funnelshift_l(0u, 1u, b >> 23);  // 2^(e & 31)
    const unsigned M = (b & 0x7FFFFFu) | 0x800000u;
    unsigned long long* c = reinterpret_cast<unsigned long long*>(acc) + (int)(b >> 28) * BLOCK;
    *c += (unsigned long long)M * pw;
  }
  template <int BLOCK, int U>
  __device__ __forceinline__ void group(const uint4* v) {
    unsigned mx = 0u;
#pragma unroll
    for (int k = 0; k < U; ++k) {
      mx = max(mx, ((v[k].x >> 23) & 0xFFu) - 1u);
      mx = max(mx, ((v[k].y >> 23) & 0xFFu) - 1u);
      mx = max(mx, ((v[k].z >> 23) & 0xFFu) - 1u);
      mx = max(mx, ((v[k].w >> 23) & 0xFFu) - 1u);
    }
    if (__builtin_expect(mx < 0xFEu, 1)) {
      notnegz = 1u;
#pragma unroll
      for (int k = 0; k < U; ++k) {
        add_normal<BLOCK>(v[k].x);
        add_normal<BLOCK>(v[k].y);
        add_normal<BLOCK>(v[k].z);
        add_normal<BLOCK>(v[k].w);
      }
    } else {
#pragma unroll
      for (int k = 0; k < U; ++k) {
        rare<BLOCK>(v[k].x);
        rare<BLOCK>(v[k].y);
        rare<BLOCK>(v[k].z);
        rare<BLOCK>(v[k].w);
      }
    }
  }
  // A term of a group that holds a zero, subnormal, Inf or NaN: normal terms
  // take the short path, zeros add nothing, the rest the general one.
  template <int BLOCK>
  __device__ __forceinline__ void rare(unsigned b) {
    if (((b >> 23) & 0xFFu) - 1u < 0xFEu) {
      notnegz = 1u;
      add_normal<BLOCK>(b);
    } else if ((b << 1) == 0u) {
      notnegz |= (b != kF32NegZero) ? 1u : 0u;
    } else {
      one<BLOCK>(b);
    }
  }
  // Unsigned carry propagation of both chunk sets (small section), the carry
  // out of chunk 7 into the top registers.
  template <int BLOCK>
  __device__ __forceinline__ void propagate() {
    unsigned long long* a = reinterpret_cast<unsigned long long*>(acc);
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      unsigned long long carry = 0ull;
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const unsigned long long x = a[(s * 8 + c) * BLOCK] + carry;
        a[(s * 8 + c) * BLOCK] = x & 0xFFFFFFFFull;
        carry = x >> 32;
      }
      if (s == 0) top_pos += carry; else top_neg += carry;
    }
  }
  __device__ __forceinline__ unsigned flags() const {
    return sflags | (notnegz ? kFlagNotNegZero : 0u);
  }
};

// One warp, chunk c in lane c (c < 11): carry propagation until canonical.
__device__ __forceinline__ void warp_normalize32(long long& v) {
  const int lane = threadIdx.x & 31;
  for (int it = 0; it < 24; ++it) {
    const long long c = (lane < kF32Chunks - 1) ? (v >> 32) : 0;
    if (!__any_sync(kFull, c != 0)) break;
    if (lane < kF32Chunks - 1) v &= 0xFFFFFFFFll;
    long long in = __shfl_up_sync(kFull, c, 1);
    if (lane == 0) in = 0;
    if (lane < kF32Chunks) v += in;
  }
}

// Correctly rounded float (ties to even) of the accumulator in lanes 0..10.
__device__ __noinline__ static unsigned warp_round32(long long v, unsigned flags,
                                                     unsigned long long nan_key) {
  if (nan_key) return nan32_from_key(nan_key);
  if ((flags & (kFlagPosInf | kFlagNegInf)) == (kFlagPosInf | kFlagNegInf)) return kF32DefaultNaN;
  if (flags & kFlagPosInf) return kF32PosInf;
  if (flags & kFlagNegInf) return kF32NegInf;
  const int lane = threadIdx.x & 31;
  warp_normalize32(v);
  const bool neg = __shfl_sync(kFull, v, kF32Chunks - 1) < 0;
  if (neg) {
    v = -v;
    warp_normalize32(v);
  }
  const unsigned nz = __ballot_sync(kFull, v != 0);
  if (nz == 0u) return ((flags & kFlagAny) && !(flags & kFlagNotNegZero)) ? kF32NegZero : 0u;
  const int h = 31 - __clz(nz);
  const unsigned long long dh = (unsigned long long)__shfl_sync(kFull, v, h);
  const unsigned long long dm = h >= 1 ? (unsigned long long)__shfl_sync(kFull, v, h - 1) : 0ull;
  const unsigned long long dl = h >= 2 ? (unsigned long long)__shfl_sync(kFull, v, h - 2) : 0ull;
  (void)lane;
  const bool sticky_low = (nz & ((h - 2) > 0 ? ((1u << (h - 2)) - 1u) : 0u)) != 0u;
  const int tb = 63 - __clzll((long long)dh);
  const int P = 32 * h + tb;  // top bit, units 2^-150
  unsigned bits;
  if (P < 25) {  // below 2^-125: exact, the pattern is the multiple of 2^-149
    const unsigned long long A = (h >= 1 ? (dm + (dh << 32)) : dh);
    bits = (unsigned)(A >> 1);
  } else {
    const unsigned __int128 W = ((unsigned __int128)dh << 64) | ((unsigned __int128)dm << 32) |
                                (unsigned __int128)dl;
    // keep 24 bits [P-23, P]; in W the top bit sits at tb + 64
    const int sh = tb + 64 - 23;
    unsigned q = (unsigned)(W >> sh);
    const bool rbit = (unsigned)(W >> (sh - 1)) & 1u;
    const unsigned __int128 rest = (((unsigned __int128)1) << (sh - 1)) - 1;
    const bool sticky = sticky_low || ((W & rest) != 0);
    if (rbit && (sticky || (q & 1u))) q += 1u;
    const unsigned e = (unsigned)(P - 23);  // biased exponent
    const unsigned long long b = ((unsigned long long)(e - 1u) << 23) + q;
    bits = b >= kF32PosInf ? kF32PosInf : (unsigned)b;
  }
  return bits | (neg ? kF32NegZero : 0u);
}

struct F32Args {
  const float* x;
  long long n;
  AccState32* g;
  float* out;
  int carry_tiles;
  int prefetch;
};

// End of a block of a binary32 sum, after its chunks are in the grid
// accumulator: the special-value record joins the grid's, and the last block
// to finish rounds once and leaves the accumulator zeroed. All threads call it.
__device__ __forceinline__ void f32_finish(const F32Args& a, unsigned f, unsigned long long nkey,
                                           unsigned& s_last) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  unsigned long long* gc = reinterpret_cast<unsigned long long*>(a.g->chunk);
  if (blockIdx.x == 0 && tid == 0 && a.n > 0) f |= kFlagAny;
  f = __reduce_or_sync(kFull, f);
  const unsigned long long key = warp_max_ull(nkey);
  if (lane == 0) {
    if (f) atomicOr(&a.g->flags, f);
    if (key) atomicMax(&a.g->nan_key, key);
  }
  __threadfence();
  __syncthreads();
  if (tid == 0) s_last = (atomicAdd(&a.g->ticket, 1u) == gridDim.x - 1) ? 1u : 0u;
  __syncthreads();
  if (!s_last || warp != 0) return;
  __threadfence();
  const long long v = lane < kF32Chunks ? (long long)atomicExch(gc + lane, 0ull) : 0;
  unsigned fl = 0u;
  unsigned long long nk = 0ull;
  if (lane == 0) {
    fl = atomicExch(&a.g->flags, 0u);
    nk = atomicExch(&a.g->nan_key, 0ull);
    atomicExch(&a.g->ticket, 0u);
  }
  fl = __shfl_sync(kFull, fl, 0);
  nk = __shfl_sync(kFull, nk, 0);
  const unsigned bits = warp_round32(v, fl, nk);
  if (lane == 0) *reinterpret_cast<unsigned*>(a.out) = bits;
}

template <int BLOCK, int UNROLL>
__global__ void __launch_bounds__(BLOCK, 1024 / BLOCK) k_sum_f32(F32Args a) {
  extern __shared__ __align__(16) long long smem32[];
  __shared__ unsigned s_last;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  SmallThread32 T;
  T.acc = smem32 + tid;
#pragma unroll
  for (int c = 0; c < 16; ++c) T.acc[c * BLOCK] = 0;
  // head: the (up to 63) elements before the first 256-byte boundary, so the
  // streamed body starts on one (as in the FP64 kernels); body: uint4 quads;
  // tail: up to 3 elements
  const int head = (int)min((long long)((256u - ((uintptr_t)a.x & 255u)) & 255u) / 4, a.n);
  const long long nq = (a.n - head) / 4;
  const int tail = (int)((a.n - head) - nq * 4);
  const uint4* xq = reinterpret_cast<const uint4*>(a.x + head);
  const unsigned* xb = reinterpret_cast<const unsigned*>(a.x);
  grid_dependency_wait();
  if (blockIdx.x == 0 && tid < 32) {  // at most 2 head terms per lane, 3 tail terms in lane 0
    for (int k = tid; k < head; k += 32) T.one<BLOCK>(xb[k]);
    if (tid == 0)
      for (int k = 0; k < tail; ++k) T.one<BLOCK>(xb[a.n - 1 - k]);
  }
  constexpr long long TQ = (long long)BLOCK * UNROLL;
  const long long ntiles = (nq + TQ - 1) / TQ;
  const long long G = gridDim.x;
  auto prefetch = [&](long long t) {
    if (t >= ntiles) return;
    const long long first = t * TQ;
    prefetch_l2(xq + first, (unsigned)(min(TQ, nq - first) * 16));
  };
  auto load = [&](long long t, uint4* buf) {
    if ((t + 1) * TQ <= nq) {  // a full tile: no bounds checks (135.5 against 140.1 us on 2e8 floats)
      const ulonglong2* p = reinterpret_cast<const ulonglong2*>(xq + t * TQ + tid);
#pragma unroll
      for (int u = 0; u < UNROLL; ++u) {
        const ulonglong2 w = ld_stream(p + u * BLOCK);
        buf[u] = make_uint4((unsigned)w.x, (unsigned)(w.x >> 32), (unsigned)w.y, (unsigned)(w.y >> 32));
      }
      return;
    }
#pragma unroll
    for (int u = 0; u < UNROLL; ++u) {
      const long long q = t * TQ + (long long)u * BLOCK + tid;
      if (q < nq) {
        const ulonglong2 w = ld_stream(reinterpret_cast<const ulonglong2*>(xq + q));
        buf[u] = make_uint4((unsigned)w.x, (unsigned)(w.x >> 32), (unsigned)w.y, (unsigned)(w.y >> 32));
      } else {
        buf[u] = make_uint4(kF32NegZero, kF32NegZero, kF32NegZero, kF32NegZero);
      }
    }
  };
  int since = 0;
  auto add = [&](const uint4* buf) {
    T.group<BLOCK, UNROLL>(buf);
    if (++since >= a.carry_tiles) {
      T.propagate<BLOCK>();
      since = 0;
    }
  };
  long long t = blockIdx.x;
  if (tid == 0)
    for (int k = 1; k <= a.prefetch; ++k) prefetch(t + k * G);
  uint4 A[UNROLL], B[UNROLL];
  if (t < ntiles) load(t, A);
  while (t < ntiles) {
    if (tid == 0 && a.prefetch > 0) prefetch(t + (a.prefetch + 1) * G);
    if (t + G < ntiles) load(t + G, B);
    add(A);
    t += G;
    if (t >= ntiles) break;
    if (tid == 0 && a.prefetch > 0) prefetch(t + (a.prefetch + 1) * G);
    if (t + G < ntiles) load(t + G, A);
    add(B);
    t += G;
  }
  __syncthreads();
  grid_launch_dependents();
  // block partial: slot s of every thread split into its low 32 bits and its
  // high part (owed to the next chunk), summed by warp s % (BLOCK / 32) and
  // added to the grid's signed chunk (s & 7) with the sign of the slot set
  constexpr int NW = BLOCK / 32;
  unsigned long long* gc = reinterpret_cast<unsigned long long*>(a.g->chunk);
  const unsigned long long* sa = reinterpret_cast<const unsigned long long*>(smem32);
  for (int sl = warp; sl < 16; sl += NW) {
    unsigned long long lo = 0ull, hi = 0ull;
#pragma unroll
    for (int k = 0; k < NW; ++k) {
      const unsigned long long v = sa[sl * BLOCK + k * 32 + lane];
      lo += v & 0xFFFFFFFFull;
      hi += v >> 32;
    }
    lo = (unsigned long long)warp_sum_ll((long long)lo);
    hi = (unsigned long long)warp_sum_ll((long long)hi);
    if (lane == 0) {
      const bool neg = sl >= 8;
      const int c = sl & 7;
      if (lo) atomicAdd(gc + c, neg ? (unsigned long long)(-(long long)lo) : lo);
      if (hi) atomicAdd(gc + c + 1, neg ? (unsigned long long)(-(long long)hi) : hi);
    }
  }
  {
    const long long top = warp_sum_ll((long long)T.top_pos - (long long)T.top_neg);
    if (lane == 0 && top) atomicAdd(gc + 8, (unsigned long long)top);
  }
  f32_finish(a, T.flags(), T.nkey, s_last);
}

// The paper's large superaccumulator for floats (Large, Fig. 4): one chunk per
// sign+exponent, 512 of them, each a 64-bit sum of 24-bit significands held as
// a 32-bit low word, added with an atomic that returns the old value, and a
// 32-bit high word that counts the carries out of it (one per 256 or more adds
// to that word). Every lane of a warp owns its own column of the planes,
// [chunk][lane], so the 32 atomics of a warp instruction always fall in 32
// different banks and never on one address, whatever the data; the warps of a
// block share the columns. A term always adds its implicit bit; zeros and
// subnormals are counted by sign and their implicit bits taken off at the
// flush, Inf and NaN land in chunks 255 and 511, which the flush ignores. The
// flush transfers chunk (s, e) = V * 2^(max(e, 1) - 150) into the signed chunks
// of the grid accumulator (chunk i weighs 2^(32 i - 150)).
constexpr int kF32LChunks = 512;
struct F32Planes {
  unsigned lo[kF32LChunks * 32];
  unsigned hi[kF32LChunks * 32];
  long long part[kF32Chunks + 1];  // the block's partial
  unsigned zeros[2];               // zero/subnormal terms of the block, by sign
};

template <int BLOCK, int UNROLL>
__global__ void __launch_bounds__(BLOCK, 1) k_sum_f32_large(F32Args a) {
  extern __shared__ __align__(16) unsigned char smem32l[];
  F32Planes& P = *reinterpret_cast<F32Planes*>(smem32l);
  __shared__ unsigned s_last;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  {
    uint4* w = reinterpret_cast<uint4*>(P.lo);
    for (int k = tid; k < 2 * kF32LChunks * 32 / 4; k += BLOCK) w[k] = make_uint4(0u, 0u, 0u, 0u);
    if (tid <= kF32Chunks) P.part[tid] = 0;
    if (tid < 2) P.zeros[tid] = 0u;
  }
  // this lane's column of the lo plane; chunk ix is at + ix * 128 bytes, its
  // hi word at + 64 KB
  const unsigned col = (unsigned)__cvta_generic_to_shared(P.lo) + 4u * (unsigned)lane;
  constexpr unsigned kHiOff = 4u * kF32LChunks * 32;
  const int head = (int)min((long long)((256u - ((uintptr_t)a.x & 255u)) & 255u) / 4, a.n);
  const long long nq = (a.n - head) / 4;
  const int tail = (int)((a.n - head) - nq * 4);
  const uint4* xq = reinterpret_cast<const uint4*>(a.x + head);
  const unsigned* xb = reinterpret_cast<const unsigned*>(a.x);
  unsigned notnegz = 0u, sflags = 0u, zpos = 0u, zneg = 0u;
  unsigned long long nkey = 0ull;
  auto add = [&](unsigned b) {  // any term
    const unsigned M = (b & 0x7FFFFFu) | 0x800000u;
    const unsigned addr = col + ((b >> 23) << 7);
    unsigned old;
    asm volatile("atom.shared.add.u32 %0, [%1], %2;" : "=r"(old) : "r"(addr), "r"(M));
    if (old + M < M) asm volatile("red.shared.add.u32 [%0], 1;" ::"r"(addr + kHiOff));
  };
  auto record = [&](unsigned b) {  // the record of a term (rare path and ends)
    const unsigned e = (b >> 23) & 0xFFu;
    notnegz |= (b != kF32NegZero) ? 1u : 0u;
    if (e == 0u) {
      if (b >> 31) ++zneg; else ++zpos;
    } else if (e == 0xFFu) {
      if (b & 0x7FFFFFu) {
        const unsigned long long k = nan32_key(b);
        nkey = k > nkey ? k : nkey;
      } else {
        sflags |= (b >> 31) ? kFlagNegInf : kFlagPosInf;
      }
    }
  };
  __syncthreads();
  grid_dependency_wait();
  if (blockIdx.x == 0 && tid < 32) {  // at most 2 head terms per lane, 3 tail terms in lane 0
    for (int k = tid; k < head; k += 32) {
      add(xb[k]);
      record(xb[k]);
    }
    if (tid == 0)
      for (int k = 0; k < tail; ++k) {
        add(xb[a.n - 1 - k]);
        record(xb[a.n - 1 - k]);
      }
  }
  constexpr long long TQ = (long long)BLOCK * UNROLL;
  const long long ntiles = (nq + TQ - 1) / TQ;
  const long long G = gridDim.x;
  auto load = [&](long long t, uint4* buf) {
#pragma unroll
    for (int u = 0; u < UNROLL; ++u) {
      const long long q = t * TQ + (long long)u * BLOCK + tid;
      if (q < nq) {
        const ulonglong2 w = ld_stream(reinterpret_cast<const ulonglong2*>(xq + q));
        buf[u] = make_uint4((unsigned)w.x, (unsigned)(w.x >> 32), (unsigned)w.y, (unsigned)(w.y >> 32));
      } else {  // padding with -0: counted as a zero by the record, so its implicit bits are
                // taken off at the flush, and it leaves the -0 record alone
        buf[u] = make_uint4(kF32NegZero, kF32NegZero, kF32NegZero, kF32NegZero);
      }
    }
  };
  // (b << 1) + 2^24 moves the exponent field to the top byte and adds one to
  // it: exponent 255 wraps to a top byte of 0, exponent 0 gives 1, every
  // normal term 2 or more, so the group is all normal exactly when the
  // minimum is at least 2^25 (one shift-add and half a three-way minimum per
  // term; measured 127 against 138 us on 2e8 floats with the exponent-field
  // maximum)
  auto group = [&](const uint4* v) {
    unsigned mn = 0xFFFFFFFFu;
#pragma unroll
    for (int k = 0; k < UNROLL; ++k) {
      mn = __vimin3_u32(mn, (v[k].x << 1) + 0x01000000u, (v[k].y << 1) + 0x01000000u);
      mn = __vimin3_u32(mn, (v[k].z << 1) + 0x01000000u, (v[k].w << 1) + 0x01000000u);
    }
#pragma unroll
    for (int k = 0; k < UNROLL; ++k) {
      add(v[k].x);
      add(v[k].y);
      add(v[k].z);
      add(v[k].w);
    }
    if (__builtin_expect(mn >= 0x02000000u, 1)) {
      notnegz = 1u;
      return;
    }
#pragma unroll
    for (int k = 0; k < UNROLL; ++k) {
      record(v[k].x);
      record(v[k].y);
      record(v[k].z);
      record(v[k].w);
    }
  };
  long long t = blockIdx.x;
  uint4 A[UNROLL], B[UNROLL];
  if (t < ntiles) load(t, A);
  while (t < ntiles) {
    if (t + G < ntiles) load(t + G, B);
    group(A);
    t += G;
    if (t >= ntiles) break;
    if (t + G < ntiles) load(t + G, A);
    group(B);
    t += G;
  }
  grid_launch_dependents();
  {
    const unsigned zp = __reduce_add_sync(kFull, zpos), zn = __reduce_add_sync(kFull, zneg);
    if (lane == 0) {
      if (zp) atomicAdd(&P.zeros[0], zp);
      if (zn) atomicAdd(&P.zeros[1], zn);
    }
  }
  __syncthreads();
  // flush: warp w takes chunks w, w + BLOCK / 32, ...; a chunk's 32 columns
  // sum to V < 2^45 (at most 2^39 terms of < 2^24 in all)
  for (int c = warp; c < kF32LChunks; c += BLOCK / 32) {
    const unsigned e = (unsigned)c & 0xFFu;
    long long v = (long long)(((unsigned long long)P.hi[c * 32 + lane] << 32) | P.lo[c * 32 + lane]);
    if (!__any_sync(kFull, v != 0)) continue;
    v = warp_sum_ll(v);
    if (e == 0xFFu) continue;  // Inf / NaN record only
    if (e == 0u) v -= (long long)P.zeros[c >> 8] << 23;  // the zeros' implicit bits
    if (lane == 0 && v != 0) {
      const unsigned ee = e ? e : 1u;
      const unsigned __int128 W = (unsigned __int128)(unsigned long long)v << (ee & 31u);
      const int i = (int)(ee >> 5);
      const bool neg = (c >> 8) != 0;
      unsigned long long* bp = reinterpret_cast<unsigned long long*>(P.part);
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const long long piece = (long long)(unsigned)(W >> (32 * j));
        if (piece) atomicAdd(bp + i + j, (unsigned long long)(neg ? -piece : piece));
      }
    }
  }
  __syncthreads();
  unsigned long long* gc = reinterpret_cast<unsigned long long*>(a.g->chunk);
  if (tid < kF32Chunks && P.part[tid] != 0) atomicAdd(gc + tid, (unsigned long long)P.part[tid]);
  f32_finish(a, sflags | (notnegz ? kFlagNotNegZero : 0u), nkey, s_last);
}

namespace {
constexpr int kF32Block = 1024;  // one block per SM: measured 4.5 % faster than two of 512
constexpr int kF32Unroll = 3;  // 135.5 us on 2e8 floats back to back (2: 154.8; 4 spills)
// The large superaccumulator: 128 KB of planes, one block of 1024 threads per
// SM, three loads per thread (768 x 4: 128.9 us, 1024 x 4: 139.3, 512 x 6:
// 140.3). Measured on 2e8 floats back to back, against the small one:
// 127.0 / 136.0 us on 2^U(-60,60), 122-123 / 135.5 us on U(-1,1) and N(0,1),
// 120.6 / 134.9 on a constant, 183 / 255 us over the full exponent range. Its
// fixed cost is about 5 us more (16.9 / 11.6 us at 2^22 floats); the two are
// level at 2^26 (53.4 / 52.7 us) and the large one is ahead at 2^27 (90.4 /
// 94.7 us), so it is the default from 5 x 2^24 values.
constexpr int kF32LBlock = 1024;
constexpr int kF32LUnroll = 3;
constexpr long long kF32LargeMin = 5ll << 24;
}  // namespace

}  // namespace xs

using namespace xs;

namespace xs {
namespace {
// One wave of `kernel` (BLOCK threads, UNROLL vectors per thread per tile);
// ID names the kernel for the once-per-device shared-memory attribute.
template <int ID, class K>
xs_status f32_launch(DeviceCtx* ctx, K kernel, int block, int unroll, size_t smem, const F32Args& a,
                     cudaStream_t s) {
  static bool attr[64] = {};  // per device
  if (ctx->device < 64 && !attr[ctx->device]) {
    XS_TRY_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr[ctx->device] = true;
  }
  int occ = 1;
  XS_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, block, smem));
  const long long tq = (long long)block * unroll;
  const long long ntiles = std::max<long long>(1, (a.n / 4 + tq - 1) / tq);
  const long long g =
      std::max<long long>(1, std::min<long long>((long long)ctx->num_sms * std::max(1, occ), ntiles));
  XS_TRY_CUDA(launch_pdl(kernel, (unsigned)g, (unsigned)block, smem, s, a));
  return set_error(XS_OK);
}
}  // namespace
}  // namespace xs

extern "C" xs_status xs_sum_f32_method_async(const float* d_values, int64_t n, float* d_out,
                                             int method, void* stream) {
  if (method < XS_METHOD_AUTO || method > XS_METHOD_LARGE) return set_error(XS_ERR_INVALID_VALUE);
  if (n < 0 || n > (int64_t(1) << 39)) return set_error(XS_ERR_INVALID_VALUE);
  xs_status st = check_device_ptr(d_out);
  if (st != XS_OK) return st;
  if (((uintptr_t)d_out & 3u) != 0u) return set_error(XS_ERR_INVALID_VALUE);
  cudaStream_t s = as_stream(stream);
  if (n == 0) {
    XS_TRY_CUDA(cudaMemsetAsync(d_out, 0, sizeof(float), s));
    return set_error(XS_OK);
  }
  if (((uintptr_t)d_values & 3u) != 0u) return set_error(XS_ERR_INVALID_VALUE);
  if ((st = check_device_ptr(d_values)) != XS_OK) return st;
  DeviceCtx* ctx = device_ctx(&st);
  if (!ctx) return st;
  Workspace* w = workspace(ctx, s, &st);
  if (!w) return st;
  static_assert(sizeof(AccState32) <= sizeof(AccState), "fits the workspace accumulator");
  F32Args a;
  a.x = d_values;
  a.n = n;
  a.g = reinterpret_cast<AccState32*>(w->acc_f32);  // zero at rest, cleared by the last block
  a.out = d_out;
  a.carry_tiles = std::max(1, (kF32CarryInterval - 7) / (4 * kF32Unroll));
  a.prefetch = prefetch_tiles(kF32Prefetch);
  const bool large = method == XS_METHOD_LARGE || (method == XS_METHOD_AUTO && n >= kF32LargeMin);
  if (large)
    return f32_launch<1>(ctx, k_sum_f32_large<kF32LBlock, kF32LUnroll>, kF32LBlock, kF32LUnroll,
                         sizeof(F32Planes), a, s);
  return f32_launch<0>(ctx, k_sum_f32<kF32Block, kF32Unroll>, kF32Block, kF32Unroll,
                       (size_t)kF32Block * 16 * sizeof(long long), a, s);
}

extern "C" xs_status xs_sum_f32_async(const float* d_values, int64_t n, float* d_out,
                                      void* stream) {
  return xs_sum_f32_method_async(d_values, n, d_out, XS_METHOD_AUTO, stream);
}

namespace xs {
// This file's debug word (xs_debug_status).
cudaError_t debug_take_f32(unsigned long long* v) { return debug_word_take(v); }
}  // namespace xs
