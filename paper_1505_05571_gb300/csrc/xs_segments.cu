// Batched segmented exact sums (CSR): one persistent launch behind a CUDA graph.
//
// Each segment is summed exactly and rounded once (abstract; small section on
// rounding). Work decomposition, computed on the device from the offsets by
// k_seg_count / k_seg_scan / k_seg_fill:
//   * long segments (length > short_max) are cut into tiles of tile_elems
//     elements; a work group (one warp by default, up to a block) sums a tile
//     with per-thread small superaccumulators (Fig. 3). A one-tile segment is
//     rounded by that group; the tiles of a longer segment meet in a
//     per-segment global accumulator through integer atomics (partial
//     superaccumulators added exactly, Discussion) and the last tile to finish
//     rounds;
//   * short segments are summed by one warp each; segments of at most two
//     finite terms take a single IEEE addition, which is correctly rounded for
//     two terms (Discussion).
// Groups take long tiles from a global cursor first, then their warps take
// short segments from a second cursor, so short work fills the tail.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <tuple>
#include <vector>

#include "xs_host.hpp"

namespace xs {

struct SegArgs {
  const double* x;
  const long long* off;  // nseg + 1
  long long nseg;
  double* out;
  long long* tile_start;       // nseg + 1: exclusive scan of the tiles of long segments
  int* slot_of;                // nseg: accumulator slot of a multi-tile segment, else -1
  long long* short_list;       // nseg: indices of short segments
  AccState* slots;             // per multi-tile segment
  unsigned long long* counters;  // [0] tiles, [1] short segments, [2] tile cursor, [3] short cursor,
                                 // [4] offsets status of the last launch (kOffBad* bits, 0 = valid)
  long long* blk;               // 3 x nblk: per-block (tiles, short, slots), then their offsets
  long long nblk;               // prep blocks of kPrepSegs segments
  int* tile_seg;                // segment of each tile, when the tiles fit in tile_cap
  long long tile_cap;
  long long tile_elems;
  long long short_max;
  int carry_groups;             // load groups between carry propagations in a tile (0: longest safe)
  int lane_max;                 // short segments up to this length are summed by one lane each
};

constexpr int kPrepThreads = 256;
constexpr int kPrepPer = 8;                              // segments per prep thread
constexpr int kPrepSegs = kPrepThreads * kPrepPer;       // segments per prep block

// Block-wide exclusive scan of one long long per thread; `total` gets the sum.
__device__ long long block_exclusive_scan(long long v, long long* total, long long* sbuf) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  long long incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const long long y = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) sbuf[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const int nw = blockDim.x >> 5;
    long long w = lane < nw ? sbuf[lane] : 0;
    long long wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const long long y = __shfl_up_sync(kFull, wi, o);
      if (lane >= o) wi += y;
    }
    if (lane < nw) sbuf[lane] = wi - w;  // exclusive warp offsets
    if (lane == 31) sbuf[32] = wi;
  }
  __syncthreads();
  const long long r = sbuf[warp] + incl - v;
  *total = sbuf[32];
  __syncthreads();
  return r;
}

// Offsets status bits (counters[4]): a segment whose start is negative or
// whose end lies below its start (its values are never read; its result is
// the default NaN), and a first offset other than 0.
constexpr unsigned long long kOffBadSegment = 1ull;
constexpr unsigned long long kOffBadFirst = 2ull;

// A segment is summed only when 0 <= off[s] <= off[s+1]: the sum of a set is
// defined for a well-formed range only, and a negative start would read
// before the values.
__device__ __forceinline__ bool segment_valid(long long start, long long end) {
  return start >= 0 && end >= start;
}

// Work lists from the offsets, in three coalesced steps. A prep block owns
// kPrepSegs consecutive segments, a thread kPrepPer of them; the order of the
// lists is the order of the segments. An invalid segment joins no list.
struct SegCounts {
  long long tiles, shorts, slots;
};
__device__ __forceinline__ SegCounts thread_counts(const SegArgs& a, long long s0, long long s1) {
  SegCounts c{0, 0, 0};
  for (long long s = s0; s < s1; ++s) {
    const long long L = a.off[s + 1] - a.off[s];
    if (!segment_valid(a.off[s], a.off[s + 1])) continue;
    if (L > a.short_max) {
      const long long t = (L + a.tile_elems - 1) / a.tile_elems;
      c.tiles += t;
      c.slots += (t > 1);
    } else {
      ++c.shorts;
    }
  }
  return c;
}

__global__ void __launch_bounds__(kPrepThreads) k_seg_count(SegArgs a) {
  __shared__ long long sbuf[33];
  const long long s0 = min((long long)blockIdx.x * kPrepSegs + (long long)threadIdx.x * kPrepPer, a.nseg);
  const long long s1 = min(s0 + kPrepPer, a.nseg);
  const SegCounts c = thread_counts(a, s0, s1);
  long long tot[3];
  block_exclusive_scan(c.tiles, &tot[0], sbuf);
  block_exclusive_scan(c.shorts, &tot[1], sbuf);
  block_exclusive_scan(c.slots, &tot[2], sbuf);
  if (threadIdx.x == 0)
    for (int k = 0; k < 3; ++k) a.blk[k * a.nblk + blockIdx.x] = tot[k];
}

// One block: exclusive scan of the block totals (in place) and the counters.
__global__ void __launch_bounds__(1024) k_seg_scan(SegArgs a) {
  __shared__ long long sbuf[33];
  for (int k = 0; k < 3; ++k) {
    long long carry = 0;
    for (long long base = 0; base < a.nblk; base += blockDim.x) {
      const long long i = base + threadIdx.x;
      const long long v = i < a.nblk ? a.blk[k * a.nblk + i] : 0;
      long long tot;
      const long long ex = block_exclusive_scan(v, &tot, sbuf);
      if (i < a.nblk) a.blk[k * a.nblk + i] = carry + ex;
      carry += tot;
    }
    if (threadIdx.x == 0) {
      if (k == 0) {
        a.counters[0] = (unsigned long long)carry;
        a.tile_start[a.nseg] = carry;
      } else if (k == 1) {
        a.counters[1] = (unsigned long long)carry;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    a.counters[2] = 0ull;
    a.counters[3] = 0ull;
    a.counters[4] = 0ull;  // k_seg_fill records what it finds
  }
}

__global__ void __launch_bounds__(kPrepThreads) k_seg_fill(SegArgs a) {
  __shared__ long long sbuf[33];
  const long long s0 = min((long long)blockIdx.x * kPrepSegs + (long long)threadIdx.x * kPrepPer, a.nseg);
  const long long s1 = min(s0 + kPrepPer, a.nseg);
  const SegCounts c = thread_counts(a, s0, s1);
  long long tot;
  long long t_off = a.blk[blockIdx.x] + block_exclusive_scan(c.tiles, &tot, sbuf);
  long long sh_off = a.blk[a.nblk + blockIdx.x] + block_exclusive_scan(c.shorts, &tot, sbuf);
  long long sl_off = a.blk[2 * a.nblk + blockIdx.x] + block_exclusive_scan(c.slots, &tot, sbuf);
  unsigned long long bad = (blockIdx.x == 0 && threadIdx.x == 0 && a.off[0] != 0) ? kOffBadFirst : 0ull;
  for (long long s = s0; s < s1; ++s) {
    const long long L = a.off[s + 1] - a.off[s];
    a.tile_start[s] = t_off;
    int slot = -1;
    if (!segment_valid(a.off[s], a.off[s + 1])) {
      reinterpret_cast<unsigned long long*>(a.out)[s] = kDefaultNaN;
      bad |= kOffBadSegment;
    } else if (L > a.short_max) {
      const long long t = (L + a.tile_elems - 1) / a.tile_elems;
      if (t_off + t <= a.tile_cap)
        for (long long k = 0; k < t; ++k) a.tile_seg[t_off + k] = (int)s;
      t_off += t;
      if (t > 1) slot = (int)(sl_off++);
    } else {
      a.short_list[sh_off++] = s;
    }
    a.slot_of[s] = slot;
  }
  if (bad) atomicOr(&a.counters[4], bad);
}

// Short segments of at most this many values are summed by one lane each
// (at most 2047 adds between carry propagations). Measured, 2e6 segments of
// 1..100 values: 0.667 ms (one warp per segment: 2.418 ms; a limit of 64:
// 1.483 ms; every term through the general add: 0.750 ms; also four loads in
// flight and no L2 prefetch: 0.889 ms); 4e6 of 1..16: 0.545 ms (4.276 ms);
// the 60,102 segments of up to 4096 values among 100,000 of log-uniform
// lengths in 1..1e6: 0.217 ms (0.240 ms). Fetching the next claim's metadata
// during the current one gained nothing and cost 30 % on those.
constexpr int kSegLaneMax = 128;
static_assert(kSegLaneMax <= 2040, "lane sums skip carry propagation");
constexpr int kPhase1Ahead = 48;  // values per thread of a tile prefetched before the block starts it

// L2 prefetch of the 16-byte-aligned part of [p, q), in pieces of at most 64 KB.
__device__ __forceinline__ void prefetch_range(const unsigned long long* p,
                                               const unsigned long long* q) {
  uintptr_t b0 = ((uintptr_t)p + 15u) & ~(uintptr_t)15u;
  const uintptr_t b1 = (uintptr_t)q & ~(uintptr_t)15u;
  while (b0 < b1) {
    const uintptr_t n = min(b1 - b0, (uintptr_t)65536u);
    prefetch_l2((const void*)b0, (unsigned)n);
    b0 += n;
  }
}

// Correctly rounded value of one thread's own chunks cmin..cmax (every other
// chunk zero; cmax < kSChunks - 2, as for sums of finite doubles), for windows
// wider than round_window takes, and clears them. The carries are propagated
// in place, a negative value is negated as a digit string, and the top eight
// digits go to round_window with an OR of the digits below them folded into
// the lowest bit of the lowest one: seven or more digits under the top, that
// bit only enters the sticky bit, so the rounding is unchanged.
template <int BLOCK>
__device__ unsigned long long round_column(long long* acc, int cmin, int cmax, unsigned flags,
                                           unsigned long long nan_key) {
  unsigned long long sp;
  if (special_result(flags, nan_key, &sp)) {
    for (int c = cmin; c <= cmax; ++c) acc[c * BLOCK] = 0;
    return sp;
  }
  long long carry = 0;
  for (int c = cmin; c <= cmax; ++c) {
    const long long x = acc[c * BLOCK] + carry;
    acc[c * BLOCK] = (long long)(unsigned)x;
    carry = x >> 32;  // arithmetic: floor division by 2^32
  }
  const bool neg = carry < 0;
  if (neg) {  // -(D + carry 2^(32 (cmax + 1))) = ~D + 1 + (-carry - 1) 2^(32 (cmax + 1))
    unsigned long long cc = 1;
    for (int c = cmin; c <= cmax; ++c) {
      const unsigned long long x = (unsigned long long)(unsigned)~(unsigned)acc[c * BLOCK] + cc;
      acc[c * BLOCK] = (long long)(unsigned)x;
      cc = x >> 32;
    }
    carry = -carry - 1 + (long long)cc;
  }
  // the magnitude: digits cmin..cmax and carry (0 <= carry < 2^32) at cmax + 1
  int m = carry != 0 ? cmax + 1 : -1;
  for (int c = cmax; m < 0 && c >= cmin; --c)
    if (acc[c * BLOCK] != 0) m = c;
  if (m < 0) return signed_zero(flags);  // the digits are all zero already
  const int p0 = max(cmin, m - 7);
  long long w[9];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int c = p0 + k;
    w[k] = c > m ? 0 : (c == cmax + 1 ? carry : acc[c * BLOCK]);
  }
  w[8] = 0;
  long long below = 0;
  for (int c = cmin; c < p0; ++c) below |= acc[c * BLOCK];
  for (int c = cmin; c <= cmax; ++c) acc[c * BLOCK] = 0;
  if (below != 0) w[0] |= 1;
  return round_window(w, m - p0 + 2, p0, flags, 0ull) | (neg ? kNegZero : 0ull);
}

// Launch shape of the segmented kernel for phase-1 work groups of W threads:
// a block of 384 threads (one per SM, 12 warps) holding 384 / W groups when W
// divides 384 -- measured on GB300, several blocks per SM accumulate about
// 10 % slower than one block of the same total size -- else one group per block.
template <int W>
struct SegShape {
  static constexpr int block = (384 % W == 0) ? 384 : W;
  static constexpr int groups = block / W;
};

template <int W, int UNROLL>
__global__ void __launch_bounds__(SegShape<W>::block, 1) k_seg_main(SegArgs a) {
  constexpr int BLOCK = SegShape<W>::block;
  constexpr int NG = SegShape<W>::groups;
  // groups of adds between carry propagations in a tile: with the head, tail
  // and padded last group, at most 2045 adds per thread
  constexpr int kCarryGroups = (kCarryInterval - 4 - 2 * UNROLL) / (2 * UNROLL);
  static_assert(W >= 32 && W % 32 == 0 && W <= 384, "whole warps, one block at most");
  // the thread that claims the next tile: warp 1 of the group, beside warp 0's
  // rounding; lane 0 when the group is one warp
  constexpr int kClaimer = W > 32 ? 32 : 0;
  extern __shared__ __align__(16) long long smem_seg[];
  __shared__ long long g_bsum[NG][kSChunks];
  __shared__ long long g_item[NG];
  __shared__ long long g_meta[NG][4];
  __shared__ unsigned g_flags[NG], g_last[NG], g_emin[NG], g_emax[NG];
  __shared__ unsigned long long g_nkey[NG];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int grp = tid / W, gt = tid - grp * W, gwarp = gt >> 5;  // group, rank and warp in it
  long long* bsum = g_bsum[grp];
  long long& s_item = g_item[grp];
  long long* s_meta = g_meta[grp];
  unsigned& s_flags = g_flags[grp];
  unsigned& s_last = g_last[grp];
  unsigned& s_emin = g_emin[grp];
  unsigned& s_emax = g_emax[grp];
  unsigned long long& s_nkey = g_nkey[grp];
  // barrier of the group's W threads (named barrier 1 + group; a warp's own
  // barrier when the group is one warp)
  auto gsync = [&]() {
    if (W == 32) __syncwarp();
    else if (NG == 1) __syncthreads();
    else asm volatile("bar.sync %0, %1;" ::"r"(1 + grp), "r"(W) : "memory");
  };
  SmallThread T;
  T.acc = smem_seg + tid;
  // The accumulators are cleared once; every merge clears again the chunks it
  // read (the window of chunks the terms touched), and the rounding scratch
  // lives outside them, so they are zero whenever a new sum starts.
  for (int c = 0; c < kSChunks; ++c) T.acc[c * BLOCK] = 0;
  const long long ntiles = (long long)a.counters[0];
  const long long nshort = (long long)a.counters[1];
  const unsigned long long* xb_all = reinterpret_cast<const unsigned long long*>(a.x);
  __syncthreads();

  // ---- phase 1: tiles of long segments, one work group of W threads each ----
  // Each group claims tiles on its own. The next tile is claimed while the
  // group merges the current one, and its start is prefetched into L2 before
  // the group moves on, so neither the claim nor a tile's first loads wait
  // behind the previous merge.
  // segment of tile t: from the table, else the last s with tile_start[s] <= t
  auto segment_of = [&](long long t) -> long long {
    if (ntiles <= a.tile_cap && XS_DCHECK(t >= 0 && t < ntiles, kDbgTableIndex)) return a.tile_seg[t];
    long long lo_s = 0, hi_s = a.nseg;  // invariant: tile_start[lo_s] <= t < tile_start[hi_s]
    while (hi_s - lo_s > 1) {
      const long long mid = (lo_s + hi_s) >> 1;
      if (a.tile_start[mid] <= t) lo_s = mid; else hi_s = mid;
    }
    return lo_s;
  };
  // where tile t lies: its segment, element range and the segment's tile count
  auto describe = [&](long long t) {
    const long long sg = segment_of(t);
    const long long ft = a.tile_start[sg];
    const long long tl = a.off[sg] + (t - ft) * a.tile_elems;
    s_meta[0] = sg;
    s_meta[1] = tl;
    s_meta[2] = min(tl + a.tile_elems, a.off[sg + 1]);
    s_meta[3] = a.tile_start[sg + 1] - ft;
  };
  if (gt == 0) {
    s_item = (long long)atomicAdd(&a.counters[2], 1ull);
    if (s_item < ntiles) describe(s_item);
  }
  for (;;) {
    for (int c = gt; c < kSChunks; c += W) bsum[c] = 0;
    if (gt == 0) {
      s_flags = 0u;
      s_nkey = 0ull;
      s_emin = 0x7FFu;
      s_emax = 0u;
    }
    gsync();
    const long long t = s_item;
    if (t >= ntiles) break;
    const long long s = s_meta[0], lo = s_meta[1], hi = s_meta[2], seg_tiles = s_meta[3];
    T.reset();
    accumulate_range<BLOCK, UNROLL, true, true>(T, a.x, lo, hi, gt, W,
                                                a.carry_groups > 0 ? min(a.carry_groups, kCarryGroups)
                                                                   : kCarryGroups);
    {
      const unsigned wmin = __reduce_min_sync(kFull, T.emin);
      const unsigned wmax = __reduce_max_sync(kFull, T.emax);
      if (lane == 0 && wmax >= wmin) {
        atomicMin(&s_emin, wmin);
        atomicMax(&s_emax, wmax);
      }
    }
    gsync();  // every thread has read s_item; the window is complete
    if (gt == kClaimer) s_item = (long long)atomicAdd(&a.counters[2], 1ull);
    const int cmin = (int)(s_emin >> kLowExpBits);
    const int cmax = s_emax >= s_emin ? (int)(s_emax >> kLowExpBits) + 1 : cmin - 1;  // empty
    unsigned f = __reduce_or_sync(kFull, T.flags());
    const unsigned long long k = warp_max_ull(T.nkey);
    if (lane == 0) {
      if (f) atomicOr(&s_flags, f);
      if (k) atomicMax(&s_nkey, k);
    }
    const long long* gacc = smem_seg + grp * W;  // the group's accumulators
    if (seg_tiles == 1) {
      group_chunk_sums<BLOCK, W>(gacc, gwarp, [&](int c, long long v) {
        atomicAdd(reinterpret_cast<unsigned long long*>(bsum + c), (unsigned long long)v);
      }, cmin, cmax);
      gsync();
      for (int c = cmin; c <= cmax; ++c) T.acc[c * BLOCK] = 0;
      constexpr int kWin = 8;  // windows up to this many chunks round in one thread
      if (cmax - cmin < kWin && cmax < kSChunks - 1) {
        if (gt == 0) {
          long long w[kWin + 1];
#pragma unroll
          for (int k = 0; k <= kWin; ++k) w[k] = cmin + k <= cmax + 1 ? bsum[cmin + k] : 0;
          const int nw = cmax >= cmin ? cmax - cmin + 2 : 0;
          reinterpret_cast<unsigned long long*>(a.out)[s] =
              round_window(w, nw, cmin, s_flags | kFlagAny, s_nkey);
        }
      } else if (gwarp == 0) {
        const long long v0 = bsum[lane], v1 = bsum[lane + 32], v2 = lane < 3 ? bsum[lane + 64] : 0;
        __syncwarp();  // bsum is the rounding scratch from here on
        const unsigned long long r = warp_round(v0, v1, v2, s_flags | kFlagAny, s_nkey, bsum, 32);
        if (lane == 0) reinterpret_cast<unsigned long long*>(a.out)[s] = r;
      }
    } else {
      AccState* g = a.slots + a.slot_of[s];
      unsigned long long* gc = reinterpret_cast<unsigned long long*>(g->chunk);
      group_chunk_sums<BLOCK, W>(gacc, gwarp, [&](int c, long long v) {
        if (v != 0) atomicAdd(gc + c, (unsigned long long)v);
      }, cmin, cmax);
      gsync();
      for (int c = cmin; c <= cmax; ++c) T.acc[c * BLOCK] = 0;
      if (gt == 0) {
        if (s_flags) atomicOr(&g->flags, s_flags);
        if (s_nkey) atomicMax(&g->nan_key, s_nkey);
        __threadfence();
        s_last = (atomicAdd(&g->ticket, 1u) == (unsigned)(seg_tiles - 1)) ? 1u : 0u;
      }
      gsync();
      if (s_last && gwarp == 0) {
        __threadfence();
        const long long v0 = (long long)atomicExch(gc + lane, 0ull);
        const long long v1 = (long long)atomicExch(gc + lane + 32, 0ull);
        const long long v2 = lane < 3 ? (long long)atomicExch(gc + lane + 64, 0ull) : 0;
        unsigned fl = 0u;
        unsigned long long key = 0ull;
        if (lane == 0) {
          fl = atomicExch(&g->flags, 0u);
          key = atomicExch(&g->nan_key, 0ull);
          atomicExch(&g->ticket, 0u);
        }
        fl = __shfl_sync(kFull, fl, 0);
        key = __shfl_sync(kFull, key, 0);
        const unsigned long long r = warp_round(v0, v1, v2, fl | kFlagAny, key, bsum, 32);
        if (lane == 0) reinterpret_cast<unsigned long long*>(a.out)[s] = r;
      }
    }
    if (gt == kClaimer) {  // the next tile: where it lies, and its first groups into L2
      const long long tn = s_item;  // beside warp 0's rounding
      if (tn < ntiles) {
        describe(tn);
        prefetch_range(xb_all + s_meta[1],
                       xb_all + min(s_meta[2], s_meta[1] + (long long)kPhase1Ahead * W));
      }
    }
    gsync();
  }

  // ---- phase 2: short segments, one warp each ----
  const unsigned long long* xb = reinterpret_cast<const unsigned long long*>(a.x);
  constexpr long long kClaim = 32;  // short segments a warp claims per cursor atomic
  for (;;) {
    long long j0 = 0;
    if (lane == 0) j0 = (long long)atomicAdd(&a.counters[3], (unsigned long long)kClaim);
    j0 = __shfl_sync(kFull, j0, 0);
    if (j0 >= nshort) break;
    const int cnt = (int)min(kClaim, nshort - j0);
    // lane q fetches the metadata of the q-th claimed segment, all at once
    long long ms = 0, mlo = 0, mhi = 0;
    if (lane < cnt) {
      ms = a.short_list[j0 + lane];
      mlo = a.off[ms];
      mhi = a.off[ms + 1];
    }
    // Segments of at most lane_max values: each lane sums the one it fetched,
    // alone, in its own accumulator column (at most lane_max adds, no carry
    // propagation), and rounds it itself (round_window, or round_column for
    // wider windows): the 32 roundings of a claim run side by side, with no
    // warp reductions.
    unsigned done = 0u;
    {
      const long long L = mhi - mlo;
      bool mine = lane < cnt && L <= (long long)a.lane_max;
      if (mine) {
        unsigned long long r = 0ull;  // +0 for an empty segment
        if (L > 0) {
          const unsigned long long b0 = __ldg(xb + mlo);
          const unsigned long long b1 = L > 1 ? __ldg(xb + mlo + 1) : kNegZero;
          if (L <= 2 && ((b0 >> 52) & 0x7FFu) != 0x7FFu && ((b1 >> 52) & 0x7FFu) != 0x7FFu) {
            // one IEEE addition is correctly rounded; x + (-0) = x keeps -0 alone
            r = (unsigned long long)__double_as_longlong(
                __dadd_rn(__longlong_as_double((long long)b0), __longlong_as_double((long long)b1)));
          } else {
            if (L >= 32) prefetch_range(xb + mlo, xb + mhi);  // the rest of it into L2
            T.reset();
            T.one<BLOCK, true>(b0);
            if (L > 1) T.one<BLOCK, true>(b1);
            long long k = mlo + 2;
            for (; k + 8 <= mhi; k += 8) {  // eight loads in flight, one normal-term test
              ulonglong2 c[4];
#pragma unroll
              for (int u = 0; u < 4; ++u) c[u] = make_ulonglong2(__ldg(xb + k + 2 * u), __ldg(xb + k + 2 * u + 1));
              T.group<BLOCK, 4, true>(c);
            }
            for (; k + 4 <= mhi; k += 4) {
              const unsigned long long c0 = __ldg(xb + k), c1 = __ldg(xb + k + 1);
              const unsigned long long c2 = __ldg(xb + k + 2), c3 = __ldg(xb + k + 3);
              T.one<BLOCK, true>(c0);
              T.one<BLOCK, true>(c1);
              T.one<BLOCK, true>(c2);
              T.one<BLOCK, true>(c3);
            }
            for (; k < mhi; ++k) T.one<BLOCK, true>(__ldg(xb + k));
            const int cmin = (int)(T.emin >> kLowExpBits);
            const int cmax = T.emax >= T.emin ? (int)(T.emax >> kLowExpBits) + 1 : cmin - 1;
            constexpr int kWin = 8;
            if (cmax - cmin < kWin && cmax < kSChunks - 1) {
              long long w[kWin + 1];
#pragma unroll
              for (int c = 0; c < kWin; ++c) {
                w[c] = 0;
                if (cmin + c <= cmax) {
                  w[c] = T.acc[(cmin + c) * BLOCK];
                  T.acc[(cmin + c) * BLOCK] = 0;
                }
              }
              w[kWin] = 0;
              const int nw = cmax >= cmin ? cmax - cmin + 2 : 0;
              r = round_window(w, nw, cmin, T.flags() | kFlagAny, T.nkey);
            } else {
              r = round_column<BLOCK>(T.acc, cmin, cmax, T.flags() | kFlagAny, T.nkey);
            }
          }
        }
        if (mine) reinterpret_cast<unsigned long long*>(a.out)[ms] = r;
      }
      done = __ballot_sync(kFull, mine);
    }
    // segment j of the claim into L2 (warp-uniform call: shuffles)
    auto prefetch_seg = [&](int j) {
      const long long plo = __shfl_sync(kFull, mlo, j & 31), phi = __shfl_sync(kFull, mhi, j & 31);
      if (lane == 0 && j < cnt && !((done >> j) & 1u)) prefetch_range(xb + plo, xb + phi);
    };
    prefetch_seg(0);
    prefetch_seg(1);
    for (int q = 0; q < cnt; ++q) {
    if ((done >> q) & 1u) continue;
    prefetch_seg(q + 2);
    const long long s = __shfl_sync(kFull, ms, q);
    const long long lo = __shfl_sync(kFull, mlo, q), hi = __shfl_sync(kFull, mhi, q);
    const long long L = hi - lo;
    if (L <= 2) {
      const unsigned long long b0 = L > 0 ? xb[lo] : 0ull;
      const unsigned long long b1 = L > 1 ? xb[lo + 1] : kNegZero;
      const bool fin = ((b0 >> 52) & 0x7FFu) != 0x7FFu && ((b1 >> 52) & 0x7FFu) != 0x7FFu;
      if (L == 0 || fin) {
        if (lane == 0) {
          // one IEEE addition is correctly rounded; x + (-0) = x keeps -0 alone
          const double r = L == 0 ? 0.0 : __dadd_rn(__longlong_as_double((long long)b0),
                                                  __longlong_as_double((long long)b1));
          a.out[s] = r;
        }
        continue;
      }
    }
    T.reset();
    int cmin = 0, cmax = kSChunks - 1;  // chunks the warp's terms can touch
    if (L <= 128) {
      // Low fixed cost for short sums (Discussion: track the chunks in use
      // instead of clearing and scanning all 67): the terms sit in registers,
      // the warp finds the range of chunk indices they touch, and only that
      // window is added into, read back and cleared again.
      unsigned long long v[4];
      int mn = kSChunks, mx = -1;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const long long idx = lo + lane + 32 * k;
        v[k] = idx < hi ? xb[idx] : kNegZero;
        const unsigned e = (unsigned)(v[k] >> 52) & 0x7FFu;
        if (e != 0x7FFu && (v[k] << 1) != 0ull) {  // finite and nonzero
          const int i = (int)((e ? e : 1u) >> kLowExpBits);
          mn = min(mn, i);
          mx = max(mx, i + 1);
        }
      }
      cmin = __reduce_min_sync(kFull, mn);
      cmax = __reduce_max_sync(kFull, mx);
      // zeros add 0 to chunks that stay zero
#pragma unroll
      for (int k = 0; k < 4; ++k) T.one<BLOCK>(v[k]);
    } else {
      accumulate_range<BLOCK, 2, false, true>(T, a.x, lo, hi, lane, 32);
      const unsigned wmin = __reduce_min_sync(kFull, T.emin);
      const unsigned wmax = __reduce_max_sync(kFull, T.emax);
      cmin = (int)(wmin >> kLowExpBits);
      cmax = wmax >= wmin ? (int)(wmax >> kLowExpBits) + 1 : cmin - 1;  // empty
    }
    // Warp sums of the window's chunks, one chunk at a time: each lane splits
    // its own chunk c into the low 32 bits and the signed high part (owed to
    // chunk c + 1) and clears it; the 32-lane sums come from 32-bit warp
    // reductions of 16-bit digits (digit sums below 2^21 in magnitude: exact).
    const unsigned f = __reduce_or_sync(kFull, T.flags()) | kFlagAny;
    const unsigned long long key = warp_max_ull(T.nkey);
    auto chunk_sums = [&](int c, long long& sum_lo, long long& sum_hi) {
      const long long u = T.acc[c * BLOCK];
      T.acc[c * BLOCK] = 0;
      const unsigned lw = (unsigned)u;
      const int hw = (int)(u >> 32);
      const unsigned l0 = __reduce_add_sync(kFull, lw & 0xFFFFu);
      const unsigned l1 = __reduce_add_sync(kFull, lw >> 16);
      const unsigned h0 = __reduce_add_sync(kFull, (unsigned)hw & 0xFFFFu);
      const int h1 = __reduce_add_sync(kFull, hw >> 16);
      sum_lo = (long long)l0 + (long long)l1 * 65536ll;
      sum_hi = (long long)h0 + (long long)h1 * 65536ll;
    };
    constexpr int kWin = 8;  // windows up to this many chunks round in one thread
    if (cmax - cmin < kWin && cmax < kSChunks - 1) {
      // the sums are the same in every lane: lane 0 rounds the window alone
      long long w[kWin + 1];
#pragma unroll
      for (int k = 0; k <= kWin; ++k) w[k] = 0;
#pragma unroll
      for (int k = 0; k < kWin; ++k) {
        if (cmin + k <= cmax) {
          long long sl, shv;
          chunk_sums(cmin + k, sl, shv);
          w[k] += sl;
          w[k + 1] += shv;
        }
      }
      if (lane == 0) {
        const int nw = cmax >= cmin ? cmax - cmin + 2 : 0;
        reinterpret_cast<unsigned long long*>(a.out)[s] = round_window(w, nw, cmin, f, key);
      }
      __syncwarp();
      continue;
    }
    // wider windows: lane L collects chunks L, L + 32 and L + 64 of the sum
    // and the warp rounds
    long long v0 = 0, v1 = 0, v2 = 0;
    auto put = [&](int k, long long val) {
      if (k < 32) { if (lane == k) v0 += val; }
      else if (k < 64) { if (lane == k - 32) v1 += val; }
      else if (lane == k - 64) v2 += val;
    };
    for (int c = cmin; c <= cmax; ++c) {
      long long sl, shv;
      chunk_sums(c, sl, shv);
      if (c == kSChunks - 1) {
        put(c, sl + shv * 4294967296ll);
      } else {
        put(c, sl);
        put(c + 1, shv);
      }
    }
    __syncwarp();  // chunks 0..2 of the warp's threads are the rounding scratch now
    const unsigned long long r = warp_round(v0, v1, v2, f, key, smem_seg + warp * 32, BLOCK);
    if (lane == 0) reinterpret_cast<unsigned long long*>(a.out)[s] = r;
    __syncwarp();
    T.acc[0] = 0;
    T.acc[BLOCK] = 0;
    if (lane < 3) T.acc[2 * BLOCK] = 0;
    __syncwarp();
    }
  }
}

namespace {

typedef void (*SegKernel)(SegArgs);
struct SegEntry {
  int block, unroll;
  SegKernel fn;
  int launch;  // threads per launched block
};
// block: the phase-1 work group (threads of the launch: SegShape<block>::block)
const SegEntry kSeg[] = {
    {128, 4, k_seg_main<128, 4>, SegShape<128>::block},
    {192, 4, k_seg_main<192, 4>, SegShape<192>::block},
    {256, 4, k_seg_main<256, 4>, SegShape<256>::block},
    {384, 4, k_seg_main<384, 4>, SegShape<384>::block},
    {192, 8, k_seg_main<192, 8>, SegShape<192>::block},
    {128, 8, k_seg_main<128, 8>, SegShape<128>::block},
    {64, 8, k_seg_main<64, 8>, SegShape<64>::block},
    {32, 8, k_seg_main<32, 8>, SegShape<32>::block},
};
constexpr int kNumSeg = sizeof(kSeg) / sizeof(kSeg[0]);

int find_seg(int block, int unroll) {
  for (int k = 0; k < kNumSeg; ++k)
    if (kSeg[k].block == block && kSeg[k].unroll == unroll) return k;
  return -1;
}

size_t seg_smem(int block) { return (size_t)block * kSChunks * sizeof(long long); }

// The longest interval, in load groups of 2 x unroll adds, between per-thread
// carry propagations inside a tile (head, tail and the padded group included).
int seg_max_carry_groups(int unroll) { return (kCarryInterval - 4 - 2 * unroll) / (2 * unroll); }

xs_seg_options default_seg_options(DeviceCtx* ctx) {
  if (ctx->have_tuned_seg) return ctx->tuned_seg;
  xs_seg_options o;
  // measured on GB300 over 100,000 segments of log-uniform lengths in 1..1e6 (58 GB),
  // with the streamed bodies on 256-byte boundaries: groups of two warps x 8
  // loads with tiles of 2^18 values and short_max 4096 take 9.53 ms (what the
  // autotuner picks); one-warp groups with tiles of 2^15, 10.54 ms (before the
  // alignment change the latter was the fastest, 10.09 ms). By length class:
  // segments up to 4096 values 0.25 ms (60,102 of them, 0.24 GB), 4097 up to
  // 2^18 2.61 ms (14.9 GB), longer ones 6.93 ms (43.2 GB, 6.24 TB/s) --
  // xs_autotune_segments picks per workload
  o.block = 64;
  o.unroll = 8;
  o.tile_elems = 1 << 18;
  o.short_max = 4096;
  o.carry_tiles = 0;
  return o;
}

xs_status resolve_options(DeviceCtx* ctx, const xs_seg_options* in, xs_seg_options* out) {
  xs_seg_options d = default_seg_options(ctx);
  xs_seg_options o = in ? *in : d;
  if (o.block == 0) o.block = d.block;
  if (o.unroll == 0) o.unroll = d.unroll;
  if (o.tile_elems == 0) o.tile_elems = d.tile_elems;
  if (o.short_max == 0) o.short_max = d.short_max;
  if (find_seg(o.block, o.unroll) < 0) return set_error(XS_ERR_NOT_SUPPORTED);
  // tiles longer than 2040 values per thread propagate carries inside the tile,
  // at most every seg_max_carry_groups(unroll) load groups
  if (o.tile_elems < 2 * o.block || o.tile_elems > (1 << 26)) return set_error(XS_ERR_INVALID_VALUE);
  if (o.carry_tiles < 0 || o.carry_tiles > seg_max_carry_groups(o.unroll)) return set_error(XS_ERR_INVALID_VALUE);
  if (o.short_max < 0 || o.short_max > 2040 * 32) return set_error(XS_ERR_INVALID_VALUE);
  *out = o;
  return XS_OK;
}

}  // namespace

}  // namespace xs

using namespace xs;

struct xs_seg_plan_s {
  int device = -1;
  SegArgs args{};
  xs_seg_options opts{};
  int kernel = -1;
  int grid = 0;
  void* mem = nullptr;  // one allocation for all work lists
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

static xs_status plan_enqueue(xs_seg_plan p, cudaStream_t s) {
  const unsigned nb = (unsigned)p->args.nblk;
  k_seg_count<<<nb, kPrepThreads, 0, s>>>(p->args);
  XS_TRY_CUDA(cudaGetLastError());
  k_seg_scan<<<1, 1024, 0, s>>>(p->args);
  XS_TRY_CUDA(cudaGetLastError());
  k_seg_fill<<<nb, kPrepThreads, 0, s>>>(p->args);
  XS_TRY_CUDA(cudaGetLastError());
  const SegEntry& K = kSeg[p->kernel];
  K.fn<<<p->grid, K.launch, seg_smem(K.launch), s>>>(p->args);
  XS_TRY_CUDA(cudaGetLastError());
  return XS_OK;
}

extern "C" {

xs_status xs_seg_plan_create(xs_seg_plan* plan, const double* d_values, const int64_t* d_offsets,
                             int64_t nseg, double* d_out, const xs_seg_options* opts,
                             void* stream) {
  if (plan == nullptr) return set_error(XS_ERR_INVALID_POINTER);
  if (nseg <= 0) return set_error(XS_ERR_INVALID_VALUE);
  if (nseg > (int64_t(1) << 31) - 2) return set_error(XS_ERR_INVALID_VALUE);
  xs_status st;
  if ((st = check_device_ptr(d_offsets)) != XS_OK) return st;
  if ((st = check_device_ptr(d_out)) != XS_OK) return st;
  if (d_values != nullptr && (st = check_device_ptr(d_values)) != XS_OK) return st;
  if (((uintptr_t)d_values & 7u) || ((uintptr_t)d_offsets & 7u) || ((uintptr_t)d_out & 7u))
    return set_error(XS_ERR_INVALID_VALUE);
  DeviceCtx* ctx = device_ctx(&st);
  if (!ctx) return st;
  xs_seg_options o;
  if ((st = resolve_options(ctx, opts, &o)) != XS_OK) return st;
  const int k = find_seg(o.block, o.unroll);
  {
    static bool attr_done[64][kNumSeg] = {};
    if (ctx->device < 64 && !attr_done[ctx->device][k]) {
      XS_TRY_CUDA(cudaFuncSetAttribute(kSeg[k].fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)seg_smem(kSeg[k].launch)));
      attr_done[ctx->device][k] = true;
    }
  }
  int occ = 0;
  XS_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kSeg[k].fn, kSeg[k].launch,
                                                            seg_smem(kSeg[k].launch)));
  if (occ < 1) return set_error(XS_ERR_NOT_SUPPORTED);
  xs_seg_plan p = new xs_seg_plan_s();
  p->device = ctx->device;
  p->opts = o;
  p->kernel = k;
  p->grid = ctx->num_sms * occ;
  // layout: counters (64 B) | tile_start (nseg+1) | short_list (nseg) | slot_of (nseg) | slots
  const size_t n = (size_t)nseg;
  const size_t bytes_ctr = 64;
  const size_t bytes_ts = (n + 1) * 8, bytes_sl = n * 8, bytes_so = ((n * 4 + 15) / 16) * 16;
  // multi-tile segments: at most total/tile, and at most nseg
  const size_t max_slots = n;
  const size_t bytes_slots = max_slots * sizeof(AccState);
  const size_t nblk = (n + kPrepSegs - 1) / kPrepSegs;
  const size_t bytes_blk = 3 * nblk * sizeof(long long);
  // tile table sized for the offsets as they are now (segments + elements / tile)
  long long last = 0;
  cudaError_t e0 = cudaMemcpy(&last, d_offsets + nseg, sizeof(long long), cudaMemcpyDeviceToHost);
  if (e0 != cudaSuccess) {
    delete p;
    return from_cuda(e0);
  }
  if (last < 0) {
    delete p;
    return set_error(XS_ERR_INVALID_VALUE);
  }
  const size_t tile_cap = n + (size_t)(last / o.tile_elems) + 1;
  const size_t bytes_tab = ((tile_cap * sizeof(int) + 15) / 16) * 16;
  const size_t total = bytes_ctr + bytes_ts + bytes_sl + bytes_so + bytes_slots + bytes_blk + bytes_tab;
  cudaError_t e = dev_alloc(&p->mem, total);
  if (e != cudaSuccess) {
    delete p;
    return from_cuda(e);
  }
  cudaStream_t s = as_stream(stream);
  e = cudaMemsetAsync(p->mem, 0, total, s);
  if (e != cudaSuccess) {
    dev_free(p->mem);
    delete p;
    return from_cuda(e);
  }
  char* base = static_cast<char*>(p->mem);
  SegArgs& a = p->args;
  a.x = d_values;
  a.off = reinterpret_cast<const long long*>(d_offsets);
  a.nseg = nseg;
  a.out = d_out;
  a.counters = reinterpret_cast<unsigned long long*>(base);
  a.tile_start = reinterpret_cast<long long*>(base + bytes_ctr);
  a.short_list = reinterpret_cast<long long*>(base + bytes_ctr + bytes_ts);
  a.slot_of = reinterpret_cast<int*>(base + bytes_ctr + bytes_ts + bytes_sl);
  a.slots = reinterpret_cast<AccState*>(base + bytes_ctr + bytes_ts + bytes_sl + bytes_so);
  a.blk = reinterpret_cast<long long*>(base + bytes_ctr + bytes_ts + bytes_sl + bytes_so + bytes_slots);
  a.nblk = (long long)nblk;
  a.tile_seg = reinterpret_cast<int*>(base + bytes_ctr + bytes_ts + bytes_sl + bytes_so + bytes_slots +
                                      bytes_blk);
  a.tile_cap = (long long)tile_cap;
  a.tile_elems = o.tile_elems;
  a.carry_groups = o.carry_tiles;
  a.short_max = o.short_max;
  a.lane_max = kSegLaneMax;
  // capture prep + main into a graph on a private stream
  cudaStream_t cs;
  e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // memset done before any replay
  if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    xs_status qs = plan_enqueue(p, cs);
    cudaError_t e2 = cudaStreamEndCapture(cs, &p->graph);
    e = (qs != XS_OK) ? cudaErrorUnknown : e2;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&p->exec, p->graph, 0);
  cudaStreamDestroy(cs);
  if (e != cudaSuccess) {
    if (p->graph) cudaGraphDestroy(p->graph);
    dev_free(p->mem);
    delete p;
    return from_cuda(e);
  }
  *plan = p;
  return set_error(XS_OK);
}

xs_status xs_seg_plan_launch(xs_seg_plan p, void* stream) {
  if (p == nullptr) return set_error(XS_ERR_INVALID_POINTER);
  XS_TRY_CUDA(cudaGraphLaunch(p->exec, as_stream(stream)));
  return set_error(XS_OK);
}

xs_status xs_seg_plan_launch_direct(xs_seg_plan p, void* stream) {
  if (p == nullptr) return set_error(XS_ERR_INVALID_POINTER);
  xs_status st = plan_enqueue(p, as_stream(stream));
  if (st != XS_OK) return st;
  return set_error(XS_OK);
}

int xs_seg_plan_kernel_launches(xs_seg_plan p) { return p ? 4 : 0; }

xs_status xs_seg_plan_check(xs_seg_plan p, void* stream) {
  if (p == nullptr) return set_error(XS_ERR_INVALID_POINTER);
  unsigned long long bad = 0ull;
  cudaStream_t s = as_stream(stream);
  XS_TRY_CUDA(cudaMemcpyAsync(&bad, &p->args.counters[4], sizeof bad, cudaMemcpyDeviceToHost, s));
  XS_TRY_CUDA(cudaStreamSynchronize(s));
  return set_error(bad ? XS_ERR_INVALID_VALUE : XS_OK);
}

xs_status xs_seg_plan_destroy(xs_seg_plan p) {
  if (p == nullptr) return set_error(XS_ERR_INVALID_POINTER);
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->graph) cudaGraphDestroy(p->graph);
  dev_free(p->mem);
  delete p;
  return set_error(XS_OK);
}

}  // extern "C"

namespace {
std::mutex g_plan_mu;
std::map<std::tuple<int, const void*, const void*, int64_t, void*, void*>, xs_seg_plan> g_plans;
}  // namespace

extern "C" {

xs_status xs_sum_each_async(const double* d_values, const int64_t* h_offsets, int64_t nseg,
                            double* d_out, void* stream) {
  if (nseg < 0) return set_error(XS_ERR_INVALID_VALUE);
  if (nseg == 0) return set_error(XS_OK);
  if (h_offsets == nullptr) return set_error(XS_ERR_INVALID_POINTER);
  if (h_offsets[0] != 0) return set_error(XS_ERR_INVALID_VALUE);
  for (int64_t k = 0; k < nseg; ++k)
    if (h_offsets[k + 1] < h_offsets[k]) return set_error(XS_ERR_INVALID_VALUE);
  xs_status st;
  if ((st = check_device_ptr(d_out)) != XS_OK) return st;
  if (h_offsets[nseg] > 0 && (st = check_device_ptr(d_values)) != XS_OK) return st;
  if (((uintptr_t)d_values & 7u) || ((uintptr_t)d_out & 7u)) return set_error(XS_ERR_INVALID_VALUE);
  cudaStream_t s = as_stream(stream);
  DeviceCtx* ctx = device_ctx(&st);
  if (!ctx) return st;
  Workspace* w = workspace(ctx, s, &st);
  if (!w) return st;
  // arguments are checked once above; each segment is then one launch of the
  // single-array kernel in the shape xs_sum_async would choose for its length
  for (int64_t k = 0; k < nseg; ++k) {
    const int64_t len = h_offsets[k + 1] - h_offsets[k];
    if (len == 0) {
      XS_TRY_CUDA(cudaMemsetAsync(d_out + k, 0, sizeof(double), s));
      continue;
    }
    st = launch_sum(ctx, d_values + h_offsets[k], len, w->acc, d_out + k, 0, default_shape(ctx, len),
                    0, s);
    if (st != XS_OK) return st;
  }
  return set_error(XS_OK);
}

xs_status xs_sum_segments(const double* d_values, const int64_t* d_offsets, int64_t nseg,
                          double* d_out, void* stream) {
  if (nseg < 0) return set_error(XS_ERR_INVALID_VALUE);
  if (nseg == 0) return set_error(XS_OK);
  int dev = -1;
  XS_TRY_CUDA(cudaGetDevice(&dev));
  const auto key = std::make_tuple(dev, (const void*)d_values, (const void*)d_offsets, nseg,
                                   (void*)d_out, stream);
  xs_seg_plan p = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_plan_mu);
    auto it = g_plans.find(key);
    if (it != g_plans.end()) p = it->second;
  }
  if (p == nullptr) {
    xs_status st = xs_seg_plan_create(&p, d_values, d_offsets, nseg, d_out, nullptr, stream);
    if (st != XS_OK) return st;
    std::lock_guard<std::mutex> lk(g_plan_mu);
    g_plans[key] = p;
  }
  return xs_seg_plan_launch(p, stream);
}

xs_status xs_autotune_segments(const double* d_values, const int64_t* d_offsets, int64_t nseg,
                               double* d_out, int reps, void* stream, xs_seg_options* best,
                               float* best_us) {
  if (reps <= 0 || nseg <= 0) return set_error(XS_ERR_INVALID_VALUE);
  xs_status st;
  DeviceCtx* ctx = device_ctx(&st);
  if (!ctx) return st;
  cudaStream_t s = as_stream(stream);
  std::vector<xs_seg_options> cands;
  const int blocks[][2] = {{128, 4}, {192, 4}, {256, 4}, {384, 4}, {192, 8}, {128, 8}, {64, 8}, {32, 8}};
  const int tiles[] = {1 << 15, 1 << 16, 1 << 17, 1 << 18, 1 << 20};
  const int shorts[] = {1024, 4096, 16384};
  for (auto& b : blocks)
    for (int t : tiles)
      for (int sm : shorts) {
        cands.push_back(xs_seg_options{b[0], b[1], t, sm, 0});
        // tiles past 2040 values per thread propagate carries: try half the interval too
        if ((long long)t > 2040LL * b[0])
          cands.push_back(xs_seg_options{b[0], b[1], t, sm, seg_max_carry_groups(b[1]) / 2});
      }
  cudaEvent_t e0, e1;
  XS_TRY_CUDA(cudaEventCreate(&e0));
  XS_TRY_CUDA(cudaEventCreate(&e1));
  float bt = 1e30f;
  xs_seg_options win = cands[0];
  std::vector<float> ts;
  for (const auto& o : cands) {
    xs_seg_plan p = nullptr;
    st = xs_seg_plan_create(&p, d_values, d_offsets, nseg, d_out, &o, stream);
    if (st == XS_ERR_NOT_SUPPORTED) continue;
    if (st != XS_OK) return st;
    if ((st = xs_seg_plan_launch(p, stream)) != XS_OK) return st;  // warm-up
    ts.clear();
    for (int r = 0; r < reps; ++r) {
      XS_TRY_CUDA(cudaEventRecord(e0, s));
      if ((st = xs_seg_plan_launch(p, stream)) != XS_OK) return st;
      XS_TRY_CUDA(cudaEventRecord(e1, s));
      XS_TRY_CUDA(cudaEventSynchronize(e1));
      float ms = 0.f;
      XS_TRY_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      ts.push_back(ms);
    }
    xs_seg_plan_destroy(p);
    std::sort(ts.begin(), ts.end());
    if (ts[ts.size() / 2] < bt) {
      bt = ts[ts.size() / 2];
      win = o;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  {
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->tuned_seg = win;
    ctx->have_tuned_seg = true;
  }
  if (best) *best = win;
  if (best_us) *best_us = bt * 1000.f;
  return set_error(XS_OK);
}

}  // extern "C"

namespace xs {
// This file's debug word (xs_debug_status).
cudaError_t debug_take_segments(unsigned long long* v) { return debug_word_take(v); }
}  // namespace xs
