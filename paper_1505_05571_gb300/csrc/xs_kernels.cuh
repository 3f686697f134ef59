// Pieces shared by the single-array kernels (sum, mean, dot product, squared
// norm): launch arguments, the split of an array into 16-byte pairs, the block
// to grid merge of partial accumulators and the last-block finish.
#pragma once

#include "xs_device.cuh"

namespace xs {

struct SumArgs {
  const double* x;
  long long n;
  AccState* g;     // global accumulator: zeroed workspace, or a handle's state
  double* out;     // mode 0: result
  int mode;        // 0: round into out and reset g; 1: normalise g in place
  int carry_tiles; // small kernel: tiles between per-thread carry propagations
  int prefetch;    // tiles of this block prefetched into L2 ahead of use (0 = off)
  unsigned long long divisor;  // mode 0: 0 rounds the sum, d >= 1 rounds the sum / d
};

// Ticket epilogue: the last block to arrive finishes the sum.
// `sc`: block shared memory the finishing warp may use as scratch (the
// accumulators are no longer needed when the block reaches this point).
// The block's adds into `g` are ordered before its ticket by the barrier and
// one device-scope fence of thread 0 (the fence is cumulative over what the
// barrier made visible to it).
static __device__ void finish_grid(const SumArgs& a, long long* sc) {
  __shared__ unsigned s_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = (atomicAdd(&a.g->ticket, 1u) == gridDim.x - 1) ? 1u : 0u;
  }
  __syncthreads();
  if (!s_last || threadIdx.x >= 32) return;
  __threadfence();
  const int lane = threadIdx.x;
  unsigned long long* ch = reinterpret_cast<unsigned long long*>(a.g->chunk);
  if (a.mode == 0) {
    long long v0 = (long long)atomicExch(ch + lane, 0ull);
    long long v1 = (long long)atomicExch(ch + lane + 32, 0ull);
    long long v2 = lane < 3 ? (long long)atomicExch(ch + lane + 64, 0ull) : 0;
    unsigned flags = 0u;
    unsigned long long key = 0ull;
    if (lane == 0) {
      flags = atomicExch(&a.g->flags, 0u);
      key = atomicExch(&a.g->nan_key, 0ull);
      atomicExch(&a.g->ticket, 0u);
    }
    flags = __shfl_sync(kFull, flags, 0);
    key = __shfl_sync(kFull, key, 0);
    const unsigned long long bits = a.divisor ? warp_round_div(v0, v1, v2, flags, key, a.divisor, sc, 32)
                                              : warp_round(v0, v1, v2, flags, key, sc, 32);
    if (lane == 0) *reinterpret_cast<unsigned long long*>(a.out) = bits;
  } else {
    long long v0 = (long long)__ldcg(ch + lane);
    long long v1 = (long long)__ldcg(ch + lane + 32);
    long long v2 = lane < 3 ? (long long)__ldcg(ch + lane + 64) : 0;
    warp_normalize(v0, v1, v2, sc, 32);
    ch[lane] = (unsigned long long)v0;
    ch[lane + 32] = (unsigned long long)v1;
    if (lane < 3) ch[lane + 64] = (unsigned long long)v2;
    if (lane == 0) a.g->ticket = 0u;
  }
}

// Finish of a mode-0 sum whose blocks recorded their chunk window in g: when
// the window holds at most 9 chunks (and no division follows) the last
// block's thread 0 reads and clears just those and rounds alone
// (round_window); otherwise the warp path.
static __device__ void finish_grid_window(const SumArgs& a, long long* sc) {
  __shared__ unsigned s_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = (atomicAdd(&a.g->ticket, 1u) == gridDim.x - 1) ? 1u : 0u;
  }
  __syncthreads();
  if (!s_last || threadIdx.x >= 32) return;
  __threadfence();
  const unsigned lo_inv = *(volatile unsigned*)&a.g->win_lo_inv;
  const unsigned hi = *(volatile unsigned*)&a.g->win_hi;
  const bool empty = lo_inv == 0u && hi == 0u;
  // a term with positional exponent e touches chunks e >> 5 and (e >> 5) + 1,
  // and the block merge carries each chunk's high part one chunk further up
  const int cmin = empty ? 0 : (int)((0x7FFu - lo_inv) >> kLowExpBits);
  const int cmax = empty ? -1 : min((int)(hi >> kLowExpBits) + 2, kSChunks - 1);  // highest written
  constexpr int kWin = 8;
  if (a.divisor == 0ull && cmax - cmin <= kWin) {
    if (threadIdx.x != 0) return;
    unsigned long long* ch = reinterpret_cast<unsigned long long*>(a.g->chunk);
    long long w[kWin + 1];
#pragma unroll
    for (int k = 0; k <= kWin; ++k)
      w[k] = cmin + k <= cmax ? (long long)atomicExch(ch + cmin + k, 0ull) : 0;
    const unsigned flags = atomicExch(&a.g->flags, 0u);
    const unsigned long long key = atomicExch(&a.g->nan_key, 0ull);
    a.g->win_lo_inv = 0u;
    a.g->win_hi = 0u;
    atomicExch(&a.g->ticket, 0u);
    *reinterpret_cast<unsigned long long*>(a.out) =
        round_window(w, cmax - cmin + 1 > 0 ? cmax - cmin + 1 : 0, cmin, flags, key);
    return;
  }
  const int lane = threadIdx.x;
  unsigned long long* ch = reinterpret_cast<unsigned long long*>(a.g->chunk);
  long long v0 = (long long)atomicExch(ch + lane, 0ull);
  long long v1 = (long long)atomicExch(ch + lane + 32, 0ull);
  long long v2 = lane < 3 ? (long long)atomicExch(ch + lane + 64, 0ull) : 0;
  unsigned flags = 0u;
  unsigned long long key = 0ull;
  if (lane == 0) {
    flags = atomicExch(&a.g->flags, 0u);
    key = atomicExch(&a.g->nan_key, 0ull);
    a.g->win_lo_inv = 0u;
    a.g->win_hi = 0u;
    atomicExch(&a.g->ticket, 0u);
  }
  flags = __shfl_sync(kFull, flags, 0);
  key = __shfl_sync(kFull, key, 0);
  const unsigned long long bits = a.divisor ? warp_round_div(v0, v1, v2, flags, key, a.divisor, sc, 32)
                                            : warp_round(v0, v1, v2, flags, key, sc, 32);
  if (lane == 0) *reinterpret_cast<unsigned long long*>(a.out) = bits;
}

// Split of the input into a head of up to 31 elements before the first
// 256-byte boundary, 16-byte pairs from there on, and an optional odd tail
// element. The streamed body starts on a 256-byte boundary: measured on GB300,
// a body that starts 8 or 128 bytes past one reads 12-30 % slower (the loads'
// 256-byte L2 fetch granules and the bulk prefetch then straddle boundaries).
struct Split {
  int head;
  bool tail;
  long long npairs;
  const ulonglong2* xv;
};
__device__ __forceinline__ Split split_input(const double* x, long long n) {
  Split s;
  s.head = (int)min((long long)((256u - ((uintptr_t)x & 255u)) & 255u) / 8, n);
  const long long body = n - s.head;
  s.npairs = body >> 1;
  s.tail = (body & 1) != 0;
  s.xv = reinterpret_cast<const ulonglong2*>(x + s.head);
  return s;
}

// L2 prefetch of tile t (clamped to the input).
template <int BLOCK, int UNROLL>
__device__ __forceinline__ void prefetch_tile(const Split& sp, long long t, long long ntiles) {
  if (t >= ntiles) return;
  const long long first = t * (long long)(BLOCK * UNROLL);
  const long long cnt = min((long long)(BLOCK * UNROLL), sp.npairs - first);
  prefetch_l2(sp.xv + first, (unsigned)(cnt * 16));
}

// Block partial -> global accumulator, plus the special-value record.
template <int BLOCK>
__device__ __forceinline__ void block_small_to_global(const long long* sm, const SumArgs& a,
                                                      unsigned flags, unsigned long long nkey) {
  unsigned long long* g = reinterpret_cast<unsigned long long*>(a.g->chunk);
  block_chunk_sums<BLOCK>(sm, [&](int c, long long v) {
    if (v != 0) atomicAdd(g + c, (unsigned long long)v);
  });
  flags = __reduce_or_sync(kFull, flags);
  nkey = warp_max_ull(nkey);
  if ((threadIdx.x & 31) == 0) {
    if (flags) atomicOr(&a.g->flags, flags);
    if (nkey) atomicMax(&a.g->nan_key, nkey);
  }
}

}  // namespace xs
