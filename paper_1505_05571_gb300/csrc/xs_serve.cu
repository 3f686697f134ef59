// Serving loop: continuous batching of exact-sum requests on one GPU.
//
// Requests (one-shot sums, session appends, session finishes) queue on the
// host. A scheduler thread admits them while an accumulator slot and the byte
// budget allow, packs every admitted request into one batch, and launches the
// batch as one persistent kernel on one of `streams` CUDA streams; up to
// `streams` batches run at once, so work submitted while others are running
// joins the next batch and overlaps with them on the device.
//
// Device side, each request becomes tiles of tile_elems elements. A work group
// (one warp by default) sums a tile with per-thread small superaccumulators
// (Fig. 3) and adds its partial into the request's accumulator slot with
// integer atomics (partials add exactly, Discussion). The last tile of a slot in a batch either normalises
// the slot in place (appends: the session's exact sum stays on the device) or
// rounds it once and clears it (finishes and one-shot sums). A session never
// has two batches in flight, so its slot is only touched by one kernel at a
// time, and a batch may carry several requests of one session.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "xs_host.hpp"

namespace xs {

struct BatchItem {
  const double* x;
  long long n;
  long long tile0;     // first global tile of this item
  long long tile_len;  // values per tile: the small tile, or the block-wide tile of a long request
  int slot;            // accumulator slot
  int slot_tiles;      // tiles of all items of this slot in the batch (ticket target)
  int res_idx;         // result index written by the slot's finisher (-1: none)
  unsigned flags;      // bit 0: the slot's group ends with a finish
};

// Tiles [0, small_tiles) are the small requests' (one-warp groups), tiles
// [small_tiles, total_tiles) the long requests' (whole blocks); items are in
// tile order, so one search finds a tile's item in either range.
struct BatchHeader {
  unsigned long long cursor;      // next small tile
  unsigned long long cursor_big;  // next long tile (starts at small_tiles)
  long long small_tiles;
  long long total_tiles;
  int nitems;
  int pad;
};

struct BatchArgs {
  const BatchItem* items;
  BatchHeader* hdr;
  AccState* slots;
  unsigned long long* results;
  long long tile_elems;
};

// Launch shape: one block of 512 threads per SM. Small requests' tiles
// (2^16 values by default) go to twelve one-warp work groups of the first 384
// threads with per-thread small superaccumulators, four loads per thread; then
// the long requests' tiles (2^21 values by default) to whole blocks with one
// large superaccumulator each (four loads per thread). Measured on GB300 with
// saturated serving of Poisson requests of 1e3..1e8 values (log-uniform), the
// one-warp groups alone reach 5.1 TB/s whatever the block shape (192 or 384
// threads, 4 loads; 8 loads: 3.3-4.5 TB/s), the same with one batch in flight
// as with three.
constexpr int kServeBlock = 384;      // threads of the small-tile phase
constexpr int kServeGroup = 32;
constexpr int kServeUnroll = 4;
constexpr int kServeBigBlock = 512;   // threads of the launch and of the long-tile phase
constexpr int kServeBigUnroll = 4;
constexpr int kServeCopies = 4;
constexpr size_t kServeSmem =
    sizeof(LargePlanes<kServeBigBlock / 32, kServeCopies>) > (size_t)kServeBlock * kSChunks * sizeof(long long)
        ? sizeof(LargePlanes<kServeBigBlock / 32, kServeCopies>)
        : (size_t)kServeBlock * kSChunks * sizeof(long long);

// L2 prefetch of the 16-byte-aligned part of [p, q), in pieces of at most 64 KB.
__device__ __forceinline__ void serve_prefetch(const double* p, const double* q) {
  uintptr_t b0 = ((uintptr_t)p + 15u) & ~(uintptr_t)15u;
  const uintptr_t b1 = (uintptr_t)q & ~(uintptr_t)15u;
  while (b0 < b1) {
    const uintptr_t n = min(b1 - b0, (uintptr_t)65536u);
    prefetch_l2((const void*)b0, (unsigned)n);
    b0 += n;
  }
}

// Last tile of a slot in a batch, one warp: round the slot once and clear it
// (a finish or a one-shot sum) or keep its exact sum in canonical form (an
// append). sc: 67 words of shared scratch.
__device__ __forceinline__ void serve_slot_finish(const BatchArgs& a, const BatchItem& it, AccState* g,
                                                  long long* sc) {
  const int lane = threadIdx.x & 31;
  unsigned long long* gc = reinterpret_cast<unsigned long long*>(g->chunk);
  __threadfence();
  if (it.flags & 1u) {  // round once and clear the slot
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
    const unsigned long long r = warp_round(v0, v1, v2, fl, key, sc, 32);
    if (lane == 0 && it.res_idx >= 0) a.results[it.res_idx] = r;
  } else {  // keep the exact sum, in canonical form
    long long v0 = (long long)__ldcg(gc + lane);
    long long v1 = (long long)__ldcg(gc + lane + 32);
    long long v2 = lane < 3 ? (long long)__ldcg(gc + lane + 64) : 0;
    warp_normalize(v0, v1, v2, sc, 32);
    gc[lane] = (unsigned long long)v0;
    gc[lane + 32] = (unsigned long long)v1;
    if (lane < 3) gc[lane + 64] = (unsigned long long)v2;
    if (lane == 0) g->ticket = 0u;
  }
}

// The small tiles [0, small_tiles), by the first BLOCK threads of the block
// (BLOCK / W independent work groups, each of which claims tiles on its own:
// one warp by default, so a group's tiles end without waiting at a barrier
// for its slowest warp). smem_srv holds the BLOCK threads' accumulators.
template <int BLOCK, int W, int UNROLL, bool WHOLE_BLOCK>
__device__ __forceinline__ void serve_small_tiles(const BatchArgs& a, long long* smem_srv) {
  static_assert(W >= 32 && W % 32 == 0 && BLOCK % W == 0, "whole warps per group");
  constexpr int NG = BLOCK / W;
  // the thread that claims the next tile: warp 1 of the group, beside warp 0's
  // rounding; lane 0 when the group is one warp
  constexpr int kClaimer = W > 32 ? 32 : 0;
  // load groups between carry propagations inside a tile longer than 2040
  // values per thread (at most 2045 adds per thread with head, tail and padding)
  constexpr int kCarryGroups = (kCarryInterval - 4 - 2 * UNROLL) / (2 * UNROLL);
  __shared__ long long g_sc[NG][kSChunks];  // rounding scratch
  __shared__ long long g_tile[NG];
  __shared__ int g_item[NG];
  __shared__ unsigned g_flags[NG], g_last[NG], g_emin[NG], g_emax[NG];
  __shared__ unsigned long long g_nkey[NG];
  const int tid = threadIdx.x, lane = tid & 31;
  const int grp = tid / W, gt = tid - grp * W, gwarp = gt >> 5;  // group, rank and warp in it
  long long* sc = g_sc[grp];
  long long& s_tile = g_tile[grp];
  int& s_item = g_item[grp];
  unsigned& s_flags = g_flags[grp];
  unsigned& s_last = g_last[grp];
  unsigned& s_emin = g_emin[grp];
  unsigned& s_emax = g_emax[grp];
  unsigned long long& s_nkey = g_nkey[grp];
  // barrier of the group (a warp's own when the group is one warp, else named
  // barrier 1 + group)
  auto gsync = [&]() {
    if (W == 32) __syncwarp();
    else if (NG == 1 && WHOLE_BLOCK) __syncthreads();
    else asm volatile("bar.sync %0, %1;" ::"r"(1 + grp), "r"(W) : "memory");
  };
  SmallThread T;
  T.acc = smem_srv + tid;
  // Accumulators are cleared once and every merge clears the window of
  // chunks it read, so they are zero whenever a tile starts.
  for (int c = 0; c < kSChunks; ++c) T.acc[c * BLOCK] = 0;
  const long long total = a.hdr->small_tiles;
  const int nitems = a.hdr->nitems;
  // the last item with tile0 <= t
  auto item_of = [&](long long t) -> int {
    int lo_i = 0, hi_i = nitems;
    while (hi_i - lo_i > 1) {
      const int mid = (lo_i + hi_i) >> 1;
      if (a.items[mid].tile0 <= t) lo_i = mid; else hi_i = mid;
    }
    return lo_i;
  };
  // The next tile is claimed and located while the group merges the current
  // one, and its start is prefetched into L2.
  if (gt == 0) {
    s_tile = (long long)atomicAdd(&a.hdr->cursor, 1ull);
    if (s_tile < total) s_item = item_of(s_tile);
  }
  for (;;) {
    if (gt == 0) {
      s_flags = 0u;
      s_nkey = 0ull;
      s_emin = 0x7FFu;
      s_emax = 0u;
    }
    gsync();
    const long long t = s_tile;
    if (t >= total) break;
    const BatchItem it = a.items[s_item];
    const long long first = (t - it.tile0) * it.tile_len;
    const long long end = min(first + it.tile_len, it.n);
    T.reset();
    if (first < end)
      accumulate_range<BLOCK, UNROLL, true, true>(T, it.x, first, end, gt, W, kCarryGroups);
    {
      const unsigned wmin = __reduce_min_sync(kFull, T.emin);
      const unsigned wmax = __reduce_max_sync(kFull, T.emax);
      if (lane == 0 && wmax >= wmin) {
        atomicMin(&s_emin, wmin);
        atomicMax(&s_emax, wmax);
      }
    }
    gsync();  // every thread has read s_tile and s_item; the window is complete
    if (gt == kClaimer) s_tile = (long long)atomicAdd(&a.hdr->cursor, 1ull);
    const int cmin = (int)(s_emin >> kLowExpBits);
    const int cmax = s_emax >= s_emin ? (int)(s_emax >> kLowExpBits) + 1 : cmin - 1;  // empty
    unsigned f = __reduce_or_sync(kFull, T.flags());
    const unsigned long long k = warp_max_ull(T.nkey);
    if (lane == 0) {
      if (f) atomicOr(&s_flags, f);
      if (k) atomicMax(&s_nkey, k);
    }
    AccState* g = a.slots + it.slot;
    unsigned long long* gc = reinterpret_cast<unsigned long long*>(g->chunk);
    group_chunk_sums<BLOCK, W>(smem_srv + grp * W, gwarp, [&](int c, long long v) {
      if (v != 0) atomicAdd(gc + c, (unsigned long long)v);
    }, cmin, cmax);
    gsync();
    for (int c = cmin; c <= cmax; ++c) T.acc[c * BLOCK] = 0;
    if (gt == 0) {
      unsigned fl = s_flags | ((it.n > 0 && t == it.tile0) ? kFlagAny : 0u);
      if (fl) atomicOr(&g->flags, fl);
      if (s_nkey) atomicMax(&g->nan_key, s_nkey);
      __threadfence();
      s_last = (atomicAdd(&g->ticket, 1u) == (unsigned)(it.slot_tiles - 1)) ? 1u : 0u;
    }
    gsync();
    if (s_last && gwarp == 0) serve_slot_finish(a, it, g, sc);
    if (gt == kClaimer) {  // where the next tile lies, and its start into L2
      const long long tn = s_tile;
      if (tn < total) {
        const int in = item_of(tn);
        s_item = in;
        const BatchItem& nx = a.items[in];
        const long long nf = (tn - nx.tile0) * nx.tile_len;
        const long long ne = min(min(nf + nx.tile_len, nx.n), nf + 48LL * W);
        if (nf < ne) serve_prefetch(nx.x + nf, nx.x + ne);
      }
    }
    gsync();
  }
}

// A batch: first the small tiles, by the first 384 threads (the other warps
// wait at the barrier), then the long tiles, each by the whole block with one
// large superaccumulator in the same shared memory (Large, Fig. 4): the block
// adds the tile into the planes, flushes them into a 67-chunk partial
// (clearing them for the next tile), adds that into the request's slot and
// takes a ticket; the slot's last tile finishes it as above.
template <int UNROLL>
__global__ void __launch_bounds__(kServeBigBlock, 1) k_serve(BatchArgs a) {
  constexpr int NW = kServeBigBlock / 32;
  extern __shared__ __align__(16) long long smem_srv[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid < kServeBlock) serve_small_tiles<kServeBlock, kServeGroup, kServeUnroll, false>(a, smem_srv);
  const long long total = a.hdr->total_tiles;
  if (a.hdr->small_tiles >= total) return;  // no long tile in this batch (uniform)
  __syncthreads();  // the small tiles' shared memory is free
  LargePlanes<NW, kServeCopies>& P = *reinterpret_cast<LargePlanes<NW, kServeCopies>*>(smem_srv);
  __shared__ long long b_sum[kSChunks];  // rounding scratch of a slot's finish
  __shared__ long long b_tile, b_next_tile;
  __shared__ int b_item, b_next_item;
  __shared__ unsigned b_flags;
  __shared__ unsigned long long b_nkey;
  constexpr int kClaimer = 32;  // warp 1 claims the next tile while its block adds the current one
  large_init(P, tid, kServeBigBlock);
  const LargeLane L = large_lane(P);
  const int nitems = a.hdr->nitems;
  auto item_of = [&](long long t) -> int {  // the last item with tile0 <= t
    int lo_i = 0, hi_i = nitems;
    while (hi_i - lo_i > 1) {
      const int mid = (lo_i + hi_i) >> 1;
      if (a.items[mid].tile0 <= t) lo_i = mid; else hi_i = mid;
    }
    return lo_i;
  };
  if (tid == 0) {
    b_tile = (long long)atomicAdd(&a.hdr->cursor_big, 1ull);
    if (b_tile < total) b_item = item_of(b_tile);
    b_flags = 0u;
    b_nkey = 0ull;
  }
  __syncthreads();
  // Three barriers per tile: after the adds, after the flush, and after the
  // partial has gone into the slot. The next tile is claimed and located, and
  // its start prefetched, while the block adds the current one; the slot's
  // ticket and its finish run in warp 0 while the other warps start the next
  // tile.
  for (;;) {
    const long long t = b_tile;
    if (t >= total) break;
    const BatchItem it = a.items[b_item];
    if (tid == kClaimer) {
      const long long tn = (long long)atomicAdd(&a.hdr->cursor_big, 1ull);
      b_next_tile = tn;
      if (tn < total) {
        const int in = item_of(tn);
        b_next_item = in;
        const BatchItem& nx = a.items[in];
        const long long nf = (tn - nx.tile0) * nx.tile_len;
        const long long ne = min(min(nf + nx.tile_len, nx.n), nf + 48LL * kServeBigBlock);
        if (nf < ne) serve_prefetch(nx.x + nf, nx.x + ne);
      }
    }
    const long long first = (t - it.tile0) * it.tile_len;
    const long long end = min(first + it.tile_len, it.n);
    LargeThread T;
    if (first < end) large_range<kServeBigBlock, UNROLL>(L, T, it.x, first, end, tid);
    {
      const unsigned zp = __reduce_add_sync(kFull, T.zpos);
      const unsigned zn = __reduce_add_sync(kFull, T.zneg);
      const unsigned f = __reduce_or_sync(kFull, T.flags());
      const unsigned long long key = warp_max_ull(T.nkey);
      if (lane == 0) {
        if (zp) atomicAdd(&P.zeros[0], zp);
        if (zn) atomicAdd(&P.zeros[1], zn);
        if (f) atomicOr(&b_flags, f);
        if (key) atomicMax(&b_nkey, key);
      }
    }
    __syncthreads();  // every add is done
    large_flush<NW, kServeCopies, true>(P);
    __syncthreads();  // every run is flushed (and its planes cleared)
    AccState* g = a.slots + it.slot;
    unsigned long long* gc = reinterpret_cast<unsigned long long*>(g->chunk);
    if (tid < kSChunks) {
      long long v = 0;
#pragma unroll
      for (int w = 0; w < NW; ++w) {
        v += P.part[w][tid];
        P.part[w][tid] = 0;
      }
      if (v != 0) atomicAdd(gc + tid, (unsigned long long)v);
    }
    if (tid < 2) P.zeros[tid] = 0u;
    unsigned fl = 0u;
    unsigned long long nk = 0ull;
    if (tid == 0) {  // this tile's record, then the next tile becomes current
      fl = b_flags | ((it.n > 0 && t == it.tile0) ? kFlagAny : 0u);
      nk = b_nkey;
      b_flags = 0u;
      b_nkey = 0ull;
      b_tile = b_next_tile;
      b_item = b_next_item;
    }
    __syncthreads();  // the partial is in the slot; the next tile is current
    if (warp == 0) {
      unsigned last = 0u;
      if (lane == 0) {
        if (fl) atomicOr(&g->flags, fl);
        if (nk) atomicMax(&g->nan_key, nk);
        __threadfence();
        last = (atomicAdd(&g->ticket, 1u) == (unsigned)(it.slot_tiles - 1)) ? 1u : 0u;
      }
      if (__shfl_sync(kFull, last, 0)) serve_slot_finish(a, it, g, b_sum);
    }
  }
}

// Rounded value of a session accumulator (normalised, state left unchanged),
// for the serial baseline. One warp.
__global__ void k_serial_round(const AccState* acc, double* out) {
  __shared__ long long sc[kSChunks];
  const int lane = threadIdx.x;
  const long long v0 = acc->chunk[lane];
  const long long v1 = acc->chunk[lane + 32];
  const long long v2 = lane < 3 ? acc->chunk[lane + 64] : 0;
  const unsigned long long bits = warp_round(v0, v1, v2, acc->flags, acc->nan_key, sc, 32);
  if (lane == 0) *reinterpret_cast<unsigned long long*>(out) = bits;
}

namespace {

using Clock = std::chrono::steady_clock;
constexpr double kNaN = __builtin_nan("");

struct Request {
  uint64_t id = 0;
  uint64_t session = 0;
  const double* x = nullptr;
  int64_t n = 0;
  bool finish = false;
  int slot = -1;
  int64_t t_submit = 0, t_admit = 0, t_launch = 0, t_done = 0;
  int32_t status = XS_ERR_NOT_READY;
  double value = kNaN;
};

struct Session {
  int slot = -1;
  bool finish_submitted = false;
  bool busy = false;  // a batch holding its requests is in flight
};

struct BatchSlot {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  void* d_mem = nullptr;  // header | items | results
  void* h_mem = nullptr;  // pinned mirror
  BatchHeader* d_hdr = nullptr;
  BatchItem* d_items = nullptr;
  unsigned long long* d_results = nullptr;
  BatchHeader* h_hdr = nullptr;
  BatchItem* h_items = nullptr;
  unsigned long long* h_results = nullptr;
  std::vector<Request*> reqs;
  std::vector<uint64_t> sessions;
  bool busy = false;
};

}  // namespace

}  // namespace xs

using namespace xs;

struct xs_server_s {
  int device = -1;
  xs_server_options opt{};
  int grid = 0;
  AccState* d_slots = nullptr;
  std::vector<int> free_slots;
  std::mutex mu;
  std::condition_variable cv_sched;
  std::condition_variable cv_done;
  std::deque<Request*> pending;
  std::unordered_map<uint64_t, Request*> reqs;
  std::unordered_map<uint64_t, Session> sessions;
  int64_t budget_free = 0;
  std::vector<BatchSlot> batches;
  std::thread thr;
  bool stop = false;
  uint64_t next_id = 1, next_session = 1;
  Clock::time_point t0;
  xs_server_stats st{};

  int64_t now() const {
    return std::chrono::duration_cast<std::chrono::nanoseconds>(Clock::now() - t0).count();
  }
  void loop();
  std::vector<Request*> admit_locked();
  void launch(BatchSlot& b);
  void complete_locked(BatchSlot& b, bool ok);
};

std::vector<Request*> xs_server_s::admit_locked() {
  std::vector<Request*> out;
  std::unordered_set<uint64_t> blocked;  // sessions whose earlier request must go first
  for (auto it = pending.begin(); it != pending.end() && (int)out.size() < opt.max_batch;) {
    Request* r = *it;
    if (r->session != 0) {
      Session& S = sessions[r->session];
      if (S.busy || blocked.count(r->session)) {
        blocked.insert(r->session);
        ++it;
        continue;
      }
    }
    const int64_t need = r->n * 8 + (r->session == 0 ? (int64_t)sizeof(AccState) : 0);
    if (need > budget_free || (r->session == 0 && free_slots.empty())) {
      if (r->session != 0) blocked.insert(r->session);
      ++it;
      continue;
    }
    budget_free -= need;
    if (r->session == 0) {
      r->slot = free_slots.back();
      free_slots.pop_back();
    } else {
      r->slot = sessions[r->session].slot;
    }
    r->t_admit = now();
    out.push_back(r);
    it = pending.erase(it);
  }
  return out;
}

void xs_server_s::launch(BatchSlot& b) {
  // groups: the requests of one slot, in submission order; smallest groups first
  std::map<int, std::vector<int>> by_slot;
  for (int k = 0; k < (int)b.reqs.size(); ++k) by_slot[b.reqs[k]->slot].push_back(k);
  std::vector<std::pair<int64_t, int>> order;
  for (auto& kv : by_slot) {
    int64_t tot = 0;
    for (int k : kv.second) tot += b.reqs[k]->n;
    order.push_back({tot, kv.first});
  }
  std::sort(order.begin(), order.end());
  // Small requests' tiles first (smallest groups first, so they finish early),
  // then long requests' block-wide tiles (largest groups first); a slot's
  // ticket counts both kinds.
  const long long te = opt.tile_elems, lt = opt.long_tile;
  auto is_long = [&](const Request* r) { return r->n >= (int64_t)opt.long_min; };
  // Long requests' tiles: long_tile values, unless the batch's long requests
  // then make fewer tiles than there are blocks (a light load); the tiles are
  // then shortened (to at least 2^16 values, a multiple of 4096) so that the
  // batch still spreads over every block, and a lone mid-size request is not
  // one block's work.
  long long long_values = 0, long_tiles_full = 0;
  for (const Request* r : b.reqs)
    if (is_long(r)) {
      long_values += r->n;
      long_tiles_full += (r->n + lt - 1) / lt;
    }
  long long long_len = lt;
  if (long_tiles_full < grid && long_values > 0) {
    const long long want = ((long_values + grid - 1) / grid + 4095) / 4096 * 4096;
    long_len = std::min(lt, std::max<long long>(std::min<long long>(lt, 1 << 16), want));
  }
  auto len_of = [&](const Request* r) -> long long { return is_long(r) ? long_len : te; };
  auto tiles_of = [&](const Request* r) {
    const long long len = len_of(r);
    return std::max<long long>(1, (r->n + len - 1) / len);
  };
  long long tile0 = 0;
  int ni = 0;
  long long small_tiles = 0;
  for (int pass = 0; pass < 2; ++pass) {
    // long tiles of the largest groups first, so the batch does not end on
    // one large request that few blocks are left to share
    if (pass == 1) std::reverse(order.begin(), order.end());
    for (auto& o : order) {
      const std::vector<int>& g = by_slot[o.second];
      int slot_tiles = 0;
      for (int k : g) slot_tiles += (int)tiles_of(b.reqs[k]);
      const bool fin = b.reqs[g.back()]->finish;
      for (int k : g) {
        const Request* r = b.reqs[k];
        if (is_long(r) != (pass == 1)) continue;
        BatchItem& it = b.h_items[ni++];
        it.x = r->x;
        it.n = r->n;
        it.tile0 = tile0;
        it.tile_len = len_of(r);
        it.slot = r->slot;
        it.slot_tiles = slot_tiles;
        it.res_idx = fin ? g.back() : -1;
        it.flags = fin ? 1u : 0u;
        tile0 += tiles_of(r);
      }
    }
    if (pass == 0) small_tiles = tile0;
  }
  b.h_hdr->cursor = 0ull;
  b.h_hdr->cursor_big = (unsigned long long)small_tiles;
  b.h_hdr->small_tiles = small_tiles;
  b.h_hdr->total_tiles = tile0;
  b.h_hdr->nitems = ni;
  const size_t bytes = sizeof(BatchHeader) + (size_t)ni * sizeof(BatchItem);
  cudaError_t e = cudaMemcpyAsync(b.d_mem, b.h_mem, bytes, cudaMemcpyHostToDevice, b.stream);
  BatchArgs a;
  a.items = b.d_items;
  a.hdr = b.d_hdr;
  a.slots = d_slots;
  a.results = b.d_results;
  a.tile_elems = te;
  const long long g = std::max<long long>(1, std::min<long long>(grid, tile0));
  if (e == cudaSuccess) {
    k_serve<kServeBigUnroll><<<(unsigned)g, kServeBigBlock, kServeSmem, b.stream>>>(a);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b.h_results, b.d_results, b.reqs.size() * sizeof(unsigned long long),
                        cudaMemcpyDeviceToHost, b.stream);
  if (e == cudaSuccess) e = cudaEventRecord(b.done, b.stream);
  const int64_t tl = now();
  std::lock_guard<std::mutex> lk(mu);
  for (Request* r : b.reqs) r->t_launch = tl;
  if (e != cudaSuccess) {
    cudaGetLastError();
    complete_locked(b, false);
  }
}

void xs_server_s::complete_locked(BatchSlot& b, bool ok) {
  const int64_t td = now();
  for (int k = 0; k < (int)b.reqs.size(); ++k) {
    Request* r = b.reqs[k];
    r->t_done = td;
    r->status = ok ? XS_OK : XS_ERR_CUDA;
    if (r->finish && ok) std::memcpy(&r->value, &b.h_results[k], sizeof(double));
    budget_free += r->n * 8;
    if (r->session == 0) {
      budget_free += (int64_t)sizeof(AccState);
      free_slots.push_back(r->slot);
    } else if (r->finish) {
      auto it = sessions.find(r->session);
      if (it != sessions.end()) {
        free_slots.push_back(it->second.slot);
        budget_free += (int64_t)sizeof(AccState);
        sessions.erase(it);
        st.open_sessions--;
      }
    }
    st.completed++;
    st.bytes_done += r->n * 8;
    st.in_flight_bytes -= r->n * 8;
  }
  for (uint64_t s : b.sessions) {
    auto it = sessions.find(s);
    if (it != sessions.end()) it->second.busy = false;
  }
  b.reqs.clear();
  b.sessions.clear();
  b.busy = false;
  cv_done.notify_all();
}

void xs_server_s::loop() {
  cudaSetDevice(device);
  std::unique_lock<std::mutex> lk(mu);
  for (;;) {
    bool progress = false;
    for (BatchSlot& b : batches) {
      if (!b.busy) continue;
      const cudaError_t q = cudaEventQuery(b.done);
      if (q == cudaErrorNotReady) continue;
      if (q != cudaSuccess) cudaGetLastError();
      complete_locked(b, q == cudaSuccess);
      progress = true;
    }
    for (BatchSlot& b : batches) {
      if (b.busy || pending.empty()) continue;
      std::vector<Request*> adm = admit_locked();
      if (adm.empty()) break;
      b.reqs = adm;
      b.busy = true;
      for (Request* r : adm) {
        if (r->session != 0) {
          Session& S = sessions[r->session];
          if (!S.busy) b.sessions.push_back(r->session);
          S.busy = true;
        }
        st.in_flight_bytes += r->n * 8;
      }
      st.batches++;
      st.queued = (int64_t)pending.size();
      lk.unlock();
      launch(b);
      lk.lock();
      progress = true;
    }
    bool any_busy = false;
    for (BatchSlot& b : batches) any_busy = any_busy || b.busy;
    if (stop && pending.empty() && !any_busy) break;
    if (!progress) {
      if (any_busy) {
        cv_sched.wait_for(lk, std::chrono::microseconds(20));
      } else {
        cv_sched.wait(lk, [&] { return stop || !pending.empty(); });
      }
    }
  }
}

extern "C" {

xs_status xs_server_create(xs_server* out, const xs_server_options* opts) {
  if (out == nullptr) return set_error(XS_ERR_INVALID_POINTER);
  xs_status st;
  DeviceCtx* ctx = device_ctx(&st);
  if (!ctx) return st;
  xs_server_options o{};
  if (opts) o = *opts;
  if (o.budget_bytes == 0) o.budget_bytes = int64_t(40) << 30;
  if (o.max_sessions == 0) o.max_sessions = 4096;
  if (o.streams == 0) o.streams = 3;
  if (o.max_batch == 0) o.max_batch = 256;
  if (o.tile_elems == 0) o.tile_elems = 1 << 16;
  // measured on GB300, saturated serving of requests of 1e3..1e8 values: long
  // requests from 2^18 values in tiles of 2^21, 6.56 TB/s (2^20 from 2^20:
  // 6.43; tiles of 2^19: 6.23; of 2^22: 6.57)
  if (o.long_min == 0) o.long_min = 1 << 18;
  if (o.long_tile == 0) o.long_tile = 1 << 21;
  // a long tile's sums of significands stay below 2^79 per chunk (the planes hold 96 bits)
  if (o.budget_bytes < 0 || o.max_sessions < 1 || o.streams < 1 || o.streams > 16 ||
      o.max_batch < 1 || o.tile_elems < 2 * kServeGroup || o.tile_elems > (1 << 26) || o.long_min < 0 ||
      o.long_tile < 2 * kServeBigBlock || o.long_tile > (1 << 26))
    return set_error(XS_ERR_INVALID_VALUE);
  xs_server s = new xs_server_s();
  s->device = ctx->device;
  s->opt = o;
  s->budget_free = o.budget_bytes;
  s->t0 = Clock::now();
  auto fail = [&](cudaError_t e) {
    for (BatchSlot& b : s->batches) {
      if (b.stream) cudaStreamDestroy(b.stream);
      if (b.done) cudaEventDestroy(b.done);
      dev_free(b.d_mem);
      host_free(b.h_mem);
    }
    dev_free(s->d_slots);
    delete s;
    return from_cuda(e);
  };
  cudaError_t e = cudaFuncSetAttribute(k_serve<kServeBigUnroll>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kServeSmem);
  int occ = 0;
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_serve<kServeBigUnroll>, kServeBigBlock, kServeSmem);
  if (e != cudaSuccess) return fail(e);
  s->grid = ctx->num_sms * std::max(1, occ);
  e = dev_alloc(&s->d_slots, (size_t)o.max_sessions * sizeof(AccState));
  if (e == cudaSuccess) e = cudaMemset(s->d_slots, 0, (size_t)o.max_sessions * sizeof(AccState));
  if (e != cudaSuccess) return fail(e);
  for (int k = o.max_sessions - 1; k >= 0; --k) s->free_slots.push_back(k);
  s->batches.resize(o.streams);
  const size_t items_bytes = (size_t)o.max_batch * sizeof(BatchItem);
  const size_t res_bytes = (size_t)o.max_batch * sizeof(unsigned long long);
  const size_t total = sizeof(BatchHeader) + items_bytes + res_bytes;
  for (BatchSlot& b : s->batches) {
    e = cudaStreamCreateWithFlags(&b.stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b.done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = dev_alloc(&b.d_mem, total);
    if (e == cudaSuccess) e = host_alloc(&b.h_mem, total, cudaHostAllocDefault);
    if (e != cudaSuccess) return fail(e);
    char* d = static_cast<char*>(b.d_mem);
    char* h = static_cast<char*>(b.h_mem);
    b.d_hdr = reinterpret_cast<BatchHeader*>(d);
    b.d_items = reinterpret_cast<BatchItem*>(d + sizeof(BatchHeader));
    b.d_results = reinterpret_cast<unsigned long long*>(d + sizeof(BatchHeader) + items_bytes);
    b.h_hdr = reinterpret_cast<BatchHeader*>(h);
    b.h_items = reinterpret_cast<BatchItem*>(h + sizeof(BatchHeader));
    b.h_results = reinterpret_cast<unsigned long long*>(h + sizeof(BatchHeader) + items_bytes);
  }
  s->thr = std::thread([s] { s->loop(); });
  *out = s;
  return set_error(XS_OK);
}

xs_status xs_server_open_session(xs_server s, uint64_t* session) {
  if (s == nullptr || session == nullptr) return set_error(XS_ERR_INVALID_POINTER);
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->free_slots.empty() || s->budget_free < (int64_t)sizeof(AccState))
    return set_error(XS_ERR_BUDGET);
  Session S;
  S.slot = s->free_slots.back();
  s->free_slots.pop_back();
  s->budget_free -= (int64_t)sizeof(AccState);
  const uint64_t id = s->next_session++;
  s->sessions[id] = S;
  s->st.open_sessions++;
  *session = id;
  return set_error(XS_OK);
}

xs_status xs_server_submit(xs_server s, const xs_request* r, uint64_t* request_id) {
  if (s == nullptr || r == nullptr || request_id == nullptr) return set_error(XS_ERR_INVALID_POINTER);
  if (r->n < 0) return set_error(XS_ERR_INVALID_VALUE);
  if (r->n > 0) {
    if (((uintptr_t)r->d_values & 7u) != 0u) return set_error(XS_ERR_INVALID_VALUE);
    const xs_status st = check_device_ptr(r->d_values);
    if (st != XS_OK) return st;
  }
  const int64_t need = r->n * 8 + (r->session == 0 ? (int64_t)sizeof(AccState) : 0);
  if (need > s->opt.budget_bytes) return set_error(XS_ERR_BUDGET);
  Request* q = new Request();
  q->session = r->session;
  q->x = r->d_values;
  q->n = r->n;
  q->finish = (r->session == 0) || (r->flags & XS_REQ_FINISH);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (r->session != 0) {
      auto it = s->sessions.find(r->session);
      if (it == s->sessions.end() || it->second.finish_submitted) {
        delete q;
        return set_error(XS_ERR_INVALID_VALUE);
      }
      if (q->finish) it->second.finish_submitted = true;
    }
    q->id = s->next_id++;
    q->t_submit = s->now();
    s->pending.push_back(q);
    s->reqs[q->id] = q;
    s->st.submitted++;
    s->st.queued = (int64_t)s->pending.size();
    *request_id = q->id;
  }
  s->cv_sched.notify_one();
  return set_error(XS_OK);
}

static void fill_result(const Request* q, xs_result* out) {
  out->status = q->status;
  out->reserved = 0;
  out->value = q->value;
  out->t_submit_ns = q->t_submit;
  out->t_admit_ns = q->t_admit;
  out->t_launch_ns = q->t_launch;
  out->t_done_ns = q->t_done;
}

xs_status xs_server_poll(xs_server s, uint64_t request_id, xs_result* out) {
  if (s == nullptr || out == nullptr) return set_error(XS_ERR_INVALID_POINTER);
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(request_id);
  if (it == s->reqs.end()) return set_error(XS_ERR_INVALID_VALUE);
  fill_result(it->second, out);
  return set_error(XS_OK);
}

xs_status xs_server_wait(xs_server s, uint64_t request_id, int64_t timeout_ns, xs_result* out) {
  if (s == nullptr || out == nullptr) return set_error(XS_ERR_INVALID_POINTER);
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(request_id);
  if (it == s->reqs.end()) return set_error(XS_ERR_INVALID_VALUE);
  Request* q = it->second;
  auto done = [&] { return q->status != XS_ERR_NOT_READY; };
  if (timeout_ns < 0) {
    s->cv_done.wait(lk, done);
  } else if (!s->cv_done.wait_for(lk, std::chrono::nanoseconds(timeout_ns), done)) {
    fill_result(q, out);
    return set_error(XS_ERR_TIMEOUT);
  }
  fill_result(q, out);
  return set_error(XS_OK);
}

xs_status xs_server_stats_get(xs_server s, xs_server_stats* out) {
  if (s == nullptr || out == nullptr) return set_error(XS_ERR_INVALID_POINTER);
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->st;
  out->queued = (int64_t)s->pending.size();
  return set_error(XS_OK);
}

xs_status xs_server_replay(xs_server s, const xs_replay_item* items, int64_t count,
                           uint64_t* request_ids, int64_t* start_ns) {
  if (s == nullptr || (count > 0 && (items == nullptr || request_ids == nullptr)))
    return set_error(XS_ERR_INVALID_POINTER);
  if (count < 0) return set_error(XS_ERR_INVALID_VALUE);
  std::unordered_map<uint64_t, uint64_t> open;  // tag -> session id
  const Clock::time_point t_start = Clock::now();
  if (start_ns) *start_ns = s->now();
  for (int64_t k = 0; k < count; ++k) {
    const xs_replay_item& it = items[k];
    const Clock::time_point due = t_start + std::chrono::nanoseconds(it.t_ns);
    for (;;) {  // sleep while far, spin for the last stretch
      const auto left = due - Clock::now();
      if (left <= std::chrono::nanoseconds(0)) break;
      if (left > std::chrono::microseconds(200)) std::this_thread::sleep_for(left / 2);
    }
    xs_request r{};
    r.d_values = it.d_values;
    r.n = it.n;
    r.flags = it.flags;
    if (it.session_tag != 0) {
      auto o = open.find(it.session_tag);
      if (o == open.end()) {
        uint64_t sid = 0;
        const Clock::time_point give_up = Clock::now() + std::chrono::seconds(60);
        for (;;) {
          const xs_status st = xs_server_open_session(s, &sid);
          if (st == XS_OK) break;
          if (st != XS_ERR_BUDGET || Clock::now() > give_up)
            return set_error(st == XS_ERR_BUDGET ? XS_ERR_TIMEOUT : st);
          std::this_thread::sleep_for(std::chrono::microseconds(20));
        }
        o = open.emplace(it.session_tag, sid).first;
      }
      r.session = o->second;
      if (it.flags & XS_REQ_FINISH) {
        const uint64_t sid = o->second;
        open.erase(o);
        r.session = sid;
      }
    }
    const xs_status st = xs_server_submit(s, &r, &request_ids[k]);
    if (st != XS_OK) return st;
  }
  return set_error(XS_OK);
}

xs_status xs_serial_replay(const xs_replay_item* items, int64_t count, double* h_values,
                           int64_t* done_ns, void* stream) {
  if (count < 0) return set_error(XS_ERR_INVALID_VALUE);
  if (count > 0 && (items == nullptr || h_values == nullptr || done_ns == nullptr))
    return set_error(XS_ERR_INVALID_POINTER);
  xs_status st;
  cudaStream_t s = as_stream(stream);
  DeviceCtx* ctx = device_ctx(&st);
  if (!ctx) return st;
  Workspace* w = workspace(ctx, s, &st);
  if (!w) return st;
  std::unordered_map<uint64_t, AccState*> open;  // session tag -> its accumulator
  auto release = [&]() {
    for (auto& kv : open) dev_free(kv.second);
    open.clear();
  };
  const Clock::time_point t0 = Clock::now();
  unsigned long long nan_bits = 0x7FF8000000000000ull;
  for (int64_t k = 0; k < count; ++k) {
    const xs_replay_item& it = items[k];
    std::memcpy(&h_values[k], &nan_bits, sizeof(double));
    if (it.n < 0) {
      release();
      return set_error(XS_ERR_INVALID_VALUE);
    }
    if (it.session_tag == 0) {  // a one-shot sum: one kernel, then wait for its result
      st = xs_sum_ex(it.d_values, it.n, stream, &h_values[k]);
      if (st != XS_OK) {
        release();
        return st;
      }
    } else {
      auto o = open.find(it.session_tag);
      if (o == open.end()) {
        AccState* a = nullptr;
        cudaError_t e = dev_alloc(&a, sizeof(AccState));
        if (e == cudaSuccess) e = cudaMemsetAsync(a, 0, sizeof(AccState), s);
        if (e != cudaSuccess) {
          dev_free(a);
          release();
          return from_cuda(e);
        }
        o = open.emplace(it.session_tag, a).first;
      }
      if (it.n > 0) {
        st = launch_sum(ctx, it.d_values, it.n, o->second, nullptr, 1, default_shape(ctx, it.n), 0, s);
        if (st != XS_OK) {
          release();
          return st;
        }
      }
      if (it.flags & XS_REQ_FINISH) {
        k_serial_round<<<1, 32, 0, s>>>(o->second, w->h_out_dev);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
          release();
          return from_cuda(e);
        }
        h_values[k] = *static_cast<volatile double*>(w->h_out);
        dev_free(o->second);
        open.erase(o);
      } else {
        const cudaError_t e = cudaStreamSynchronize(s);  // one request at a time
        if (e != cudaSuccess) {
          release();
          return from_cuda(e);
        }
      }
    }
    done_ns[k] = std::chrono::duration_cast<std::chrono::nanoseconds>(Clock::now() - t0).count();
  }
  release();
  return set_error(XS_OK);
}

xs_status xs_server_destroy(xs_server s) {
  if (s == nullptr) return set_error(XS_ERR_INVALID_POINTER);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_sched.notify_all();
  if (s->thr.joinable()) s->thr.join();
  for (BatchSlot& b : s->batches) {
    cudaStreamSynchronize(b.stream);
    cudaStreamDestroy(b.stream);
    cudaEventDestroy(b.done);
    dev_free(b.d_mem);
    host_free(b.h_mem);
  }
  dev_free(s->d_slots);
  for (auto& kv : s->reqs) delete kv.second;
  delete s;
  return set_error(XS_OK);
}

}  // extern "C"

namespace xs {
// This file's debug word (xs_debug_status).
cudaError_t debug_take_serve(unsigned long long* v) { return debug_word_take(v); }
}  // namespace xs
