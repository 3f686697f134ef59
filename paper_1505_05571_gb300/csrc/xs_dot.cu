// Exact dot product and squared norm: every product is rounded to the nearest
// double (an ordinary IEEE multiply), and the products are summed exactly and
// rounded once -- the paper's squared-norm and dot-product functions
// (performance section, norm and dot timings). The multiply is fused into the
// streaming small-superaccumulator kernel, so the inputs are read once.
//
// Reading: a NaN product (NaN input, or Inf times 0) enters the sum as the
// default quiet NaN 0x7FF8000000000000, since the payload an IEEE multiply
// returns for NaN operands differs between processors.
#include <cuda_runtime.h>

#include <algorithm>

#include "xs_host.hpp"
#include "xs_kernels.cuh"

namespace xs {

struct DotArgs {
  SumArgs s;          // s.x is the first vector
  const double* y;    // second vector (dot); unused for the squared norm
};

// The rounded product's bits. Nothing consumes them until the next tile, so
// the FP64 latency stays off the warp's path; a NaN product (exponent 2047)
// always takes the general path, where canon_nan replaces it.
__device__ __forceinline__ unsigned long long product_bits(unsigned long long a,
                                                           unsigned long long b) {
  return (unsigned long long)__double_as_longlong(
      __dmul_rn(__longlong_as_double((long long)a), __longlong_as_double((long long)b)));
}
__device__ __forceinline__ unsigned long long canon_nan(unsigned long long p) {
  return ((p & 0x7FFFFFFFFFFFFFFFull) > kPosInf) ? kDefaultNaN : p;
}

// Pair p (elements head + 2p, head + 2p + 1) of the second vector.
template <bool YVEC>
__device__ __forceinline__ ulonglong2 load_y(const double* y, long long p) {
  if (YVEC) return ld_stream(reinterpret_cast<const ulonglong2*>(y) + p);
  const unsigned long long* yb = reinterpret_cast<const unsigned long long*>(y);
  return make_ulonglong2(ld_stream1(yb + 2 * p), ld_stream1(yb + 2 * p + 1));
}

// L2 prefetch of the 16-byte-aligned part of y's pairs [first, first + cnt).
__device__ __forceinline__ void prefetch_y(const double* y, long long first, long long cnt) {
  const uintptr_t lo = ((uintptr_t)(y + 2 * first) + 15u) & ~(uintptr_t)15u;
  const uintptr_t hi = ((uintptr_t)(y + 2 * (first + cnt))) & ~(uintptr_t)15u;
  if (hi > lo) prefetch_l2((const void*)lo, (unsigned)(hi - lo));
}

// KIND 0: sum of x[i] * y[i]; KIND 1: sum of x[i] * x[i].
template <int BLOCK, int UNROLL, int KIND, bool YVEC>
__global__ void __launch_bounds__(BLOCK, 1) k_dot_small(DotArgs d) {
  extern __shared__ __align__(16) long long smem_dot[];
  const SumArgs& a = d.s;
  const int tid = threadIdx.x;
  SmallThread T;
  T.acc = smem_dot + tid;
  for (int c = 0; c < kSChunks; ++c) T.acc[c * BLOCK] = 0;

  const Split sp = split_input(a.x, a.n);
  const double* yb = d.y + sp.head;  // y aligned with x's pairs
  auto y_at = [&](long long i) -> unsigned long long {
    return (unsigned long long)__double_as_longlong(KIND == 0 ? d.y[i] : a.x[i]);
  };
  constexpr long long TP = (long long)BLOCK * UNROLL;
  const long long ntiles = (sp.npairs + TP - 1) / TP;
  const long long G = gridDim.x;
  auto prefetch = [&](long long t) {
    if (t >= ntiles) return;
    prefetch_tile<BLOCK, UNROLL>(sp, t, ntiles);
    if (KIND == 0) prefetch_y(yb, t * TP, min(TP, sp.npairs - t * TP));
  };
  auto load = [&](long long t, ulonglong2* X, ulonglong2* Y) {
    const long long base = t * TP + tid;
#pragma unroll
    for (int u = 0; u < UNROLL; ++u) {
      const long long p = base + (long long)u * BLOCK;
      if (p < sp.npairs) {
        X[u] = ld_stream(sp.xv + p);
        if (KIND == 0) Y[u] = load_y<YVEC>(yb, p);
      } else {  // -0 * +0 = -0 adds nothing and leaves the signed-zero record alone
        X[u] = make_ulonglong2(kNegZero, kNegZero);
        if (KIND == 0) Y[u] = make_ulonglong2(0ull, 0ull);
      }
    }
  };
  // Products of a tile, issued one tile before they are added: the narrow
  // FP64 pipe's latency overlaps the previous tile's accumulation.
  auto multiply = [&](const ulonglong2* X, const ulonglong2* Y, ulonglong2* P) {
#pragma unroll
    for (int u = 0; u < UNROLL; ++u) {
      if (KIND == 0) {
        P[u] = make_ulonglong2(product_bits(X[u].x, Y[u].x), product_bits(X[u].y, Y[u].y));
      } else {
        P[u] = make_ulonglong2(product_bits(X[u].x, X[u].x), product_bits(X[u].y, X[u].y));
      }
    }
  };
  // Adds the products P of one tile while the products Pn of the next tile are
  // computed between the adds (same basic block), so the narrow FP64 pipe
  // works alongside the integer pipes instead of stalling the warp.
  int since = 0;
  auto add_mul = [&](const ulonglong2* P, const ulonglong2* X, const ulonglong2* Y,
                     ulonglong2* Pn, bool next) {
    unsigned e[2 * UNROLL];
    unsigned mx = 0u;
#pragma unroll
    for (int k = 0; k < UNROLL; ++k) {
      e[2 * k] = ((unsigned)(P[k].x >> 32) >> 20) & 0x7FFu;
      e[2 * k + 1] = ((unsigned)(P[k].y >> 32) >> 20) & 0x7FFu;
      mx = max(mx, e[2 * k] - 1u);
      mx = max(mx, e[2 * k + 1] - 1u);
    }
    const ulonglong2* Yk = KIND == 0 ? Y : X;
    if (__builtin_expect(mx < 0x7FEu, 1)) {
      T.notnegz = 1u;
#pragma unroll
      for (int k = 0; k < UNROLL; ++k) {
        if (next) Pn[k].x = product_bits(X[k].x, Yk[k].x);
        sacc_add_normal<BLOCK>(T.acc, (unsigned)P[k].x, (unsigned)(P[k].x >> 32), e[2 * k]);
        if (next) Pn[k].y = product_bits(X[k].y, Yk[k].y);
        sacc_add_normal<BLOCK>(T.acc, (unsigned)P[k].y, (unsigned)(P[k].y >> 32), e[2 * k + 1]);
      }
    } else {
#pragma unroll
      for (int k = 0; k < UNROLL; ++k) {
        if (next) Pn[k] = make_ulonglong2(product_bits(X[k].x, Yk[k].x), product_bits(X[k].y, Yk[k].y));
        T.one<BLOCK>(canon_nan(P[k].x));
        T.one<BLOCK>(canon_nan(P[k].y));
      }
    }
    if (++since >= a.carry_tiles) {
      sacc_propagate(T.acc, BLOCK);
      since = 0;
    }
  };
  long long t = blockIdx.x;
  if (tid == 0)
    for (int k = 0; k <= a.prefetch; ++k) prefetch(t + k * G);
  grid_dependency_wait();
  if (blockIdx.x == 0 && tid < 32) {  // head (one element per lane) and tail
    const unsigned long long* xb = reinterpret_cast<const unsigned long long*>(a.x);
    if (tid < sp.head) T.one<BLOCK>(canon_nan(product_bits(xb[tid], y_at(tid))));
    if (tid == 0 && sp.tail) T.one<BLOCK>(canon_nan(product_bits(xb[a.n - 1], y_at(a.n - 1))));
  }
  ulonglong2 XA[UNROLL], YA[UNROLL], XB[UNROLL], YB[UNROLL], PA[UNROLL], PB[UNROLL];
  if (t < ntiles) {
    load(t, XA, YA);
    if (t + G < ntiles) load(t + G, XB, YB);
    multiply(XA, YA, PA);
  }
  while (t < ntiles) {
    // PA: products of tile t; XB/YB: tile t + G; XA/YA are free
    if (tid == 0 && a.prefetch > 0) prefetch(t + (a.prefetch + 2) * G);
    if (t + 2 * G < ntiles) load(t + 2 * G, XA, YA);
    add_mul(PA, XB, YB, PB, t + G < ntiles);
    t += G;
    if (t >= ntiles) break;
    // PB: products of tile t; XA/YA: tile t + G
    if (tid == 0 && a.prefetch > 0) prefetch(t + (a.prefetch + 2) * G);
    if (t + 2 * G < ntiles) load(t + 2 * G, XB, YB);
    add_mul(PB, XA, YA, PA, t + G < ntiles);
    t += G;
  }
  __syncthreads();
  grid_launch_dependents();
  unsigned f = T.flags();
  if (blockIdx.x == 0 && tid == 0 && a.n > 0) f |= kFlagAny;
  block_small_to_global<BLOCK>(smem_dot, a, f, T.nkey);
  finish_grid(a, smem_dot);
}

// The same products into the paper's large superaccumulator (Large, Fig. 4):
// one block-wide set of sign+exponent chunks in shared memory, as in the
// single-array large kernel. A product that is zero, subnormal, Inf or NaN
// sends its group through the record (the default NaN for a NaN product); its
// significand lands in a chunk the flush ignores (Inf, NaN) or is taken off
// with the zero counts.
template <int BLOCK>
constexpr int dot_large_copies() { return BLOCK >= 512 ? 4 : (BLOCK >= 256 ? 2 : 1); }
template <int BLOCK>
constexpr int dot_large_blocks() { return BLOCK >= 512 ? 1 : (BLOCK >= 256 ? 2 : 4); }
template <int BLOCK>
constexpr size_t dot_large_smem() { return sizeof(LargePlanes<BLOCK / 32, dot_large_copies<BLOCK>()>); }

template <int BLOCK, int UNROLL, int KIND, bool YVEC>
__global__ void __launch_bounds__(BLOCK, dot_large_blocks<BLOCK>()) k_dot_large(DotArgs d) {
  constexpr int NW = BLOCK / 32;
  constexpr int R = dot_large_copies<BLOCK>();
  extern __shared__ __align__(16) unsigned char smem_dotl[];
  LargePlanes<NW, R>& P = *reinterpret_cast<LargePlanes<NW, R>*>(smem_dotl);
  const SumArgs& a = d.s;
  const int tid = threadIdx.x;
  const Split sp = split_input(a.x, a.n);
  const double* yb = d.y + sp.head;  // y aligned with x's pairs
  auto y_at = [&](long long i) -> unsigned long long {
    return (unsigned long long)__double_as_longlong(KIND == 0 ? d.y[i] : a.x[i]);
  };
  constexpr long long TP = (long long)BLOCK * UNROLL;
  const long long ntiles = (sp.npairs + TP - 1) / TP;
  const long long nfull = sp.npairs / TP;
  const long long G = gridDim.x;
  auto prefetch = [&](long long t) {
    if (t >= ntiles) return;
    prefetch_tile<BLOCK, UNROLL>(sp, t, ntiles);
    if (KIND == 0) prefetch_y(yb, t * TP, min(TP, sp.npairs - t * TP));
  };
  auto load = [&](long long t, ulonglong2* X, ulonglong2* Y) {  // a full tile
    const long long base = t * TP + tid;
#pragma unroll
    for (int u = 0; u < UNROLL; ++u) {
      X[u] = ld_stream(sp.xv + base + (long long)u * BLOCK);
      if (KIND == 0) Y[u] = load_y<YVEC>(yb, base + (long long)u * BLOCK);
    }
  };
  long long t = blockIdx.x;
  if (tid == 0)
    for (int k = 0; k <= a.prefetch; ++k) prefetch(t + k * G);
  large_init(P, tid, BLOCK);
  const LargeLane L = large_lane(P);
  __syncthreads();
  grid_dependency_wait();
  LargeThread T;
  auto add = [&](const ulonglong2* X, const ulonglong2* Y) {
    ulonglong2 Pr[UNROLL];
#pragma unroll
    for (int u = 0; u < UNROLL; ++u) {
      const ulonglong2 yv = KIND == 0 ? Y[u] : X[u];
      Pr[u] = make_ulonglong2(product_bits(X[u].x, yv.x), product_bits(X[u].y, yv.y));
    }
    const unsigned mx = large_group_add<UNROLL>(L, Pr);
    if (__builtin_expect(mx >= 0x7FE00000u, 0)) {
#pragma unroll
      for (int u = 0; u < UNROLL; ++u) Pr[u] = make_ulonglong2(canon_nan(Pr[u].x), canon_nan(Pr[u].y));
    }
    T.group_record<UNROLL>(mx, Pr);
  };
  auto one = [&](unsigned long long xv, unsigned long long yv) {
    const unsigned long long p = canon_nan(product_bits(xv, yv));
    large_one_add(L, p);
    T.term(p);
  };
  ulonglong2 XA[UNROLL], YA[UNROLL], XB[UNROLL], YB[UNROLL];
  if (t < nfull) load(t, XA, YA);
  if (blockIdx.x == 0 && tid < 32) {  // head (one element per lane) and tail
    const unsigned long long* xb = reinterpret_cast<const unsigned long long*>(a.x);
    if (tid < sp.head) one(xb[tid], y_at(tid));
    if (tid == 0 && sp.tail) one(xb[a.n - 1], y_at(a.n - 1));
  }
  while (t < nfull) {
    if (tid == 0 && a.prefetch > 0) prefetch(t + (a.prefetch + 1) * G);
    if (t + G < nfull) load(t + G, XB, YB);
    add(XA, YA);
    t += G;
    if (t >= nfull) break;
    if (tid == 0 && a.prefetch > 0) prefetch(t + (a.prefetch + 1) * G);
    if (t + G < nfull) load(t + G, XA, YA);
    add(XB, YB);
    t += G;
  }
  if (t == nfull && nfull < ntiles) {  // the ragged last tile, term by term
    const long long base = t * TP + tid;
#pragma unroll
    for (int u = 0; u < UNROLL; ++u) {
      const long long q = base + (long long)u * BLOCK;
      if (q < sp.npairs) {
        const ulonglong2 xv = ld_stream(sp.xv + q);
        const ulonglong2 yv = KIND == 0 ? load_y<YVEC>(yb, q) : xv;
        one(xv.x, yv.x);
        one(xv.y, yv.y);
      }
    }
  }
  grid_launch_dependents();
  {  // zero/subnormal counts of the block (their spurious implicit bits)
    const unsigned zp = __reduce_add_sync(kFull, T.zpos);
    const unsigned zn = __reduce_add_sync(kFull, T.zneg);
    if ((tid & 31) == 0) {
      if (zp) atomicAdd(&P.zeros[0], zp);
      if (zn) atomicAdd(&P.zeros[1], zn);
    }
  }
  __syncthreads();
  large_flush(P);
  __syncthreads();
  if (tid < kSChunks) {
    long long v = 0;
#pragma unroll
    for (int w = 0; w < NW; ++w) v += P.part[w][tid];
    if (v != 0) atomicAdd(reinterpret_cast<unsigned long long*>(&a.g->chunk[tid]), (unsigned long long)v);
  }
  unsigned f = __reduce_or_sync(kFull, T.flags());
  const unsigned long long key = warp_max_ull(T.nkey);
  if ((tid & 31) == 0) {
    if (blockIdx.x == 0 && tid == 0 && a.n > 0) f |= kFlagAny;
    if (f) atomicOr(&a.g->flags, f);
    if (key) atomicMax(&a.g->nan_key, key);
  }
  finish_grid(a, reinterpret_cast<long long*>(P.copies));
}

namespace {

constexpr int kDotBlock = 384;
constexpr int kDotUnroll = 4;
// The large superaccumulator for products: launch shapes and the size from
// which XS_METHOD_AUTO takes it. Measured on 1e8 pairs (us, against the
// small method): x and y at the same 16-byte offset 219.2 with 512 x 2
// (256.6; 512 x 4: 227.5, 768 x 2: 225.9, 256 x 4: 229.4); y one element off
// 247.8 with 768 x 2 (388.8; 512 x 2: 270.3); squared norm 204.9 (215.7).
// From 2^21 values the large method is ahead in all three cases (aligned dot
// 12.0 / 13.3 us, y one element off 13.9 / 14.8, squared norm 11.7 / 12.4;
// at 2^26 150 / 176, 167 / 261, 140 / 149).
constexpr int kDotLBlock = 512;    // x and y pairs aligned alike (and the squared norm)
constexpr int kDotLBlockY1 = 768;  // y read element by element
constexpr int kDotLUnroll = 2;
constexpr long long kDotLargeMin = 1ll << 21;
typedef void (*DotKernel)(DotArgs);

DotKernel dot_kernel(int kind, bool yvec) {
  if (kind == 1) return k_dot_small<kDotBlock, kDotUnroll, 1, true>;
  return yvec ? k_dot_small<kDotBlock, kDotUnroll, 0, true> : k_dot_small<kDotBlock, kDotUnroll, 0, false>;
}

template <int BLOCK, int UNROLL>
DotKernel dot_large_kernel(int kind, bool yvec) {
  if (kind == 1) return k_dot_large<BLOCK, UNROLL, 1, true>;
  return yvec ? k_dot_large<BLOCK, UNROLL, 0, true> : k_dot_large<BLOCK, UNROLL, 0, false>;
}

xs_status launch_dot(const double* x, const double* y, int64_t n, double* d_out, int kind,
                     int method, void* stream) {
  xs_status st;
  if (method < XS_METHOD_AUTO || method > XS_METHOD_LARGE) return set_error(XS_ERR_INVALID_VALUE);
  if (n < 0) return set_error(XS_ERR_INVALID_VALUE);
  if ((st = check_device_ptr(d_out)) != XS_OK) return st;
  if (((uintptr_t)d_out & 7u) != 0u) return set_error(XS_ERR_INVALID_VALUE);
  cudaStream_t s = as_stream(stream);
  if (n == 0) {
    XS_TRY_CUDA(cudaMemsetAsync(d_out, 0, sizeof(double), s));
    return set_error(XS_OK);
  }
  if (((uintptr_t)x & 7u) != 0u || (kind == 0 && ((uintptr_t)y & 7u) != 0u))
    return set_error(XS_ERR_INVALID_VALUE);
  if ((st = check_device_ptr(x)) != XS_OK) return st;
  if (kind == 0 && (st = check_device_ptr(y)) != XS_OK) return st;
  DeviceCtx* ctx = device_ctx(&st);
  if (!ctx) return st;
  Workspace* w = workspace(ctx, s, &st);
  if (!w) return st;
  // y shares x's pairs when both sit at the same offset within 16 bytes
  const bool yvec = kind == 1 || ((((uintptr_t)x) ^ ((uintptr_t)y)) & 15u) == 0u;
  const bool large = method == XS_METHOD_LARGE || (method == XS_METHOD_AUTO && n >= kDotLargeMin);
  DotKernel fn = dot_kernel(kind, yvec);
  int block = kDotBlock, unroll = kDotUnroll;
  size_t smem = (size_t)kDotBlock * kSChunks * sizeof(long long);
  if (large && yvec) {
    fn = dot_large_kernel<kDotLBlock, kDotLUnroll>(kind, yvec);
    block = kDotLBlock;
    unroll = kDotLUnroll;
    smem = dot_large_smem<kDotLBlock>();
  } else if (large) {
    fn = dot_large_kernel<kDotLBlockY1, kDotLUnroll>(kind, yvec);
    block = kDotLBlockY1;
    unroll = kDotLUnroll;
    smem = dot_large_smem<kDotLBlockY1>();
  }
  static bool attr[64][6] = {};
  const int slot = (kind == 1 ? 2 : (yvec ? 0 : 1)) + (large ? 3 : 0);
  if (ctx->device < 64 && !attr[ctx->device][slot]) {
    XS_TRY_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr[ctx->device][slot] = true;
  }
  int occ = 1;
  XS_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, block, smem));
  const long long tp = (long long)block * unroll;
  const long long ntiles = std::max<long long>(1, (n / 2 + tp - 1) / tp);
  const long long g = std::max<long long>(1, std::min<long long>((long long)ctx->num_sms * std::max(1, occ), ntiles));
  DotArgs d;
  d.s.x = x;
  d.s.n = n;
  d.s.g = w->acc;
  d.s.out = d_out;
  d.s.mode = 0;
  d.s.carry_tiles = std::max(1, (kCarryInterval - 2) / (2 * kDotUnroll));
  d.s.prefetch = prefetch_tiles(kDotPrefetch);
  d.s.divisor = 0ull;
  d.y = kind == 0 ? y : x;
  XS_TRY_CUDA(launch_pdl(fn, (unsigned)g, (unsigned)block, smem, s, d));
  return set_error(XS_OK);
}

}  // namespace

}  // namespace xs

using namespace xs;

extern "C" {

xs_status xs_dot_async(const double* d_x, const double* d_y, int64_t n, double* d_out,
                       void* stream) {
  return launch_dot(d_x, d_y, n, d_out, 0, XS_METHOD_AUTO, stream);
}

xs_status xs_norm2_async(const double* d_x, int64_t n, double* d_out, void* stream) {
  return launch_dot(d_x, nullptr, n, d_out, 1, XS_METHOD_AUTO, stream);
}

xs_status xs_dot_method_async(const double* d_x, const double* d_y, int64_t n, double* d_out,
                              int method, void* stream) {
  return launch_dot(d_x, d_y, n, d_out, 0, method, stream);
}

xs_status xs_norm2_method_async(const double* d_x, int64_t n, double* d_out, int method,
                                void* stream) {
  return launch_dot(d_x, nullptr, n, d_out, 1, method, stream);
}

}  // extern "C"

namespace xs {
// This file's debug word (xs_debug_status).
cudaError_t debug_take_dot(unsigned long long* v) { return debug_word_take(v); }
}  // namespace xs
