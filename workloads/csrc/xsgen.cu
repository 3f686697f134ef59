// Device twin of workloads/gen.py: the same SplitMix64 draws and bit recipes,
// so large synthetic inputs can be generated in HBM instead of on the host.
// It holds no summation arithmetic. Keys and permutation constants are
// computed on the host (workloads/gen.py) and passed in.
#include <cstdint>
#include <cuda_runtime.h>

namespace {

constexpr unsigned long long kGamma = 0x9E3779B97F4A7C15ull;

__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__device__ __forceinline__ unsigned long long draw(unsigned long long key, unsigned long long i) {
  return mix64(key + (i + 1ull) * kGamma);
}
__device__ __forceinline__ unsigned long long expsel(unsigned long long v, unsigned long long span) {
  return ((v >> 32) * span) >> 32;
}
__device__ __forceinline__ unsigned long long band_bits(unsigned long long u, unsigned long long v,
                                                        int lo, int hi) {
  const unsigned long long e = expsel(v, (unsigned long long)(hi - lo)) + (unsigned long long)(lo + 1023);
  return (u & 0x8000000000000000ull) | (e << 52) | (u & 0x000FFFFFFFFFFFFFull);
}
__device__ __forceinline__ unsigned long long full_bits(unsigned long long u, unsigned long long v,
                                                        unsigned long long emax_excl) {
  const unsigned long long e = expsel(v, emax_excl);
  return (u & 0x8000000000000000ull) | (e << 52) | (u & 0x000FFFFFFFFFFFFFull);
}

struct Keys {
  unsigned long long sm, exp, sm2, exp2;
};

__global__ void k_band(unsigned long long* out, long long start, long long count, Keys k, int lo,
                       int hi) {
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < count;
       j += (long long)gridDim.x * blockDim.x) {
    const unsigned long long i = (unsigned long long)(start + j);
    out[j] = band_bits(draw(k.sm, i), draw(k.exp, i), lo, hi);
  }
}

__global__ void k_full(unsigned long long* out, long long start, long long count, Keys k) {
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < count;
       j += (long long)gridDim.x * blockDim.x) {
    const unsigned long long i = (unsigned long long)(start + j);
    out[j] = full_bits(draw(k.sm, i), draw(k.exp, i), 2047ull);
  }
}

// X[i] = base[pi^{-1}(i)], pi^{-1}(i) = (i - b) * a_inv mod 2^n_log2.
__global__ void k_paired(unsigned long long* out, long long start, long long count, Keys k,
                         int n_log2, unsigned long long a_inv, unsigned long long b) {
  const unsigned long long mask = (1ull << n_log2) - 1ull;
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < count;
       j += (long long)gridDim.x * blockDim.x) {
    const unsigned long long i = (unsigned long long)(start + j);
    const unsigned long long kk = ((i - b) * a_inv) & mask;
    const unsigned long long jj = kk >> 1;
    const unsigned long long vj = full_bits(draw(k.sm, jj), draw(k.exp, jj), 2047ull);
    const bool big = ((vj >> 52) & 0x7FFull) >= 1000ull;
    const unsigned long long fresh = full_bits(draw(k.sm2, jj), draw(k.exp2, jj), 1000ull);
    const unsigned long long partner = big ? (vj ^ 0x8000000000000000ull) : fresh;
    out[j] = (kk & 1ull) ? partner : vj;
  }
}

__global__ void k_cancel(unsigned long long* out, long long start, long long count, Keys k,
                         int n_log2, unsigned long long a_inv, unsigned long long b) {
  const unsigned long long mask = (1ull << n_log2) - 1ull;
  const unsigned long long half = 1ull << (n_log2 - 1);
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < count;
       j += (long long)gridDim.x * blockDim.x) {
    const unsigned long long i = (unsigned long long)(start + j);
    const unsigned long long kk = ((i - b) * a_inv) & mask;
    unsigned long long r;
    if (kk < half) {
      const unsigned long long jj = kk >> 1;
      r = band_bits(draw(k.sm, jj), draw(k.exp, jj), 990, 1000);
      if (kk & 1ull) r ^= 0x8000000000000000ull;
    } else {
      r = band_bits(draw(k.sm2, kk), draw(k.exp2, kk), -60, 60);
    }
    out[j] = r;
  }
}

int grid_for(long long count) {
  long long g = (count + 255) / 256;
  return (int)(g > 65536 ? 65536 : (g < 1 ? 1 : g));
}

}  // namespace

extern "C" {

int xsg_band(void* out, long long start, long long count, unsigned long long key_sm,
             unsigned long long key_exp, int lo, int hi, void* stream) {
  Keys k{key_sm, key_exp, 0, 0};
  k_band<<<grid_for(count), 256, 0, (cudaStream_t)stream>>>((unsigned long long*)out, start, count,
                                                             k, lo, hi);
  return (int)cudaGetLastError();
}

int xsg_full_range(void* out, long long start, long long count, unsigned long long key_sm,
                   unsigned long long key_exp, void* stream) {
  Keys k{key_sm, key_exp, 0, 0};
  k_full<<<grid_for(count), 256, 0, (cudaStream_t)stream>>>((unsigned long long*)out, start, count, k);
  return (int)cudaGetLastError();
}

int xsg_paired(void* out, long long start, long long count, unsigned long long key_sm,
               unsigned long long key_exp, unsigned long long key_sm2, unsigned long long key_exp2,
               int n_log2, unsigned long long a_inv, unsigned long long b, void* stream) {
  Keys k{key_sm, key_exp, key_sm2, key_exp2};
  k_paired<<<grid_for(count), 256, 0, (cudaStream_t)stream>>>((unsigned long long*)out, start,
                                                               count, k, n_log2, a_inv, b);
  return (int)cudaGetLastError();
}

int xsg_cancel(void* out, long long start, long long count, unsigned long long key_sm,
               unsigned long long key_exp, unsigned long long key_sm2, unsigned long long key_exp2,
               int n_log2, unsigned long long a_inv, unsigned long long b, void* stream) {
  Keys k{key_sm, key_exp, key_sm2, key_exp2};
  k_cancel<<<grid_for(count), 256, 0, (cudaStream_t)stream>>>((unsigned long long*)out, start,
                                                               count, k, n_log2, a_inv, b);
  return (int)cudaGetLastError();
}

}  // extern "C"
