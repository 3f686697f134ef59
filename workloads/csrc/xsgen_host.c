/* Host twin of workloads/gen.py for large index ranges: the same SplitMix64
 * draws and bit recipe, written in plain C and spread over OpenMP threads, so
 * tests can regenerate tens of GB of inputs on the host in seconds (numpy
 * runs single-threaded). It holds no summation arithmetic. Keys are computed
 * by workloads/gen.py and passed in; a CPU test checks this file against the
 * numpy recipe bit for bit. */
#include <stdint.h>

#define GAMMA 0x9E3779B97F4A7C15ull

static inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

/* out[j] = pow2_band_bits(draw(key_sm, start + j), draw(key_exp, start + j), lo, hi)
 * for j in [0, count): uniform sign and 52-bit mantissa, unbiased exponent
 * lo + floor((v >> 32) * (hi - lo) / 2^32). */
void xgh_band(uint64_t* out, int64_t start, int64_t count, uint64_t key_sm, uint64_t key_exp,
              int lo, int hi) {
  const uint64_t span = (uint64_t)(int64_t)(hi - lo);
  const uint64_t bias = (uint64_t)(int64_t)(lo + 1023);
#pragma omp parallel for schedule(static)
  for (int64_t j = 0; j < count; ++j) {
    const uint64_t i = (uint64_t)(start + j) + 1u;
    const uint64_t u = mix64(key_sm + i * GAMMA);
    const uint64_t v = mix64(key_exp + i * GAMMA);
    const uint64_t e = (((v >> 32) * span) >> 32) + bias;
    out[j] = (u & 0x8000000000000000ull) | (e << 52) | (u & 0x000FFFFFFFFFFFFFull);
  }
}
