// xs_sum_noalloc: the single-array exact sum for callers that must not
// allocate device memory.
//
// The one piece of scratch the single-array kernel needs -- the 560-byte grid
// accumulator that every block adds its partial into and that the last block
// rounds and clears -- lives here in a file-scope static __device__ array
// instead of a cudaMalloc'ed per-stream workspace. The module holds it on
// every GPU that loads the library until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "xs_host.hpp"

namespace xs {

// Scratch of xs_sum_noalloc: one grid accumulator per device.
static __device__ __align__(256) AccState g_noalloc_scratch[1];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
AccState* g_noalloc_addr[kMaxDevices] = {};  // device address of the scratch, once set up
int g_noalloc_grid[kMaxDevices] = {};

// Once per device, with that device current: the scratch's device address
// (the host-side symbol is only a stand-in and must never reach a kernel),
// and the grid of the fixed launch shape.
xs_status noalloc_setup(int dev, AccState** addr, int* grid) {
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (g_noalloc_addr[dev] == nullptr) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) return from_cuda(e != cudaSuccess ? e : cudaErrorUnknown);
    int g = 0;
    const xs_status st = small_fixed_grid(&g);
    if (st != XS_OK) return st;
    g_noalloc_grid[dev] = g;
    g_noalloc_addr[dev] = static_cast<AccState*>(p);
  }
  *addr = g_noalloc_addr[dev];
  *grid = g_noalloc_grid[dev];
  return XS_OK;
}

}  // namespace

}  // namespace xs

using namespace xs;

extern "C" xs_status xs_sum_noalloc(const double* d_values, int64_t n, double* d_out,
                                    void* stream) {
  if (n < 0 || n > XS_NOALLOC_MAX_TERMS) return set_error(XS_ERR_INVALID_VALUE);
  if (d_out == nullptr || ((uintptr_t)d_out & 7u) != 0u) return set_error(XS_ERR_INVALID_POINTER);
  xs_status st = check_device_ptr(d_out);
  if (st != XS_OK) return st;
  cudaStream_t s = as_stream(stream);
  if (n == 0) {
    XS_TRY_CUDA(cudaMemsetAsync(d_out, 0, sizeof(double), s));
    return set_error(XS_OK);
  }
  if (((uintptr_t)d_values & 7u) != 0u) return set_error(XS_ERR_INVALID_VALUE);
  if ((st = check_device_ptr(d_values)) != XS_OK) return st;
  int dev = 0;
  XS_TRY_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return set_error(XS_ERR_NOT_SUPPORTED);
  AccState* acc = nullptr;
  int grid = 0;
  if ((st = noalloc_setup(dev, &acc, &grid)) != XS_OK) return st;
  // The scratch keeps whatever the previous call left; the kernel needs a
  // zero accumulator and ticket, so clear them first (a memset, not an
  // allocation).
  XS_TRY_CUDA(cudaMemsetAsync(acc, 0, sizeof(AccState), s));
  if ((st = launch_small_fixed(d_values, n, acc, d_out, grid, s)) != XS_OK) return st;
  return set_error(XS_OK);
}

namespace xs {
// This file's debug word (xs_debug_status).
cudaError_t debug_take_noalloc(unsigned long long* v) { return debug_word_take(v); }
}  // namespace xs
