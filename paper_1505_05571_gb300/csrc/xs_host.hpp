// Host-side runtime shared by the library's translation units: error state,
// per-device context, per-stream workspaces and launch helpers.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <mutex>
#include <vector>

#include "../../include/xsum.h"
#include "xs_device.cuh"

namespace xs {

xs_status set_error(xs_status s);
xs_status from_cuda(cudaError_t e);  // records and maps a CUDA error

#define XS_TRY_CUDA(call)                        \
  do {                                           \
    cudaError_t _e = (call);                     \
    if (_e != cudaSuccess) return from_cuda(_e); \
  } while (0)

// Every device and pinned-host allocation of the library goes through these
// four calls. They count the allocations held (xs_debug_live_allocations) and
// let a test make the k-th next one fail as an out-of-memory error
// (xs_debug_fail_allocation), so each caller's unwinding can be checked.
cudaError_t dev_alloc(void** p, size_t bytes);
void dev_free(void* p);
cudaError_t host_alloc(void** p, size_t bytes, unsigned flags);
void host_free(void* p);
template <typename T>
cudaError_t dev_alloc(T** p, size_t bytes) {
  return dev_alloc(reinterpret_cast<void**>(p), bytes);
}
template <typename T>
cudaError_t host_alloc(T** p, size_t bytes, unsigned flags) {
  return host_alloc(reinterpret_cast<void**>(p), bytes, flags);
}

// Each translation unit's debug word, read and cleared (always 0 outside a
// -DXS_DEBUG build): the codes of the checks its kernels saw fail.
cudaError_t debug_take_core(unsigned long long* v);
cudaError_t debug_take_segments(unsigned long long* v);
cudaError_t debug_take_serve(unsigned long long* v);
cudaError_t debug_take_dot(unsigned long long* v);
cudaError_t debug_take_f32(unsigned long long* v);
cudaError_t debug_take_noalloc(unsigned long long* v);

// Device pointer check (cudaPointerGetAttributes): host or unregistered
// memory is rejected.
xs_status check_device_ptr(const void* p);

// Work space of one (device, stream) pair. Allocated zeroed; every kernel that
// uses `acc` leaves it zeroed again (the last block resets what it read).
struct Workspace {
  AccState* acc = nullptr;        // grid accumulator of xs_sum
  AccState* acc_host = nullptr;   // accumulator of xs_sum_host
  AccState* acc_f32 = nullptr;    // grid accumulator of the FP32 sum (its smaller layout)
  double* d_out = nullptr;        // device result slot
  double* h_out = nullptr;        // mapped pinned result slot (host view)
  double* h_out_dev = nullptr;    // the same slot as kernels address it
  // xs_sum_host staging ring
  double* stage[2] = {nullptr, nullptr};
  size_t stage_elems = 0;
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t full[2] = {nullptr, nullptr};
  cudaEvent_t free_[2] = {nullptr, nullptr};
  // inexact comparison sum: per-block partials and the ticket behind them
  double* inexact_partial = nullptr;
};

struct SumShape {
  int method;
  int block;
  int unroll;
};

struct DeviceCtx {
  int device = -1;
  int num_sms = 0;
  std::mutex mu;
  std::map<cudaStream_t, Workspace*> ws;
  // tuned single-array choice per size class (log2 n)
  std::map<int, SumShape> tuned_sum;
  // tuned segmented options (one entry; 0 fields = defaults)
  bool have_tuned_seg = false;
  xs_seg_options tuned_seg{};
  std::vector<int> occupancy;  // resident blocks per SM of each compiled shape
};

DeviceCtx* device_ctx(xs_status* st);  // context of the current device
Workspace* workspace(DeviceCtx* ctx, cudaStream_t s, xs_status* st);

// Launch of the single-array kernel into a target accumulator.
// mode 0: round into d_out and reset the target; mode 1: normalise the target
// in place (accumulator handles).
xs_status launch_sum(DeviceCtx* ctx, const double* d_values, int64_t n, AccState* target,
                     double* d_out, int mode, SumShape shape, int grid, cudaStream_t s,
                     unsigned long long divisor = 0);
SumShape default_shape(DeviceCtx* ctx, int64_t n);
xs_status launch_small_fixed(const double* d_values, int64_t n, AccState* target, double* d_out,
                             int grid, cudaStream_t s);
xs_status small_fixed_grid(int* grid);

// L2 prefetch distance (tiles ahead of each block) that a kernel family uses:
// the process-wide setting of xs_set_prefetch_tiles, else `builtin`.
int prefetch_tiles(int builtin);
constexpr int kSumPrefetch = 3;  // FP64 sum and mean kernels
constexpr int kDotPrefetch = 3;  // dot and squared-norm kernels
constexpr int kF32Prefetch = 0;  // binary32 sum kernel (measured: prefetching made it re-read 12 %)

// Launch with programmatic stream serialization: the grid may be scheduled
// while the previous kernel on the stream finishes. Every kernel launched this
// way calls grid_dependency_wait() before its first global-memory access
// (other than L2 prefetches).
template <typename... P, typename... A>
cudaError_t launch_pdl(void (*kernel)(P...), unsigned grid, unsigned block, size_t smem,
                       cudaStream_t s, A&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<A&&>(args)...);
}

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

}  // namespace xs
