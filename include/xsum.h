/*
 * xsum.h -- C ABI of the GB300 exact FP64 summation library (libxsum.so).
 *
 * Every entry point sums IEEE-754 binary64 values EXACTLY and rounds the exact
 * sum once to the nearest double, ties to even, as in R. M. Neal, "Fast Exact
 * Summation Using Small and Large Superaccumulators" (2015): abstract and
 * Introduction (problem statement), section "Exact summation using a small
 * superaccumulator" (67-chunk accumulator, carry propagation, rounding),
 * section "Faster exact summation of many terms with a large
 * superaccumulator" (4096-chunk accumulator, transfers), and the Discussion
 * (merging partial accumulators; results finite whenever the rounded exact sum
 * is representable).
 *
 * Result rules (identical for every entry point and every launch shape; the
 * result never depends on order, block size or grid size):
 *   - any NaN input: the NaN with the largest 51-bit payload, a positive one
 *     preferred on ties, returned with the quiet bit set;
 *   - else +Inf and -Inf both present: the quiet NaN 0x7FF8000000000000;
 *   - else +Inf or -Inf present: that infinity (the finite part is ignored);
 *   - else an exact zero: -0.0 when there is at least one term and every term
 *     is -0.0, otherwise +0.0 (an empty sum is +0.0);
 *   - else the exact sum rounded to nearest, ties to even, +-Inf when its
 *     magnitude is at least 2^1024 - 2^970.
 *
 * Conventions:
 *   - Pointers named d_* are CUDA device pointers (cudaMalloc, cudaMallocAsync
 *     or managed memory) of the current device; h_* are host pointers.
 *     Value arrays must be 8-byte aligned; they need not be 16-byte aligned.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream). Asynchronous calls only enqueue work on it.
 *   - The caller owns every buffer and stream; the library never writes its
 *     inputs and never frees caller memory. Library objects (handles, plans,
 *     servers) own their own device memory until destroyed.
 *   - The library keeps a small workspace per (device, stream), created on the
 *     first call that needs it. Calls on one stream are ordered; do not issue
 *     two library calls that share a workspace or a handle from two host
 *     threads at once.
 *   - Errors: functions return an xs_status and also record it as the calling
 *     thread's last error (xs_get_last_error). XS_ERR_INVALID_VALUE: n < 0,
 *     misaligned pointer, malformed offsets detected on the host, bad option;
 *     XS_ERR_INVALID_POINTER: NULL where data is needed, or a host pointer where
 *     a device pointer is required; XS_ERR_OUT_OF_MEMORY: a library allocation
 *     failed; XS_ERR_CUDA: any other CUDA runtime error.
 *   - There is no CPU fallback: without a usable CUDA device every compute
 *     call fails with XS_ERR_CUDA.
 */
#ifndef XSUM_H
#define XSUM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum xs_status {
  XS_OK = 0,
  XS_ERR_INVALID_VALUE = 1,
  XS_ERR_INVALID_POINTER = 2,
  XS_ERR_OUT_OF_MEMORY = 3,
  XS_ERR_CUDA = 4,
  XS_ERR_TIMEOUT = 5,
  XS_ERR_BUDGET = 6,
  XS_ERR_NOT_SUPPORTED = 7,
  XS_ERR_NOT_READY = 8
} xs_status;

/* Accumulation method of a single-array sum. */
typedef enum xs_method {
  XS_METHOD_AUTO = 0,  /* tuned choice by size (xs_autotune_sum), else built-in default */
  XS_METHOD_SMALL = 1, /* per-thread small superaccumulators (small-superaccumulator section) */
  XS_METHOD_LARGE = 2  /* per-block large superaccumulator + transfers (large section) */
} xs_method;

/* Version string of the library. */
const char* xs_version(void);

/* Last status recorded by a call on the calling thread; and its text. */
xs_status xs_get_last_error(void);
const char* xs_status_string(xs_status s);

/* ---------------------------------------------------------------------------
 * Single array
 * ------------------------------------------------------------------------- */

/* Exact sum of d_values[0..n), rounded once (abstract; Discussion).
 * Blocks the host until the result is ready (stream-ordered). Returns a quiet
 * NaN and records the error on failure. */
double xs_sum(const double* d_values, int64_t n, void* stream);

/* Same, with a status; *h_out receives the result. */
xs_status xs_sum_ex(const double* d_values, int64_t n, void* stream, double* h_out);

/* Asynchronous form: enqueues one kernel on `stream` that writes the rounded
 * exact sum to the device double *d_out. `method` is an xs_method. */
xs_status xs_sum_async(const double* d_values, int64_t n, double* d_out, int method,
                       void* stream);

/* Asynchronous form with an explicit launch shape (used by the autotuner and
 * the tests; every shape gives the same bits). method: XS_METHOD_SMALL or
 * XS_METHOD_LARGE; block: threads per block; unroll: 16-byte loads per thread
 * per tile; grid: blocks (0 = one wave). XS_ERR_NOT_SUPPORTED for a shape that
 * is not compiled in (see xs_list_configs). */
xs_status xs_sum_async_config(const double* d_values, int64_t n, double* d_out, int method,
                              int block, int unroll, int grid, void* stream);

/* Launch shape that XS_METHOD_AUTO uses for n elements on the current device:
 * the autotuned choice for n's size class if there is one, else the built-in
 * default. */
xs_status xs_default_shape(int64_t n, int* method, int* block, int* unroll);

/* L2 prefetch distance of the sum, mean, dot, squared-norm and binary32
 * kernels, in tiles of each block (0 disables, at most 64; -1, the initial
 * setting, gives each kernel its built-in distance). A process-wide tuning
 * knob. */
xs_status xs_set_prefetch_tiles(int tiles);

/* Number of compiled launch shapes, and shape k as (method, block, unroll). */
int xs_list_configs(int* methods, int* blocks, int* unrolls, int capacity);

/* Host-buffer form: h_values[0..n) stays in host memory; the library copies it
 * to the device in pipelined chunks (pinned host memory gives full speed) and
 * accumulates each chunk while the next one is in flight. Blocking. */
xs_status xs_sum_host(const double* h_values, int64_t n, double* h_out, void* stream);

/* Correctly rounded exact MEAN: the exact sum divided by n, rounded once to
 * nearest, ties to even, straight from the superaccumulator (Discussion:
 * rounding the value of a small superaccumulator divided by a positive
 * integer; the Introduction's motivating example is the sample mean). Unlike
 * rounding the sum and then dividing, this is the correctly rounded mean, and
 * it never overflows even when the sum would. Specials as for the sum; n == 0
 * writes the default quiet NaN 0x7FF8000000000000. Asynchronous; *d_out on
 * the device. */
xs_status xs_mean_async(const double* d_values, int64_t n, double* d_out, void* stream);

/* Exact dot product: each product d_x[i] * d_y[i] is rounded to the nearest
 * double (IEEE multiply), the n products are summed exactly and the sum is
 * rounded once (performance section: squared norm and dot product computed
 * with the superaccumulator summation). Reading: a NaN product (NaN input, or
 * Inf times 0) counts as the default quiet NaN 0x7FF8000000000000. The two
 * vectors may have different 16-byte alignment. Asynchronous; *d_out on the
 * device. */
xs_status xs_dot_async(const double* d_x, const double* d_y, int64_t n, double* d_out,
                       void* stream);
/* Exact squared norm: the sum of the rounded squares d_x[i] * d_x[i], rounded
 * once (same passage). */
xs_status xs_norm2_async(const double* d_x, int64_t n, double* d_out, void* stream);
/* The same two with the method chosen (an xs_method): XS_METHOD_SMALL, the
 * products into per-thread small superaccumulators; XS_METHOD_LARGE, into one
 * large superaccumulator per block (Large, Fig. 4); XS_METHOD_AUTO, what
 * xs_dot_async and xs_norm2_async use (the large one from 2^21 values). Same
 * bits whatever the method; XS_ERR_INVALID_VALUE for any other method. */
xs_status xs_dot_method_async(const double* d_x, const double* d_y, int64_t n, double* d_out,
                              int method, void* stream);
xs_status xs_norm2_method_async(const double* d_x, int64_t n, double* d_out, int method,
                                void* stream);

/* Exact sum of binary32 values, rounded once to the nearest float, ties to
 * even -- the single-precision variant with a smaller superaccumulator
 * (Introduction). Same result rules as the double sum, with float constants:
 * largest 22-bit NaN payload, default NaN 0x7FC00000, overflow when
 * |sum| >= 2^128 - 2^103. d_values 4-byte aligned; *d_out is a device float;
 * n <= 2^39 (XS_ERR_INVALID_VALUE above). Asynchronous. */
xs_status xs_sum_f32_async(const float* d_values, int64_t n, float* d_out, void* stream);
/* The same sum with the method chosen (an xs_method): XS_METHOD_SMALL, the
 * small superaccumulator per thread (sixteen unsigned sign-split chunks);
 * XS_METHOD_LARGE, the large superaccumulator per block (one chunk per
 * sign+exponent, 512, Large, Fig. 4, each lane of a warp adding into its own
 * column of 32-bit words); XS_METHOD_AUTO, what xs_sum_f32_async uses (the large
 * one from 5 x 2^24 values). Same bits whatever the method. */
xs_status xs_sum_f32_method_async(const float* d_values, int64_t n, float* d_out, int method,
                                  void* stream);

/* Inexact plain FP64 sum (a comparison baseline only, NOT exact: the rounding
 * after each addition depends on the launch shape). Writes *d_out. */
xs_status xs_inexact_sum_async(const double* d_values, int64_t n, double* d_out, void* stream);

/* Times every compiled shape of both methods on this input (CUDA events,
 * `reps` repetitions after one warm-up, median) and records the fastest as the
 * XS_METHOD_AUTO choice for arrays of this size class (log2 n) on the current
 * device. Outputs the winner and its median time in microseconds. */
xs_status xs_autotune_sum(const double* d_values, int64_t n, int reps, void* stream,
                          int* best_method, int* best_block, int* best_unroll, float* best_us);

/* Largest n that xs_sum_noalloc accepts: 2^45 terms, a chosen cap (the
 * headroom the CPU oracle is sized for), far inside what the accumulator
 * holds. Every per-thread, block and grid chunk bound of the kernel is
 * independent of n (carries propagate every <= 2047 adds; block partials stay
 * below 2^41 per chunk), except the top chunk, which carries the sum's high
 * part: |sum| < n 2^1024 and the top chunk weighs 2^1037, so it stays below
 * n 2^-13 + 2^32 < 2^63 in magnitude for any n below 2^75. */
#define XS_NOALLOC_MAX_TERMS (((int64_t)1) << 45)

/* Exact sum for callers that cannot allocate device memory. The paper has no
 * counterpart: it is a packaging of the single-array sum for such callers.
 *
 * Every other entry point may call cudaMalloc on first use (a per-stream work
 * space). Some callers must not let a library do that: code inside a host
 * application or framework that owns all device memory through its own pool
 * and budget (a hidden cudaMalloc escapes its accounting, and cudaFree
 * synchronizes the whole device), latency-bound loops that cannot afford an
 * allocation's unpredictable cost, and processes whose device memory is
 * already full. This entry point performs no cudaMalloc, cudaFree,
 * cudaMallocHost or other allocating call (torch's allocator included).
 *
 * Its only scratch is one 560-byte accumulator per device, a static device
 * array inside the library that every GPU which loads the library holds until
 * the process exits. The caller passes the input d_values[0..n) and the
 * device result slot *d_out, as for xs_sum_async; the call is asynchronous on
 * `stream`. Each call first clears the accumulator (cudaMemsetAsync), then
 * launches the sum, which leaves it cleared again.
 *
 * - The first call on a device looks up that device's address of the
 *   accumulator (with the device current); make that first call before any
 *   stream capture on that device.
 * - Every call on a device shares the one accumulator: calls that overlap on
 *   the GPU (different streams, or different host threads without ordering)
 *   race and give wrong results. Order them on one stream.
 * - n > XS_NOALLOC_MAX_TERMS returns XS_ERR_INVALID_VALUE; other errors as
 *   for xs_sum_async. */
xs_status xs_sum_noalloc(const double* d_values, int64_t n, double* d_out, void* stream);

/* ---------------------------------------------------------------------------
 * Batched segmented sums (CSR)
 * ------------------------------------------------------------------------- */

/* d_out[k] = exact sum of d_values[d_offsets[k] .. d_offsets[k+1]) for
 * k < nseg. d_offsets (nseg + 1 int64, device) must start at 0 and never
 * decrease. The device checks them on every launch: a segment whose start is
 * negative or whose end lies below its start is not read and gets the default
 * quiet NaN 0x7FF8000000000000, and the plan records the fault (see
 * xs_seg_plan_check); offsets past the end of d_values cannot be detected
 * and must not occur. One persistent launch behind a CUDA
 * graph cached per (values, offsets, nseg, out, stream); asynchronous. The
 * first call for a new key allocates and captures, so make it outside any
 * stream capture. */
xs_status xs_sum_segments(const double* d_values, const int64_t* d_offsets, int64_t nseg,
                          double* d_out, void* stream);

/* Comparison baseline of the batched form (not a faster path): the same
 * segment sums as xs_sum_segments, computed as one single-array kernel launch
 * per segment, issued from a C loop on `stream` in the launch shape
 * xs_sum_async would choose for each length. Offsets are HOST int64 (nseg + 1,
 * starting at 0, non-decreasing: checked on the host, XS_ERR_INVALID_VALUE
 * otherwise); arguments are checked once, not per segment. An empty segment
 * writes +0.0 with a memset. Asynchronous; same bits as xs_sum_segments. */
xs_status xs_sum_each_async(const double* d_values, const int64_t* h_offsets, int64_t nseg,
                            double* d_out, void* stream);

/* Explicit plan: owns the work lists and the instantiated graph. */
typedef struct xs_seg_plan_s* xs_seg_plan;
/* Tunables of the segmented kernel; zero fields take the tuned or default value. */
typedef struct xs_seg_options {
  int block;         /* threads per work group of a long-segment tile: 128, 192, 256 or 384
                        with unroll 4; 32, 64, 128 or 192 with unroll 8. Groups smaller than
                        384 threads share one 384-thread block (twelve groups of one warp,
                        six of two, three of 128, two of 192); default 64, two warps */
  int unroll;        /* 16-byte loads per thread per load group; default 8 */
  int tile_elems;    /* elements per work item of a long segment (2 x block .. 2^26);
                        default 2^18 */
  int short_max;     /* segments up to this length (at most 65,280) are summed by one warp;
                        default 4096 */
  int carry_tiles;   /* load groups (2 x unroll adds per thread each) between per-thread carry
                        propagations inside a tile longer than 2040 values per thread; 0 gives
                        the longest interval that keeps 2047 adds, larger values are rejected */
} xs_seg_options;
xs_status xs_seg_plan_create(xs_seg_plan* plan, const double* d_values, const int64_t* d_offsets,
                             int64_t nseg, double* d_out, const xs_seg_options* opts,
                             void* stream);
xs_status xs_seg_plan_launch(xs_seg_plan plan, void* stream); /* replays the graph */
xs_status xs_seg_plan_launch_direct(xs_seg_plan plan, void* stream); /* same kernels, no graph */
int xs_seg_plan_kernel_launches(xs_seg_plan plan); /* kernels per launch */
/* Waits for `stream` and reports what the plan's last launch found in the
 * offsets: XS_ERR_INVALID_VALUE if the first offset was not 0 or some segment
 * was malformed (those segments hold the default NaN), else XS_OK. */
xs_status xs_seg_plan_check(xs_seg_plan plan, void* stream);
xs_status xs_seg_plan_destroy(xs_seg_plan plan);

/* Times candidate xs_seg_options on this input and records the fastest for
 * later plans on this device; writes the winner and its median time. */
xs_status xs_autotune_segments(const double* d_values, const int64_t* d_offsets, int64_t nseg,
                               double* d_out, int reps, void* stream, xs_seg_options* best,
                               float* best_us);

/* ---------------------------------------------------------------------------
 * Serving loop: continuous batching of sum and append requests
 *
 * Each request is summed exactly and rounded once (abstract); a session keeps
 * its running exact sum in a device-resident accumulator between requests and
 * rounds only when finished (Discussion: partial superaccumulators are added
 * exactly). A scheduler thread admits queued requests while an accumulator
 * slot and the byte budget allow, packs the admitted ones into one persistent
 * batch launch per scheduling round (smallest requests first), and keeps up to
 * `streams` batches in flight, so requests that arrive while others run join
 * the next batch and their work overlaps on the device. Results are the same
 * bits as the request alone.
 * ------------------------------------------------------------------------- */

typedef struct xs_server_s* xs_server;

typedef struct xs_server_options {
  int64_t budget_bytes; /* admission budget: 8 n bytes per admitted request until it completes,
                           plus 560 B per open accumulator (0 = 40 GB) */
  int max_sessions;     /* accumulator slots, shared by sessions and one-shot sums (0 = 4096) */
  int streams;          /* batches in flight at once (0 = 3) */
  int max_batch;        /* requests per batch launch (0 = 256) */
  int tile_elems;       /* elements per work item of a one-warp group (64 .. 2^26; 0 = 65536) */
  int long_min;         /* requests of at least this many values are summed in block-wide tiles,
                           one large superaccumulator per block (Large, Fig. 4); 0 = 2^18 */
  int long_tile;        /* values per block-wide tile (1024 .. 2^26; 0 = 2^21) */
} xs_server_options;

/* xs_request.flags */
#define XS_REQ_FINISH 1u /* after adding the data: round the session, return it, close it */

typedef struct xs_request {
  uint64_t session;       /* 0 = one-shot sum of the data; else an id from xs_server_open_session */
  const double* d_values; /* device array, read when the request runs: keep it valid until done */
  int64_t n;
  uint32_t flags;         /* XS_REQ_FINISH (implied for one-shot sums) */
  uint32_t reserved;
} xs_request;

typedef struct xs_result {
  int32_t status;  /* XS_OK when done; XS_ERR_NOT_READY while queued or running */
  int32_t reserved;
  double value;    /* rounded exact sum of a one-shot or finishing request (NaN for appends) */
  int64_t t_submit_ns, t_admit_ns, t_launch_ns, t_done_ns; /* server clock, ns since creation */
} xs_result;

typedef struct xs_server_stats {
  int64_t submitted, completed, batches, bytes_done;
  int64_t queued, in_flight_bytes, open_sessions;
} xs_server_stats;

/* Creates the server on the current device: allocates the slot pool and the
 * per-stream batch buffers, starts the scheduler thread. */
xs_status xs_server_create(xs_server* s, const xs_server_options* opts);
/* Reserves an accumulator slot for a session (XS_ERR_BUDGET if none is free). */
xs_status xs_server_open_session(xs_server s, uint64_t* session);
/* Queues a request (thread-safe). Requests of one session apply in submission
 * order. XS_ERR_BUDGET if 8 n alone exceeds the budget; XS_ERR_INVALID_POINTER
 * for a non-device array; XS_ERR_INVALID_VALUE for an unknown or finished
 * session. */
xs_status xs_server_submit(xs_server s, const xs_request* r, uint64_t* request_id);
/* Non-blocking: out->status is XS_ERR_NOT_READY until the request is done. */
xs_status xs_server_poll(xs_server s, uint64_t request_id, xs_result* out);
/* Blocks up to timeout_ns (< 0: no limit); XS_ERR_TIMEOUT if still not done. */
xs_status xs_server_wait(xs_server s, uint64_t request_id, int64_t timeout_ns, xs_result* out);
xs_status xs_server_stats_get(xs_server s, xs_server_stats* out);

/* One request of a replayed arrival trace. */
typedef struct xs_replay_item {
  int64_t t_ns;           /* submit time, ns after the replay starts (non-decreasing) */
  uint64_t session_tag;   /* 0 = one-shot sum; else items with the same tag form one session,
                             opened at its first item */
  const double* d_values; /* device array */
  int64_t n;
  uint32_t flags;         /* XS_REQ_FINISH on a session's last item */
  uint32_t reserved;
} xs_replay_item;

/* Submits items[0..count) at their times from the calling thread (a load
 * generator that keeps microsecond timing, which a scripting language cannot),
 * writing each request id. *start_ns receives the replay start on the server
 * clock, so item k arrived at *start_ns + items[k].t_ns. Opening a session
 * waits up to 60 s for a free slot (XS_ERR_TIMEOUT after that). Returns after
 * the last submit; collect results with xs_server_wait. */
xs_status xs_server_replay(xs_server s, const xs_replay_item* items, int64_t count,
                           uint64_t* request_ids, int64_t* start_ns);
/* Comparison baseline of the serving loop (not a server): runs the requests of
 * items[0..count) one at a time in order, each alone, ignoring the arrival
 * times, from a C loop on `stream`. A one-shot item is one single-array sum
 * whose result the loop waits for; a session item (same session_tag) is
 * appended to that session's own device accumulator and waited for, and the
 * session's finishing item is rounded once (Discussion: partial
 * superaccumulators add exactly). h_values[k] receives the rounded sum of a
 * one-shot or finishing item (quiet NaN for appends); done_ns[k] the time, ns
 * since the call started, at which item k completed. Allocates one 560-byte
 * accumulator per open session (freed when it finishes or on return). */
xs_status xs_serial_replay(const xs_replay_item* items, int64_t count, double* h_values,
                           int64_t* done_ns, void* stream);

/* Waits for every queued and running request, stops the thread, frees. */
xs_status xs_server_destroy(xs_server s);

/* ---------------------------------------------------------------------------
 * Device-resident accumulators (partial sums that are merged exactly,
 * Discussion; canonical form after carry propagation, small section)
 * ------------------------------------------------------------------------- */

#define XS_ACC_BYTES 560 /* exported state: 67 int64 chunks + flags + NaN key */

typedef struct xs_acc_s* xs_acc;
xs_status xs_acc_create(xs_acc* h, void* stream);        /* allocates; value: empty sum */
xs_status xs_acc_init(xs_acc h, void* stream);           /* reset to the empty sum */
xs_status xs_acc_add(xs_acc h, const double* d_values, int64_t n, void* stream); /* append */
xs_status xs_acc_merge(xs_acc dst, xs_acc src, void* stream); /* dst += src; src unchanged */
xs_status xs_acc_round(xs_acc h, double* d_out, void* stream); /* async; state unchanged */
/* Correctly rounded (accumulated value) / divisor, divisor >= 1 (e.g. the
 * mean of everything appended); async; state unchanged. */
xs_status xs_acc_round_div(xs_acc h, int64_t divisor, double* d_out, void* stream);
xs_status xs_acc_export(xs_acc h, void* h_buf, void* stream); /* XS_ACC_BYTES, blocking */
xs_status xs_acc_import(xs_acc h, const void* h_buf, void* stream); /* blocking */
xs_status xs_acc_destroy(xs_acc h);
void* xs_acc_device_state(xs_acc h); /* device address of the 560-byte state */

/* ---------------------------------------------------------------------------
 * Test hooks (no counterpart in the paper): allocation-failure injection
 * ------------------------------------------------------------------------- */

/* Makes the k-th next device or pinned-host allocation of the library (k >= 1;
 * 1 = the next one) fail as if memory were exhausted, so every entry point's
 * XS_ERR_OUT_OF_MEMORY path and its unwinding can be tested; k = 0 disarms.
 * Process-wide; not for production use. */
xs_status xs_debug_fail_allocation(int64_t k);
/* Number of device and pinned-host allocations the library currently holds
 * (workspaces, handles, plans, servers): a failed call must leave it as it
 * was. */
int64_t xs_debug_live_allocations(void);

/* 1 if this library was built with -DXS_DEBUG (build.py's debug build), else 0.
 * In that build the kernels check their chunk indices (small accumulator
 * chunks 0..66, large accumulator indices 0..4095, flushed pieces inside the
 * small accumulator), the add bound between carry propagations (at most 2047
 * adds, and every chunk within what they can reach) and the segmented tile
 * table index; a failed check skips the access it guards and records a code. */
int xs_is_debug_build(void);
/* Waits for the device, then stores in *codes the OR of the codes recorded
 * since the last call (1 small chunk index, 2 carry interval, 4 chunk bound,
 * 8 large index, 16 flush index, 32 table index) and clears them. Always 0
 * outside the debug build. XS_ERR_INVALID_POINTER if codes is NULL. */
xs_status xs_debug_status(uint64_t* codes);

#ifdef __cplusplus
}
#endif

#endif /* XSUM_H */
