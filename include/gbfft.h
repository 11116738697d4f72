/*
 * gbfft -- batched complex FFT for one NVIDIA GB300 (sm_103a), C ABI.
 *
 * Method: Bergach, Kofman, de Simone, Tissot, Syska, "Efficient FFT mapping on
 * GPU for radar processing application: modeling and implementation" (2015).
 *   Sec. 2.1      the DFT X(k) = sum_n x(n) w_N^{nk}, w_N = exp(-2 pi i / N);
 *                 the backward transform flips the exponent's sign; twiddle
 *                 factors are precomputed and stored; mixed-radix stages.
 *   Sec. 3.2      radix clustering bounded by on-chip storage; per-(radix,
 *                 start stage) stage costs; shortest path over the schedule
 *                 digraph picks the radix schedule; Eq. 1 bandwidth bound.
 *   Sec. 3.3      transforms larger than one on-chip block are split and
 *                 merged (four-step: column FFTs, twiddle, row FFTs).
 *   Sec. 3.4      one transform per compute unit, global memory touched only at
 *                 the first read and the last write; blocked transpose.
 *   Sec. 3.1      the radar application: FFTs, a transpose, FFTs (2D frame).
 *
 * Conventions shared by every entry point:
 *   - Data are complex64: interleaved (re, im) IEEE float32, 8 bytes per
 *     element, natural order in and out (complex32, 4 bytes per element, for
 *     plans and jobs of precision FFT_PREC_TC_FP16_C32).
 *   - 1D: element i of transform b is at b*n[0] + i.
 *     2D: n = {rows, cols}; frame b is row-major [rows][cols] (cols
 *     contiguous) at b*rows*cols.
 *   - direction FFT_FORWARD (-1) uses exp(-2 pi i nk/N); FFT_INVERSE (+1) uses
 *     exp(+2 pi i nk/N) and is NOT normalised: inverse(forward(x)) = N x.
 *   - Pointers named `in`/`out` are device pointers owned by the caller,
 *     aligned to the element size (8 bytes; 4 for complex32).  `in` is never written.  in == out (in place) is allowed.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *   - Errors are returned as fft_status_t and never abort; fft_last_error()
 *     gives a human-readable message for the calling thread.  No entry point
 *     falls back to the CPU: without a usable CUDA device plan creation fails
 *     with FFT_ERR_CUDA.
 */
#ifndef GBFFT_H
#define GBFFT_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define GBFFT_API __attribute__((visibility("default")))
#else
#define GBFFT_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fft_plan_s* fft_plan_t; /* opaque; owned by the library */

typedef enum {
  FFT_OK = 0,
  FFT_ERR_INVALID_ARG = 1,      /* null pointer, bad enum, misaligned pointer */
  FFT_ERR_UNSUPPORTED_SIZE = 2, /* n not a power of two, or outside 2^0 .. 2^24 */
  FFT_ERR_OUT_OF_MEMORY = 3,    /* device allocation for tables / workspace failed */
  FFT_ERR_CUDA = 4,             /* a CUDA call failed (message in fft_last_error) */
  FFT_ERR_TIMEOUT = 5,          /* a bounded wait gave up */
  FFT_ERR_BAD_PLAN = 6,         /* null or destroyed plan, or plan/device mismatch */
  FFT_ERR_NOT_IMPLEMENTED = 7   /* a valid request this build does not provide */
} fft_status_t;

enum { FFT_FORWARD = -1, FFT_INVERSE = +1 };

/*
 * Precision classes.  Data are complex64 (two FP32 values, 8 bytes) in every
 * class but FFT_PREC_TC_FP16_C32; the tensor-core classes compute each
 * radix-16 stage as a dense 16-point DFT matmul on the tensor cores with FP32
 * accumulation (twiddles stay FP32), after a radix-2/4/8 FP32 stage when the
 * length is not a power of 16, for batched 1D lengths 2^4 .. 2^14 in one pass
 * and 2^15 .. 2^24 in six steps (transpose, tensor-core rows of N1, transpose
 * with the twiddle w_N^{n2 k1}, rows of N2, transpose; N = N1 N2, a workspace
 * of 2 min(batch, c) n elements, c = max(1, 2^28 / n)):
 *   FFT_PREC_TC_FP16    stage inputs and DFT matrix rounded to FP16 (each
 *                       stage's input scaled by 1/16, exactly undone at the end)
 *   FFT_PREC_TC_BF16    rounded to BF16
 *   FFT_PREC_TC_BF16X3  split x = x_hi + x_lo, F = F_hi + F_lo in BF16 and
 *                       x_hi F_hi + x_hi F_lo + x_lo F_hi accumulated (about
 *                       16 significant bits per product: near-FP32 accuracy)
 *   FFT_PREC_TC_FP16_C32  the FP16 class with input and output stored as
 *                       complex32: FP16 real and imaginary parts interleaved,
 *                       4 bytes per element, so a transform moves half the
 *                       bytes of the complex64 classes.  The output is rounded
 *                       to FP16 once more; a value beyond the FP16 range
 *                       (|v| > 65504) becomes an infinity.  Buffers need
 *                       4-byte alignment.  Plans, fft_execute,
 *                       fft_execute_graph, fft_execute_host (byte counts of 4
 *                       per element) and the server take it.
 */
enum {
  FFT_PREC_FP32 = 0,     /* FP32 data, FP32 arithmetic, FP64-generated twiddles */
  FFT_PREC_TC_FP16 = 1,
  FFT_PREC_TC_BF16 = 2,
  FFT_PREC_TC_BF16X3 = 3,
  FFT_PREC_TC_FP16_C32 = 4
};

/*
 * Create a plan for `batch` transforms of shape n[0..dims) (dims 1 or 2),
 * direction FFT_FORWARD / FFT_INVERSE, precision FFT_PREC_*.
 * Each length must be a power of two; 1D n[0] in [1, 2^24]; 2D rows and cols in
 * [1, 2^14].  batch >= 0 (batch 0 gives a plan whose execute does nothing).
 * The plan is bound to the CUDA device current at creation.  It allocates its
 * twiddle tables and, for 1D n > 2^14, a workspace of min(batch, c)*n
 * complex64 with c = max(1, 2^28 / n) (query with fft_plan_workspace_bytes):
 * such plans run larger batches in sub-batches of c transforms, one after the
 * other on the stream, which bounds the working set of their strided passes.
 * Nothing is allocated by fft_execute.
 * Sec. 2.1 (DFT, direction), Sec. 3.2 (block size from on-chip limits,
 * radix schedule), Sec. 3.3 (split into passes).
 */
GBFFT_API fft_status_t fft_plan_create(fft_plan_t* plan, const int64_t* n, int dims, int64_t batch,
                             int direction, int precision);

/*
 * Options for fft_plan_create_ex.  Zero-initialise and set what you need;
 * a zero field means "library default".
 *   autotune      1: time candidate radix schedules / tile shapes on this GPU at
 *                 plan creation and keep the fastest (Sec. 3.2: stage costs are
 *                 benchmarked, the shortest path over the schedule digraph is
 *                 taken, then checked against whole-pass timings).
 *   radix         elements per thread (2, 4, 8 or 16): the largest radix of the
 *                 on-chip block (Sec. 3.2 "Insights").
 *   schedule      log2 of the radix of each stage of the first pass, LSB-first
 *                 nibbles, terminated by a zero nibble; e.g. 0x344 = radix
 *                 16, 16, 8 (in that order).  Must sum to the pass length.
 *   max_block_log2  largest on-chip block 2^k (default from shared memory);
 *                 smaller values force multi-pass splits (testing).
 *   tile          transforms per thread block for passes that allow a choice.
 *   generic       1: run every pass with the run-time-parameter kernel even
 *                 where a compile-time specialisation of the shape exists.
 *   variant       kernel variant: 0 library choice, 1 register kernel (one
 *                 tile per block), 2 TMA-staged kernel (batched contiguous
 *                 N = 2^12..2^14, where the library's own choice is the
 *                 staged kernel for 2^13 and 2^14 and the register kernel
 *                 for 2^12: the next transform is copied into shared
 *                 memory while the current one is computed), 3 register
 *                 kernel on a persistent grid that prefetches its next tile
 *                 into L2 (every pass with a compile-time shape: contiguous
 *                 tiles, and the strided column tiles of two-pass and 2D
 *                 plans), 4 as 2 but without tensor maps: the column tiles
 *                 of strided passes copy their rows with per-thread 16-byte
 *                 copies instead of tensor-map (TMA) boxes and write their
 *                 output with register stores only.
 *   epilogue      how a two-pass 1D plan finds the twiddle w_N^{n2 k1} applied
 *                 between its passes: 0 library choice, 1 two small tables
 *                 (w = hi[m >> b] * lo[m mod 2^b]), 2 one table of N entries laid
 *                 out like the first pass's output (coalesced loads, N*8 bytes
 *                 more plan memory), 3 computed in-kernel from the exact FP32
 *                 angle 2m/N with sincospi, 4 factored: the first pass's last
 *                 stage writes k1 = jb + i*Ns, and w_N^{n2 k1} is computed as
 *                 w_N^{n2 jb} * (w_N^{n2 Ns})^i (two sincospi per butterfly,
 *                 the powers by products; no table).
 *   split_log2    two-pass 1D plans: log2 of the first (column) pass length N1
 *                 (0 = library choice, N1 <= N2).
 */
typedef struct {
  int autotune;
  int radix;
  uint32_t schedule;
  int max_block_log2;
  int tile;
  int generic;      /* 1: never use the compile-time specialised kernels (testing) */
  int variant;      /* kernel variant, see above */
  int epilogue;     /* four-step twiddle source, see above */
  int split_log2;   /* two-pass split N = N1 * N2, log2 N1 */
  int reserved[4];
} fft_plan_options_t;

GBFFT_API fft_status_t fft_plan_create_ex(fft_plan_t* plan, const int64_t* n, int dims, int64_t batch,
                                int direction, int precision,
                                const fft_plan_options_t* options);

/*
 * Enqueue the transform of `in` into `out` on `stream` (device pointers, see
 * the conventions above).  Asynchronous: returns after enqueueing; no host
 * synchronisation and no allocation.  A plan may be used from several host
 * threads only on distinct streams and only if no two executions overlap on
 * the device when the plan has a workspace (multi-pass 1D).
 * Sec. 3.4 (each pass reads and writes global memory once).
 */
GBFFT_API fft_status_t fft_execute(fft_plan_t plan, const void* in, void* out, void* stream);

/*
 * Host-memory variant: copy `host_in` (batch transforms, pinned or pageable)
 * to the device buffer `dev_in`, transform into `dev_out`, copy `dev_out` back
 * to `host_out`, all on `stream`, split into chunks of whole transforms so that
 * copies in both directions overlap the kernels.  dev_in / dev_out are caller-
 * owned device buffers of the full problem size (dev_in may equal dev_out).
 * Asynchronous like fft_execute; host buffers must stay valid until the stream
 * reaches this point.  Chunking applies to 1D plans; 2D plans run whole.
 */
GBFFT_API fft_status_t fft_execute_host(fft_plan_t plan, const void* host_in, void* host_out,
                              void* dev_in, void* dev_out, void* stream);

/*
 * Same transform as fft_execute, replayed from a CUDA graph: the first call for
 * a given (in, out) pair captures the plan's launches into a graph (on a
 * private stream) and instantiates it; later calls with the same pair launch
 * that graph on `stream`, which costs one launch instead of one per pass.
 * Up to 8 pairs are kept per plan (least recently used is replaced).  The
 * first call for a pair does the capture work; make it before any capture
 * the caller itself runs on `stream`.
 */
GBFFT_API fft_status_t fft_execute_graph(fft_plan_t plan, const void* in, void* out, void* stream);

/* Release the plan, its tables and workspace.  Null is accepted. */
GBFFT_API fft_status_t fft_plan_destroy(fft_plan_t plan);

/* Bytes of device workspace owned by the plan (0 for single-pass plans). */
GBFFT_API fft_status_t fft_plan_workspace_bytes(fft_plan_t plan, size_t* bytes);

/* Kernel launches one fft_execute enqueues. */
GBFFT_API fft_status_t fft_plan_launch_count(fft_plan_t plan, int* launches);

/*
 * JSON description of the plan (passes, radix schedules, tile shapes, grid,
 * shared memory; "kernels": per pass the kernel bound to it -- "staged" (the
 * TMA / cp.async staged kernel, used when the source is 16-byte aligned, else
 * the compile-time kernel of the shape), "compile_time", "generic",
 * "tensor_core" or "copy" -- with its persistent-grid size and L2-prefetch
 * flag) written to buf (NUL-terminated, truncated to len).  Returns
 * FFT_ERR_INVALID_ARG if buf is too small for the whole text.
 */
GBFFT_API fft_status_t fft_plan_describe(fft_plan_t plan, char* buf, size_t len);

/*
 * Same planning as fft_plan_create_ex but for a hypothetical device and with
 * no CUDA call at all: sm_count and smem_optin_bytes describe the GPU.  Writes
 * the plan's JSON description.  Lets the planner be checked on a host without
 * a GPU.
 */
GBFFT_API fft_status_t fft_plan_dry_run(const int64_t* n, int dims, int64_t batch, int direction,
                              int precision, const fft_plan_options_t* options, int sm_count,
                              int smem_optin_bytes, char* buf, size_t len);

/* Wait for the stream-ordered work of the plan's last execute and report any
 * asynchronous CUDA error it raised. */
GBFFT_API fft_status_t fft_plan_sync_status(fft_plan_t plan, void* stream);

/* -------------------------------------------------- fast convolution --
 * Matched filtering of radar lines (Sec. 2.2, the range-Doppler processing
 * chain of the SAR application: range compression correlates each received
 * range line with the transmitted chirp; azimuth compression does the same
 * along each range bin with the azimuth chirp).  Each line goes through one
 * kernel pass: forward DFT, multiply by a filter spectrum, unnormalised
 * inverse DFT, read once from and written once to HBM:
 *
 *     out_line = scale * IDFT( H_line . DFT(in_line) )
 *
 * IDFT is the unnormalised inverse (exponent +2 pi i nk/N); scale = 1/N makes
 * this the circular convolution of the line with the filter's impulse
 * response, and H = conj(DFT(chirp)) makes it the matched filter (circular
 * cross-correlation with the chirp).  For 2D plans (n = {rows, cols}) the
 * rows (range, cols points each) are filtered first, then the columns
 * (azimuth, rows points each); the result is back in the signal domain.
 * Range-cell migration correction is not part of this step.
 */
typedef struct {
  /* Filter spectrum, complex64 in device memory owned by the caller; it must
   * stay valid and unchanged for the plan's lifetime (the plan keeps the
   * pointer, not a copy).  8-byte aligned. */
  const void* h;
  /* 1: one filter of N points for every line, h[k] for k < N.
   * Otherwise one filter per line, laid out like one frame of the data with
   * each line's filter along that line: 1D (lines = batch): h[b*N + k];
   * 2D rows filter (lines = rows): h[r*cols + k]; 2D columns filter
   * (lines = cols): h[k*cols + c].  Any other value is FFT_ERR_INVALID_ARG. */
  int64_t lines;
  /* Factor applied with the filter (1/N gives the normalised inverse). */
  float scale;
  int32_t reserved; /* 0 */
} fft_filter_t;

/*
 * Plan a fast convolution of `batch` 1D lines of length n[0] (dims = 1) or of
 * `batch` frames n = {rows, cols} (dims = 2) with filters[0 .. dims-1]
 * (filters[0] along the columns / the only dimension, filters[1] along the
 * rows of a 2D frame).  Every length must be a power of two in [2, 2^14] (one
 * line per on-chip block); longer lines return FFT_ERR_NOT_IMPLEMENTED.  FP32
 * only.  Execute with fft_execute / fft_execute_host / fft_execute_graph;
 * in == out is allowed.  options may be NULL; radix, schedule, tile, generic
 * and variant (3: persistent grid prefetching each block's next tile into L2)
 * apply, autotune is ignored.
 */
GBFFT_API fft_status_t fft_conv_plan_create(fft_plan_t* plan, const int64_t* n, int dims,
                                            int64_t batch, const fft_filter_t* filters,
                                            const fft_plan_options_t* options);

/* fft_plan_dry_run for a convolution plan (filters[d].h may be NULL here). */
GBFFT_API fft_status_t fft_conv_plan_dry_run(const int64_t* n, int dims, int64_t batch,
                                             const fft_filter_t* filters,
                                             const fft_plan_options_t* options, int sm_count,
                                             int smem_optin_bytes, char* buf, size_t len);

/*
 * Allocation-free execution.  The paper has no counterpart: this entry point
 * exists for callers that may not allocate GPU memory while they run -- a
 * real-time radar loop that reserves all of its memory at start-up and cannot
 * afford cudaMalloc's blocking and device synchronisation later, or code
 * embedded in a framework that owns the device-memory budget.  It transforms
 * `batch` contiguous 1D sequences of length n from `in` to `out` on `stream`
 * (same data conventions as fft_execute) without a plan, and allocates
 * nothing: the twiddle tables and the between-pass workspace live in one array
 * the library reserves statically on every GPU that loads it (64 MiB of
 * workspace plus 512 KiB of tables, held until the process exits).
 *   - n is a power of two in [1, 2^23].  For n > 2^14 (two passes) n*batch
 *     must be at most 2^23 complex elements; larger problems return
 *     FFT_ERR_UNSUPPORTED_SIZE (create a plan instead).
 *   - The first call on a device looks up the array's device address; make
 *     that first call before any stream capture begins.  The address is kept
 *     for the life of the process: resetting the device (cudaDeviceReset, or
 *     a reset of its primary context) while the library is loaded is not
 *     supported.
 *   - Every call uses the same array and leaves its contents behind.  Calls
 *     whose GPU work overlaps (different streams, several host threads) race
 *     and corrupt each other's results: serialise them.  Each call clears the
 *     status word it uses and writes the workspace before reading it; the
 *     twiddle tables are regenerated whenever the table layout differs from
 *     the one the previous call on the device left.
 *   - The library remembers, per device and in host memory only, the plan of
 *     the last (n, batch, direction) it was called with, so a loop that calls
 *     with one shape plans and prepares its kernels once.
 *   - Errors in the arguments and in enqueueing are returned.  The staged
 *     kernels' bounded waits for their own copies into shared memory (about
 *     0.5 s each, far above any copy's duration) are not reported by this
 *     entry point: if one ever gave up, the call would return FFT_OK with part
 *     of the output unwritten.  Callers that need that guarantee create a plan
 *     and check fft_plan_sync_status.
 */
GBFFT_API fft_status_t fft_execute_noalloc(int64_t n, int64_t batch, int direction,
                                           const void* in, void* out, void* stream);

/* ------------------------------------------------------- serving loop --
 * Continuous batching of FFT jobs on one GPU (the paper's top level, Sec. 3.4:
 * a batch of independent transforms spread over the compute units, each
 * reading and writing the shared memory hierarchy once, with a dataflow model
 * of reads, compute and writes).  Jobs reference caller-owned device buffers.
 * A worker thread admits jobs in arrival order while the bytes they hold when
 * running (input + output + workspace) fit the memory budget, coalesces every
 * waiting job of the same shape, direction and precision into one launch (for
 * batched 1D single-pass FP32 shapes: one kernel over all their buffers),
 * spreads launches over several streams so they overlap (small groups on the
 * stream whose queued work is estimated to end first; groups large enough to
 * fill the GPU alone one after another on the first stream), and keeps plans
 * and twiddle tables resident per shape.  Jobs that arrive while others run are admitted
 * as soon as memory frees up.  When the oldest waiting job does not fit, later
 * jobs that fit may start first if, by an estimate of run times from the bytes
 * each job moves, they cannot delay it (backfilling; strict_order turns this
 * off).
 */
typedef struct fft_server_s* fft_server_t;

typedef struct {
  size_t memory_budget_bytes; /* default 64 GiB */
  int streams;                /* default 4 */
  int max_group;              /* most jobs coalesced into one group, default 256 */
  int max_running;            /* most groups on the GPU at once, default 4 x streams */
  int fail_workspace_alloc;   /* testing: workspace allocations fail (host-side fault) */
  int strict_order;           /* 1: admit strictly in arrival order (no backfilling) */
  int large_group_log2;       /* groups of at least 2^k complex elements in total run on
                                 the first stream, one after another, and smaller ones on
                                 the others (0: k = 23; -1: every group may go to any
                                 stream).  Large groups fill the GPU on their own; run
                                 concurrently, their working sets add up and the strided
                                 passes lose bandwidth (measured: 4 streams 3.26 TB/s
                                 against 3.98 TB/s on one, same job mix) */
  int reserved[5];
} fft_server_options_t;

typedef struct {
  int dims;          /* 1 or 2 */
  int64_t n[2];      /* lengths as in fft_plan_create */
  int64_t batch;     /* >= 1 */
  int direction;     /* FFT_FORWARD / FFT_INVERSE */
  int precision;     /* FFT_PREC_* */
  const void* in;    /* device, batch x n complex64, untouched until the job ends */
  void* out;         /* device, same size */
} fft_job_t;

typedef struct {
  int status;        /* fft_status_t of the job */
  double latency_ms; /* submit -> completion observed */
  double queue_ms;   /* submit -> launch */
} fft_job_result_t;

typedef struct {
  uint64_t submitted, completed, failed;
  uint64_t launches;        /* kernel-level launches issued */
  uint64_t groups;          /* admitted groups */
  uint64_t coalesced_jobs;  /* jobs that shared a coalesced launch */
  uint64_t workspace_allocations;
  size_t peak_bytes_in_flight, budget_bytes;
  double p50_ms, p99_ms, mean_ms, max_ms; /* latency of completed jobs (the most recent 2^20) */
  double wall_s;            /* first submit -> last completion */
  double gflops;            /* 5 N log2 N of completed jobs / wall_s */
  uint64_t backfilled_jobs; /* jobs admitted ahead of an older waiting job */
  double host_launch_s;     /* worker thread time spent enqueueing groups */
  double group_stream_s;    /* sum over completed groups of the time from their first
                               launch to their completion on their stream (CUDA events);
                               above wall_s when groups overlap on the device */
} fft_server_stats_t;

/* Start a server on the current device (options may be NULL). */
GBFFT_API fft_status_t fft_server_create(fft_server_t* server, const fft_server_options_t* options);
/* Queue a job; returns a ticket.  Shape errors and jobs larger than the budget
 * are rejected here. */
GBFFT_API fft_status_t fft_server_submit(fft_server_t server, const fft_job_t* job, uint64_t* ticket);
/* Wait for a job (timeout_s < 0: no limit); FFT_ERR_TIMEOUT if it is not done
 * in time (it keeps running).  Each ticket can be waited for once. */
GBFFT_API fft_status_t fft_server_wait(fft_server_t server, uint64_t ticket, double timeout_s,
                                       fft_job_result_t* result);
/* Hold (paused = 1) or resume (0) admissions: jobs submitted while held are
 * queued and then considered together, so a burst of same-shape jobs is
 * coalesced; running work is unaffected. */
GBFFT_API fft_status_t fft_server_pause(fft_server_t server, int paused);
/* Wait until nothing is queued or running. */
GBFFT_API fft_status_t fft_server_drain(fft_server_t server, double timeout_s);
GBFFT_API fft_status_t fft_server_stats(fft_server_t server, fft_server_stats_t* stats);
/* Stop the worker, wait for running work, free plans and workspaces. */
GBFFT_API fft_status_t fft_server_destroy(fft_server_t server);

/* ------------------------------------------------ persistent work queue --
 * A persistent batch kernel fed by a device-visible job queue (Sec. 3.4: the
 * top-level batch handed to every compute unit, here without one kernel
 * launch per job).  One queue serves one transform shape: batched 1D FP32
 * transforms of length n (a power of two, 2 .. 2^12), up to max_batch per
 * job, in one direction.  Jobs are descriptors (in, out, batch) written by
 * the host into a ring of `slots` entries in mapped pinned host memory; a
 * worker kernel launched cooperatively (all of its blocks resident at once)
 * on the queue's own stream polls the ring, and for each job every block
 * computes its share of the tiles; the last block to finish publishes the
 * job's completion in the ring.  Jobs complete in ticket order.
 *
 * The worker runs while jobs keep arriving: when no job arrives for about
 * 2^16 polls (tens of milliseconds) or fft_queue_destroy asks it to stop, it
 * exits, and the next submit or wait launches it again.  Every wait in the
 * worker is bounded.  While it runs it holds its blocks' SMs (the `blocks`
 * of fft_queue_create: 0 = one per tile of a max_batch job, at most what the
 * GPU holds at once) and a device-wide synchronisation waits for it to go
 * idle.  The queue allocates at creation only; submit and wait allocate
 * nothing.  Calls on one queue are thread-safe; a wait polls its job's
 * completion without holding the queue's lock, so other threads can submit
 * meanwhile.
 */
typedef struct fft_queue_s* fft_queue_t;

/* Create a queue on the current device.  slots: ring entries (1 .. 4096;
 * 0 = 64).  blocks: worker blocks (0 = automatic).  n outside 2 .. 2^12 (or
 * not a power of two): FFT_ERR_NOT_IMPLEMENTED / FFT_ERR_UNSUPPORTED_SIZE. */
GBFFT_API fft_status_t fft_queue_create(fft_queue_t* queue, int64_t n, int64_t max_batch,
                                        int direction, int slots, int blocks);
/* Append a job: `batch` (1 .. max_batch) transforms from `in` to `out`
 * (device pointers, 8-byte aligned, complex64; in == out allowed).  The
 * worker runs on the queue's own stream and is not ordered after any other
 * stream: `in` must hold its data when submit is called (the stream that
 * wrote it synchronised).  The buffers must stay valid and `in` unchanged
 * until the job completes.
 * Returns its ticket (1, 2, 3, ...).  When the ring is full, waits (up to
 * about one second) for the oldest job's slot; FFT_ERR_TIMEOUT if it stays
 * busy. */
GBFFT_API fft_status_t fft_queue_submit(fft_queue_t queue, const void* in, void* out,
                                        int64_t batch, uint64_t* ticket);
/* Wait until job `ticket` has completed (timeout_s < 0: no limit): FFT_OK,
 * FFT_ERR_TIMEOUT (still pending), FFT_ERR_INVALID_ARG (ticket never
 * issued), or FFT_ERR_CUDA (the worker failed).  Once it returns FFT_OK the
 * job's output is complete in device memory. */
GBFFT_API fft_status_t fft_queue_wait(fft_queue_t queue, uint64_t ticket, double timeout_s);
/* Counters: worker launches so far and jobs completed. */
GBFFT_API fft_status_t fft_queue_info(fft_queue_t queue, int64_t* worker_launches,
                                      uint64_t* completed);
/* Stop the worker once the jobs already submitted are done, then free the
 * queue. */
GBFFT_API fft_status_t fft_queue_destroy(fft_queue_t queue);

/* ---------------------------------------------------- synthetic inputs --
 * Seeded test signals generated on the device (the paper's workloads are
 * synthetic radar data; this fills the uniform-noise inputs of the benchmarks
 * without a host round trip).  Writes `count` complex64 values to the device
 * buffer `out` (8-byte aligned), element j with real and imaginary parts
 * uniform in [-1, 1) from a counter-based hash (SplitMix64 at stream indices
 * 2 (first + j) and 2 (first + j) + 1 for `seed`), so out = values
 * first .. first + count - 1 of one endless seeded sequence: slices can be
 * generated separately.  Asynchronous on `stream`.  No plan is involved. */
GBFFT_API fft_status_t fft_fill_uniform(void* out, int64_t count, uint64_t seed, uint64_t first,
                                        void* stream);

/* Message of the last failure on the calling thread ("" if none). */
GBFFT_API const char* fft_last_error(void);

/* Diagnostic of the device-side bounded waits.  Every wait in the library's
 * kernels (the staged kernels' and the tensor-core kernel's waits on an
 * mbarrier, the work queue's polls) gives up after a fixed number of polls,
 * sets a status word and returns instead of hanging.  This call runs that
 * wait where it must run out: one block whose threads wait on an mbarrier
 * that nothing completes, with the library's wait loop limited to `polls`
 * polls (1 .. 2^22; 2^22 is the limit the kernels use, about 0.5 s), then
 * reads the status word back.  *gave_up = 1 is the expected result; the call
 * synchronises the current device and leaves it usable.  FFT_ERR_INVALID_ARG
 * for polls outside that range or a null gave_up; FFT_ERR_CUDA if no device. */
GBFFT_API fft_status_t fft_wait_selftest(uint32_t polls, int* gave_up);

/* ------------------------------------------------ schedule model (host) --
 * Sec. 3.2 "FFT performance model": a radix schedule for N = 2^L is a path in
 * the digraph whose nodes are stage indices 0..L and whose edge s -> s+log2(r)
 * means "radix r starting at stage s"; under the stage-independence hypothesis
 * a schedule costs the sum of its edges' benchmarked costs, and the cheapest
 * schedule is the shortest source-to-sink path (Dijkstra).
 *
 * `radix_logs`  allowed log2(radix) values, e.g. {1, 2, 3} for radices 2, 4, 8.
 * `cost`        cost[j * log2n + s] = cost of radix 2^radix_logs[j] starting
 *               at stage s (entries whose edge would overrun the sink are
 *               ignored; a negative or NaN entry removes that edge).
 * These functions touch no GPU.
 */

/* Number of distinct schedules (source-to-sink paths). */
GBFFT_API fft_status_t fft_schedule_count(int log2n, const int* radix_logs, int n_radix, uint64_t* count);

/* Cheapest schedule: writes its radix logs in stage order to path_logs
 * (capacity path_cap) and their number to path_len, total to total_cost. */
GBFFT_API fft_status_t fft_schedule_shortest_path(int log2n, const int* radix_logs, int n_radix,
                                        const double* cost, int* path_logs, int path_cap,
                                        int* path_len, double* total_cost);

/* Cost of a given schedule (radix logs in stage order) under the same model. */
GBFFT_API fft_status_t fft_schedule_path_cost(int log2n, const int* radix_logs, int n_radix,
                                    const double* cost, const int* path_logs, int path_len,
                                    double* total_cost);

/* Sec. 3.2 Eq. 1: bandwidth-bound FFT throughput in GFLOP/s (5 N log2 N
 * convention) for bandwidth `gbs` GB/s when every complex sample of
 * `bytes_per_sample` bytes crosses the bandwidth-limited link `passes` times
 * (the paper's form is bytes_per_sample = 8, passes = 1). */
GBFFT_API double fft_bandwidth_bound_gflops(int64_t n, double gbs, double bytes_per_sample, double passes);

#ifdef __cplusplus
}
#endif

#endif /* GBFFT_H */
