// Persistent work queue (C ABI in include/gbfft.h, fft_queue_*): a batch
// kernel that stays resident and takes its jobs from a ring of descriptors in
// mapped pinned host memory, instead of one kernel launch per job (the
// top-level batch of Sec. 3.4 handed to every compute unit).
//
// Protocol, per ticket t (1, 2, ...; ring slot s = (t - 1) mod slots):
//   host    writes in / out / batch of slot s, then releases seq = t;
//   block 0 polls seq (acquire, system scope, bounded), copies the
//           descriptor into the slot's device record `go` and releases
//           go.ticket = t (device scope); after too many empty polls, or
//           when the host sets the stop word, it releases go.ticket = QUIT
//           instead and the worker ends;
//   others  poll go.ticket (acquire, device scope, bounded) and follow
//           block 0's decision, so either every block runs job t or none;
//   all     compute their tiles of the job (grid-strided), then count
//           themselves done; the last block releases ring done = t (system
//           scope) for the host.
// The host reuses a slot only after its previous job is done, so go and the
// block counter of a slot are never live for two tickets.  The worker is
// launched cooperatively (all blocks resident: none waits on a block that
// cannot run), and relaunched by the host when it has exited with jobs pending.
#include <cuda_runtime.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <mutex>
#include <thread>

#include "../../include/gbfft.h"
#include "exec.h"
#include "kernels.h"
#include "kernels_impl.cuh"
#include "planner.h"
#include "queue_ring.h"
#include "trace.h"

namespace gbfft {
fft_status_t set_error(fft_status_t st, const char* msg);
}

using namespace gbfft;

namespace {

constexpr uint32_t kQueueMagic = 0x51554555u;
constexpr uint64_t kQuit = ~0ull;
constexpr uint32_t kIdlePolls = 1u << 16;   // block 0: empty polls before the worker ends
constexpr uint64_t kFollowPolls = 1ull << 21;  // other blocks: polls of go before giving up

struct alignas(64) QSlot {  // mapped pinned host memory
  uint64_t seq;    // ticket of the job in the slot (host: release)
  uint64_t done;   // ticket of the last job of the slot completed (device: release)
  uint64_t in, out;
  int64_t batch;
};
struct alignas(64) QHeader {  // mapped pinned host memory, before the slots
  uint32_t stop;
};
struct alignas(64) QGo {  // device memory, one per slot
  uint64_t ticket;  // t, or kQuit
  uint64_t in, out;
  int64_t batch;
};

struct QueueArgs {
  QSlot* ring;            // device alias of the ring
  const QHeader* header;  // device alias of the header
  QGo* go;
  int* cnt;               // blocks done with the slot's current ticket
  int* status;            // set when a block gave up following block 0
  int slots;
  uint64_t first_ticket;
};

// ---------------------------------------------------------------- device --

__device__ __forceinline__ uint64_t ld_acquire_sys(const void* p) {
  uint64_t v;
  asm volatile("ld.acquire.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint32_t ld_acquire_sys32(const void* p) {
  uint32_t v;
  asm volatile("ld.acquire.sys.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint64_t ld_relaxed_sys(const void* p) {
  uint64_t v;
  asm volatile("ld.relaxed.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_sys(void* p, uint64_t v) {
  asm volatile("st.release.sys.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ uint64_t ld_acquire_gpu(const void* p) {
  uint64_t v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint64_t ld_relaxed_gpu(const void* p) {
  uint64_t v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed_gpu(void* p, uint64_t v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void st_release_gpu(void* p, uint64_t v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Blocks of at most 256 threads: the queue's single-pass plans (R = 16 up to
// 4096 points with 256 threads per tile; shorter lengths 64 threads).  TR:
// the compile-time shape of the length where one exists (kernel_shapes.h),
// else every parameter from the descriptor.
template <int R, class TR>
__global__ void __launch_bounds__(256)
queue_worker(const __grid_constant__ PassDesc d0, const __grid_constant__ QueueArgs q) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cf* sm = reinterpret_cast<cf*>(smem_raw);
  __shared__ uint64_t s_ticket, s_in, s_out;
  // the block's copy of the pass descriptor; each job sets its count
  __shared__ PassDesc d;
  const int tid = threadIdx.x;
  if (tid == 0) d = d0;
  for (uint64_t t = q.first_ticket;; ++t) {
    const int s = (int)((t - 1) % (uint64_t)q.slots);
    QGo* g = q.go + s;
    if (tid == 0) {
      uint64_t got = kQuit;
      if (blockIdx.x == 0) {
        for (uint32_t it = 0; it < kIdlePolls; ++it) {
          if (ld_acquire_sys(&q.ring[s].seq) == t) {
            got = t;
            break;
          }
          if (ld_acquire_sys32(&q.header->stop)) break;
          if (it > 1024) __nanosleep(256);  // tight polls first: latency of a busy queue
        }
        if (got == t) {
          st_relaxed_gpu(&g->in, ld_relaxed_sys(&q.ring[s].in));
          st_relaxed_gpu(&g->out, ld_relaxed_sys(&q.ring[s].out));
          st_relaxed_gpu(&g->batch, ld_relaxed_sys(&q.ring[s].batch));
        }
        st_release_gpu(&g->ticket, got);
      } else {
        bool seen = false;
        for (uint64_t it = 0; it < kFollowPolls; ++it) {
          const uint64_t v = ld_acquire_gpu(&g->ticket);
          if (v == t || v == kQuit) {
            got = v;
            seen = true;
            break;
          }
          if (it > 1024) __nanosleep(256);
        }
        if (!seen) atomicExch(q.status, 1);  // block 0 never decided: leave (got = QUIT)
      }
      s_ticket = got;
      if (got == t) {
        s_in = ld_relaxed_gpu(&g->in);
        s_out = ld_relaxed_gpu(&g->out);
        const int64_t batch = (int64_t)ld_relaxed_gpu(&g->batch);
        d.count_inner = batch;
        d.tiles_inner = d.tiles = (batch + d.G - 1) / d.G;
      }
    }
    __syncthreads();
    if (s_ticket != t) return;  // the same decision in every block
    const cf* in = reinterpret_cast<const cf*>(s_in);
    cf* out = reinterpret_cast<cf*>(s_out);
    for (int64_t tile = blockIdx.x; tile < d.tiles; tile += gridDim.x)
      pass_tile<R, MAP_ROWS, MAP_ROWS, TR>(in, out, d, tile, sm, tid);
    __syncthreads();  // this block's stores are issued; s_* is rewritten next
    if (tid == 0) {
      __threadfence();
      if (atomicAdd(q.cnt + s, 1) == (int)gridDim.x - 1) {
        q.cnt[s] = 0;  // the slot's next ticket starts after the host has seen `done`
        __threadfence_system();
        st_release_sys(&q.ring[s].done, t);
      }
    }
  }
}

const void* worker_fn(int R, const PassDesc& d) {
#define GB_TRY(LOGL, SCHED, NST, RR, G, LM, SM, CONTIG, EPI)                                     \
  if (shape_matches(d, R, MAP_ROWS, MAP_ROWS, LOGL, SCHED, NST, RR, G, LM, SM, CONTIG, EPI))     \
    return (const void*)queue_worker<RR, CtTraits<LOGL, SCHED, NST, RR, G, CONTIG, EPI>>;
  GB_SHAPES_CONTIG(GB_TRY)
#undef GB_TRY
  switch (R) {
    case 2: return (const void*)queue_worker<2, RtTraits>;
    case 4: return (const void*)queue_worker<4, RtTraits>;
    case 8: return (const void*)queue_worker<8, RtTraits>;
    case 16: return (const void*)queue_worker<16, RtTraits>;
    default: return nullptr;
  }
}

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

std::atomic<uint64_t>* seq_of(QSlot* s) { return reinterpret_cast<std::atomic<uint64_t>*>(&s->seq); }
std::atomic<uint64_t>* done_of(QSlot* s) {
  return reinterpret_cast<std::atomic<uint64_t>*>(&s->done);
}

}  // namespace

struct fft_queue_s {
  uint32_t magic = kQueueMagic;
  int device = -1;
  PlanSpec spec;
  PassDesc d0{};
  const void* fn = nullptr;
  int block = 0, grid = 0;
  size_t smem = 0;
  int slots = 0;
  int64_t max_batch = 0;
  void* tables = nullptr;  // twiddles, then the status word
  void* dev = nullptr;     // go records, block counters
  void* host = nullptr;    // header + ring (mapped pinned)
  QHeader* header = nullptr;
  QSlot* ring = nullptr;
  QueueArgs args{};
  cudaStream_t stream = nullptr;
  uint64_t issued = 0, completed = 0;
  int64_t launches = 0;
  bool failed = false;
  std::mutex mu;
};

namespace {

bool queue_ok(fft_queue_t q) { return q && q->magic == kQueueMagic; }

void free_queue(fft_queue_t q) {
  if (q->stream) cudaStreamDestroy(q->stream);
  if (q->host) cudaFreeHost(q->host);
  if (q->dev) cudaFree(q->dev);
  if (q->tables) cudaFree(q->tables);
  q->magic = 0;
  delete q;
}

fft_status_t cuda_err(cudaError_t e, const char* what) {
  char b[256];
  snprintf(b, sizeof b, "%s: %s", what, cudaGetErrorString(e));
  cudaGetLastError();
  return set_error(FFT_ERR_CUDA, b);
}

void update_completed(fft_queue_t q) {
  q->completed = ring_completed(q->completed, q->issued, q->slots, [q](int slot) {
    return done_of(q->ring + slot)->load(std::memory_order_acquire);
  });
}

// Launches the worker when it is not running and jobs are pending.
fft_status_t ensure_worker(fft_queue_t q) {
  if (q->failed) return set_error(FFT_ERR_CUDA, "the queue's worker failed earlier");
  cudaError_t e = cudaStreamQuery(q->stream);
  if (e == cudaErrorNotReady) return FFT_OK;  // running
  if (e != cudaSuccess) {
    q->failed = true;
    return cuda_err(e, "queue worker");
  }
  update_completed(q);
  if (q->completed >= q->issued) return FFT_OK;
  if (q->launches > 0) {
    int st = 0;
    e = cudaMemcpy(&st, q->args.status, sizeof st, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_err(e, "queue status");
    if (st) {
      q->failed = true;
      return set_error(FFT_ERR_TIMEOUT, "a worker block gave up waiting for the queue's leader");
    }
  }
  // fresh decision records and counters for this launch
  e = cudaMemsetAsync(q->dev, 0, (size_t)q->slots * (sizeof(QGo) + sizeof(int)), q->stream);
  if (e != cudaSuccess) return cuda_err(e, "queue reset");
  q->args.first_ticket = q->completed + 1;
  void* params[] = {&q->d0, &q->args};
  e = cudaLaunchCooperativeKernel(q->fn, dim3(q->grid), dim3(q->block), params, q->smem,
                                  q->stream);
  if (e != cudaSuccess) {
    q->failed = true;
    return cuda_err(e, "queue worker launch");
  }
  ++q->launches;
  return FFT_OK;
}

}  // namespace

extern "C" {

fft_status_t fft_queue_create(fft_queue_t* queue, int64_t n, int64_t max_batch, int direction,
                              int slots, int blocks) {
  if (!queue) return set_error(FFT_ERR_INVALID_ARG, "queue output pointer is null");
  *queue = nullptr;
  if (n < 2 || n > 4096)
    return set_error(n < 1 ? FFT_ERR_UNSUPPORTED_SIZE : FFT_ERR_NOT_IMPLEMENTED,
                     "the work queue takes 1D lengths 2 .. 2^12");
  if ((n & (n - 1)) != 0) return set_error(FFT_ERR_UNSUPPORTED_SIZE, "n must be a power of two");
  if (max_batch < 1) return set_error(FFT_ERR_INVALID_ARG, "max_batch must be >= 1");
  if (slots == 0) slots = 64;
  if (slots < 1 || slots > 4096) return set_error(FFT_ERR_INVALID_ARG, "slots must be 1 .. 4096");
  if (blocks < 0) return set_error(FFT_ERR_INVALID_ARG, "blocks must be >= 0");
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_err(e, "no usable CUDA device");
  cudaDeviceProp prop;
  e = cudaGetDeviceProperties(&prop, dev);
  if (e != cudaSuccess) return cuda_err(e, "cudaGetDeviceProperties");
  int coop = 0;
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  if (!coop) return set_error(FFT_ERR_NOT_IMPLEMENTED, "device has no cooperative launch");
  Caps caps;
  caps.sm_count = prop.multiProcessorCount;
  caps.smem_optin = (int)prop.sharedMemPerBlockOptin;
  caps.max_block = prop.maxThreadsPerBlock;

  fft_queue_t q = new (std::nothrow) fft_queue_s();
  if (!q) return set_error(FFT_ERR_OUT_OF_MEMORY, "host allocation of the queue failed");
  q->device = dev;
  q->slots = slots;
  q->max_batch = max_batch;
  fft_plan_options_t opt{};
  opt.variant = 1;  // the register kernel's tiles (one tile per block at a time)
  make_plan(q->spec, &n, 1, max_batch, direction, FFT_PREC_FP32, &opt, caps);
  if (q->spec.status != FFT_OK) {
    fft_status_t st = q->spec.status;
    char msg[256];
    snprintf(msg, sizeof msg, "%s", q->spec.error);
    delete q;
    return set_error(st, msg);
  }
  const PassSpec& p = q->spec.passes[0];
  const bool one_pass = q->spec.passes.size() == 1 && p.kind == PASS_FFT && p.batch_is_tiles;
  if (one_pass) q->d0 = pass_desc(p, 0, max_batch, max_batch);
  q->fn = one_pass ? worker_fn(p.R, q->d0) : nullptr;
  if (!q->fn) {
    delete q;
    return set_error(FFT_ERR_NOT_IMPLEMENTED, "no single-pass register plan for this length");
  }
  q->block = p.block;
  q->smem = p.smem;
  if ((e = cudaStreamCreateWithFlags(&q->stream, cudaStreamNonBlocking)) != cudaSuccess ||
      (e = cudaMalloc(&q->tables, (size_t)q->spec.table_elems * 8 + 16)) != cudaSuccess ||
      (e = cudaMalloc(&q->dev, (size_t)slots * (sizeof(QGo) + sizeof(int)))) != cudaSuccess ||
      (e = cudaHostAlloc(&q->host, sizeof(QHeader) + (size_t)slots * sizeof(QSlot),
                         cudaHostAllocMapped)) != cudaSuccess) {
    fft_status_t st = cuda_err(e, "queue allocation");
    free_queue(q);
    return st == FFT_ERR_CUDA ? FFT_ERR_OUT_OF_MEMORY : st;
  }
  memset(q->host, 0, sizeof(QHeader) + (size_t)slots * sizeof(QSlot));
  q->header = static_cast<QHeader*>(q->host);
  q->ring = reinterpret_cast<QSlot*>(static_cast<char*>(q->host) + sizeof(QHeader));
  void* dhost = nullptr;
  if ((e = cudaHostGetDevicePointer(&dhost, q->host, 0)) != cudaSuccess) {
    fft_status_t st = cuda_err(e, "device view of the queue ring");
    free_queue(q);
    return st;
  }
  int* status = reinterpret_cast<int*>(static_cast<char*>(q->tables) + q->spec.table_elems * 8);
  e = cudaMemsetAsync(status, 0, 16, q->stream);
  if (e == cudaSuccess) e = enqueue_tables(q->spec, static_cast<cf*>(q->tables), q->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(q->stream);
  if (e == cudaSuccess && q->smem > 48 * 1024)
    e = cudaFuncSetAttribute(q->fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)q->smem);
  int per_sm = 0;
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, q->fn, q->block, q->smem);
  if (e != cudaSuccess || per_sm < 1) {
    fft_status_t st = e != cudaSuccess ? cuda_err(e, "queue setup")
                                       : set_error(FFT_ERR_CUDA, "worker block does not fit an SM");
    free_queue(q);
    return st;
  }
  q->d0.tw = static_cast<const cf*>(q->tables);
  q->d0.status = status;
  const int64_t resident = (int64_t)per_sm * caps.sm_count;
  const int64_t tiles = (max_batch + p.G - 1) / p.G;
  q->grid = (int)std::min<int64_t>(blocks > 0 ? blocks : tiles, resident);
  q->args.ring = reinterpret_cast<QSlot*>(static_cast<char*>(dhost) + sizeof(QHeader));
  q->args.header = static_cast<const QHeader*>(dhost);
  q->args.go = static_cast<QGo*>(q->dev);
  q->args.cnt = reinterpret_cast<int*>(static_cast<char*>(q->dev) + (size_t)slots * sizeof(QGo));
  q->args.status = status;
  q->args.slots = slots;
  *queue = q;
  return FFT_OK;
}

fft_status_t fft_queue_submit(fft_queue_t q, const void* in, void* out, int64_t batch,
                              uint64_t* ticket) {
  TraceRange trace("fft_queue_submit");
  if (!queue_ok(q)) return set_error(FFT_ERR_BAD_PLAN, "null or destroyed queue");
  if (!ticket) return set_error(FFT_ERR_INVALID_ARG, "ticket output pointer is null");
  if (!in || !out) return set_error(FFT_ERR_INVALID_ARG, "in/out must be device pointers");
  if (((uintptr_t)in & 7) || ((uintptr_t)out & 7))
    return set_error(FFT_ERR_INVALID_ARG, "in/out must be 8-byte aligned (complex64)");
  if (batch < 1 || batch > q->max_batch)
    return set_error(FFT_ERR_INVALID_ARG, "batch must be 1 .. the queue's max_batch");
  std::lock_guard<std::mutex> lock(q->mu);
  const uint64_t t = q->issued + 1;
  QSlot* s = q->ring + (t - 1) % (uint64_t)q->slots;
  {
    // the slot's previous job must be done before it is rewritten
    const double limit = now_s() + 1.0;
    for (uint32_t it = 0; !ring_slot_free(t, q->slots, done_of(s)->load(std::memory_order_acquire));
         ++it) {
      if ((it & 63) == 0) {
        fft_status_t st = ensure_worker(q);
        if (st != FFT_OK) return st;
        if (now_s() > limit)
          return set_error(FFT_ERR_TIMEOUT, "queue full: its oldest job is still running");
      }
      std::this_thread::yield();
    }
  }
  s->in = (uint64_t)(uintptr_t)in;
  s->out = (uint64_t)(uintptr_t)out;
  s->batch = batch;
  seq_of(s)->store(t, std::memory_order_release);
  q->issued = t;
  *ticket = t;
  return ensure_worker(q);
}

fft_status_t fft_queue_wait(fft_queue_t q, uint64_t ticket, double timeout_s) {
  if (!queue_ok(q)) return set_error(FFT_ERR_BAD_PLAN, "null or destroyed queue");
  int slots = 0;
  {
    std::lock_guard<std::mutex> lock(q->mu);
    if (ticket < 1 || ticket > q->issued) return set_error(FFT_ERR_INVALID_ARG, "unknown ticket");
    slots = q->slots;
  }
  // the ticket is complete once its slot's done word reaches it (queue_ring.h);
  // polled without the lock, so other threads can submit meanwhile
  const std::atomic<uint64_t>* done = done_of(q->ring + (ticket - 1) % (uint64_t)slots);
  const double limit = timeout_s < 0 ? 1e300 : now_s() + timeout_s;
  for (uint32_t it = 0;; ++it) {
    if (done->load(std::memory_order_acquire) >= ticket) return FFT_OK;
    if ((it & 255) == 255) {
      // a worker that ended just before this job arrived is started again
      std::lock_guard<std::mutex> lock(q->mu);
      fft_status_t st = ensure_worker(q);
      if (st != FFT_OK) return st;
      if (now_s() > limit) return set_error(FFT_ERR_TIMEOUT, "job not finished before the timeout");
    }
  }
}

fft_status_t fft_queue_info(fft_queue_t q, int64_t* worker_launches, uint64_t* completed) {
  if (!queue_ok(q)) return set_error(FFT_ERR_BAD_PLAN, "null or destroyed queue");
  std::lock_guard<std::mutex> lock(q->mu);
  update_completed(q);
  if (worker_launches) *worker_launches = q->launches;
  if (completed) *completed = q->completed;
  return FFT_OK;
}

fft_status_t fft_queue_destroy(fft_queue_t q) {
  if (!queue_ok(q)) return set_error(FFT_ERR_BAD_PLAN, "null or destroyed queue");
  fft_status_t st = FFT_OK;
  {
    std::lock_guard<std::mutex> lock(q->mu);
    // jobs already submitted run first: the worker takes a job that is in
    // the ring before it looks at the stop word
    st = ensure_worker(q);
    reinterpret_cast<std::atomic<uint32_t>*>(&q->header->stop)->store(1, std::memory_order_release);
    cudaError_t e = cudaStreamSynchronize(q->stream);  // the worker ends within one poll
    if (e != cudaSuccess && st == FFT_OK) st = cuda_err(e, "queue worker");
  }
  free_queue(q);
  return st;
}

}  // extern "C"
