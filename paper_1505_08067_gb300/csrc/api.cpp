// C ABI of the library (include/gbfft.h).  Plans own their device twiddle
// tables and workspace; fft_execute only enqueues kernels.
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/gbfft.h"
#include "autotune.h"
#include "exec.h"
#include "kernels.h"
#include "planner.h"
#include "trace.h"

using namespace gbfft;

namespace {

// Message of the last failure on this thread (fixed storage: reporting an
// error never allocates).
thread_local char g_err[512];

fft_status_t fail(fft_status_t st, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
  return st;
}

fft_status_t cuda_fail(cudaError_t e, const char* what) {
  return fail(FFT_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

constexpr uint32_t kMagic = 0x47424646u;  // "GBFF"

}  // namespace

struct fft_plan_s {
  uint32_t magic = kMagic;
  int device = -1;
  PlanSpec spec;
  Caps caps;
  void* tables = nullptr;  // cf[spec.table_elems], then the status word
  int* status = nullptr;   // set by kernels whose bounded waits give up
  void* work = nullptr;    // cf[spec.work_elems]
  PassLaunch launches[kMaxPasses];  // whole-batch launches, device pointers filled
  // lazily created resources of fft_execute_host
  cudaStream_t s_h2d = nullptr, s_k = nullptr, s_d2h = nullptr;
  cudaEvent_t ev_start = nullptr, ev_h2d = nullptr, ev_k = nullptr, ev_end = nullptr;
  std::mutex host_mu;
  // captured executions (fft_execute_graph), keyed by (in, out)
  struct GraphEntry {
    const void* in = nullptr;
    void* out = nullptr;
    cudaGraphExec_t exec = nullptr;
    uint64_t last_use = 0;
  };
  static constexpr int kGraphs = 8;
  GraphEntry graphs[kGraphs];
  uint64_t graph_clock = 0;
  cudaStream_t s_capture = nullptr;
  std::mutex graph_mu;
};

namespace {

bool plan_ok(fft_plan_t p) { return p && p->magic == kMagic; }

fft_status_t query_caps(Caps& caps, int& device) {
  cudaError_t e = cudaGetDevice(&device);
  if (e != cudaSuccess) return cuda_fail(e, "no usable CUDA device");
  cudaDeviceProp prop;
  e = cudaGetDeviceProperties(&prop, device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceProperties");
  caps.sm_count = prop.multiProcessorCount;
  caps.smem_optin = (int)prop.sharedMemPerBlockOptin;
  caps.max_block = prop.maxThreadsPerBlock;
  return FFT_OK;
}

int64_t elems_per_batch(const PlanSpec& s) { return s.dims == 1 ? s.n[0] : s.n[0] * s.n[1]; }

fft_status_t build_plan(fft_plan_t* out, const int64_t* n, int dims, int64_t batch, int direction,
                        int precision, const fft_plan_options_t* opt,
                        const ConvSpec* conv = nullptr, const void* const* filters = nullptr) {
  if (!out) return fail(FFT_ERR_INVALID_ARG, "plan output pointer is null");
  *out = nullptr;
  Caps caps;
  int dev = -1;
  fft_status_t st = query_caps(caps, dev);
  if (st != FFT_OK) return st;
  PlanSpec spec;
  make_plan(spec, n, dims, batch, direction, precision, opt, caps, conv);
  if (spec.status != FFT_OK) return fail(spec.status, "%s", spec.error);
  if (conv) {
    for (int d = 0; d < dims; ++d) spec.filter[d] = filters[d];
  } else if (opt && opt->autotune && precision == FFT_PREC_FP32) {
    // choose the options on this GPU, then plan with them
    fft_plan_options_t chosen{};
    char report[sizeof spec.tuning];
    st = autotune_options(n, dims, batch, direction, *opt, caps, dev, &chosen, report,
                          sizeof report);
    if (st != FFT_OK) return st;
    make_plan(spec, n, dims, batch, direction, precision, &chosen, caps);
    if (spec.status != FFT_OK) return fail(spec.status, "%s", spec.error);
    memcpy(spec.tuning, report, sizeof spec.tuning);
  }
  fft_plan_t p = new (std::nothrow) fft_plan_s();
  if (!p) return fail(FFT_ERR_OUT_OF_MEMORY, "host allocation of the plan failed");
  p->device = dev;
  p->caps = caps;
  p->spec = spec;
  cudaError_t e;
  e = cudaMalloc(&p->tables, (size_t)spec.table_elems * 8 + 16);
  if (e != cudaSuccess) {
    delete p;
    cudaGetLastError();
    return fail(FFT_ERR_OUT_OF_MEMORY, "twiddle tables: %s", cudaGetErrorString(e));
  }
  p->status = reinterpret_cast<int*>(static_cast<char*>(p->tables) + (size_t)spec.table_elems * 8);
  e = cudaMemset(p->status, 0, 16);
  if (e != cudaSuccess) {
    cudaFree(p->tables);
    delete p;
    return cuda_fail(e, "status word");
  }
  if (spec.work_elems > 0) {
    e = cudaMalloc(&p->work, (size_t)spec.work_elems * 8);
    if (e != cudaSuccess) {
      cudaFree(p->tables);
      delete p;
      cudaGetLastError();
      return fail(FFT_ERR_OUT_OF_MEMORY, "workspace of %lld bytes: %s",
                  (long long)spec.work_elems * 8, cudaGetErrorString(e));
    }
  }
  // tables on the legacy stream, waited for alone (work of the caller on
  // non-blocking streams is not waited for)
  e = enqueue_tables(spec, static_cast<cf*>(p->tables), 0);
  if (e == cudaSuccess) e = cudaStreamSynchronize(0);
  if (e == cudaSuccess)
    e = bind_launches(p->spec, p->caps, static_cast<const cf*>(p->tables), p->status, p->launches);
  if (e != cudaSuccess) {
    fft_plan_destroy(p);
    return cuda_fail(e, "twiddle generation");
  }

  *out = p;
  return FFT_OK;
}

}  // namespace

// Used by autotune.cpp to report failures through fft_last_error.
namespace gbfft {
fft_status_t set_error(fft_status_t st, const char* msg) { return fail(st, "%s", msg); }
}  // namespace gbfft

extern "C" {

fft_status_t fft_plan_create(fft_plan_t* plan, const int64_t* n, int dims, int64_t batch,
                             int direction, int precision) {
  TraceRange r("fft_plan_create");
  return build_plan(plan, n, dims, batch, direction, precision, nullptr);
}

fft_status_t fft_plan_create_ex(fft_plan_t* plan, const int64_t* n, int dims, int64_t batch,
                                int direction, int precision, const fft_plan_options_t* options) {
  TraceRange r("fft_plan_create");
  return build_plan(plan, n, dims, batch, direction, precision, options);
}

// Data pointers are aligned to the plan's element size (complex64 or complex32).
static bool aligned_io(const PlanSpec& s, const void* p) {
  return ((uintptr_t)p % (uintptr_t)elem_bytes(s.precision)) == 0;
}

fft_status_t fft_execute(fft_plan_t plan, const void* in, void* out, void* stream) {
  TraceRange r("fft_execute");
  if (!plan_ok(plan)) return fail(FFT_ERR_BAD_PLAN, "null or destroyed plan");
  if (plan->spec.batch == 0) return FFT_OK;
  if (!in || !out) return fail(FFT_ERR_INVALID_ARG, "in/out must be device pointers");
  if (!aligned_io(plan->spec, in) || !aligned_io(plan->spec, out))
    return fail(FFT_ERR_INVALID_ARG, "in/out must be aligned to the element size (%d bytes)",
                elem_bytes(plan->spec.precision));
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev != plan->device)
    return fail(FFT_ERR_BAD_PLAN, "plan was created on device %d, current device is %d",
                plan->device, dev);
  e = enqueue_passes(plan->spec, plan->launches, in, out, plan->work, 0, plan->spec.batch,
                     static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
  return FFT_OK;
}

fft_status_t fft_execute_host(fft_plan_t plan, const void* host_in, void* host_out, void* dev_in,
                              void* dev_out, void* stream) {
  TraceRange r("fft_execute_host");
  if (!plan_ok(plan)) return fail(FFT_ERR_BAD_PLAN, "null or destroyed plan");
  const PlanSpec& s = plan->spec;
  if (s.batch == 0) return FFT_OK;
  if (!host_in || !host_out || !dev_in || !dev_out)
    return fail(FFT_ERR_INVALID_ARG, "null buffer");
  if (!aligned_io(s, dev_in) || !aligned_io(s, dev_out))
    return fail(FFT_ERR_INVALID_ARG, "device buffers must be aligned to the element size");
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev != plan->device) return fail(FFT_ERR_BAD_PLAN, "plan/device mismatch");
  std::lock_guard<std::mutex> lock(plan->host_mu);
  cudaStream_t user = static_cast<cudaStream_t>(stream);
  if (!plan->s_h2d) {
    const unsigned fl = cudaStreamNonBlocking;
    if ((e = cudaStreamCreateWithFlags(&plan->s_h2d, fl)) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&plan->s_k, fl)) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&plan->s_d2h, fl)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&plan->ev_start, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&plan->ev_h2d, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&plan->ev_k, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&plan->ev_end, cudaEventDisableTiming)) != cudaSuccess)
      return cuda_fail(e, "stream/event creation for host execution");
  }
  const int64_t E = elems_per_batch(s);
  const size_t per = (size_t)E * elem_bytes(s.precision);
  // chunks of whole batch entries, about 32 MiB each (1D only; 2D runs whole)
  int64_t chunk = s.batch;
  if (s.dims == 1) chunk = std::max<int64_t>(1, (int64_t)((32u << 20) / per));
  chunk = std::min(chunk, s.batch);
  if ((e = cudaEventRecord(plan->ev_start, user)) != cudaSuccess) return cuda_fail(e, "record");
  cudaStreamWaitEvent(plan->s_h2d, plan->ev_start, 0);
  cudaStreamWaitEvent(plan->s_k, plan->ev_start, 0);
  cudaStreamWaitEvent(plan->s_d2h, plan->ev_start, 0);
  const char* hi = static_cast<const char*>(host_in);
  char* ho = static_cast<char*>(host_out);
  char* di = static_cast<char*>(dev_in);
  char* dout = static_cast<char*>(dev_out);
  char* wk = static_cast<char*>(plan->work);
  for (int64_t b0 = 0; b0 < s.batch; b0 += chunk) {
    const int64_t nb = std::min(chunk, s.batch - b0);
    const size_t off = (size_t)b0 * per, bytes = (size_t)nb * per;
    if ((e = cudaMemcpyAsync(di + off, hi + off, bytes, cudaMemcpyHostToDevice, plan->s_h2d)) !=
        cudaSuccess)
      return cuda_fail(e, "host-to-device copy");
    cudaEventRecord(plan->ev_h2d, plan->s_h2d);
    cudaStreamWaitEvent(plan->s_k, plan->ev_h2d, 0);
    // the chunks run one after the other on s_k, so each reuses the workspace
    // from its start
    e = enqueue_passes(s, plan->launches, di + off, dout + off, wk, b0, nb, plan->s_k);
    if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
    cudaEventRecord(plan->ev_k, plan->s_k);
    cudaStreamWaitEvent(plan->s_d2h, plan->ev_k, 0);
    if ((e = cudaMemcpyAsync(ho + off, dout + off, bytes, cudaMemcpyDeviceToHost, plan->s_d2h)) !=
        cudaSuccess)
      return cuda_fail(e, "device-to-host copy");
  }
  cudaEventRecord(plan->ev_end, plan->s_d2h);
  if ((e = cudaStreamWaitEvent(user, plan->ev_end, 0)) != cudaSuccess)
    return cuda_fail(e, "join");
  return FFT_OK;
}

fft_status_t fft_execute_graph(fft_plan_t plan, const void* in, void* out, void* stream) {
  TraceRange r("fft_execute_graph");
  if (!plan_ok(plan)) return fail(FFT_ERR_BAD_PLAN, "null or destroyed plan");
  if (plan->spec.batch == 0) return FFT_OK;
  if (!in || !out) return fail(FFT_ERR_INVALID_ARG, "in/out must be device pointers");
  if (!aligned_io(plan->spec, in) || !aligned_io(plan->spec, out))
    return fail(FFT_ERR_INVALID_ARG, "in/out must be aligned to the element size (%d bytes)",
                elem_bytes(plan->spec.precision));
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev != plan->device) return fail(FFT_ERR_BAD_PLAN, "plan/device mismatch");
  std::lock_guard<std::mutex> lock(plan->graph_mu);
  fft_plan_s::GraphEntry* hit = nullptr;
  fft_plan_s::GraphEntry* victim = &plan->graphs[0];
  for (auto& g : plan->graphs) {
    if (g.exec && g.in == in && g.out == out) hit = &g;
    if (!g.exec || g.last_use < victim->last_use) victim = &g;
  }
  if (!hit) {
    if (!plan->s_capture) {
      e = cudaStreamCreateWithFlags(&plan->s_capture, cudaStreamNonBlocking);
      if (e != cudaSuccess) return cuda_fail(e, "capture stream");
    }
    cudaGraph_t graph = nullptr;
    e = cudaStreamBeginCapture(plan->s_capture, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(e, "begin capture");
    cudaError_t le = enqueue_passes(plan->spec, plan->launches, in, out, plan->work, 0,
                                    plan->spec.batch, plan->s_capture);
    e = cudaStreamEndCapture(plan->s_capture, &graph);
    if (le != cudaSuccess || e != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      return cuda_fail(le != cudaSuccess ? le : e, "graph capture");
    }
    if (victim->exec) cudaGraphExecDestroy(victim->exec);
    victim->exec = nullptr;
    e = cudaGraphInstantiate(&victim->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      victim->exec = nullptr;
      return cuda_fail(e, "graph instantiation");
    }
    victim->in = in;
    victim->out = out;
    hit = victim;
  }
  hit->last_use = ++plan->graph_clock;
  e = cudaGraphLaunch(hit->exec, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "graph launch");
  return FFT_OK;
}

fft_status_t fft_plan_destroy(fft_plan_t plan) {
  if (!plan) return FFT_OK;
  if (!plan_ok(plan)) return fail(FFT_ERR_BAD_PLAN, "destroyed or foreign plan");
  plan->magic = 0;
  int cur = -1;
  cudaGetDevice(&cur);
  if (cur != plan->device && plan->device >= 0) cudaSetDevice(plan->device);
  for (auto& g : plan->graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  if (plan->s_capture) cudaStreamDestroy(plan->s_capture);
  if (plan->s_h2d) {
    cudaStreamSynchronize(plan->s_h2d);
    cudaStreamSynchronize(plan->s_k);
    cudaStreamSynchronize(plan->s_d2h);
    cudaStreamDestroy(plan->s_h2d);
    cudaStreamDestroy(plan->s_k);
    cudaStreamDestroy(plan->s_d2h);
    cudaEventDestroy(plan->ev_start);
    cudaEventDestroy(plan->ev_h2d);
    cudaEventDestroy(plan->ev_k);
    cudaEventDestroy(plan->ev_end);
  }
  if (plan->tables) cudaFree(plan->tables);
  if (plan->work) cudaFree(plan->work);
  if (cur >= 0 && cur != plan->device) cudaSetDevice(cur);
  delete plan;
  return FFT_OK;
}

fft_status_t fft_plan_workspace_bytes(fft_plan_t plan, size_t* bytes) {
  if (!plan_ok(plan)) return fail(FFT_ERR_BAD_PLAN, "null or destroyed plan");
  if (!bytes) return fail(FFT_ERR_INVALID_ARG, "bytes is null");
  *bytes = (size_t)plan->spec.work_elems * 8;
  return FFT_OK;
}

fft_status_t fft_plan_launch_count(fft_plan_t plan, int* launches) {
  if (!plan_ok(plan)) return fail(FFT_ERR_BAD_PLAN, "null or destroyed plan");
  if (!launches) return fail(FFT_ERR_INVALID_ARG, "launches is null");
  *launches = plan->spec.batch == 0 ? 0 : (int)plan->spec.passes.size();
  return FFT_OK;
}

static fft_status_t copy_text(const std::string& t, char* buf, size_t len) {
  if (!buf || len == 0) return fail(FFT_ERR_INVALID_ARG, "buffer is null or empty");
  size_t n = std::min(len - 1, t.size());
  memcpy(buf, t.data(), n);
  buf[n] = 0;
  if (t.size() >= len) return fail(FFT_ERR_INVALID_ARG, "buffer too small (%zu bytes needed)",
                                   t.size() + 1);
  return FFT_OK;
}

fft_status_t fft_plan_describe(fft_plan_t plan, char* buf, size_t len) {
  if (!plan_ok(plan)) return fail(FFT_ERR_BAD_PLAN, "null or destroyed plan");
  // the planner's description plus, per pass, the kernel bound to it
  std::string t = describe(plan->spec);
  std::string k = ",\"kernels\":[";
  for (int i = 0; i < plan->spec.passes.size(); ++i) {
    const PassSpec& p = plan->spec.passes[i];
    const PassLaunch& l = plan->launches[i];
    const char* kind = p.kind == PASS_COPY        ? "copy"
                       : p.kind == PASS_TRANSPOSE ? "transpose"
                       : p.tc_prec        ? (p.variant == 1 ? "tensor_core_warp_mma"
                                                                : "tensor_core_tcgen05")
                       : l.has_staged     ? "staged"  // for a 16-byte-aligned source
                       : l.specialised    ? "compile_time"
                                          : "generic";
    char b[160];
    snprintf(b, sizeof b, "%s{\"kernel\":\"%s\",\"conv\":%d,\"persistent_grid\":%d,"
             "\"ctas_per_sm\":%d,\"l2_prefetch\":%d}", i ? "," : "", kind, p.conv,
             l.persistent_grid, l.ctas_per_sm, (int)l.d.l2_prefetch);
    k += b;
  }
  k += "]";
  t.insert(t.size() - 1, k);
  return copy_text(t, buf, len);
}

fft_status_t fft_plan_dry_run(const int64_t* n, int dims, int64_t batch, int direction,
                              int precision, const fft_plan_options_t* options, int sm_count,
                              int smem_optin_bytes, char* buf, size_t len) {
  if (sm_count <= 0 || smem_optin_bytes <= 0)
    return fail(FFT_ERR_INVALID_ARG, "device description must be positive");
  Caps caps;
  caps.sm_count = sm_count;
  caps.smem_optin = smem_optin_bytes;
  PlanSpec spec;
  make_plan(spec, n, dims, batch, direction, precision, options, caps);
  if (spec.status != FFT_OK) return fail(spec.status, "%s", spec.error);
  return copy_text(describe(spec), buf, len);
}

static fft_status_t conv_spec(const fft_filter_t* filters, int dims, bool need_ptr, ConvSpec& cs,
                              const void** ptrs) {
  if (!filters) return fail(FFT_ERR_INVALID_ARG, "filters is null");
  if (dims != 1 && dims != 2) return fail(FFT_ERR_INVALID_ARG, "dims must be 1 or 2");
  for (int d = 0; d < dims; ++d) {
    const fft_filter_t& f = filters[d];
    if (f.lines < 1) return fail(FFT_ERR_INVALID_ARG, "filter %d: lines must be >= 1", d);
    if (!(f.scale == f.scale)) return fail(FFT_ERR_INVALID_ARG, "filter %d: scale is NaN", d);
    if (need_ptr) {
      if (!f.h) return fail(FFT_ERR_INVALID_ARG, "filter %d: h is null", d);
      if ((uintptr_t)f.h & 7) return fail(FFT_ERR_INVALID_ARG, "filter %d: h must be 8-byte aligned", d);
      cudaPointerAttributes a;
      cudaError_t e = cudaPointerGetAttributes(&a, f.h);
      if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(FFT_ERR_INVALID_ARG, "filter %d: h is not a CUDA pointer", d);
      }
      if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)
        return fail(FFT_ERR_INVALID_ARG, "filter %d: h must be device (or managed) memory", d);
    }
    cs.lines[d] = f.lines;
    cs.scale[d] = f.scale;
    ptrs[d] = f.h;
  }
  return FFT_OK;
}

fft_status_t fft_conv_plan_create(fft_plan_t* plan, const int64_t* n, int dims, int64_t batch,
                                  const fft_filter_t* filters, const fft_plan_options_t* options) {
  TraceRange r("fft_conv_plan_create");
  if (!plan) return fail(FFT_ERR_INVALID_ARG, "plan output pointer is null");
  *plan = nullptr;
  ConvSpec cs;
  const void* ptrs[2] = {nullptr, nullptr};
  fft_status_t st = conv_spec(filters, dims, true, cs, ptrs);
  if (st != FFT_OK) return st;
  return build_plan(plan, n, dims, batch, FFT_FORWARD, FFT_PREC_FP32, options, &cs, ptrs);
}

fft_status_t fft_conv_plan_dry_run(const int64_t* n, int dims, int64_t batch,
                                   const fft_filter_t* filters, const fft_plan_options_t* options,
                                   int sm_count, int smem_optin_bytes, char* buf, size_t len) {
  if (sm_count <= 0 || smem_optin_bytes <= 0)
    return fail(FFT_ERR_INVALID_ARG, "device description must be positive");
  ConvSpec cs;
  const void* ptrs[2] = {nullptr, nullptr};
  fft_status_t st = conv_spec(filters, dims, false, cs, ptrs);
  if (st != FFT_OK) return st;
  Caps caps;
  caps.sm_count = sm_count;
  caps.smem_optin = smem_optin_bytes;
  PlanSpec spec;
  make_plan(spec, n, dims, batch, FFT_FORWARD, FFT_PREC_FP32, options, caps, &cs);
  if (spec.status != FFT_OK) return fail(spec.status, "%s", spec.error);
  return copy_text(describe(spec), buf, len);
}

fft_status_t fft_plan_sync_status(fft_plan_t plan, void* stream) {
  if (!plan_ok(plan)) return fail(FFT_ERR_BAD_PLAN, "null or destroyed plan");
  cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "stream synchronisation");
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "asynchronous error");
  int flag = 0;
  e = cudaMemcpy(&flag, plan->status, sizeof flag, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "status word");
  if (flag) {
    cudaMemset(plan->status, 0, sizeof flag);
    return fail(FFT_ERR_TIMEOUT, "a kernel gave up waiting for its TMA copy (bounded wait)");
  }
  return FFT_OK;
}

const char* fft_last_error(void) { return g_err; }

fft_status_t fft_schedule_count(int log2n, const int* radix_logs, int n_radix, uint64_t* count) {
  if (log2n < 0 || log2n > 60 || !radix_logs || n_radix <= 0 || !count)
    return fail(FFT_ERR_INVALID_ARG, "bad schedule-count arguments");
  *count = count_schedules(log2n, radix_logs, n_radix);
  return FFT_OK;
}

fft_status_t fft_schedule_shortest_path(int log2n, const int* radix_logs, int n_radix,
                                        const double* cost, int* path_logs, int path_cap,
                                        int* path_len, double* total_cost) {
  if (log2n < 1 || !radix_logs || n_radix <= 0 || !cost || !path_logs || !path_len ||
      !total_cost)
    return fail(FFT_ERR_INVALID_ARG, "bad shortest-path arguments");
  std::vector<int> path;
  double total = 0;
  if (!shortest_schedule(log2n, radix_logs, n_radix, cost, path, total))
    return fail(FFT_ERR_INVALID_ARG, "no schedule reaches the sink");
  if ((int)path.size() > path_cap) return fail(FFT_ERR_INVALID_ARG, "path capacity too small");
  for (size_t i = 0; i < path.size(); ++i) path_logs[i] = path[i];
  *path_len = (int)path.size();
  *total_cost = total;
  return FFT_OK;
}

fft_status_t fft_schedule_path_cost(int log2n, const int* radix_logs, int n_radix,
                                    const double* cost, const int* path_logs, int path_len,
                                    double* total_cost) {
  if (log2n < 1 || !radix_logs || n_radix <= 0 || !cost || !path_logs || path_len <= 0 ||
      !total_cost)
    return fail(FFT_ERR_INVALID_ARG, "bad path-cost arguments");
  double t = 0;
  if (!schedule_cost(log2n, radix_logs, n_radix, cost, path_logs, path_len, t))
    return fail(FFT_ERR_INVALID_ARG, "path is not a source-to-sink schedule");
  *total_cost = t;
  return FFT_OK;
}

double fft_bandwidth_bound_gflops(int64_t n, double gbs, double bytes_per_sample, double passes) {
  if (n < 2 || gbs <= 0 || bytes_per_sample <= 0 || passes <= 0) return 0.0;
  double lg = 0;
  for (int64_t v = n; v > 1; v >>= 1) lg += 1;
  // samples per second the link sustains times the flops each sample carries
  return 5.0 * (double)n * lg * gbs / (bytes_per_sample * passes * (double)n);
}

}  // extern "C"
