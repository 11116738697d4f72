// Plan-time autotuner.  Bergach et al. choose the FFT variant in two steps:
// an analytic / benchmark-based model first (Sec. 3.2: the on-chip block size
// from the limits of the compute unit; the cost of every (radix, start stage)
// pair benchmarked on its own; the shortest source-to-sink path of the
// schedule digraph under the stage-independence hypothesis), then runtime
// validation of the whole computation, because the model only loosely
// predicts the cost of data movement (abstract; Sec. 5).  Here:
//
//   1. model   - the block limit comes from the device's shared memory
//                (planner); for single-pass plans the per-(radix, stage) costs
//                are measured with the stage micro-kernel and Dijkstra gives
//                the model's radix schedule;
//   2. validate - whole plans are timed on this GPU for a small set of
//                candidates: the model's schedule, the default schedule, the
//                kernel variants, tile sizes, and for two-pass plans the
//                N = N1 * N2 split and the source of the four-step twiddle.
//
// The fastest candidate's options are kept (per device, shape and direction),
// in memory and, if GBFFT_WISDOM names a file, on disk.  GBFFT_BUILD_ID (set by
// the build: a hash of the library's sources) is part of every key.
#include "autotune.h"

#include <cuda_runtime.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <limits>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "exec.h"
#include "kernels.h"

#ifndef GBFFT_BUILD_ID
#define GBFFT_BUILD_ID "unversioned"
#endif

namespace gbfft {

namespace {

struct DevBuf {
  void* p = nullptr;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
  cudaError_t alloc(size_t bytes) { return cudaMalloc(&p, bytes > 0 ? bytes : 16); }
};

struct Ev {
  cudaEvent_t a = nullptr, b = nullptr;
  Ev() {
    cudaEventCreate(&a);
    cudaEventCreate(&b);
  }
  ~Ev() {
    cudaEventDestroy(a);
    cudaEventDestroy(b);
  }
};

constexpr double kInf = std::numeric_limits<double>::infinity();

int ilog2(int64_t v) {
  int l = 0;
  while ((int64_t(1) << l) < v) ++l;
  return l;
}

uint32_t pack_schedule(const Sched& s) {
  uint32_t c = 0;
  for (int i = 0; i < s.size() && i < 8; ++i) c |= (uint32_t)s[i] << (4 * i);
  return c;
}

std::string opts_key(const fft_plan_options_t& o) {
  char b[160];
  snprintf(b, sizeof b, "%d %d %u %d %d %d %d %d %d", o.radix, o.tile, o.schedule, o.max_block_log2,
           o.generic, o.variant, o.epilogue, o.split_log2, o.autotune);
  return b;
}

std::string opts_json(const fft_plan_options_t& o) {
  char b[200];
  snprintf(b, sizeof b,
           "{\"radix\":%d,\"tile\":%d,\"schedule\":%u,\"variant\":%d,\"epilogue\":%d,"
           "\"split_log2\":%d}",
           o.radix, o.tile, o.schedule, o.variant, o.epilogue, o.split_log2);
  return b;
}

// ------------------------------------------------ stage costs (Sec. 3.2) --

// Per-element time (ns) of radix 2^j starting at stage s of a length-2^logL
// contiguous pass with R elements per thread and G transforms per block,
// measured in isolation.  cost[(j-1) * logL + s]; -1 where the edge overruns.
cudaError_t measure_stage_costs(const PassSpec& pass, const Caps& caps, cudaStream_t st,
                                std::vector<double>& cost, std::vector<int>& radix_logs) {
  const int logL = pass.logL, L = 1 << logL;
  const int logR = ilog2(pass.R);
  radix_logs.clear();
  for (int j = 1; j <= logR; ++j) radix_logs.push_back(j);
  cost.assign((size_t)logR * logL, -1.0);
  const int pitch = L + (L >> 4) + std::max(1, 16 / pass.G);
  const int smem_elems = pass.G * pitch;
  const size_t smem = (size_t)smem_elems * 8;
  if (smem > (size_t)caps.smem_optin) return cudaSuccess;
  DevBuf table, sink;
  cudaError_t e = table.alloc((size_t)L * 8 * 2);
  if (e != cudaSuccess) return e;
  if ((e = sink.alloc(64 * 1024)) != cudaSuccess) return e;
  Ev ev;
  for (int j = 1; j <= logR; ++j) {
    const int r = 1 << j;
    for (int s = 0; s + j <= logL; ++s) {
      const int Ns = 1 << s;
      // stage table: entry i*Ns + k = w_{Ns*r}^{i*k}
      if ((e = launch_twiddle_gen(table.p, (int64_t)Ns * r, (int64_t)Ns * r, 0, Ns, 1, st)) !=
          cudaSuccess)
        return e;
      PassDesc d = pass_desc(pass, 0, 1, 1);
      d.nst = 15;
      d.rlog[1] = j;
      d.tw_off[1] = 0;
      d.tw = static_cast<const cf*>(table.p);
      d.pitch = pitch;
      d.smem_elems = smem_elems;
      d.conj_in = d.conj_out = 0;
      const int block = pass.G * (L / pass.R);
      const int grid = caps.sm_count * 2;
      const int reps = 16;
      if ((e = launch_stage_bench(pass.R, d, Ns, reps, grid, block, smem, sink.p, st)) !=
          cudaSuccess)
        return e;
      cudaEventRecord(ev.a, st);
      for (int it = 0; it < 3; ++it)
        if ((e = launch_stage_bench(pass.R, d, Ns, reps, grid, block, smem, sink.p, st)) !=
            cudaSuccess)
          return e;
      cudaEventRecord(ev.b, st);
      if ((e = cudaEventSynchronize(ev.b)) != cudaSuccess) return e;
      float ms = 0;
      cudaEventElapsedTime(&ms, ev.a, ev.b);
      const double elems = 3.0 * reps * grid * (double)pass.G * L;
      cost[(size_t)(j - 1) * logL + s] = ms * 1e6 / elems;
    }
  }
  return cudaSuccess;
}

// ---------------------------------------------------- whole-plan timing --

double time_candidate(const fft_plan_options_t& o, const int64_t* n, int dims, int64_t batch,
                      int direction, const Caps& caps, void* in, void* out, cudaStream_t st) {
  static PlanSpec s;  // large; tuning runs under the cache mutex
  make_plan(s, n, dims, batch, direction, FFT_PREC_FP32, &o, caps);
  if (s.status != FFT_OK) return kInf;
  DevBuf tables, work;
  if (tables.alloc((size_t)s.table_elems * 8 + 16) != cudaSuccess) return kInf;
  if (s.work_elems && work.alloc((size_t)s.work_elems * 8) != cudaSuccess) return kInf;
  int* status = reinterpret_cast<int*>(static_cast<char*>(tables.p) + (size_t)s.table_elems * 8);
  cudaMemsetAsync(status, 0, 16, st);
  PassLaunch launches[kMaxPasses];
  if (enqueue_tables(s, static_cast<cf*>(tables.p), st) != cudaSuccess) return kInf;
  if (bind_launches(s, caps, static_cast<const cf*>(tables.p), status, launches) != cudaSuccess)
    return kInf;
  for (int it = 0; it < 2; ++it)
    if (enqueue_passes(s, launches, in, out, work.p, 0, batch, st) != cudaSuccess) return kInf;
  Ev ev;
  const int reps = 5;
  cudaEventRecord(ev.a, st);
  for (int it = 0; it < reps; ++it)
    if (enqueue_passes(s, launches, in, out, work.p, 0, batch, st) != cudaSuccess) return kInf;
  cudaEventRecord(ev.b, st);
  if (cudaEventSynchronize(ev.b) != cudaSuccess) {
    cudaGetLastError();
    return kInf;
  }
  float ms = 0;
  cudaEventElapsedTime(&ms, ev.a, ev.b);
  return ms / reps;
}

// ----------------------------------------------------------- the cache --

std::mutex g_mu;
std::map<std::string, fft_plan_options_t> g_cache;
bool g_wisdom_loaded = false;

const char* wisdom_path() {
  const char* p = getenv("GBFFT_WISDOM");
  return (p && *p) ? p : nullptr;
}

void load_wisdom() {
  if (g_wisdom_loaded) return;
  g_wisdom_loaded = true;
  const char* path = wisdom_path();
  if (!path) return;
  FILE* f = fopen(path, "r");
  if (!f) return;
  char line[512];
  while (fgets(line, sizeof line, f)) {
    char key[256];
    fft_plan_options_t o{};
    if (sscanf(line, "%255[^|]| %d %d %u %d %d %d %d %d", key, &o.radix, &o.tile, &o.schedule,
               &o.max_block_log2, &o.generic, &o.variant, &o.epilogue, &o.split_log2) == 9)
      g_cache[key] = o;
  }
  fclose(f);
}

void save_wisdom(const std::string& key, const fft_plan_options_t& o) {
  const char* path = wisdom_path();
  if (!path) return;
  FILE* f = fopen(path, "a");
  if (!f) return;
  fprintf(f, "%s| %d %d %u %d %d %d %d %d\n", key.c_str(), o.radix, o.tile, o.schedule,
          o.max_block_log2, o.generic, o.variant, o.epilogue, o.split_log2);
  fclose(f);
}

}  // namespace

fft_status_t autotune_options(const int64_t* n, int dims, int64_t batch, int direction,
                              const fft_plan_options_t& base, const Caps& caps, int device,
                              fft_plan_options_t* chosen, char* report, size_t report_len) {
  fft_plan_options_t b = base;
  b.autotune = 0;
  *chosen = b;
  if (report && report_len) report[0] = 0;
  if (batch == 0) return FFT_OK;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) {
    cudaGetLastError();
    return set_error(FFT_ERR_CUDA, "autotune: cudaGetDeviceProperties failed");
  }
  // keyed by the library build, the driver, the device and the shape: a
  // result tuned by another build or driver is not reused
  int driver = 0;
  if (cudaDriverGetVersion(&driver) != cudaSuccess) cudaGetLastError();
  char keybuf[256];
  snprintf(keybuf, sizeof keybuf, "%s/%d/%s/%d %d %lld %lld %lld %d %s", GBFFT_BUILD_ID, driver,
           prop.name, prop.multiProcessorCount, dims, (long long)n[0],
           (long long)(dims > 1 ? n[1] : 1), (long long)batch, direction, opts_key(b).c_str());
  const std::string key = keybuf;
  std::lock_guard<std::mutex> lock(g_mu);
  load_wisdom();
  auto hit = g_cache.find(key);
  if (hit != g_cache.end()) {
    *chosen = hit->second;
    if (report && report_len) snprintf(report, report_len, "{\"cached\":%s}", opts_json(*chosen).c_str());
    return FFT_OK;
  }

  // default plan (the analytic choice) and trial buffers
  static PlanSpec def;
  make_plan(def, n, dims, batch, direction, FFT_PREC_FP32, &b, caps);
  if (def.status != FFT_OK) return set_error(def.status, def.error);
  const int64_t E = dims == 1 ? n[0] : n[0] * n[1];
  const int64_t trial = std::min<int64_t>(batch, std::max<int64_t>(1, (int64_t(1) << 25) / E));
  DevBuf in, out;
  if (in.alloc((size_t)(trial * E) * 8) != cudaSuccess ||
      out.alloc((size_t)(trial * E) * 8) != cudaSuccess) {
    cudaGetLastError();
    return set_error(FFT_ERR_OUT_OF_MEMORY, "autotune: trial buffers");
  }
  cudaStream_t st;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess)
    return set_error(FFT_ERR_CUDA, "autotune: stream");
  cudaMemsetAsync(in.p, 0, (size_t)(trial * E) * 8, st);

  std::vector<fft_plan_options_t> cand;
  cand.push_back(b);
  std::string model_json = "null";
  const int logN = ilog2(n[0]);
  const PassSpec& p0 = def.passes[0];
  if (dims == 1 && def.passes.size() == 1 && p0.kind == PASS_FFT && p0.batch_is_tiles) {
    // kernel variants and tile sizes
    for (int v : {1, 2, 3}) {
      if (v == 2 && (logN < 12 || logN > 14)) continue;
      fft_plan_options_t o = b;
      o.variant = v;
      cand.push_back(o);
    }
    if (!b.tile && logN <= 11) {
      for (int g : {p0.G / 2, p0.G * 2}) {
        if (g < 1 || g * (p0.logL > 0 ? (1 << p0.logL) / p0.R : 1) > caps.max_block) continue;
        fft_plan_options_t o = b;
        o.tile = g;
        o.variant = 1;
        cand.push_back(o);
      }
    }
    // the paper's model: stage costs, then the shortest path
    if (!b.schedule && p0.logL >= 2) {
      std::vector<double> cost;
      std::vector<int> logs;
      if (measure_stage_costs(p0, caps, st, cost, logs) == cudaSuccess) {
        std::vector<int> path;
        double total = 0;
        if (shortest_schedule(p0.logL, logs.data(), (int)logs.size(), cost.data(), path, total) &&
            (int)path.size() <= 8) {
          Sched ms;
          for (int v : path) ms.push_back(v);
          std::string pj = "[";
          for (size_t i = 0; i < path.size(); ++i) pj += (i ? "," : "") + std::to_string(1 << path[i]);
          pj += "]";
          char mb[256];
          snprintf(mb, sizeof mb, "{\"schedule\":%s,\"cost_ns_per_element\":%.4f}", pj.c_str(),
                   total);
          model_json = mb;
          if (pack_schedule(ms) != pack_schedule(p0.rlogs)) {
            fft_plan_options_t o = b;
            o.schedule = pack_schedule(ms);
            o.radix = p0.R;
            cand.push_back(o);
          }
        }
      } else {
        cudaGetLastError();
      }
    }
  } else if (dims == 1 && def.passes.size() == 2) {
    // split N = N1 * N2, four-step twiddle source, and the persistent grid
    // with L2 prefetch of the next tile (variant 3)
    const int l1d = def.passes[0].logL;
    for (int l1 = l1d - 1; l1 <= l1d + 1; ++l1)
      for (int ep : {2, 3, 4})
        for (int v : {0, 3}) {
          if (ep == 2 && logN > 22) continue;
          fft_plan_options_t o = b;
          o.split_log2 = l1;
          o.epilogue = ep;
          o.variant = v;
          cand.push_back(o);
        }
  } else if (dims == 2) {
    for (int v : {1, 2, 3}) {
      fft_plan_options_t o = b;
      o.variant = v;
      cand.push_back(o);
    }
  }

  double best = kInf;
  std::string tried = "[";
  for (size_t i = 0; i < cand.size(); ++i) {
    const double ms = time_candidate(cand[i], n, dims, trial, direction, caps, in.p, out.p, st);
    char tb[320];
    snprintf(tb, sizeof tb, "%s{\"opts\":%s,\"ms\":%.5f}", i ? "," : "",
             opts_json(cand[i]).c_str(), ms < kInf ? ms : -1.0);
    tried += tb;
    if (ms < best) {
      best = ms;
      *chosen = cand[i];
    }
  }
  tried += "]";
  cudaStreamSynchronize(st);
  cudaStreamDestroy(st);
  cudaGetLastError();
  if (!(best < kInf)) return set_error(FFT_ERR_CUDA, "autotune: no candidate ran");
  g_cache[key] = *chosen;
  save_wisdom(key, *chosen);
  if (report && report_len)
    snprintf(report, report_len,
             "{\"trial_batch\":%lld,\"model\":%s,\"candidates\":%s,\"chosen\":%s}",
             (long long)trial, model_json.c_str(), tried.c_str(), opts_json(*chosen).c_str());
  return FFT_OK;
}

}  // namespace gbfft
