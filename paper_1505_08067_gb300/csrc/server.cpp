// Serving loop: continuous batching of FFT jobs on one GPU (C ABI in
// include/gbfft.h, fft_server_*).
//
// A worker thread owns the device side.  It repeatedly
//   1. polls the completion events of running groups, marks their jobs done
//      (latency = completion seen - submit) and frees their bytes;
//   2. asks the scheduler (scheduler.h) for groups that fit the memory budget
//      (backfilling by estimated run times unless strict order is asked for)
//      and launches each on the stream whose queued work is estimated to end
//      first: jobs of one contiguous single-pass FP32 shape in one coalesced
//      kernel launch (job table in the kernel parameters), other jobs as their
//      plan's passes, one after the other, on the group's stream;
//   3. sleeps briefly when nothing changed.
// Plans (twiddle tables) stay resident per job key; multi-pass workspaces are
// stream-ordered allocations from the server's own memory pool (allocated on
// the group's stream before its passes, freed on it after them: no
// device-wide synchronisation, memory reused once the freeing stream has
// passed it).  Groups on different streams overlap on the device.
// Everything a running group holds counts against the budget.
#include <cuda_runtime.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/gbfft.h"
#include "exec.h"
#include "kernels.h"
#include "planner.h"
#include "scheduler.h"
#include "trace.h"

namespace gbfft {
fft_status_t set_error(fft_status_t st, const char* msg);
}

using namespace gbfft;

namespace {

constexpr uint32_t kServerMagic = 0x53525646u;
// Run-time estimate of a job for the scheduler: its algorithmic bytes (one
// read and one write of each element per pass) at an effective rate, plus a
// launch overhead.
constexpr double kEstBytesPerS = 3.0e12;
constexpr double kEstLaunchS = 6e-6;
constexpr size_t kLatencyWindow = size_t(1) << 20;  // latency samples kept for p50 / p99

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct KeyLess {
  bool operator()(const JobKey& a, const JobKey& b) const {
    if (a.dims != b.dims) return a.dims < b.dims;
    if (a.n0 != b.n0) return a.n0 < b.n0;
    if (a.n1 != b.n1) return a.n1 < b.n1;
    if (a.direction != b.direction) return a.direction < b.direction;
    return a.precision < b.precision;
  }
};

struct PlanEntry {
  PlanSpec spec;            // planned for a large batch; per-job descriptors rescale it
  void* tables = nullptr;   // twiddles + status word
  int* status = nullptr;
  PassLaunch launches[kMaxPasses];
  bool groupable = false;   // contiguous single-pass FP32: coalesced launches
  int64_t elems = 0;        // complex elements per batch entry
  int64_t work_per_entry = 0;  // workspace elements per batch entry (two-pass plans)
};

struct JobRec {
  fft_job_t job;
  double t_submit = 0, t_launch = 0, t_done = 0;
  int status = -1;  // -1 waiting / running, else fft_status_t
};

struct Running {
  SchedGroup group;
  cudaEvent_t start = nullptr;  // recorded on the group's stream before its launches
  cudaEvent_t done = nullptr;   // after them
};

}  // namespace

struct fft_server_s {
  uint32_t magic = kServerMagic;
  int device = -1;
  Caps caps;
  fft_server_options_t opt{};
  Scheduler sched;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::thread worker;
  bool stop = false;
  bool paused = false;  // admissions held (fft_server_pause)
  std::vector<cudaStream_t> streams;
  std::vector<double> stream_free;  // estimated time each stream's queued work ends
  std::map<JobKey, PlanEntry*, KeyLess> plans;
  std::unordered_map<uint64_t, JobRec> jobs;
  std::vector<Running> running;
  cudaMemPool_t ws_pool = nullptr;  // stream-ordered workspace allocations
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> free_events;  // (start, done) pairs
  uint64_t next_id = 1;
  uint64_t submitted = 0, completed = 0, failed = 0, launches = 0, coalesced = 0;
  std::vector<double> latencies;  // the most recent kLatencyWindow completions (a ring)
  size_t latency_next = 0;
  double first_submit = 0, last_done = 0, flops = 0;
  size_t ws_allocs = 0;
  double host_launch_s = 0;   // worker time spent enqueueing groups
  double group_stream_s = 0;  // sum over completed groups of start -> done on their stream

  fft_server_s(size_t budget, int max_group, size_t group_bytes, bool backfill)
      : sched(budget, max_group, group_bytes, backfill) {}
};

namespace {

int64_t job_elems(const fft_job_t& j) { return j.dims == 1 ? j.n[0] : j.n[0] * j.n[1]; }

double job_flops(const fft_job_t& j) {
  const double e = (double)job_elems(j);
  double lg = 0;
  for (int64_t v = job_elems(j); v > 1; v >>= 1) lg += 1;
  return 5.0 * e * lg * (double)j.batch;
}

// Plan for a job key (created once, kept resident).  Called by the worker.
PlanEntry* plan_for(fft_server_t s, const JobKey& k, fft_status_t* st) {
  auto it = s->plans.find(k);
  if (it != s->plans.end()) return it->second;
  PlanEntry* pe = new PlanEntry();
  int64_t n[2] = {k.n0, k.n1};
  // a large nominal batch gives the full tile shape; jobs rescale the descriptors
  const int64_t elems = k.dims == 1 ? k.n0 : k.n0 * k.n1;
  const int64_t nominal = std::max<int64_t>(1, (int64_t(1) << 24) / elems);
  make_plan(pe->spec, n, k.dims, nominal, k.direction, k.precision, nullptr, s->caps);
  if (pe->spec.status != FFT_OK) {
    *st = pe->spec.status;
    delete pe;
    return nullptr;
  }
  cudaError_t e = cudaMalloc(&pe->tables, (size_t)pe->spec.table_elems * 8 + 16);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *st = FFT_ERR_OUT_OF_MEMORY;
    delete pe;
    return nullptr;
  }
  pe->status = reinterpret_cast<int*>(static_cast<char*>(pe->tables) + pe->spec.table_elems * 8);
  // tables on the legacy stream, waited for alone: the server's streams are
  // non-blocking, so groups already running are not waited for
  e = cudaMemsetAsync(pe->status, 0, 16, 0);
  if (e == cudaSuccess) e = enqueue_tables(pe->spec, static_cast<cf*>(pe->tables), 0);
  if (e == cudaSuccess) e = cudaStreamSynchronize(0);
  if (e == cudaSuccess)
    e = bind_launches(pe->spec, s->caps, static_cast<const cf*>(pe->tables), pe->status,
                      pe->launches);
  if (e != cudaSuccess) {
    cudaFree(pe->tables);
    delete pe;
    *st = FFT_ERR_CUDA;
    return nullptr;
  }
  // jobs of any batch run the two-pass plans in sub-batches (the plan was made
  // for the nominal batch, below the sub-batch size)
  if (k.dims == 1 && pe->spec.work_elems > 0) pe->spec.chunk_batch = two_pass_chunk(elems);
  const PassSpec& p0 = pe->spec.passes[0];
  pe->groupable = k.dims == 1 && pe->spec.passes.size() == 1 && p0.kind == PASS_FFT &&
                  p0.batch_is_tiles && p0.tc_prec == 0;
  pe->elems = elems;
  pe->work_per_entry = pe->spec.work_elems / nominal;
  s->plans[k] = pe;
  return pe;
}

// Workspaces come in power-of-two size classes (at most 2x the request; the
// budget accounts for the class size), allocated in stream order from the
// server's pool, which keeps its memory (release threshold: never) so that
// steady-state allocations map no new pages.
size_t ws_class(size_t bytes) {
  size_t c = 1 << 20;
  while (c < bytes) c <<= 1;
  return c;
}

void* ws_get(fft_server_t s, size_t bytes, cudaStream_t st) {
  if (s->opt.fail_workspace_alloc) return nullptr;  // host-side fault injection
  void* p = nullptr;
  if (cudaMallocFromPoolAsync(&p, ws_class(bytes), s->ws_pool, st) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  ++s->ws_allocs;
  return p;
}

// Launch one admitted group on a stream.  Returns false if it could not.
bool launch_group(fft_server_t s, Running& r) {
  const SchedGroup& g = r.group;
  const JobKey key = g.jobs[0].key;
  fft_status_t pst = FFT_OK;
  PlanEntry* pe = plan_for(s, key, &pst);
  const double t = now_s();
  auto fail_all = [&](fft_status_t st) {
    for (const SchedJob& j : g.jobs) {
      JobRec& rec = s->jobs[j.id];
      rec.status = st;
      rec.t_done = now_s();
      ++s->failed;
    }
  };
  if (!pe) {
    fail_all(pst);
    return false;
  }
  // large groups in order on the first stream; the others on the stream
  // whose queued work is estimated to end first (the first one too when
  // there is no other, or when large groups are not set apart)
  int64_t group_elems = 0;
  for (const SchedJob& j : g.jobs) group_elems += job_elems(s->jobs[j.id].job) * j.batch;
  const int lg = s->opt.large_group_log2 == 0 ? 23 : s->opt.large_group_log2;
  const bool apart = lg > 0 && s->streams.size() > 1;
  size_t si = 0;
  if (!(apart && group_elems >= (int64_t(1) << std::min(lg, 62)))) {
    const size_t first = apart ? 1 : 0;
    si = first;
    for (size_t i = first + 1; i < s->streams.size(); ++i)
      if (s->stream_free[i] < s->stream_free[si]) si = i;
  }
  cudaStream_t st = s->streams[si];
  s->stream_free[si] = std::max(s->stream_free[si], t) + g.cost;
  if (s->free_events.empty()) {
    cudaEvent_t a = nullptr, b = nullptr;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
      cudaGetLastError();
      if (a) cudaEventDestroy(a);
      fail_all(FFT_ERR_CUDA);
      return false;
    }
    s->free_events.emplace_back(a, b);
  }
  r.start = s->free_events.back().first;
  r.done = s->free_events.back().second;
  s->free_events.pop_back();
  cudaEventRecord(r.start, st);
  TraceRange trace("fft_server launch group");
  cudaError_t e = cudaSuccess;
  if (pe->groupable && g.jobs.size() > 1) {
    // one coalesced launch per kMaxGroup jobs
    const PassSpec& p0 = pe->spec.passes[0];
    PassDesc d0 = pe->launches[0].d;
    for (size_t b = 0; b < g.jobs.size() && e == cudaSuccess; b += kMaxGroup) {
      GroupTable gt{};
      int64_t tiles = 0;
      for (size_t i = b; i < g.jobs.size() && gt.n < kMaxGroup; ++i) {
        const JobRec& rec = s->jobs[g.jobs[i].id];
        GroupEntry& ge = gt.e[gt.n++];
        ge.in = static_cast<const cf*>(rec.job.in);
        ge.out = static_cast<cf*>(rec.job.out);
        ge.count = rec.job.batch;
        ge.tiles = (rec.job.batch + p0.G - 1) / p0.G;
        ge.tile_begin = tiles;
        tiles += ge.tiles;
      }
      const int grid = (int)std::min<int64_t>(tiles, (int64_t)s->caps.sm_count * 16);
      e = launch_grouped(p0.R, d0, gt, grid, p0.block, p0.smem, st);
      ++s->launches;
    }
    s->coalesced += g.jobs.size();
  } else {
    for (const SchedJob& j : g.jobs) {
      const JobRec& rec = s->jobs[j.id];
      void* ws = nullptr;
      const int64_t ws_entries =
          pe->spec.chunk_batch > 0 ? std::min(rec.job.batch, pe->spec.chunk_batch) : rec.job.batch;
      const size_t wsb = (size_t)pe->work_per_entry * 8 * (size_t)ws_entries;
      if (wsb) {
        ws = ws_get(s, wsb, st);
        if (!ws) {
          e = cudaErrorMemoryAllocation;
          break;
        }
      }
      // a six-step plan's second buffer follows this job's first one
      e = enqueue_passes(pe->spec, pe->launches, rec.job.in, rec.job.out, ws, 0, rec.job.batch, st,
                         pe->spec.work2_off > 0 ? ws_entries * pe->elems : -1);
      if (ws) cudaFreeAsync(ws, st);  // after the passes, in stream order
      ++s->launches;
      if (e != cudaSuccess) break;
    }
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    s->free_events.emplace_back(r.start, r.done);
    r.start = r.done = nullptr;
    fail_all(e == cudaErrorMemoryAllocation ? FFT_ERR_OUT_OF_MEMORY : FFT_ERR_CUDA);
    return false;
  }
  cudaEventRecord(r.done, st);
  for (const SchedJob& j : g.jobs) s->jobs[j.id].t_launch = t;
  return true;
}

void worker_loop(fft_server_t s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lock(s->mu);
  while (!s->stop) {
    bool progress = false;
    // 1. completions
    for (size_t i = 0; i < s->running.size();) {
      Running& r = s->running[i];
      cudaError_t q = cudaEventQuery(r.done);
      if (q == cudaErrorNotReady) {
        ++i;
        continue;
      }
      const double t = now_s();
      for (const SchedJob& j : r.group.jobs) {
        JobRec& rec = s->jobs[j.id];
        rec.t_done = t;
        if (q == cudaSuccess) {
          rec.status = FFT_OK;
          ++s->completed;
          const double ms = (t - rec.t_submit) * 1e3;
          if (s->latencies.size() < kLatencyWindow) s->latencies.push_back(ms);
          else s->latencies[s->latency_next] = ms;
          s->latency_next = (s->latency_next + 1) % kLatencyWindow;
          s->flops += job_flops(rec.job);
        } else {
          rec.status = FFT_ERR_CUDA;
          ++s->failed;
        }
      }
      if (q != cudaSuccess) cudaGetLastError();
      float gms = 0;
      if (q == cudaSuccess && cudaEventElapsedTime(&gms, r.start, r.done) == cudaSuccess)
        s->group_stream_s += gms * 1e-3;
      else
        cudaGetLastError();
      s->last_done = t;
      s->sched.finished(r.group);
      s->free_events.emplace_back(r.start, r.done);
      s->running.erase(s->running.begin() + i);
      progress = true;
    }
    if (progress) s->cv_done.notify_all();
    // 2. launches
    SchedGroup g;
    while (!s->paused && (int)s->running.size() < s->opt.max_running &&
           s->sched.next(g, now_s())) {
      Running r;
      r.group = g;
      const double tl = now_s();
      const bool launched = launch_group(s, r);
      s->host_launch_s += now_s() - tl;
      if (launched) {
        s->running.push_back(std::move(r));
      } else {
        s->sched.finished(g);
        s->cv_done.notify_all();
      }
      progress = true;
    }
    // 3. wait
    if (!progress) {
      if (s->running.empty() && s->sched.waiting() == 0)
        s->cv_work.wait_for(lock, std::chrono::milliseconds(50));
      else {
        lock.unlock();
        std::this_thread::sleep_for(std::chrono::microseconds(20));
        lock.lock();
      }
    }
  }
}

bool server_ok(fft_server_t s) { return s && s->magic == kServerMagic; }

}  // namespace

extern "C" {

fft_status_t fft_server_create(fft_server_t* server, const fft_server_options_t* options) {
  if (!server) return set_error(FFT_ERR_INVALID_ARG, "server output pointer is null");
  *server = nullptr;
  fft_server_options_t o{};
  if (options) o = *options;
  if (o.memory_budget_bytes == 0) o.memory_budget_bytes = (size_t)64 << 30;
  if (o.streams <= 0) o.streams = 4;
  if (o.max_group <= 0) o.max_group = 256;
  if (o.max_running <= 0) o.max_running = 4 * o.streams;
  if (o.streams > 64) return set_error(FFT_ERR_INVALID_ARG, "at most 64 streams");
  if (o.large_group_log2 < -1 || o.large_group_log2 > 40)
    return set_error(FFT_ERR_INVALID_ARG, "large_group_log2 must be -1, 0 or 1..40");
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return set_error(FFT_ERR_CUDA, "no usable CUDA device");
  }
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess)
    return set_error(FFT_ERR_CUDA, "cudaGetDeviceProperties");
  fft_server_t s = new (std::nothrow) fft_server_s(o.memory_budget_bytes, o.max_group,
                                                    o.memory_budget_bytes, o.strict_order == 0);
  if (!s) return set_error(FFT_ERR_OUT_OF_MEMORY, "host allocation of the server failed");
  s->opt = o;
  s->device = dev;
  s->caps.sm_count = prop.multiProcessorCount;
  s->caps.smem_optin = (int)prop.sharedMemPerBlockOptin;
  s->caps.max_block = prop.maxThreadsPerBlock;
  for (int i = 0; i < o.streams; ++i) {
    cudaStream_t st;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      for (cudaStream_t x : s->streams) cudaStreamDestroy(x);
      delete s;
      return set_error(FFT_ERR_CUDA, "stream creation");
    }
    s->streams.push_back(st);
    s->stream_free.push_back(0.0);
  }
  cudaMemPoolProps pp{};
  pp.allocType = cudaMemAllocationTypePinned;
  pp.location.type = cudaMemLocationTypeDevice;
  pp.location.id = dev;
  if (cudaMemPoolCreate(&s->ws_pool, &pp) != cudaSuccess) {
    cudaGetLastError();
    for (cudaStream_t x : s->streams) cudaStreamDestroy(x);
    delete s;
    return set_error(FFT_ERR_CUDA, "workspace memory pool creation");
  }
  uint64_t keep = ~uint64_t(0);
  cudaMemPoolSetAttribute(s->ws_pool, cudaMemPoolAttrReleaseThreshold, &keep);
  s->worker = std::thread(worker_loop, s);
  *server = s;
  return FFT_OK;
}

fft_status_t fft_server_submit(fft_server_t s, const fft_job_t* job, uint64_t* ticket) {
  TraceRange trace("fft_server_submit");
  if (!server_ok(s)) return set_error(FFT_ERR_BAD_PLAN, "null or destroyed server");
  if (!job || !ticket) return set_error(FFT_ERR_INVALID_ARG, "job and ticket are required");
  // validate the shape with the planner (host only)
  PlanSpec probe;
  make_plan(probe, job->n, job->dims, 1, job->direction, job->precision, nullptr, s->caps);
  if (probe.status != FFT_OK) return set_error(probe.status, probe.error);
  if (job->batch < 1) return set_error(FFT_ERR_INVALID_ARG, "batch must be >= 1");
  if (!job->in || !job->out) return set_error(FFT_ERR_INVALID_ARG, "in/out must be device buffers");
  const int eb = elem_bytes(job->precision);  // complex64, or complex32
  if (((uintptr_t)job->in % eb) || ((uintptr_t)job->out % eb))
    return set_error(FFT_ERR_INVALID_ARG, "in/out must be aligned to the element size");
  const int64_t e = job_elems(*job) * job->batch;
  // workspace of one sub-batch (two-pass plans run large batches in sub-batches)
  const int64_t ws_entries =
      probe.work_elems > 0 ? std::min<int64_t>(job->batch, two_pass_chunk(job_elems(*job))) : 0;
  const size_t ws = (size_t)probe.work_elems * 8 * (size_t)ws_entries;
  const size_t bytes = (size_t)e * 2 * eb + (ws ? ws_class(ws) : 0);
  std::lock_guard<std::mutex> lock(s->mu);
  SchedJob sj;
  sj.id = s->next_id++;
  sj.key.dims = job->dims;
  sj.key.n0 = job->n[0];
  sj.key.n1 = job->dims > 1 ? job->n[1] : 1;
  sj.key.direction = job->direction;
  sj.key.precision = job->precision;
  sj.batch = job->batch;
  sj.bytes = bytes;
  sj.groupable = probe.passes.size() == 1 && probe.passes[0].batch_is_tiles &&
                 probe.passes[0].tc_prec == 0 && job->dims == 1;
  sj.t_submit = now_s();
  sj.cost = (double)e * 2.0 * eb * (double)probe.passes.size() / kEstBytesPerS + kEstLaunchS;
  if (!s->sched.submit(sj))
    return set_error(FFT_ERR_OUT_OF_MEMORY, "job needs more bytes than the server's budget");
  JobRec rec;
  rec.job = *job;
  rec.t_submit = sj.t_submit;
  s->jobs[sj.id] = rec;
  if (s->submitted++ == 0) s->first_submit = sj.t_submit;
  *ticket = sj.id;
  s->cv_work.notify_one();
  return FFT_OK;
}

fft_status_t fft_server_wait(fft_server_t s, uint64_t ticket, double timeout_s,
                             fft_job_result_t* result) {
  if (!server_ok(s)) return set_error(FFT_ERR_BAD_PLAN, "null or destroyed server");
  std::unique_lock<std::mutex> lock(s->mu);
  auto it = s->jobs.find(ticket);
  if (it == s->jobs.end()) return set_error(FFT_ERR_INVALID_ARG, "unknown ticket");
  const auto deadline = std::chrono::steady_clock::now() +
                        std::chrono::duration_cast<std::chrono::steady_clock::duration>(
                            std::chrono::duration<double>(timeout_s < 0 ? 1e9 : timeout_s));
  while (it->second.status < 0) {
    if (s->cv_done.wait_until(lock, deadline) == std::cv_status::timeout &&
        it->second.status < 0)
      return set_error(FFT_ERR_TIMEOUT, "job not finished before the timeout");
    it = s->jobs.find(ticket);
  }
  const JobRec& rec = it->second;
  if (result) {
    result->status = rec.status;
    result->latency_ms = (rec.t_done - rec.t_submit) * 1e3;
    result->queue_ms = rec.t_launch > 0 ? (rec.t_launch - rec.t_submit) * 1e3 : -1.0;
  }
  const int st = rec.status;
  s->jobs.erase(it);
  return st == FFT_OK ? FFT_OK : set_error((fft_status_t)st, "job failed");
}

fft_status_t fft_server_drain(fft_server_t s, double timeout_s) {
  if (!server_ok(s)) return set_error(FFT_ERR_BAD_PLAN, "null or destroyed server");
  std::unique_lock<std::mutex> lock(s->mu);
  const auto deadline = std::chrono::steady_clock::now() +
                        std::chrono::duration_cast<std::chrono::steady_clock::duration>(
                            std::chrono::duration<double>(timeout_s < 0 ? 1e9 : timeout_s));
  while (s->sched.waiting() > 0 || !s->running.empty()) {
    if (s->cv_done.wait_until(lock, deadline) == std::cv_status::timeout &&
        (s->sched.waiting() > 0 || !s->running.empty()))
      return set_error(FFT_ERR_TIMEOUT, "server did not drain before the timeout");
  }
  return FFT_OK;
}

fft_status_t fft_server_stats(fft_server_t s, fft_server_stats_t* out) {
  if (!server_ok(s)) return set_error(FFT_ERR_BAD_PLAN, "null or destroyed server");
  if (!out) return set_error(FFT_ERR_INVALID_ARG, "stats pointer is null");
  std::lock_guard<std::mutex> lock(s->mu);
  memset(out, 0, sizeof *out);
  out->submitted = s->submitted;
  out->completed = s->completed;
  out->failed = s->failed;
  out->launches = s->launches;
  out->coalesced_jobs = s->coalesced;
  out->groups = s->sched.groups();
  out->peak_bytes_in_flight = s->sched.peak_in_flight();
  out->budget_bytes = s->sched.budget();
  out->workspace_allocations = s->ws_allocs;
  out->backfilled_jobs = s->sched.backfilled();
  out->host_launch_s = s->host_launch_s;
  out->group_stream_s = s->group_stream_s;
  std::vector<double> l = s->latencies;
  if (!l.empty()) {
    std::sort(l.begin(), l.end());
    auto pct = [&](double p) { return l[std::min(l.size() - 1, (size_t)(p * (double)(l.size() - 1) + 0.5))]; };
    out->p50_ms = pct(0.50);
    out->p99_ms = pct(0.99);
    out->max_ms = l.back();
    double sum = 0;
    for (double v : l) sum += v;
    out->mean_ms = sum / (double)l.size();
  }
  out->wall_s = s->last_done > s->first_submit ? s->last_done - s->first_submit : 0.0;
  out->gflops = out->wall_s > 0 ? s->flops / out->wall_s / 1e9 : 0.0;
  return FFT_OK;
}

fft_status_t fft_server_pause(fft_server_t s, int paused) {
  if (!server_ok(s)) return set_error(FFT_ERR_BAD_PLAN, "null or destroyed server");
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->paused = paused != 0;
  }
  s->cv_work.notify_all();
  return FFT_OK;
}

fft_status_t fft_server_destroy(fft_server_t s) {
  if (!s) return FFT_OK;
  if (!server_ok(s)) return set_error(FFT_ERR_BAD_PLAN, "destroyed or foreign server");
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->stop = true;
    s->paused = false;
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  for (cudaStream_t st : s->streams) cudaStreamSynchronize(st);
  for (Running& r : s->running) {
    if (r.start) cudaEventDestroy(r.start);
    if (r.done) cudaEventDestroy(r.done);
  }
  if (s->ws_pool) cudaMemPoolDestroy(s->ws_pool);
  for (auto& ev : s->free_events) {
    cudaEventDestroy(ev.first);
    cudaEventDestroy(ev.second);
  }
  for (auto& kv : s->plans) {
    cudaFree(kv.second->tables);
    delete kv.second;
  }
  for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
  s->magic = 0;
  delete s;
  return FFT_OK;
}

}  // extern "C"
