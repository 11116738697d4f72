// Per-call cost of the C ABI for a small batched transform (N = 1024 x 64,
// 512 KiB), measured from C so that no language binding sits in the loop.
//
//   call_latency [n] [batch] [reps]
//
// For fft_execute, fft_execute_graph, fft_execute_noalloc, and for an empty
// kernel launch as the floor of any launch on this device, it prints one JSON
// object with, per entry point:
//   host_us          host time to enqueue one call (calls back to back)
//   device_us        device time per call, CUDA events around the same loop
//                    (back to back: launch gaps included)
//   round_trip_us    median of single calls each followed by a stream
//                    synchronize (enqueue + execution + completion seen)
// and for the persistent work queue (fft_queue_*, same shape):
//   round_trip_us    median of single jobs, submit then wait
//   per_job_us       jobs submitted back to back, time per job until the
//                    last one is seen complete
// Exit status 0 on success, 1 on any library or CUDA error.
#include <cuda_runtime.h>
#include <stdio.h>
#include <stdlib.h>

#include <algorithm>
#include <chrono>
#include <vector>

#include "gbfft.h"

__global__ void empty_kernel() {}

static double now_us() {
  using namespace std::chrono;
  return duration<double, std::micro>(steady_clock::now().time_since_epoch()).count();
}

#define CK(x)                                                                      \
  do {                                                                             \
    cudaError_t e_ = (x);                                                          \
    if (e_ != cudaSuccess) {                                                       \
      fprintf(stderr, "%s:%d %s: %s\n", __FILE__, __LINE__, #x, cudaGetErrorString(e_)); \
      exit(1);                                                                     \
    }                                                                              \
  } while (0)

static void ok(fft_status_t s, const char* what) {
  if (s != FFT_OK) {
    fprintf(stderr, "%s failed: %d %s\n", what, (int)s, fft_last_error());
    exit(1);
  }
}

struct Result {
  double host_us, device_us, round_trip_us;
};

template <class F>
static Result measure(cudaStream_t st, int reps, F fn) {
  cudaEvent_t a, b;
  CK(cudaEventCreate(&a));
  CK(cudaEventCreate(&b));
  for (int i = 0; i < 50; ++i) fn();
  CK(cudaStreamSynchronize(st));
  CK(cudaEventRecord(a, st));
  const double t0 = now_us();
  for (int i = 0; i < reps; ++i) fn();
  const double t1 = now_us();
  CK(cudaEventRecord(b, st));
  CK(cudaEventSynchronize(b));
  float ms = 0;
  CK(cudaEventElapsedTime(&ms, a, b));
  std::vector<double> rt;
  for (int i = 0; i < 300; ++i) {
    const double t = now_us();
    fn();
    CK(cudaStreamSynchronize(st));
    rt.push_back(now_us() - t);
  }
  std::sort(rt.begin(), rt.end());
  CK(cudaEventDestroy(a));
  CK(cudaEventDestroy(b));
  return {(t1 - t0) / reps, ms * 1e3 / reps, rt[rt.size() / 2]};
}

int main(int argc, char** argv) {
  int64_t n = argc > 1 ? atoll(argv[1]) : 1024;
  int64_t batch = argc > 2 ? atoll(argv[2]) : 64;
  int reps = argc > 3 ? atoi(argv[3]) : 2000;
  if (n < 1 || batch < 1 || reps < 1) {
    fprintf(stderr, "usage: call_latency [n] [batch] [reps]\n");
    return 1;
  }
  const size_t bytes = (size_t)(n * batch) * 8;
  void *in = nullptr, *out = nullptr;
  CK(cudaMalloc(&in, bytes));
  CK(cudaMalloc(&out, bytes));
  CK(cudaMemset(in, 0x3c, bytes));  // finite values (0.0115 in every float)
  cudaStream_t st;
  CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  fft_plan_t plan = nullptr;
  ok(fft_plan_create(&plan, &n, 1, batch, FFT_FORWARD, FFT_PREC_FP32), "fft_plan_create");
  int launches = 0;
  ok(fft_plan_launch_count(plan, &launches), "fft_plan_launch_count");

  fft_status_t last = FFT_OK;
  const Result ex = measure(st, reps, [&] { last = fft_execute(plan, in, out, st); });
  ok(last, "fft_execute");
  const Result gr = measure(st, reps, [&] { last = fft_execute_graph(plan, in, out, st); });
  ok(last, "fft_execute_graph");
  const Result na =
      measure(st, reps, [&] { last = fft_execute_noalloc(n, batch, FFT_FORWARD, in, out, st); });
  ok(last, "fft_execute_noalloc");
  const Result e1 = measure(st, reps, [&] { empty_kernel<<<1, 32, 0, st>>>(); });
  CK(cudaGetLastError());
  const Result e64 = measure(st, reps, [&] { empty_kernel<<<64, 256, 0, st>>>(); });
  CK(cudaGetLastError());
  ok(fft_plan_sync_status(plan, st), "fft_plan_sync_status");

  // persistent work queue: the worker stays resident while jobs keep coming
  double q_rt = -1, q_per = -1;
  int64_t q_launches = 0;
  if (n >= 2 && n <= 4096) {
    fft_queue_t q = nullptr;
    ok(fft_queue_create(&q, n, batch, FFT_FORWARD, 64, 0), "fft_queue_create");
    uint64_t t = 0;
    for (int i = 0; i < 50; ++i) {
      ok(fft_queue_submit(q, in, out, batch, &t), "fft_queue_submit");
      ok(fft_queue_wait(q, t, 10.0), "fft_queue_wait");
    }
    std::vector<double> rt;
    for (int i = 0; i < 300; ++i) {
      const double t0 = now_us();
      ok(fft_queue_submit(q, in, out, batch, &t), "fft_queue_submit");
      ok(fft_queue_wait(q, t, 10.0), "fft_queue_wait");
      rt.push_back(now_us() - t0);
    }
    std::sort(rt.begin(), rt.end());
    q_rt = rt[rt.size() / 2];
    const double t0 = now_us();
    for (int i = 0; i < reps; ++i) ok(fft_queue_submit(q, in, out, batch, &t), "fft_queue_submit");
    ok(fft_queue_wait(q, t, 30.0), "fft_queue_wait");
    q_per = (now_us() - t0) / reps;
    uint64_t done = 0;
    ok(fft_queue_info(q, &q_launches, &done), "fft_queue_info");
    ok(fft_queue_destroy(q), "fft_queue_destroy");
  }

  auto js = [](const char* name, const Result& r, bool comma) {
    printf("\"%s\":{\"host_us\":%.3f,\"device_us\":%.3f,\"round_trip_us\":%.3f}%s", name, r.host_us,
           r.device_us, r.round_trip_us, comma ? "," : "");
  };
  printf("{\"n\":%lld,\"batch\":%lld,\"reps\":%d,\"launches_per_call\":%d,\"calls\":{",
         (long long)n, (long long)batch, reps, launches);
  js("fft_execute", ex, true);
  js("fft_execute_graph", gr, true);
  js("fft_execute_noalloc", na, true);
  js("empty_kernel_1x32", e1, true);
  js("empty_kernel_64x256", e64, false);
  printf("},\"fft_queue\":{\"round_trip_us\":%.3f,\"per_job_us\":%.3f,\"worker_launches\":%lld}}\n",
         q_rt, q_per, (long long)q_launches);
  fft_plan_destroy(plan);
  CK(cudaStreamDestroy(st));
  CK(cudaFree(in));
  CK(cudaFree(out));
  return 0;
}
