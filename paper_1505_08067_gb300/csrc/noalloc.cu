// fft_execute_noalloc: the batched 1D transform without a plan and without any
// device allocation.
//
// Who needs it: callers that are not allowed to allocate GPU memory once they
// are running -- for example a radar processing loop that reserves all of its
// memory at start-up and must not stall later (cudaMalloc can block and
// synchronise the device), or code that runs inside a host framework that owns
// the whole device-memory budget and forbids allocations behind its back.
// Such callers still own their input and output buffers; everything else the
// transform needs (twiddle tables and, for lengths above 2^14, the workspace
// between the two passes) lives in one array reserved statically below.
//
// The array is a file-scope __device__ variable, so every GPU that loads this
// library holds it until the process exits.  Host code must not use its name
// as an address (on the host it is only a stand-in): the device address is
// looked up with cudaGetSymbolAddress once per device, the first time this
// entry point runs on that device, and cached.
//
// Host-side state per device (static, no heap): the device address, and the
// plan and bound launches of the last shape called, so that a loop calling
// with one shape pays the planning and kernel preparation once; the twiddle
// tables in the array are regenerated only when the table layout changes.
#include <cuda_runtime.h>
#include <string.h>

#include <mutex>

#include "../../include/gbfft.h"
#include "exec.h"
#include "trace.h"

namespace gbfft {
fft_status_t set_error(fft_status_t st, const char* msg);
}

using namespace gbfft;

namespace {

constexpr int64_t kWorkElems = int64_t(1) << 23;   // 64 MiB of complex64 workspace
constexpr int64_t kTableElems = int64_t(1) << 16;  // 512 KiB of twiddle factors
constexpr int kMaxDevices = 64;

static __device__ __align__(256) float2 g_noalloc_scratch[kWorkElems + kTableElems];

struct DeviceState {
  void* addr = nullptr;      // device address of g_noalloc_scratch
  bool have_shape = false;   // spec / launches hold the last (n, batch, direction)
  int64_t n = 0, batch = 0;
  int direction = 0;
  PlanSpec spec;
  PassLaunch launches[kMaxPasses];
  bool tables_valid = false;  // the array holds the tables of `spec` (segment list below)
  SmallVec<TwSegment, 40> table_layout;
};

std::mutex g_mu;
DeviceState g_state[kMaxDevices];

bool same_tables(const SmallVec<TwSegment, 40>& a, const SmallVec<TwSegment, 40>& b) {
  if (a.size() != b.size()) return false;
  for (int i = 0; i < a.size(); ++i) {
    const TwSegment &x = a[i], &y = b[i];
    if (x.off != y.off || x.count != y.count || x.den != y.den || x.mult != y.mult ||
        x.mode != y.mode || x.r != y.r)
      return false;
  }
  return true;
}

// Device address of the scratch array on `dev` (which must be current).
fft_status_t scratch_address(DeviceState& ds) {
  if (ds.addr) return FFT_OK;
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || !p) {
    cudaGetLastError();
    return set_error(FFT_ERR_CUDA, "fft_execute_noalloc: cudaGetSymbolAddress of the static "
                                   "scratch array failed");
  }
  ds.addr = p;
  return FFT_OK;
}

}  // namespace

extern "C" fft_status_t fft_execute_noalloc(int64_t n, int64_t batch, int direction,
                                            const void* in, void* out, void* stream) {
  TraceRange trace("fft_execute_noalloc");
  if (n < 1 || (n & (n - 1)) || n > kWorkElems)
    return set_error(FFT_ERR_UNSUPPORTED_SIZE,
                     "fft_execute_noalloc: n must be a power of two between 1 and 2^23");
  if (direction != FFT_FORWARD && direction != FFT_INVERSE)
    return set_error(FFT_ERR_INVALID_ARG, "direction must be FFT_FORWARD or FFT_INVERSE");
  if (batch < 0) return set_error(FFT_ERR_INVALID_ARG, "batch must be >= 0");
  if (batch == 0) return FFT_OK;
  if (!in || !out) return set_error(FFT_ERR_INVALID_ARG, "in/out must be device pointers");
  if (((uintptr_t)in & 7) || ((uintptr_t)out & 7))
    return set_error(FFT_ERR_INVALID_ARG, "in/out must be 8-byte aligned (complex64)");
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return set_error(FFT_ERR_CUDA, "no usable CUDA device");
  }
  if (dev < 0 || dev >= kMaxDevices)
    return set_error(FFT_ERR_INVALID_ARG, "fft_execute_noalloc supports device ids 0..63");
  std::lock_guard<std::mutex> lock(g_mu);
  DeviceState& ds = g_state[dev];
  fft_status_t st = scratch_address(ds);
  if (st != FFT_OK) return st;
  cf* work = static_cast<cf*>(ds.addr);
  cf* tables = work + kWorkElems;
  int* status = reinterpret_cast<int*>(tables + (kTableElems - 2));
  cudaStream_t cs = static_cast<cudaStream_t>(stream);

  if (!(ds.have_shape && ds.n == n && ds.batch == batch && ds.direction == direction)) {
    ds.have_shape = false;
    Caps caps;
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess)
      caps.sm_count = v;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) == cudaSuccess)
      caps.smem_optin = v;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxThreadsPerBlock, dev) == cudaSuccess)
      caps.max_block = v;
    fft_plan_options_t opt{};
    opt.epilogue = 4;  // four-step twiddles computed in-kernel: no N-entry table in static memory
    make_plan(ds.spec, &n, 1, batch, direction, FFT_PREC_FP32, &opt, caps);
    if (ds.spec.status != FFT_OK) return set_error(ds.spec.status, ds.spec.error);
    if (ds.spec.work_elems > kWorkElems)
      return set_error(FFT_ERR_UNSUPPORTED_SIZE,
                       "fft_execute_noalloc: n * batch needs more than the 64 MiB static "
                       "workspace (at most 2^23 complex elements when n > 2^14); use "
                       "fft_plan_create");
    if (ds.spec.table_elems + 2 > kTableElems)
      return set_error(FFT_ERR_UNSUPPORTED_SIZE,
                       "fft_execute_noalloc: twiddle tables exceed the static area");
    cudaError_t e = bind_launches(ds.spec, caps, tables, status, ds.launches);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return set_error(FFT_ERR_CUDA, cudaGetErrorString(e));
    }
    ds.have_shape = true;
    ds.n = n;
    ds.batch = batch;
    ds.direction = direction;
  }

  // the status word the staged kernels set when a bounded wait gives up:
  // cleared on the caller's stream, so a give-up of an earlier call does not
  // linger (an asynchronous memset allocates nothing)
  cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int), cs);
  if (e == cudaSuccess && !(ds.tables_valid && same_tables(ds.table_layout, ds.spec.tables))) {
    ds.tables_valid = false;
    e = enqueue_tables(ds.spec, tables, cs);
    if (e == cudaSuccess) {
      ds.table_layout = ds.spec.tables;
      ds.tables_valid = true;
    }
  }
  if (e == cudaSuccess) e = enqueue_passes(ds.spec, ds.launches, in, out, work, 0, batch, cs);
  if (e != cudaSuccess) {
    cudaGetLastError();
    ds.tables_valid = false;
    ds.have_shape = false;
    return set_error(FFT_ERR_CUDA, cudaGetErrorString(e));
  }
  return FFT_OK;
}
