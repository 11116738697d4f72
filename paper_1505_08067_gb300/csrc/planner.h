// Host-side planning: turns (n, dims, batch, direction) and the GPU's limits
// into a list of passes.  No CUDA calls here, so the planner runs on any host.
#pragma once
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/gbfft.h"
#include "fft_core.h"

namespace gbfft {

// Fixed-capacity array: planning needs no heap allocation (a plan never has
// more than 15 stages per pass, 4 passes or 40 twiddle segments).
template <class T, int N>
struct SmallVec {
  T v[N];
  int n = 0;
  void push_back(const T& x) {
    if (n < N) v[n++] = x;
  }
  void clear() { n = 0; }
  void assign(int count, const T& x) {
    n = count < N ? count : N;
    for (int i = 0; i < n; ++i) v[i] = x;
  }
  int size() const { return n; }
  bool empty() const { return n == 0; }
  T& operator[](int i) { return v[i]; }
  const T& operator[](int i) const { return v[i]; }
  T* begin() { return v; }
  T* end() { return v + n; }
  const T* begin() const { return v; }
  const T* end() const { return v + n; }
  static constexpr int capacity() { return N; }
};
using Sched = SmallVec<int, 15>;

enum { BUF_IN = 0, BUF_OUT = 1, BUF_WORK = 2, BUF_WORK2 = 3 };
enum { PASS_FFT = 0, PASS_COPY = 1, PASS_TRANSPOSE = 2 };
constexpr int kMaxPasses = 6;

struct Caps {
  int sm_count = 152;
  int smem_optin = 232448;  // bytes of dynamic shared memory a block may opt into
  int max_block = 1024;
};

struct PassSpec {
  int kind = PASS_FFT;
  int logL = 0;
  int R = 1;
  int G = 1;
  int lmap = MAP_ROWS, smap = MAP_ROWS;
  Sched rlogs;                 // radix schedule, stage order
  int64_t tiles = 0, tiles_inner = 1, count_inner = 0;
  int64_t outer = 1;           // number of outer indices (batch of a multi-pass plan)
  Strides in{}, out{};
  int src = BUF_IN, dst = BUF_OUT;
  int conj_in = 0, conj_out = 0;
  int epi = 0, epi_logN = 0, epi_lo_bits = 0;
  int block = 0;
  int pitch = 0;
  int smem_elems = 0;
  size_t smem = 0;
  int grid = 0;
  int variant = 0;              // contiguous passes: 0 auto, 1 register, 2 staged, 3 L2 prefetch
  int conv = 0;                 // fast convolution pass (see PassDesc::conv)
  int h_dim = 0;                // which dimension's filter
  int64_t h_lines = 1;          // 1 or the lines per frame along this dimension
  float h_scale = 1.f;
  int tc_prec = 0;              // tensor-core class (FFT_PREC_TC_*), 0 for FP32
  int io16 = 0;                 // tensor-core pass with complex32 (FP16) input and output
  bool batch_is_tiles = false;  // contiguous pass: batch maps to tiles of G transforms
  int64_t units_per_batch = 1;  // contiguous pass: transforms per batch entry
  // PASS_COPY
  int64_t copy_count = 0, copy_in_stride = 1, copy_out_stride = 1;
  // PASS_TRANSPOSE: per batch entry, the tr_rows x tr_cols row-major matrix at
  // the source is written as its tr_cols x tr_rows transpose; with tr_logN > 0
  // element (r, c) is first multiplied by exp(tr_sign * 2 pi i r c / 2^tr_logN)
  // (the six-step twiddle).
  int64_t tr_rows = 0, tr_cols = 0;
  int tr_logN = 0, tr_sign = -1;
  // twiddle-table offsets (complex entries) inside the plan's table allocation
  SmallVec<int32_t, 15> tw_off;  // per stage (stage 0 unused)
  int64_t epi_hi_off = 0, epi_lo_off = 0;
};

struct TwSegment {  // one twiddle_gen launch (mode 0: exponent (j / r) * (j % r))
  int64_t off, count, den, mult;
  int mode, r;
};

// Fast convolution (matched filtering) along every dimension of a plan:
// per dimension, the number of distinct filters (1, or one per line of a
// frame along that dimension) and the factor applied with the filter.
struct ConvSpec {
  int64_t lines[2] = {1, 1};
  float scale[2] = {1.f, 1.f};
};

struct PlanSpec {
  int dims = 1;
  int64_t n[2] = {1, 1};
  int64_t batch = 0;
  int direction = FFT_FORWARD;
  int precision = FFT_PREC_FP32;
  int max_block_log2 = 14;
  bool generic_only = false;  // never pick compile-time specialisations
  bool conv = false;          // fast-convolution plan (make_plan with a ConvSpec)
  const void* filter[2] = {nullptr, nullptr};  // device filter spectra per dimension
  SmallVec<PassSpec, kMaxPasses> passes;
  SmallVec<TwSegment, 40> tables;
  int64_t table_elems = 0;
  int64_t work_elems = 0;
  // two-pass 1D plans execute in sub-batches of at most chunk_batch transforms
  // (0: no sub-batching); work_elems holds one sub-batch
  int64_t chunk_batch = 0;
  // six-step plans: the second workspace buffer starts work2_off elements in
  int64_t work2_off = 0;
  fft_status_t status = FFT_OK;
  char error[256] = {0};
  char tuning[4096] = {0};  // autotuner report (JSON), empty if not tuned
};

// Elements a two-pass 1D plan executes at once: larger batches run in
// sub-batches.  The strided column passes touch many pages at once; measured
// on GB300, 2^22 x 256 (24 GiB with input, output and workspace) ran at 59% of
// the HBM bandwidth as one launch sequence and at 83% in two sub-batches,
// 2^20 x 1024 at 84% against 89% in sub-batches of 2^28 elements.
constexpr int64_t kTwoPassChunkElems = int64_t(1) << 28;

// Sub-batch (transforms) of a two-pass 1D plan of length n.
inline int64_t two_pass_chunk(int64_t n) {
  const int64_t c = kTwoPassChunkElems / (n > 0 ? n : 1);
  return c > 0 ? c : 1;
}

// Largest on-chip block 2^k for these limits: the shared-memory exchange
// buffer (with its padding) must fit one block, and at most 1024 threads of
// 16 elements each hold it.
int block_log2_limit(const Caps& caps);

// Default radix schedule of a length-2^logL pass with 2^logR elements per
// thread: as many full-radix stages as fit, the remainder radix last.
Sched default_schedule(int logL, int logR);

// Heap-free: fills `s` in place.  With `conv`, every dimension is a fast
// convolution pass (direction is ignored; the plan's filters are bound later).
// Bytes of one data element of a plan or job of this precision: complex64,
// or complex32 for FFT_PREC_TC_FP16_C32.
inline int elem_bytes(int precision) { return precision == FFT_PREC_TC_FP16_C32 ? 4 : 8; }

void make_plan(PlanSpec& s, const int64_t* n, int dims, int64_t batch, int direction,
               int precision, const fft_plan_options_t* opt, const Caps& caps,
               const ConvSpec* conv = nullptr);

// Rebuild one pass for a different radix / schedule / tile (autotuner); keeps
// geometry.  Returns false if the combination is invalid.
bool reshape_pass(PassSpec& p, int R, const Sched& rlogs, int G, const Caps& caps);

// Fill PassDesc (without device pointers) for a pass restricted to
// batch entries [b0, b0 + nb).
PassDesc pass_desc(const PassSpec& p, int64_t b0, int64_t nb, int64_t n_total);

std::string describe(const PlanSpec& s);

// Schedule digraph (Sec. 3.2).
uint64_t count_schedules(int log2n, const int* radix_logs, int n_radix);
bool shortest_schedule(int log2n, const int* radix_logs, int n_radix, const double* cost,
                       std::vector<int>& path, double& total);
bool schedule_cost(int log2n, const int* radix_logs, int n_radix, const double* cost,
                   const int* path, int len, double& total);

}  // namespace gbfft
