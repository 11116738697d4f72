// Host-side launch interface of the device kernels in kernels.cu.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

#include "fft_core.h"

namespace gbfft {

// Job table of a coalesced launch (see stockham_grouped): up to kMaxGroup jobs
// of one contiguous single-pass shape, each with its own buffers.
constexpr int kMaxGroup = 64;
struct GroupEntry {
  const cf* in;
  cf* out;
  int64_t tile_begin;  // first tile of this job in the launch
  int64_t tiles;       // tiles of this job
  int64_t count;       // transforms of this job
};
struct GroupTable {
  int n;
  GroupEntry e[kMaxGroup];
};

// Everything needed to launch one stockham_pass.
struct PassLaunch {
  PassDesc d;
  int R;            // elements per thread (register radix): 2, 4, 8 or 16
  int lmap, smap;   // thread maps of the load (and middle) stages and of the store
  int grid, block;  // grid size (tiles are grid-strided) and threads per block
  size_t smem;      // dynamic shared memory in bytes
  const void* fn = nullptr;  // resolved kernel (specialised or generic)
  bool specialised = false;
  bool has_staged = false;   // a staged kernel exists for this shape (see below)
  int persistent_grid = 0;   // nonzero: grid capped at resident blocks (L2-prefetch variant)
  int ctas_per_sm = 0;       // persistent kernels: resident blocks per SM the grid assumes
  struct StagedLaunchData {
    const void* fn = nullptr;
    int grid = 0, block = 0;
    int max_grid = 0;  // resident blocks per SM x SMs (persistent grid)
    size_t smem = 0;
    bool map_in = false;   // input in column tiles (tensor-map box loads possible)
    bool map_out = false;  // output in column tiles (tensor-map box stores possible)
    bool tmap = false;     // use tensor maps where the layout allows
  } staged;
};

// The staged kernel for a pass (one contiguous transform or G columns per
// block, TMA copy of the next tile); used when the source is 16-byte aligned.
using StagedLaunch = PassLaunch::StagedLaunchData;

// Fills `s` if a staged kernel exists for this pass shape (contiguous
// transforms, or column tiles of a strided pass) and thread maps.
bool resolve_staged(const PassDesc& d, int lmap, int smap, bool generic_only, StagedLaunch* s);
// Opt-in shared memory and a persistent grid of (blocks per SM) x SMs.
cudaError_t prepare_staged(StagedLaunch& s, int64_t tiles, int sm_count);
cudaError_t launch_staged(const StagedLaunch& s, const PassDesc& d, const void* in, void* out,
                          cudaStream_t st);
// Encodes d.tmap_in (map_in) and d.tmap_out (map_out) for column tiles over
// `in` / `out` and sets d.tmap_*_ok; false if neither could be encoded (the
// pass's layout or the driver does not allow it).
bool encode_cols_maps(PassDesc& d, bool map_in, bool map_out, const void* in, void* out);

// Kernel for this pass shape: a compile-time specialisation when one matches,
// else the generic kernel for (R, maps).
const void* resolve_kernel(int R, int lmap, int smap, const PassDesc& d, bool generic_only,
                           bool* specialised);

// Tensor-core class kernel for length 2^logL (4, 8, 12) and FFT_PREC_TC_*:
// the warp-level MMA form.
const void* resolve_tc(int logL, int prec);
// The tcgen05 form for length 2^logL (4 .. 14); *smem = the shared memory it
// needs (the plan may ask for more to bound the CTAs per SM).
const void* resolve_umma(int logL, int prec, size_t* smem);
// Tensor-memory columns one tcgen05 block of length 2^logL allocates.
int umma_tmem_cols(int logL);
// Blocks of `fn` one SM holds at once by its registers, shared memory and
// threads (from the kernel's attributes and the device's limits), and by
// tensor memory when tmem_cols > 0 (512 columns per SM).
cudaError_t resident_blocks(const void* fn, int block, size_t smem, int tmem_cols, int* blocks);
// The tcgen05 form of the FP16 class with complex32 input and output.
const void* resolve_umma_c32(int logL, size_t* smem);
// The kernel of a tensor-core pass of the given variant (0 tcgen05, 1 warp MMA);
// io16: complex32 input and output (tcgen05, FP16 only).
inline const void* resolve_tc_pass(int logL, int prec, int variant, int io16 = 0) {
  size_t sm = 0;
  if (io16) return variant == 0 && prec == 1 ? resolve_umma_c32(logL, &sm) : nullptr;  // FP16
  return variant == 1 ? resolve_tc(logL, prec) : resolve_umma(logL, prec, &sm);
}

// Six-step transposes (transpose.cu): per batch entry, rows x cols -> cols x
// rows, optionally multiplying element (r, c) by exp(sign 2 pi i r c / 2^logN)
// first (logN > 0); complex64, or complex32 with h16.  rows and cols are
// multiples of 32.
cudaError_t launch_transpose(const void* in, void* out, int64_t batch, int64_t rows, int64_t cols,
                             int logN, int sign, int h16, int sm_count, cudaStream_t st);

// Per-kernel attributes a launch needs (opt-in shared memory); call once after
// resolving, before the first launch_pass.
cudaError_t prepare_launch(PassLaunch& p);

cudaError_t launch_pass(const PassLaunch& p, const void* in, void* out, cudaStream_t st);
cudaError_t occupancy(const PassLaunch& p, int* ctas_per_sm);
// Times one Stockham stage in isolation (see stage_bench).
cudaError_t launch_stage_bench(int R, const PassDesc& d, int Ns, int reps, int grid, int block,
                               size_t smem, void* sink, cudaStream_t st);
// One launch over the jobs of `gt` with the generic row kernel of R elements
// per thread; d0 is the pass descriptor of one job (tables, shape, strides).
cudaError_t launch_grouped(int R, const PassDesc& d0, const GroupTable& gt, int grid, int block,
                           size_t smem, cudaStream_t st);
cudaError_t launch_copy(const void* in, void* out, int64_t count, int64_t in_stride,
                        int64_t out_stride, cudaStream_t st);
cudaError_t launch_twiddle_gen(void* out, int64_t count, int64_t den, int mode, int r,
                               int64_t mult, cudaStream_t st);

}  // namespace gbfft
