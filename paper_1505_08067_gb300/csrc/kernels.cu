// Device kernels of the batched complex FFT (sm_103a).
//
//  stockham_pass<R, LMAP, SMAP, TR>  one pass of a batched transform: every
//      transform of length L <= 2^14 (or a tile of G of them) lives on one SM,
//      each thread holds R elements in registers, radix stages exchange through
//      shared memory, global memory is read once and written once
//      (Bergach et al. Sec. 3.4 "one FFT per EU": only the first read and the
//      last write touch the memory hierarchy).  The output can be written
//      transposed and multiplied by the four-step twiddle w_N^{n2 k1}, which is
//      how passes of a split transform are joined (Sec. 3.3).  TR = RtTraits
//      is the generic kernel; CtTraits instantiations fix the hot shapes at
//      compile time.
//  twiddle_gen                   FP64 roots of unity rounded once to FP32
//      (the precomputed twiddle table of Sec. 2.1).
//  copy_kernel                   length-1 transforms (the DFT is the identity).
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>
#include <mutex>

#include "kernels_impl.cuh"

namespace gbfft {

// out[i] = in[i] for `count` transforms of length 1 with the given strides.
__global__ void copy_kernel(const cf* __restrict__ in, cf* out, int64_t count, int64_t in_stride,
                            int64_t out_stride) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i * out_stride] = in[i * in_stride];
}

// Twiddle tables in FP64, rounded once to FP32.  Entry j of `count`:
//   mode 0 (stage table):  exponent = (j / r) * (j % r)
//   mode 1 (power table):  exponent = j * mult
// value = exp(-2 pi i * (exponent mod den) / den).  The exponent is reduced as
// an integer, so sincospi receives an exact argument in [0, 2).
__global__ void twiddle_gen(float2* out, int64_t count, int64_t den, int mode, int r,
                            int64_t mult) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < count;
       j += (int64_t)gridDim.x * blockDim.x) {
    int64_t e = (mode == 0) ? (j / r) * (j % r) : j * mult;
    e %= den;
    double s, c;
    sincospi(2.0 * (double)e / (double)den, &s, &c);
    out[j] = make_float2((float)c, (float)(-s));
  }
}

// ------------------------------------------------------------------ host --

static KernelFn generic_kernel(int R, int lmap, int smap) {
  if (lmap == MAP_ROWS && smap == MAP_ROWS) return (KernelFn)generic_kernel_rows(R);
  if (lmap == MAP_COLS && smap == MAP_COLS) return (KernelFn)generic_kernel_cols(R);
  if (lmap == MAP_ROWS && smap == MAP_COLS) return (KernelFn)generic_kernel_transposing(R);
  return nullptr;
}

const void* resolve_kernel(int R, int lmap, int smap, const PassDesc& d, bool generic_only,
                           bool* specialised) {
  if (d.conv) {
    if (lmap != smap) return nullptr;  // convolution passes keep their layout
    return resolve_conv_kernel(R, lmap, d, generic_only, specialised);
  }
  if (!generic_only) {
    const void* f = resolve_contig_shape(R, lmap, smap, d);
    if (!f) f = resolve_fourstep_shape(R, lmap, smap, d);
    if (f) {
      if (specialised) *specialised = true;
      return f;
    }
  }
  if (specialised) *specialised = false;
  return (const void*)generic_kernel(R, lmap, smap);
}

bool resolve_staged(const PassDesc& d, int lmap, int smap, bool generic_only, StagedLaunch* s) {
  if (generic_only) return false;
  if (lmap == MAP_COLS) {
    s->map_in = s->map_out = true;
    // convolutions over column tiles: only with per-column filters staged
    // by tile (a shared filter keeps the register kernel)
    return (!d.conv || cols_filter_staged(d)) && resolve_staged_cols_shape(d, lmap, smap, s);
  }
  if (lmap == MAP_ROWS && smap == MAP_COLS) {
    s->map_out = true;
    return !d.conv && resolve_staged_trans_shape(d, lmap, smap, s);
  }
  if (lmap != MAP_ROWS || smap != MAP_ROWS) return false;
  return d.conv ? resolve_conv_staged_shape(d, s) : resolve_staged_shape(d, s);
}

cudaError_t prepare_staged(StagedLaunch& s, int64_t tiles, int sm_count) {
  cudaError_t e = cudaFuncSetAttribute(s.fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)s.smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, s.fn, s.block, s.smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  int64_t g = (int64_t)per_sm * sm_count;
  s.max_grid = (int)g;
  s.grid = (int)(g < tiles ? g : tiles);
  return cudaSuccess;
}

// cuTensorMapEncodeTiled from the driver (no link-time dependency on libcuda).
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    else
      (void)cudaGetLastError();
  });
  return fn;
}

// Tensor map for the column tiles of pass `d` over buffer `p` with strides
// `st` (d.in or d.out): rows of st.e complex64 elements, boxes of G columns x
// `box_rows` rows.  False when the layout does not allow it (cols_map_rows),
// `p` is not 16-byte aligned, or the encoder refuses.
static bool encode_cols_map(const PassDesc& d, const Strides& st, const void* p, int box_rows,
                            unsigned char (&map)[128]) {
  int64_t rows = 0;
  if (!cols_map_rows(d, st, rows) || ((uintptr_t)p & 15)) return false;
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return false;
  static_assert(sizeof(CUtensorMap) == sizeof(map), "tensor map size");
  const cuuint64_t dims[2] = {(cuuint64_t)st.e, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)st.e * 8};
  const cuuint32_t box[2] = {(cuuint32_t)d.G, (cuuint32_t)box_rows};
  const cuuint32_t elem_strides[2] = {1, 1};
  CUtensorMap m;
  if (enc(&m, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, const_cast<void*>(p), dims, strides, box,
          elem_strides, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
          CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return false;
  memcpy(map, &m, sizeof(m));
  return true;
}

// Tensor map of the filter frame of a convolution over column tiles
// (cols_filter_staged): dims {in.e, L}, boxes of G columns x min(L, 256) rows.
static bool encode_filter_map(PassDesc& d) {
  const int L = 1 << d.logL;
  if (!cols_filter_staged(d) || ((uintptr_t)d.h & 15)) return false;
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)d.in.e, (cuuint64_t)L};
  const cuuint64_t strides[1] = {(cuuint64_t)d.in.e * 8};
  const cuuint32_t box[2] = {(cuuint32_t)d.G, (cuuint32_t)(L < 256 ? L : 256)};
  const cuuint32_t elem_strides[2] = {1, 1};
  CUtensorMap m;
  if (enc(&m, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, const_cast<cf*>(d.h), dims, strides, box,
          elem_strides, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
          CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return false;
  memcpy(d.tmap_h, &m, sizeof(m));
  return true;
}

bool encode_cols_maps(PassDesc& d, bool map_in, bool map_out, const void* in, void* out) {
  const int L = 1 << d.logL;
  d.tmap_in_ok = map_in && encode_cols_map(d, d.in, in, L < 256 ? L : 256, d.tmap_in);
  d.tmap_out_ok =
      map_out && encode_cols_map(d, d.out, out, L / 2 < 256 ? L / 2 : 256, d.tmap_out);
  d.tmap_h_ok = map_in && d.tmap_in_ok && encode_filter_map(d);
  return d.tmap_in_ok || d.tmap_out_ok;
}

cudaError_t launch_staged(const StagedLaunch& s, const PassDesc& d, const void* in, void* out,
                          cudaStream_t st) {
  KernelFn k = reinterpret_cast<KernelFn>(const_cast<void*>(s.fn));
  if (!k || s.grid < 1) return cudaErrorInvalidValue;
  PassDesc dm = d;
  if (s.tmap && (s.map_in || s.map_out)) {
    const bool mo = s.map_out && cols_store_map(d);
    encode_cols_maps(dm, s.map_in, mo, in, out);
  }
  k<<<s.grid, s.block, s.smem, st>>>(static_cast<const cf*>(in), static_cast<cf*>(out), dm);
  return cudaGetLastError();
}

cudaError_t prepare_launch(PassLaunch& p) {
  if (!p.fn) return cudaErrorInvalidValue;
  if (p.smem > 48 * 1024)
    return cudaFuncSetAttribute(p.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem);
  return cudaSuccess;
}

cudaError_t launch_pass(const PassLaunch& p, const void* in, void* out, cudaStream_t st) {
  KernelFn k = reinterpret_cast<KernelFn>(const_cast<void*>(p.fn));
  if (!k) return cudaErrorInvalidValue;
  k<<<p.grid, p.block, p.smem, st>>>(static_cast<const cf*>(in), static_cast<cf*>(out), p.d);
  return cudaGetLastError();
}

cudaError_t occupancy(const PassLaunch& p, int* ctas_per_sm) {
  KernelFn k = reinterpret_cast<KernelFn>(const_cast<void*>(p.fn));
  if (!k) return cudaErrorInvalidValue;
  if (p.smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute((const void*)k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)p.smem);
    if (e != cudaSuccess) return e;
  }
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, (const void*)k, p.block,
                                                       p.smem);
}

cudaError_t resident_blocks(const void* fn, int block, size_t smem, int tmem_cols, int* blocks) {
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, fn);
  if (e != cudaSuccess) return e;
  int dev = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  int regs_sm = 0, smem_sm = 0, threads_sm = 0, blocks_sm = 0, reserved = 0;
  cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&threads_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
  cudaDeviceGetAttribute(&blocks_sm, cudaDevAttrMaxBlocksPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
  const int warps = (block + 31) / 32;
  const int regs_warp = ((fa.numRegs * 32 + 255) / 256) * 256;  // allocated per warp in 256s
  int n = blocks_sm;
  if (regs_warp > 0) n = std::min(n, regs_sm / (regs_warp * warps));
  n = std::min(n, threads_sm / block);
  const size_t per_block = smem + fa.sharedSizeBytes + (size_t)reserved;
  if (per_block > 0) n = std::min(n, (int)((size_t)smem_sm / per_block));
  if (tmem_cols > 0) n = std::min(n, 512 / tmem_cols);
  *blocks = std::max(n, 0);
  return cudaSuccess;
}

cudaError_t launch_stage_bench(int R, const PassDesc& d, int Ns, int reps, int grid, int block,
                               size_t smem, void* sink, cudaStream_t st) {
  const void* f = nullptr;
  switch (R) {
    case 2: f = (const void*)stage_bench<2>; break;
    case 4: f = (const void*)stage_bench<4>; break;
    case 8: f = (const void*)stage_bench<8>; break;
    case 16: f = (const void*)stage_bench<16>; break;
    default: return cudaErrorInvalidValue;
  }
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  using BenchFn = void (*)(PassDesc, int, int, cf*);
  reinterpret_cast<BenchFn>(const_cast<void*>(f))<<<grid, block, smem, st>>>(d, Ns, reps,
                                                                                 static_cast<cf*>(sink));
  return cudaGetLastError();
}

cudaError_t launch_grouped(int R, const PassDesc& d0, const GroupTable& gt, int grid, int block,
                           size_t smem, cudaStream_t st) {
  if (gt.n < 1 || gt.n > kMaxGroup) return cudaErrorInvalidValue;
  const void* f = nullptr;
  switch (R) {
    case 2: f = (const void*)stockham_grouped<2>; break;
    case 4: f = (const void*)stockham_grouped<4>; break;
    case 8: f = (const void*)stockham_grouped<8>; break;
    case 16: f = (const void*)stockham_grouped<16>; break;
    default: return cudaErrorInvalidValue;
  }
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  using GFn = void (*)(PassDesc, GroupTable);
  reinterpret_cast<GFn>(const_cast<void*>(f))<<<grid, block, smem, st>>>(d0, gt);
  return cudaGetLastError();
}

cudaError_t launch_copy(const void* in, void* out, int64_t count, int64_t in_stride,
                        int64_t out_stride, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  int64_t blocks = (count + 255) / 256;
  if (blocks > 65535) blocks = 65535;
  copy_kernel<<<(int)blocks, 256, 0, st>>>(static_cast<const cf*>(in), static_cast<cf*>(out),
                                           count, in_stride, out_stride);
  return cudaGetLastError();
}

cudaError_t launch_twiddle_gen(void* out, int64_t count, int64_t den, int mode, int r,
                               int64_t mult, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  int64_t blocks = (count + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  twiddle_gen<<<(int)blocks, 256, 0, st>>>(static_cast<float2*>(out), count, den, mode, r, mult);
  return cudaGetLastError();
}

}  // namespace gbfft
