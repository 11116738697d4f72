// Device kernels of the batched complex FFT (sm_103a).
//
//  stockham_pass<R, LMAP, SMAP>  one pass of a batched transform: every
//      transform of length L <= 2^14 (or a tile of G of them) lives on one SM,
//      each thread holds R elements in registers, radix stages exchange through
//      shared memory, global memory is read once and written once
//      (Bergach et al. Sec. 3.4 "one FFT per EU": only the first read and the
//      last write touch the memory hierarchy).  The output can be written
//      transposed and multiplied by the four-step twiddle w_N^{n2 k1}, which is
//      how passes of a split transform are joined (Sec. 3.3).
//  twiddle_gen                   FP64 roots of unity rounded once to FP32
//      (the precomputed twiddle table of Sec. 2.1).
//  copy_kernel                   length-1 transforms (the DFT is the identity).
#include <cuda_runtime.h>

#include "fft_stage.h"
#include "kernels.h"

namespace gbfft {

struct DevMem {
  // Input is read exactly once: stream it past L1 with an evict-first hint.
  GB_HD static cf ldg(const cf* p, int64_t off) {
#ifdef __CUDA_ARCH__
    float2 r = __ldcs(reinterpret_cast<const float2*>(p) + off);
    return mk(r.x, r.y);
#else
    return p[off];
#endif
  }
  GB_HD static void stg(cf* p, int64_t off, cf v) {
#ifdef __CUDA_ARCH__
    *(reinterpret_cast<float2*>(p) + off) = make_float2(v.x, v.y);
#else
    p[off] = v;
#endif
  }
  GB_HD static cf ldtw(const cf* p) {
#ifdef __CUDA_ARCH__
    float2 r = __ldg(reinterpret_cast<const float2*>(p));
    return mk(r.x, r.y);
#else
    return *p;
#endif
  }
  GB_HD static cf lds(const cf* s, int i) { return s[i]; }
  GB_HD static void sts(cf* s, int i, cf v) { s[i] = v; }
};

template <int R, int LMAP, int SMAP>
__global__ void __launch_bounds__(1024)
stockham_pass(const cf* __restrict__ in, cf* out, const __grid_constant__ PassDesc d) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cf* sm = reinterpret_cast<cf*>(smem_raw);
  using B = PassBody<R, LMAP, SMAP, DevMem>;
  const int tid = threadIdx.x;
  for (int64_t tile = blockIdx.x; tile < d.tiles; tile += gridDim.x) {
    const typename B::Tile tl = B::tile_of(d, tile);
    cf v[R];
    B::first(v, d, in, out, sm, tl, tid);
    int Ns = 1 << d.rlog[0];
    for (int s = 1; s < d.nst; ++s) {
      __syncthreads();
      B::read(v, d, s, Ns, out, sm, tl, tid);
      if (s < d.nst - 1) {
        __syncthreads();
        B::write(v, d, s, Ns, sm, tid);
      }
      Ns <<= d.rlog[s];
    }
    __syncthreads();  // shared memory is reused by the next tile
  }
}

// out[i] = in[i] for `count` transforms of length 1 with the given strides.
__global__ void copy_kernel(const cf* __restrict__ in, cf* out, int64_t count, int64_t in_stride,
                            int64_t out_stride) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i * out_stride] = in[i * in_stride];
}

// Twiddle tables in FP64, rounded once to FP32.  Segment j of `count`:
//   mode 0 (stage table, radix r):  exponent = (j / r) * (j % r)
//   mode 1 (power table):           exponent = j * mult
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

template <int R, int LMAP, int SMAP>
static cudaError_t launch_t(const PassDesc& d, const cf* in, cf* out, int grid, int block,
                            size_t smem, cudaStream_t st) {
  auto k = stockham_pass<R, LMAP, SMAP>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
  }
  k<<<grid, block, smem, st>>>(in, out, d);
  return cudaGetLastError();
}

template <int LMAP, int SMAP>
static cudaError_t launch_maps(int R, const PassDesc& d, const cf* in, cf* out, int grid,
                               int block, size_t smem, cudaStream_t st) {
  switch (R) {
    case 2: return launch_t<2, LMAP, SMAP>(d, in, out, grid, block, smem, st);
    case 4: return launch_t<4, LMAP, SMAP>(d, in, out, grid, block, smem, st);
    case 8: return launch_t<8, LMAP, SMAP>(d, in, out, grid, block, smem, st);
    case 16: return launch_t<16, LMAP, SMAP>(d, in, out, grid, block, smem, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_pass(const PassLaunch& p, const void* in, void* out, cudaStream_t st) {
  const cf* i = static_cast<const cf*>(in);
  cf* o = static_cast<cf*>(out);
  if (p.lmap == MAP_ROWS && p.smap == MAP_ROWS)
    return launch_maps<MAP_ROWS, MAP_ROWS>(p.R, p.d, i, o, p.grid, p.block, p.smem, st);
  if (p.lmap == MAP_COLS && p.smap == MAP_COLS)
    return launch_maps<MAP_COLS, MAP_COLS>(p.R, p.d, i, o, p.grid, p.block, p.smem, st);
  if (p.lmap == MAP_ROWS && p.smap == MAP_COLS)
    return launch_maps<MAP_ROWS, MAP_COLS>(p.R, p.d, i, o, p.grid, p.block, p.smem, st);
  return cudaErrorInvalidValue;
}

cudaError_t kernel_attributes(int R, int lmap, int smap, cudaFuncAttributes* attr) {
#define GB_ATTR(RR, A, B_) \
  if (R == RR && lmap == A && smap == B_) return cudaFuncGetAttributes(attr, stockham_pass<RR, A, B_>);
  GB_ATTR(2, 0, 0) GB_ATTR(4, 0, 0) GB_ATTR(8, 0, 0) GB_ATTR(16, 0, 0)
  GB_ATTR(2, 1, 1) GB_ATTR(4, 1, 1) GB_ATTR(8, 1, 1) GB_ATTR(16, 1, 1)
  GB_ATTR(2, 0, 1) GB_ATTR(4, 0, 1) GB_ATTR(8, 0, 1) GB_ATTR(16, 0, 1)
#undef GB_ATTR
  return cudaErrorInvalidValue;
}

cudaError_t occupancy(int R, int lmap, int smap, int block, size_t smem, int* ctas_per_sm) {
#define GB_OCC(RR, A, B_)                                                                   \
  if (R == RR && lmap == A && smap == B_) {                                                 \
    auto k = stockham_pass<RR, A, B_>;                                                      \
    if (smem > 48 * 1024) {                                                                 \
      cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                           (int)smem);                                      \
      if (e != cudaSuccess) return e;                                                       \
    }                                                                                       \
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, k, block, smem);      \
  }
  GB_OCC(2, 0, 0) GB_OCC(4, 0, 0) GB_OCC(8, 0, 0) GB_OCC(16, 0, 0)
  GB_OCC(2, 1, 1) GB_OCC(4, 1, 1) GB_OCC(8, 1, 1) GB_OCC(16, 1, 1)
  GB_OCC(2, 0, 1) GB_OCC(4, 0, 1) GB_OCC(8, 0, 1) GB_OCC(16, 0, 1)
#undef GB_OCC
  return cudaErrorInvalidValue;
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
