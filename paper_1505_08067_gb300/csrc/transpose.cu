// Batched transpose with an optional twiddle multiply: the transposes of a
// six-step plan (Sec. 3.3 split into passes; Sec. 3.4 blocked transpose
// through on-chip memory).  Per batch entry the rows x cols row-major matrix
// at `in` is written as its cols x rows transpose at `out`; with logN > 0,
// element (r, c) is first multiplied by exp(sign * 2 pi i r c / 2^logN)
// (r c < 2^logN: the exponent is exact, the angle 2 r c / 2^logN too; a
// thread's rows r, r + 8, r + 16, r + 24 of one column take the powers of
// exp(sign 2 pi i 8 c / 2^logN), at most three further roundings).
// Elements are complex64, or complex32 (FP16 pairs) with H.
//
// 32 x 32 tiles through shared memory (one padding column: the column reads
// of a half warp fall into distinct bank pairs); 256 threads moving 4
// elements each (plain complex64) or 128 threads moving 8 (complex32, and
// the twiddle transpose), loads and stores both along rows of 32
// consecutive elements.  Persistent grid over all tiles of all batch
// entries.
#include <cuda_runtime.h>

#include <algorithm>

#include "kernels_impl.cuh"
#include "tc_stage.h"

namespace gbfft {

namespace {

template <bool H>
__device__ __forceinline__ cf tr_load(const void* p, int64_t i) {
  if (H) {  // an FP16 pair (real in the low half), widened exactly
    const uint32_t r = __ldcs(static_cast<const unsigned int*>(p) + i);
    float x, y;
    asm("{\n\t.reg .b16 l, h;\n\tmov.b32 {l, h}, %2;\n\tcvt.f32.f16 %0, l;\n\tcvt.f32.f16 %1, h;\n\t}"
        : "=f"(x), "=f"(y)
        : "r"(r));
    return mk(x, y);
  }
  const float2 v = __ldcs(static_cast<const float2*>(p) + i);
  return mk(v.x, v.y);
}

template <bool H>
__device__ __forceinline__ void tr_store(void* p, int64_t i, cf v) {
  if (H) static_cast<uint32_t*>(p)[i] = pack_rn<TC_FP16>(v.x, v.y);
  else static_cast<float2*>(p)[i] = make_float2(v.x, v.y);
}

// THREADS = 32 x WY: each thread moves 32 / WY elements of a tile, rows
// r0 + WY i of one column.  Plain complex64: WY = 8, four elements.
// complex32: WY = 4, eight elements, so that a warp keeps as many bytes in
// flight as with complex64 (four 4-byte loads per thread held the complex32
// transpose to about 60% of the HBM bandwidth).  With the twiddle: WY = 4
// as well, which spreads each thread's two sincospi over eight elements.
template <bool H, bool TW>
__global__ void __launch_bounds__(H || TW ? 128 : 256)
transpose_kernel(const void* __restrict__ in, void* __restrict__ out, int64_t batch, int64_t rows,
                 int64_t cols, int logN, int sign) {
  constexpr int WY = H || TW ? 4 : 8, PER = 32 / WY;
  __shared__ cf tile[32][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x WY
  const int64_t trow = rows / 32, tcol = cols / 32, per = trow * tcol;
  for (int64_t t = blockIdx.x; t < batch * per; t += gridDim.x) {
    const int64_t b = t / per, rt = (t - b * per) / tcol, ct = t - b * per - rt * tcol;
    const int64_t base = b * rows * cols;
    // the thread's elements share column c and step WY rows: their
    // twiddles are w^{r c} (w^{WY c})^i, two sincospi and a running product
    const int64_t c = ct * 32 + tx, r0 = rt * 32 + ty;
    cf w = mk(1.f, 0.f), step = mk(1.f, 0.f);
    if (TW) {
      w = DevMem::rotor(r0 * c, logN);  // exp(-2 pi i r c / N), r c < N
      step = DevMem::rotor(WY * c, logN);
      if (sign > 0) {
        w = cconj(w);
        step = cconj(step);
      }
    }
    cf v[PER];
#pragma unroll
    for (int i = 0; i < PER; ++i) v[i] = tr_load<H>(in, base + (r0 + WY * i) * cols + c);
#pragma unroll
    for (int i = 0; i < PER; ++i) {
      if (TW) {
        v[i] = cmul(v[i], w);
        w = cmul(w, step);
      }
      tile[ty + WY * i][tx] = v[i];
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < PER; ++i) {
      const int64_t c = ct * 32 + ty + WY * i, r = rt * 32 + tx;
      tr_store<H>(out, base + c * rows + r, tile[tx][ty + WY * i]);
    }
    __syncthreads();  // the tile is reused
  }
}

}  // namespace

cudaError_t launch_transpose(const void* in, void* out, int64_t batch, int64_t rows, int64_t cols,
                             int logN, int sign, int h16, int sm_count, cudaStream_t st) {
  if (batch <= 0) return cudaSuccess;
  if (rows % 32 || cols % 32 || rows < 32 || cols < 32) return cudaErrorInvalidValue;
  const int64_t tiles = batch * (rows / 32) * (cols / 32);
  // eight 256-thread blocks (plain complex64) or sixteen 128-thread blocks
  // per SM
  const int per_sm = h16 || logN > 0 ? 16 : 8;
  const int grid =
      (int)std::min<int64_t>(tiles, (int64_t)(sm_count > 0 ? sm_count : 152) * per_sm);
#define GB_TR(HH, TT) \
  transpose_kernel<HH, TT><<<grid, HH || TT ? 128 : 256, 0, st>>>(in, out, batch, rows, cols, logN, sign)
  if (h16) {
    if (logN > 0) GB_TR(true, true);
    else GB_TR(true, false);
  } else {
    if (logN > 0) GB_TR(false, true);
    else GB_TR(false, false);
  }
#undef GB_TR
  return cudaGetLastError();
}

}  // namespace gbfft
