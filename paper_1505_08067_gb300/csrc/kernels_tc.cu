// Tensor-core class kernels (see tc_stage.h): batched contiguous transforms of
// length L = 16, 256 or 4096 whose radix-16 stages run as DFT matmuls on the
// tensor cores.  One tile = 4096 complex elements (4096 / L transforms) per
// 256-thread block; two shared buffers of 4096 complex (64 KB, dynamic) hold
// the tile between stages.
#include <cuda_runtime.h>

#include "kernels_impl.cuh"
#include "tc_stage.h"

namespace gbfft {

template <int PREC>
__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1) {
  if (PREC == TC_FP16)
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
  else
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// One MMA group: y = DFT16 of each of the group's 16 butterflies (real block
// form, 8 MMAs; 24 for the split-BF16x3 variant).
template <int PREC>
__device__ __forceinline__ void tc_group(const cf (&x)[8], const uint32_t (&bh)[2][4][2],
                                         const uint32_t (&bl)[2][4][2], cf (&y)[8]) {
  constexpr int P = PREC == TC_BF16X3 ? TC_BF16 : PREC;
  constexpr bool SPLIT = PREC == TC_BF16X3;
  float acc[4][4] = {};
#pragma unroll
  for (int kb = 0; kb < 2; ++kb) {
    uint32_t a[4], alo[4];
    tc_a_frag<P, SPLIT>(x, kb, a, alo);
#pragma unroll
    for (int nb = 0; nb < 4; ++nb) {
      mma16816<P>(acc[nb], a, bh[kb][nb][0], bh[kb][nb][1]);
      if (SPLIT) {
        mma16816<P>(acc[nb], a, bl[kb][nb][0], bl[kb][nb][1]);
        mma16816<P>(acc[nb], alo, bh[kb][nb][0], bh[kb][nb][1]);
      }
    }
  }
  tc_outputs(acc, y);
}

// Stage S reads buffer S & 1's predecessor and writes the other one (ping-pong),
// so a group's outputs go out right after its MMAs; one barrier per stage.
// The backward transform's swaps are run-time selects at the first load and
// the last store (one copy of the tile code).
template <int LOGL, int PREC, int S>
__device__ __forceinline__ void tc_stage(const PassDesc& d, const cf* gin, cf* gout, cf* sm,
                                         const cf* stg, const uint32_t (&bh)[2][4][2],
                                         const uint32_t (&bl)[2][4][2], int w, int lane,
                                         int valid) {
  constexpr int P = PREC == TC_BF16X3 ? TC_BF16 : PREC;
  using B = TcBody<LOGL, P, DevMem>;
  const cf* src = S == 0 ? stg : sm + ((S + 1) & 1) * 4096;  // staging, or stage S-1's output
  cf* dst = sm + (S & 1) * 4096;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    cf x[8], y[8];
    B::template gather<S>(x, d, gin, src, w, h, lane, valid, d.conj_in != 0);
    tc_group<PREC>(x, bh, bl, y);
    B::template scatter<S>(y, gout, dst, w, h, lane, valid, d.conj_out != 0);
  }
  __syncthreads();
}

// Copy the valid transforms of tile `tile` into the staging buffer (one
// thread): bulk copies of kChunk elements, each to its padded place.
template <class B>
__device__ __forceinline__ void tc_stage_in(const cf* in, const PassDesc& d, int64_t tile,
                                            cf* stg, uint64_t* bar) {
  constexpr int TPC = 4096 / B::L;
  const int64_t first = tile * TPC;
  const int64_t rem = d.count_inner - first;
  const int nv = rem < TPC ? (int)rem : TPC;
  const int chunks = nv * B::L / B::kChunk;
  const uint32_t bytes = (uint32_t)(nv * B::L * 8);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
  const cf* src = in + first * B::L;
  for (int c = 0; c < chunks; ++c)
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_u32(stg + c * (B::kChunk + 2))),
        "l"(src + c * B::kChunk), "r"((uint32_t)(B::kChunk * 8)), "r"(smem_u32(bar))
        : "memory");
}

// Two blocks per SM (at most 128 registers a thread).  Persistent: each block
// builds the DFT-matrix fragments once and copies its next tile into a padded
// staging buffer (bulk copies, mbarrier with a bounded wait) while the
// current one is computed; a source that is not 16-byte aligned is read from
// global memory instead.
template <int LOGL, int PREC>
__global__ void __launch_bounds__(256, 2)
stockham_tc(const cf* __restrict__ in, cf* out, const __grid_constant__ PassDesc d) {
  constexpr int P = PREC == TC_BF16X3 ? TC_BF16 : PREC;
  using B = TcBody<LOGL, P, DevMem>;
  extern __shared__ __align__(16) unsigned char smem_tc[];
  cf* sm = reinterpret_cast<cf*>(smem_tc);  // two buffers of 4096 complex
  cf* stg = sm + 8192;                      // staging, B::kStageSlots complex
  uint64_t* bar = reinterpret_cast<uint64_t*>(stg + B::kStageSlots);
  constexpr int TPC = 4096 >> LOGL;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const bool staged = (reinterpret_cast<uintptr_t>(in) & 15) == 0;
  uint32_t bh[2][4][2], bl[2][4][2];
#pragma unroll
  for (int kb = 0; kb < 2; ++kb)
#pragma unroll
    for (int nb = 0; nb < 4; ++nb) {
      tc_b_frag<P>(lane, kb, nb, 0, bh[kb][nb][0], bh[kb][nb][1]);
      if (PREC == TC_BF16X3) tc_b_frag<P>(lane, kb, nb, 1, bl[kb][nb][0], bl[kb][nb][1]);
      else bl[kb][nb][0] = bl[kb][nb][1] = 0;
    }
  if (tid == 0) mbar_init(bar, 1);
  __syncthreads();
  if (staged && tid == 0 && blockIdx.x < d.tiles) tc_stage_in<B>(in, d, blockIdx.x, stg, bar);
  uint32_t parity = 0;
  for (int64_t tile = blockIdx.x; tile < d.tiles; tile += gridDim.x) {
    const int64_t first = tile * TPC;
    const int64_t rem = d.count_inner - first;
    const int valid = rem < TPC ? (int)rem : TPC;
    const cf* gin = in + first * (1 << LOGL);
    cf* gout = out + first * (1 << LOGL);
    if (staged) {
      const bool ok = mbar_wait(bar, parity, kWaitPolls);
      if (__syncthreads_or(!ok)) {
        if (tid == 0) {
          atomicExch(d.status, 1);
          mbar_wait(bar, parity, kWaitPolls);  // let the copy in flight land before leaving
        }
        return;
      }
      parity ^= 1u;
    }
    tc_stage<LOGL, PREC, 0>(d, gin, gout, sm, staged ? stg : nullptr, bh, bl, w, lane, valid);
    // every thread has read the staging buffer: start the next tile's copy
    if (staged && tid == 0 && tile + gridDim.x < d.tiles)
      tc_stage_in<B>(in, d, tile + gridDim.x, stg, bar);
    constexpr int NST = LOGL / 4;
    if constexpr (NST > 1) tc_stage<LOGL, PREC, 1>(d, gin, gout, sm, stg, bh, bl, w, lane, valid);
    if constexpr (NST > 2) tc_stage<LOGL, PREC, 2>(d, gin, gout, sm, stg, bh, bl, w, lane, valid);
  }
}

const void* resolve_tc(int logL, int prec) {
#define GB_TC(LG, P) \
  if (logL == LG && prec == P) return (const void*)stockham_tc<LG, P>;
  GB_TC(4, 1) GB_TC(4, 2) GB_TC(4, 3)
  GB_TC(8, 1) GB_TC(8, 2) GB_TC(8, 3)
  GB_TC(12, 1) GB_TC(12, 2) GB_TC(12, 3)
#undef GB_TC
  return nullptr;
}

}  // namespace gbfft
