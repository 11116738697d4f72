// Kernel templates shared by the translation units that instantiate them
// (kernels.cu: generic kernels and launch glue; shapes_contig.cu and
// shapes_fourstep.cu: compile-time shapes).  See kernels.cu for an overview.
#pragma once
#include <cuda_runtime.h>

#include "fft_split.h"
#include "fft_stage.h"
#include "kernel_shapes.h"
#include "kernels.h"

namespace gbfft {

using KernelFn = void (*)(const cf*, cf*, PassDesc);

struct DevMem {
  // Input is read exactly once: stream it with an evict-first hint.
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
  // w_N^m for 0 <= m < N = 2^logN <= 2^24: the angle 2m/N is exact in FP32.
  GB_HD static cf rotor(int64_t m, int logN) {
#ifdef __CUDA_ARCH__
    float s, c;
    sincospif(__int2float_rn((int)m) * __int_as_float((127 + 1 - logN) << 23), &s, &c);
    return mk(c, -s);
#else
    (void)m;
    (void)logN;
    return mk(1.f, 0.f);
#endif
  }
};

// One tile of a pass: load, every stage, store.
template <int R, int LMAP, int SMAP, class TR>
__device__ __forceinline__ void pass_tile(const cf* __restrict__ in, cf* out, const PassDesc& d,
                                          int64_t tile, cf* sm, int tid) {
  using B = PassBody<R, LMAP, SMAP, DevMem, TR>;
  const typename B::Tile tl = B::tile_of(d, tile);
  cf v[R];
  B::first(v, d, in, out, sm, tl, tid);
  int Ns = 1 << TR::rlog(d, 0);
  if constexpr (TR::kMaxStages < 15) {
#pragma unroll
    for (int s = 1; s < TR::kMaxStages; ++s) {
      __syncthreads();
      B::read(v, d, s, Ns, out, sm, tl, tid);
      if (s < TR::kMaxStages - 1) {
        __syncthreads();
        B::write(v, d, s, Ns, sm, tid);
      }
      Ns <<= TR::rlog(d, s);
    }
  } else {
#pragma unroll 1
    for (int s = 1; s < d.nst; ++s) {
      __syncthreads();
      B::read(v, d, s, Ns, out, sm, tl, tid);
      if (s < d.nst - 1) {
        __syncthreads();
        B::write(v, d, s, Ns, sm, tid);
      }
      Ns <<= d.rlog[s];
    }
  }
  __syncthreads();  // shared memory is reused by the next tile
}

__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2::evict_last [%0];" ::"l"(p));
}

// Pull the input of tile `tile` into L2 (persistent grids: a block's next
// tile streams in while the current one is computed, so its stage-0 loads hit
// L2 instead of DRAM).  Two tile layouts: G whole contiguous transforms (one
// 128-byte line per thread and pass of the loop), or G adjacent columns of a
// strided pass (the first and last line of each row's G elements).
template <class TR>
__device__ __forceinline__ void prefetch_tile(const cf* in, const PassDesc& d, int64_t tile,
                                              int tid) {
  const int64_t L = int64_t(1) << TR::logL(d);
  const int64_t outer = tile / d.tiles_inner, inner = tile - outer * d.tiles_inner;
  const cf* base = in + outer * d.in.o + inner * d.in.t;
  if (TR::in_e(d) == 1 && TR::in_g(d) == L) {
    const int64_t left = (d.count_inner - inner * TR::G(d)) * L;  // ragged last tile
    const int64_t valid = min((int64_t)TR::G(d) * L, left);
    const char* b = reinterpret_cast<const char*>(base);
    for (int64_t line = tid; line * 16 < valid; line += blockDim.x) prefetch_l2(b + line * 128);
  } else if (TR::in_g(d) == 1) {
    const int64_t gl = min((int64_t)TR::G(d), d.count_inner - inner * TR::G(d)) - 1;
    for (int64_t a = tid; a < L; a += blockDim.x) {
      const cf* row = base + a * TR::in_e(d);
      prefetch_l2(row);
      prefetch_l2(row + gl);
    }
  }
}

// Stages s = 1 .. nst-1 of one round of a convolution tile.  Round 1 keeps
// the last stage's results in registers; round 2 stores them (swap undone).
template <int R, int MAP, class TR, bool ROUND1>
__device__ __forceinline__ void conv_stages(cf (&v)[R], const PassDesc& d, cf* out, cf* sm,
                                            const typename PassBody<R, MAP, MAP, DevMem, TR>::Tile& tl,
                                            int tid) {
  using B = PassBody<R, MAP, MAP, DevMem, TR>;
  int Ns = 1 << TR::rlog(d, 0);
  if constexpr (TR::kMaxStages < 15) {
#pragma unroll
    for (int s = 1; s < TR::kMaxStages; ++s) {
      __syncthreads();
      if (ROUND1) B::read_nostore(v, d, s, Ns, sm, tl, tid);
      else B::template read_s<true>(v, d, s, Ns, out, sm, tl, tid);
      if (s < TR::kMaxStages - 1) {
        __syncthreads();
        B::write(v, d, s, Ns, sm, tid);
      }
      Ns <<= TR::rlog(d, s);
    }
  } else {
#pragma unroll 1
    for (int s = 1; s < d.nst; ++s) {
      __syncthreads();
      if (ROUND1) B::read_nostore(v, d, s, Ns, sm, tl, tid);
      else B::template read_s<true>(v, d, s, Ns, out, sm, tl, tid);
      if (s < d.nst - 1) {
        __syncthreads();
        B::write(v, d, s, Ns, sm, tid);
      }
      Ns <<= d.rlog[s];
    }
  }
}

// One tile of a fast-convolution pass: out = h_scale * IDFT(H . DFT(in)) per
// line, the tile read once and written once (see PassBody's conv phases).
template <int R, int MAP, class TR>
__device__ __forceinline__ void conv_tile(const cf* __restrict__ in, cf* out, const PassDesc& d,
                                          int64_t tile, cf* sm, int tid) {
  using B = PassBody<R, MAP, MAP, DevMem, TR>;
  const typename B::Tile tl = B::tile_of(d, tile);
  cf v[R];
  B::first_nostore(v, d, in, sm, tl, tid);
  conv_stages<R, MAP, TR, true>(v, d, out, sm, tl, tid);
  if (B::conv_in_regs(d)) {
    B::conv_regs(v, d, tl, tid);
  } else {
    __syncthreads();  // every round-1 read of shared memory is done
    B::conv_mid(v, d, sm, tl, tid);
    __syncthreads();
    B::first_smem(v, d, sm, tid);
  }
  if (TR::nst(d) == 1) {
    B::store_first(v, d, out, tl, tid);
  } else {
    __syncthreads();  // stage 0 of round 2 rewrites the slots it read
    B::write(v, d, 0, 1, sm, tid);
    conv_stages<R, MAP, TR, false>(v, d, out, sm, tl, tid);
  }
  __syncthreads();  // shared memory is reused by the next tile
}

template <int R, int MAP, class TR>
__global__ void __launch_bounds__(1024)
stockham_conv(const cf* __restrict__ in, cf* out, const __grid_constant__ PassDesc d) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cf* sm = reinterpret_cast<cf*>(smem_raw);
  for (int64_t tile = blockIdx.x; tile < d.tiles; tile += gridDim.x) {
    if (d.l2_prefetch && tile + gridDim.x < d.tiles)
      prefetch_tile<TR>(in, d, tile + gridDim.x, threadIdx.x);
    conv_tile<R, MAP, TR>(in, out, d, tile, sm, threadIdx.x);
  }
}

// Coalesced launch of several same-shape jobs (separate buffers): the job
// table rides in the kernel parameters; tile t belongs to the job whose range
// [tile_begin, next tile_begin) contains it.
template <int R>
__global__ void __launch_bounds__(1024)
stockham_grouped(const __grid_constant__ PassDesc d0, const __grid_constant__ GroupTable gt) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cf* sm = reinterpret_cast<cf*>(smem_raw);
  const int tid = threadIdx.x;
  const int64_t total = gt.e[gt.n - 1].tile_begin + gt.e[gt.n - 1].tiles;
  int j = 0;
  for (int64_t tile = blockIdx.x; tile < total; tile += gridDim.x) {
    while (j + 1 < gt.n && gt.e[j + 1].tile_begin <= tile) ++j;  // tiles only grow
    PassDesc d = d0;
    d.count_inner = gt.e[j].count;
    d.tiles_inner = d.tiles = gt.e[j].tiles;
    pass_tile<R, MAP_ROWS, MAP_ROWS, RtTraits>(gt.e[j].in, gt.e[j].out, d,
                                               tile - gt.e[j].tile_begin, sm, tid);
  }
}

template <int R, int LMAP, int SMAP, class TR>
__global__ void __launch_bounds__(1024)
stockham_pass(const cf* __restrict__ in, cf* out, const __grid_constant__ PassDesc d) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cf* sm = reinterpret_cast<cf*>(smem_raw);
  using B = PassBody<R, LMAP, SMAP, DevMem, TR>;
  const int tid = threadIdx.x;
  for (int64_t tile = blockIdx.x; tile < d.tiles; tile += gridDim.x) {
    const typename B::Tile tl = B::tile_of(d, tile);
    if (d.l2_prefetch && tile + gridDim.x < d.tiles) prefetch_tile<TR>(in, d, tile + gridDim.x, tid);
    cf v[R];
    B::first(v, d, in, out, sm, tl, tid);
    int Ns = 1 << TR::rlog(d, 0);
    if constexpr (TR::kMaxStages < 15) {
      // compile-time schedule: unrolled, every radix and offset a constant
#pragma unroll
      for (int s = 1; s < TR::kMaxStages; ++s) {
        __syncthreads();
        B::read(v, d, s, Ns, out, sm, tl, tid);
        if (s < TR::kMaxStages - 1) {
          __syncthreads();
          B::write(v, d, s, Ns, sm, tid);
        }
        Ns <<= TR::rlog(d, s);
      }
    } else {
#pragma unroll 1
      for (int s = 1; s < d.nst; ++s) {
        __syncthreads();
        B::read(v, d, s, Ns, out, sm, tl, tid);
        if (s < d.nst - 1) {
          __syncthreads();
          B::write(v, d, s, Ns, sm, tid);
        }
        Ns <<= d.rlog[s];
      }
    }
    __syncthreads();  // shared memory is reused by the next tile
  }
}

// ------------------------------------------------------- staged pass --
// TMA bulk copy global -> shared, mbarrier completion (sm_90+ PTX).

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Expect `bytes` on the barrier and start the copies (one thread).  src and
// dst are 16-byte aligned and bytes is a multiple of 16.
__device__ __forceinline__ void tma_load(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
  const uint32_t b = smem_u32(bar);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(bytes)
               : "memory");
  constexpr uint32_t kChunk = 32768;
  for (uint32_t off = 0; off < bytes; off += kChunk) {
    const uint32_t n = bytes - off < kChunk ? bytes - off : kChunk;
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_u32(static_cast<char*>(dst) + off)),
        "l"(static_cast<const char*>(src) + off), "r"(n), "r"(b)
        : "memory");
  }
}

// Wait for phase `parity` of the barrier; gives up after `limit` polls.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint32_t limit) {
  const uint32_t b = smem_u32(bar);
  for (uint32_t it = 0; it < limit; ++it) {
    uint32_t done;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; "
        "selp.u32 %0, 1, 0, p; }"
        : "=r"(done)
        : "r"(b), "r"(parity)
        : "memory");
    if (done) return true;
    if (it > 64) __nanosleep(128);
  }
  return false;
}

constexpr uint32_t kWaitPolls = 1u << 22;  // ~0.5 s of polling before giving up

// Input base of a staged tile: one contiguous transform, or G adjacent
// columns (tile = (outer, inner) as in PassDesc).
template <class SH>
__device__ __forceinline__ const cf* staged_src(const cf* in, const PassDesc& d, int64_t tile) {
  if constexpr (SH::kG == 1) {
    return in + tile * SH::kL;
  } else {
    const int64_t outer = tile / d.tiles_inner, inner = tile - outer * d.tiles_inner;
    return in + outer * d.in.o + inner * d.in.t;
  }
}

// Column tiles: every thread copies its share of the tile's L rows (G*8
// bytes each, row a from src + a*e to st + a*G) in 16-byte asynchronous
// copies, then has the barrier count its arrival once they have landed (the
// barrier of a column kernel expects one arrival per thread).  Plain per-thread
// copies: a bulk copy with different addresses in each lane would be issued
// one lane at a time.
template <class SH>
__device__ __forceinline__ void copy_rows(cf* st, const cf* src, int64_t e, uint64_t* bar,
                                          int tid) {
  constexpr int CH = SH::kG * 8 / 16;  // 16-byte chunks per row
  static_assert(CH >= 1 && SH::kG * 8 % 16 == 0, "rows must be whole 16-byte chunks");
  for (int c = tid; c < SH::kL * CH; c += SH::kT) {
    const int a = c / CH, j = c - a * CH;
    const char* g = reinterpret_cast<const char*>(src + a * e) + 16 * j;
    char* sdst = reinterpret_cast<char*>(st + a * SH::kG) + 16 * j;
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(sdst)), "l"(g)
                 : "memory");
  }
  asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// Row tiles of a transposing pass: G contiguous rows of L elements, one bulk
// copy each (one thread), to pitched rows st + g*(L + kRowPad).
template <class SH>
__device__ __forceinline__ void stage_rows(cf* st, const cf* src, uint64_t* bar) {
  const uint32_t b = smem_u32(bar);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b),
               "r"((uint32_t)(SH::kG * SH::kL * 8))
               : "memory");
  for (int g = 0; g < SH::kG; ++g)
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_u32(st + g * (SH::kL + SH::kRowPad))),
        "l"(src + g * SH::kL), "r"((uint32_t)(SH::kL * 8)), "r"(b)
        : "memory");
}

// Column tiles, tensor-map form: one thread copies the tile's L rows of G
// elements as boxes of min(L, 256) rows (d.tmap_in), landing in the same
// interleaved layout as copy_rows (element a of column g at a*G + g); the
// barrier expects this thread's one arrival with the tile's bytes.
template <class SH>
__device__ __forceinline__ void tma_cols(cf* st, const PassDesc& d, int64_t tile, uint64_t* bar) {
  constexpr int BR = SH::kL < 256 ? SH::kL : 256;
  static_assert(SH::kL % BR == 0 && SH::kG * 8 % 16 == 0, "whole boxes of 16-byte rows");
  int32_t x, y;
  tma_tile_coords(d, d.in, tile, x, y);
  const uint32_t b = smem_u32(bar);
  const uint64_t map = reinterpret_cast<uint64_t>(&d.tmap_in[0]);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b),
               "r"((uint32_t)(SH::kL * SH::kG * 8))
               : "memory");
  for (int j = 0; j < SH::kL / BR; ++j)
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(st + j * BR * SH::kG)),
        "l"(map), "r"(x), "r"(y + j * BR), "r"(b)
        : "memory");
}

// Fast convolution over column tiles (cols_filter_staged, d.tmap_h_ok): the
// filters of the tile's G columns (all L rows) copied by tensor-map boxes over
// h into `st`, in the data's interleaved layout; one arrival with the bytes.
template <class SH>
__device__ __forceinline__ void tma_filter(cf* st, const PassDesc& d, int64_t col0,
                                           uint64_t* bar) {
  constexpr int BR = SH::kL < 256 ? SH::kL : 256;
  const uint32_t b = smem_u32(bar);
  const uint64_t map = reinterpret_cast<uint64_t>(&d.tmap_h[0]);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b),
               "r"((uint32_t)(SH::kL * SH::kG * 8))
               : "memory");
  for (int j = 0; j < SH::kL / BR; ++j)
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(st + j * BR * SH::kG)),
        "l"(map), "r"((int32_t)col0), "r"(j * BR), "r"(b)
        : "memory");
}

// Column tiles, tensor-map store of rows [0, L/2) of tile `tile` from xs (box
// layout, SplitBody::store_half_smem) as boxes of min(L/2, 256) rows
// (d.tmap_out).  Called by one thread after a barrier that follows every
// thread's writes and proxy fence.  Does not wait: the caller's thread 0
// waits for the copies to have read xs (cp.async.bulk.wait_group.read)
// before the barrier that precedes the next write to xs.
template <class SH>
__device__ __forceinline__ void tma_store_half0(const cf* xs, const PassDesc& d, int64_t tile) {
  constexpr int HL = SH::kL / 2, BR = HL < 256 ? HL : 256;
  static_assert(HL % BR == 0 && SH::kG * 8 % 16 == 0, "whole boxes of 16-byte rows");
  int32_t x, y;
  tma_tile_coords(d, d.out, tile, x, y);
  const uint64_t map = reinterpret_cast<uint64_t>(&d.tmap_out[0]);
  for (int j = 0; j < HL / BR; ++j)
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::
                     "l"(map), "r"(x), "r"(y + j * BR), "r"(smem_u32(xs + j * BR * SH::kG))
                 : "memory");
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}

// Column-tile output: the first half of the rows through the exchange buffer
// x and tensor-map box stores (asynchronous), the second half by register
// stores while those copies run -- half the strided store instructions, and
// no wait for the copies (x is next written one tile later).
template <class SH, bool SWAP>
__device__ __forceinline__ void store_cols_tma(const cf (&v)[SH::kR], const PassDesc& d, cf* x,
                                               cf* o, int64_t tile, int64_t col0, int tid) {
  using B = SplitBody<SH, DevMem>;
  B::template store_half_smem<SWAP, 0>(v, d, x, col0, tid);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncthreads();
  if (tid == 0) tma_store_half0<SH>(x, d, tile);
  B::template store_half<SWAP, 1>(v, d, o, col0, tid);
}

// HOLD: the exchanged stages' roots in `rt` were loaded before the first tile.
// `on_free` runs on every thread once every thread of the block has passed
// the first barrier (so has read its stage-0 inputs from staging).
template <class SH, int S, bool HOLD, class OnFree>
__device__ __forceinline__ void split_exchange(cf (&v)[SH::kR], const PassDesc& d, cf* x, int tid,
                                               typename SplitBody<SH, DevMem>::Roots& rt,
                                               OnFree on_free) {
  using B = SplitBody<SH, DevMem>;
  auto& r = B::template roots_of<S>(rt);
  if constexpr (SH::kPowTw && !HOLD) B::template roots<S>(r, d, tid);
  if constexpr (SH::kPrefetchFused && S == SH::kExchanges - 1) B::fused_roots(rt.fr, d, tid);
  B::template write_half<S, 0>(v, x, tid);
  __syncthreads();
  on_free();
  B::template read_half<S, 0>(v, x, tid);
  __syncthreads();
  B::template write_half<S, 1>(v, x, tid);
  __syncthreads();
  B::template read_half<S, 1>(v, x, tid);
  B::template compute<S>(v, d, tid, r);
  __syncthreads();
}

struct NoOp {
  __device__ void operator()() const {}
};

// The exchanges after stages 0 .. kExchanges-1; the first one runs
// `on_free` (the copy of the next tile, or of the filters, into the staging
// buffer) once staging has been read; unless HOLD, each loads the twiddle
// roots of the stage after it into `rt`; the last one loads those of a fused
// radix-2 last stage (SplitShape::kPrefetchFused).
template <class SH, bool HOLD, class OnFree>
__device__ __forceinline__ void split_round(cf (&v)[SH::kR], const PassDesc& d, cf* x, int tid,
                                            typename SplitBody<SH, DevMem>::Roots& rt,
                                            OnFree on_free) {
  static_assert(SH::kExchanges >= 1, "at least one exchange");
  split_exchange<SH, 0, HOLD>(v, d, x, tid, rt, on_free);
  if constexpr (SH::kExchanges > 1) split_exchange<SH, 1, HOLD>(v, d, x, tid, rt, NoOp{});
  if constexpr (SH::kExchanges > 2) split_exchange<SH, 2, HOLD>(v, d, x, tid, rt, NoOp{});
}

// Start the copy of tile `t` into the staging buffer (one contiguous
// transform, G rows, or G columns by tensor-map boxes or row copies).
template <class SH>
__device__ __forceinline__ void stage_tile(cf* st, const cf* in, const PassDesc& d, int64_t t,
                                           uint64_t* bar, int tid) {
  if constexpr (SH::kG == 1) {
    if (tid == 0) tma_load(st, staged_src<SH>(in, d, t), SH::kL * 8, bar);
  } else if constexpr (SH::kRowsIn) {
    if (tid == 0) stage_rows<SH>(st, staged_src<SH>(in, d, t), bar);
  } else if (d.tmap_in_ok) {
    if (tid == 0) tma_cols<SH>(st, d, t, bar);
  } else {
    copy_rows<SH>(st, staged_src<SH>(in, d, t), d.in.e, bar, tid);
  }
}

// One tile per block (a contiguous transform, or G adjacent columns of a
// strided pass), persistent over tiles; the next tile streams into shared
// memory by bulk copies while this one is computed.  CONV: fast convolution
// of each line (forward stages, filter, forward stages on swapped data; see
// SplitBody::conv_middle).
template <class SH, int MINB, bool CONV = false>
__global__ void __launch_bounds__(SH::kT, MINB)
stockham_staged(const cf* __restrict__ in, cf* out, const __grid_constant__ PassDesc d) {
  extern __shared__ __align__(128) unsigned char smem_staged[];
  cf* st = reinterpret_cast<cf*>(smem_staged);
  cf* x = st + SH::kStageElems;
  uint64_t* bar = reinterpret_cast<uint64_t*>(x + SH::kHalfSlots);
  using B = SplitBody<SH, DevMem>;
  const int tid = threadIdx.x;
  const int64_t step = gridDim.x;
  int64_t tile = blockIdx.x;
  // one arrival (thread 0's expect_tx for bulk or tensor-map copies) for
  // contiguous transforms, row tiles and column tiles with a tensor map; one
  // per thread (its row copies) for other column tiles
  const bool one_arrival = SH::kG == 1 || SH::kRowsIn || d.tmap_in_ok;
  if (tid == 0) mbar_init(bar, one_arrival ? 1 : SH::kT);
  __syncthreads();
  if (tile < d.tiles) stage_tile<SH>(st, in, d, tile, bar, tid);  // uniform over the block
  // twiddle roots: loaded once here (kHold, kHoldFused) or per tile
  constexpr bool kHold = SH::kHoldRoots && !CONV;
  constexpr bool kHoldFused = SH::kHoldFused && !CONV;
  typename B::Roots rt;
  if constexpr (kHold) {
    B::template roots<0>(rt.r0, d, tid);
    if constexpr (SH::kExchanges > 1) B::template roots<1>(rt.r1, d, tid);
    if constexpr (SH::kExchanges > 2) B::template roots<2>(rt.r2, d, tid);
  }
  if constexpr (kHoldFused) B::fused_roots(rt.fr, d, tid);
  constexpr bool kFrReady = SH::kPrefetchFused || kHoldFused;
  uint32_t parity = 0;
  for (; tile < d.tiles; tile += step) {
    // the previous tile's tensor-map stores must have read x before this
    // tile's exchanges write it (the barrier below orders the rest)
    if (SH::kG > 1 && tid == 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
    const bool ok = mbar_wait(bar, parity, kWaitPolls);
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        atomicExch(d.status, 1);
        mbar_wait(bar, parity, kWaitPolls);  // let the copy in flight land before leaving
        if constexpr (SH::kG > 1) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
      }
      return;
    }
    parity ^= 1u;
    const int64_t next = tile + step < d.tiles ? tile + step : -1;
    cf* o;
    int64_t col0;  // G == 1: the line (tile); else the first column of the tile
    if constexpr (SH::kG == 1) {
      o = out + tile * SH::kL;
      col0 = tile;
    } else {
      const int64_t outer = tile / d.tiles_inner, inner = tile - outer * d.tiles_inner;
      o = out + outer * d.out.o + inner * d.out.t;
      col0 = inner * SH::kG;
    }
    // a convolution over column tiles with per-line filters stages the tile's
    // filters once the data has been read, and the next tile once the
    // filters have (its copy then overlaps the second round only).  Lines
    // of a range convolution keep reading their filter from global memory
    // (staging it as well measured 0.166 against 0.162 ms per frame).
    const bool fstage = CONV && SH::kG > 1 && d.tmap_h_ok && d.tmap_in_ok;
    cf v[SH::kR];
    if (d.conj_in) B::template first<true>(v, st, tid);
    else B::template first<false>(v, st, tid);
    split_round<SH, kHold>(v, d, x, tid, rt, [&] {
      if (fstage) {
        if constexpr (SH::kG > 1) {
          if (tid == 0) tma_filter<SH>(st, d, col0, bar);
        }
      } else if (next >= 0) {
        stage_tile<SH>(st, in, d, next, bar, tid);  // staging has been read
      }
    });
    if constexpr (CONV) {
      if (fstage) {
        const bool fok = mbar_wait(bar, parity, kWaitPolls);
        if (__syncthreads_or(!fok)) {
          if (tid == 0) {
            atomicExch(d.status, 1);
            mbar_wait(bar, parity, kWaitPolls);  // let the copy in flight land before leaving
            asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
          }
          return;
        }
        parity ^= 1u;
        B::conv_middle(v, d, col0, tid, st);
        split_round<SH, kHold>(v, d, x, tid, rt, [&] {
          if (next >= 0) stage_tile<SH>(st, in, d, next, bar, tid);  // the filters have been read
        });
      } else {
        B::conv_middle(v, d, col0, tid);
        split_round<SH, kHold>(v, d, x, tid, rt, NoOp{});
      }
      if constexpr (SH::kFuseLast) {
        B::template store_fused<true, kFrReady>(v, d, o, col0, tid, rt.fr);
      } else if (SH::kG > 1 && d.tmap_out_ok) {
        if constexpr (SH::kG > 1) store_cols_tma<SH, true>(v, d, x, o, tile, col0, tid);
      } else {
        B::template store<true>(v, d, o, col0, tid);
      }
    } else if constexpr (SH::kFuseLast) {
      if (d.conj_out) B::template store_fused<true, kFrReady>(v, d, o, col0, tid, rt.fr);
      else B::template store_fused<false, kFrReady>(v, d, o, col0, tid, rt.fr);
    } else if (SH::kG > 1 && d.tmap_out_ok) {
      if constexpr (SH::kG > 1) {
        if (d.conj_out) store_cols_tma<SH, true>(v, d, x, o, tile, col0, tid);
        else store_cols_tma<SH, false>(v, d, x, o, tile, col0, tid);
      }
    } else {
      if (d.conj_out) B::template store<true>(v, d, o, col0, tid);
      else B::template store<false>(v, d, o, col0, tid);
    }
  }
  // tensor-map stores: the last ones have read shared memory; let them land
  if (SH::kG > 1 && tid == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}


// Stage micro-benchmark (Bergach et al. Sec. 3.2: every (radix, start stage)
// pair is timed on its own): repeats stage 1 of descriptor `d` -- radix
// 2^d.rlog[1] after stages whose radices multiply to Ns -- on shared memory,
// `reps` times: read + twiddle + DFT, barrier, write, barrier.  No global
// traffic except the twiddle loads the real stage makes.
template <int R>
__global__ void __launch_bounds__(1024)
stage_bench(const __grid_constant__ PassDesc d, int Ns, int reps, cf* sink) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cf* sm = reinterpret_cast<cf*>(smem_raw);
  using B = PassBody<R, MAP_ROWS, MAP_ROWS, DevMem, RtTraits>;
  const int tid = threadIdx.x;
  for (int i = tid; i < d.smem_elems; i += blockDim.x) sm[i] = mk(1e-3f * (float)(i & 1023), 1.f);
  __syncthreads();
  cf v[R];
  typename B::Tile tl;
  tl.outer = 0;
  tl.inner = 0;
  for (int rep = 0; rep < reps; ++rep) {
    B::read(v, d, 1, Ns, nullptr, sm, tl, tid);
    __syncthreads();
    B::write(v, d, 1, Ns, sm, tid);
    __syncthreads();
  }
  if (v[0].x == 12345.f && v[0].y == -12345.f) sink[blockIdx.x] = v[0];
}

template <int R, int LMAP, int SMAP, class TR>
KernelFn kfn() {
  return stockham_pass<R, LMAP, SMAP, TR>;
}

template <class SH, int MINB, bool CONV = false>
KernelFn staged_fn() {
  return stockham_staged<SH, MINB, CONV>;
}

// Fast-convolution kernels (conv.cu): a compile-time shape if one matches,
// else the generic kernel for (R, map).
const void* resolve_conv_kernel(int R, int map, const PassDesc& d, bool generic_only,
                                bool* specialised);

// Generic (run-time-parameter) kernels by thread maps, one translation unit each.
const void* generic_kernel_rows(int R);         // rows -> rows
const void* generic_kernel_cols(int R);         // columns -> columns
const void* generic_kernel_transposing(int R);  // rows -> columns

// Resolvers of the compile-time shapes, one per translation unit.
const void* resolve_contig_shape(int R, int lmap, int smap, const PassDesc& d);
const void* resolve_fourstep_shape(int R, int lmap, int smap, const PassDesc& d);
bool resolve_staged_shape(const PassDesc& d, StagedLaunch* s);
bool resolve_conv_staged_shape(const PassDesc& d, StagedLaunch* s);
bool resolve_staged_cols_shape(const PassDesc& d, int lmap, int smap, StagedLaunch* s);
bool resolve_staged_trans_shape(const PassDesc& d, int lmap, int smap, StagedLaunch* s);

}  // namespace gbfft
