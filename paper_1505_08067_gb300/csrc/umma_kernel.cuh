// Tensor-core class on tcgen05 (see umma_stage.h): batched contiguous
// transforms of length L = 2^4 .. 2^14 whose radix-16 stages are 16-point
// DFT matmuls issued as UMMA instructions (operands in shared memory through
// matrix descriptors, FP32 accumulators in tensor memory), with an optional
// radix-2/4/8 first stage in FP32 registers.
//
// One CTA of 256 threads (8 warps; 512 at 2^14) owns a tile of T = max(L, 4096) elements
// at a time, on a persistent grid.  Per tile:
//   load     every thread reads its share of the tile (radix-r0 first stage
//            in registers when L is not a power of 16), twiddles, rounds to
//            FP16/BF16 and stores the stage-0 A operand in shared memory.
//            Tiles of 4096 elements (L <= 2^12; not the split class) from a
//            16-byte-aligned input are read from a staging buffer in shared
//            memory, which a bulk copy (TMA) fills with the CTA's next tile
//            while this one goes through its stages; the others from global
//            memory (the next tile prefetched into L2 where that measured
//            faster);
//   stage t  thread 0 issues the UMMAs of the stage (T/2048 row blocks x 2
//            K halves; x3 for the split-BF16 class) and commits them to an
//            mbarrier; all threads wait (bounded), each warp reads its rows
//            of D from tensor memory (tcgen05.ld, one butterfly's 16 outputs
//            per thread), and either twiddles, rounds and stores them as the
//            next stage's A operand, or writes them to global memory.
// The shared-memory writes are made visible to the tensor cores with
// fence.proxy.async before the barrier that precedes each issue; tensor-memory
// reads finish (tcgen05.wait::ld) before the barrier after which the next
// stage overwrites the accumulators.
//
// Every wait is bounded: a give-up sets the pass's status word, waits (again
// bounded) for the UMMAs and the staging copy in flight, frees the tensor
// memory and returns.
//
// Input and output are complex64, or complex32 (FP16 re, im; 4 bytes per
// element) when the kernel's H parameter is set: the loader widens each FP16
// pair to FP32 and the last stage rounds its FP32 results to FP16 pairs.
// The kernels are instantiated in kernels_umma.cu (complex64) and
// kernels_umma_c32.cu (complex32).
#pragma once
#include <cuda_runtime.h>

#include <type_traits>

#include "kernels_impl.cuh"
#include "umma_stage.h"

namespace gbfft {

// ------------------------------------------------------------ PTX wrappers --

__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   smem_u32(slot)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}

__device__ __forceinline__ void tc05_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc05_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// generic-proxy shared-memory writes -> visible to the tensor cores
__device__ __forceinline__ void fence_smem_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// D[tmem] (+)= A[desc] . B[desc]; kind::f16, M = 128, N = 32, K = 16.
__device__ __forceinline__ void umma16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                       uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}

// Brings [p, p + bytes) into L2 ahead of its loads (a bulk prefetch: no
// shared memory, no completion to wait for).  Both 16-byte aligned.
__device__ __forceinline__ void prefetch_l2(const void* p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// The mbarrier completes one phase when every UMMA this thread issued is done.
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

// 16 consecutive FP32 columns of this thread's tensor-memory lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// 32 consecutive FP32 columns of this thread's tensor-memory lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// --------------------------------------------------------------- operands --

// Device memory policy of the per-thread body: the pass kernels' global
// accesses plus 32-bit shared stores at byte addresses.
// The stores carry no memory clobber, so the compiler may hoist the next
// global or twiddle loads above them (with the clobber every load waited for
// the store before it); the fence and barrier before each UMMA issue order
// them for the tensor cores.
struct UmmaDevMem : DevMem {
  static constexpr bool kHalfIO = false;
  __device__ __forceinline__ static void sts32(uint32_t saddr, uint32_t v) {
    asm volatile("st.shared.b32 [%0], %1;" ::"r"(saddr), "r"(v));
  }
  __device__ __forceinline__ static const cf* at(const cf* p, int64_t e) { return p + e; }
  __device__ __forceinline__ static cf* at(cf* p, int64_t e) { return p + e; }
  __device__ __forceinline__ static cf ldg_sw(const cf* p, int64_t off, bool swap) {
    const cf v = ldg(p, off);
    return swap ? mk(v.y, v.x) : v;
  }
  __device__ __forceinline__ static void stg_sw(cf* p, int64_t off, cf v, bool swap) {
    stg(p, off, swap ? mk(v.y, v.x) : v);
  }
};

// An FP16 pair (real in the low half) widened to FP32: exact.
__device__ __forceinline__ cf unpack_f16x2(uint32_t r) {
  float x, y;
  asm("{\n\t.reg .b16 l, h;\n\tmov.b32 {l, h}, %2;\n\tcvt.f32.f16 %0, l;\n\tcvt.f32.f16 %1, h;\n\t}"
      : "=f"(x), "=f"(y)
      : "r"(r));
  return mk(x, y);
}

// complex32 storage: element offsets count 4-byte FP16 pairs, and the body's
// `cf*` base pointers carry byte addresses of such arrays.  A swap of the two
// halves is one byte permutation of the packed pair.
struct UmmaDevMemH : UmmaDevMem {
  static constexpr bool kHalfIO = true;
  __device__ __forceinline__ static const cf* at(const cf* p, int64_t e) {
    return reinterpret_cast<const cf*>(reinterpret_cast<const uint32_t*>(p) + e);
  }
  __device__ __forceinline__ static cf* at(cf* p, int64_t e) {
    return reinterpret_cast<cf*>(reinterpret_cast<uint32_t*>(p) + e);
  }
  __device__ __forceinline__ static cf ldg_sw(const cf* p, int64_t off, bool swap) {
    return unpack_f16x2(ldg_pair(p, off, swap));
  }
  // the packed pair itself, halves swapped when asked
  __device__ __forceinline__ static uint32_t ldg_pair(const cf* p, int64_t off, bool swap) {
    const uint32_t r = __ldcs(reinterpret_cast<const unsigned int*>(p) + off);
    return __byte_perm(r, 0u, swap ? 0x1032u : 0x3210u);
  }
  __device__ __forceinline__ static void stg_sw(cf* p, int64_t off, cf v, bool swap) {
    reinterpret_cast<uint32_t*>(p)[off] =
        __byte_perm(pack_rn<TC_FP16>(v.x, v.y), 0u, swap ? 0x1032u : 0x3210u);
  }
};

// The loader's reads from the staging buffer (shared memory, same element
// offsets as the tile in global memory) instead of global memory.
template <class Base>
struct UmmaStagedMem : Base {
  __device__ __forceinline__ static uint32_t ldg_pair(const cf* p, int64_t off, bool swap) {
    const uint32_t r = reinterpret_cast<const uint32_t*>(p)[off];
    return __byte_perm(r, 0u, swap ? 0x1032u : 0x3210u);
  }
  __device__ __forceinline__ static cf ldg_sw(const cf* p, int64_t off, bool swap) {
    if constexpr (Base::kHalfIO) {
      return unpack_f16x2(ldg_pair(p, off, swap));
    } else {
      const float2 v = reinterpret_cast<const float2*>(p)[off];
      return swap ? mk(v.y, v.x) : mk(v.x, v.y);
    }
  }
};

template <int LOGL, int PREC, bool H = false>
struct Umma {
  using G = UmmaGeo<LOGL>;
  using Mem = std::conditional_t<H, UmmaDevMemH, UmmaDevMem>;
  using Body = UmmaBody<LOGL, PREC, Mem>;
  using BodyS = UmmaBody<LOGL, PREC, UmmaStagedMem<Mem>>;  // loader from the staging buffer
  static constexpr int P = Body::P;
  static constexpr bool SPLIT = Body::SPLIT;
  static constexpr int SMEM = (SPLIT ? 2 : 1) * G::A_BYTES + 2 * G::B_BYTES + 16;

  // UMMAs of one stage: every row block, both K halves (three products each
  // for the split class), then a commit to the stage's mbarrier.
  static __device__ __forceinline__ void issue(uint32_t tmem, uint32_t a_hi, uint32_t a_lo,
                                               uint32_t b_hi, uint32_t b_lo, uint64_t* bar) {
    const uint32_t idesc = umma_idesc(P == TC_FP16 ? 0 : 1);
#pragma unroll
    for (int rb = 0; rb < G::RB; ++rb) {
      const uint32_t dt = tmem + 32u * rb;
#pragma unroll
      for (int ks = 0; ks < 2; ++ks) {
        const uint32_t ao = (uint32_t)rb * 8192u + 32u * ks;
        umma16(dt, umma_smem_desc(a_hi + ao), umma_smem_desc(b_hi + 32u * ks), idesc, ks);
        if (SPLIT) {
          umma16(dt, umma_smem_desc(a_hi + ao), umma_smem_desc(b_lo + 32u * ks), idesc, 1);
          umma16(dt, umma_smem_desc(a_lo + ao), umma_smem_desc(b_hi + 32u * ks), idesc, 1);
        }
      }
    }
    umma_commit(bar);
  }

  // Outputs of tensor-core stage t: each thread reads the 16 outputs of the
  // butterfly in its tensor-memory lane, for each of its warp's row blocks.
  template <int t>
  static __device__ __forceinline__ void epilogue(const PassDesc& d, cf* gout, int valid,
                                                  uint32_t tmem, uint32_t a_hi, uint32_t a_lo,
                                                  int warp, int lane) {
    const int q = warp & 3;
#pragma unroll 1
    for (int rb = warp >> 2; rb < G::RB; rb += G::NWARP / 4) {
      const uint32_t ta = tmem + ((uint32_t)(q * 32) << 16) + 32u * rb;
      const int m = rb * 128 + q * 32 + lane;
      typename Body::RowPart rp = Body::template row_part<t>(d, m);
      uint32_t r[16];
      tmem_ld16(ta, r);  // outputs 0..7
      Body::template epilogue_part<t, 0, 8>(d, gout, valid, rp, r, a_hi, a_lo);
      tmem_ld16(ta + 16u, r);  // outputs 8..15
      Body::template epilogue_part<t, 8, 8>(d, gout, valid, rp, r, a_hi, a_lo);
    }
  }
};

template <int LOGL, int PREC, bool H>
__global__ void __launch_bounds__(32 * umma_warps(LOGL), umma_warps(LOGL) == 16 ? 2 : 4)
stockham_umma(const cf* __restrict__ in, cf* out, const __grid_constant__ PassDesc d) {
  using U = Umma<LOGL, PREC, H>;
  using Body = typename U::Body;
  using Mem = typename U::Mem;
  constexpr int ESZ = H ? 4 : 8;  // bytes per stored element
  using G = typename U::G;
  extern __shared__ __align__(1024) unsigned char smem_umma[];
  // 1 KB-aligned base (the 64-byte swizzle repeats every 512 bytes)
  const uint32_t base = (smem_u32(smem_umma) + 1023u) & ~1023u;
  unsigned char* gbase = smem_umma + (base - smem_u32(smem_umma));
  const uint32_t a_hi = base;
  const uint32_t a_lo = base + G::A_BYTES;
  const uint32_t b_hi = base + (U::SPLIT ? 2 : 1) * G::A_BYTES;
  const uint32_t b_lo = b_hi + G::B_BYTES;
  uint64_t* bar = reinterpret_cast<uint64_t*>(gbase + (b_lo + G::B_BYTES - base));
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 1);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // staging buffer (umma_staging_bytes): 128-byte aligned after the above
  constexpr bool kStaged = umma_staging_bytes(LOGL, ESZ, U::SPLIT) > 0;
  constexpr uint32_t kStageBytes = kStaged ? (uint32_t)G::T * ESZ : 0u;
  const uint32_t st_rel = ((b_lo + G::B_BYTES - base) + 16u + 127u) & ~127u;
  const cf* stg = reinterpret_cast<const cf*>(gbase + st_rel);
  uint64_t* lbar = reinterpret_cast<uint64_t*>(gbase + st_rel + kStageBytes);
  const bool staged = kStaged && (reinterpret_cast<uintptr_t>(in) & 15) == 0;
  // bytes of tile t's valid transforms (every transform L * ESZ >= 64 bytes)
  auto tile_bytes = [&](int64_t t) -> uint32_t {
    const int64_t rem = d.count_inner - t * G::TPT;
    return (uint32_t)((rem < G::TPT ? rem : G::TPT) * G::L * ESZ);
  };

  if (warp == 0) tmem_alloc(tslot, G::TMEM_COLS);
  // the DFT matrix (and its low part) in the B layout, once per CTA
  for (int e = tid; e < 1024; e += G::THREADS) {
    const int n = e >> 5, k = e & 31;
    const float v = umma_dft_entry(k, n);
    const uint16_t h = U::P == TC_FP16 ? f32_to_f16_bits(v) : f32_to_bf16_bits(v);
    *reinterpret_cast<uint16_t*>(gbase + (b_hi - base) + umma_boff(n, k)) = h;
    if (U::SPLIT)
      *reinterpret_cast<uint16_t*>(gbase + (b_lo - base) + umma_boff(n, k)) =
          f32_to_bf16_bits(v - bf16_bits_to_f32(h));
  }
  if (tid == 0) {
    mbar_init(bar, 1);
    if (kStaged) mbar_init(lbar, 1);
  }
  fence_smem_async();
  tc05_fence_before();
  __syncthreads();
  tc05_fence_after();
  const uint32_t tmem = *tslot;
  // the first tile's copy; `pending`: a copy is in flight that no wait has seen
  bool pending = staged && blockIdx.x < d.tiles;
  if (pending && tid == 0)
    tma_load(const_cast<cf*>(stg), Mem::at(in, (int64_t)blockIdx.x * G::TPT * G::L),
             tile_bytes(blockIdx.x), lbar);
  uint32_t lparity = 0;

  // the loader's parts of this thread's blocks of items
  const int et = umma_load_item<LOGL>(lane, warp);
  auto parts = [&](int b) { return Body::block_part_of(et, b); };
  auto parts_s = [&](int b) { return U::BodyS::block_part_of(et, b); };

  uint32_t parity = 0;
  bool failed = false;
  for (int64_t tile = blockIdx.x; tile < d.tiles && !failed; tile += gridDim.x) {
    const int64_t first = tile * G::TPT;
    const int64_t rem = d.count_inner - first;
    const int valid = rem < G::TPT ? (int)rem : G::TPT;
    const cf* gin = Mem::at(in, first * G::L);
    cf* gout = Mem::at(out, first * G::L);
    // the tile this CTA takes next, into L2 while this one is computed
    // (whole 16-byte units inside the tile only; none for a ragged tile).
    // Measured per form: it pays for complex32 storage, for tiles of 4096
    // elements and for the split class at 2^13; for complex64 FP16 / BF16 at
    // 2^13 and 2^14 and the split class at 2^14 it costs 5-18% (at 2^14 with
    // it, DRAM reads were 17% above the tile bytes: prefetched lines read
    // again).
    constexpr bool kPrefetchL2 = H || LOGL < 13 || (U::SPLIT && LOGL == 13);
    if (kPrefetchL2 && !staged && tid == 0 && tile + gridDim.x < d.tiles) {
      const int64_t nfirst = (tile + gridDim.x) * G::TPT;
      if (nfirst + G::TPT <= d.count_inner) {
        const uintptr_t a = reinterpret_cast<uintptr_t>(Mem::at(in, nfirst * G::L));
        const uintptr_t a16 = (a + 15) & ~uintptr_t(15);
        const uintptr_t e16 = (a + (uintptr_t)G::T * ESZ) & ~uintptr_t(15);
        if (e16 > a16) prefetch_l2(reinterpret_cast<const void*>(a16), (uint32_t)(e16 - a16));
      }
    }
    bool direct = true;
    if constexpr (kStaged) {
      if (staged) {
        const bool ok = mbar_wait(lbar, lparity, kWaitPolls);
        if (__syncthreads_or(!ok)) {
          if (tid == 0) atomicExch(d.status, 1);
          failed = true;
          break;
        }
        lparity ^= 1u;
        pending = false;
        if (valid == G::TPT) U::BodyS::template load_tile<true>(d, stg, valid, a_hi, a_lo, parts_s);
        else U::BodyS::template load_tile<false>(d, stg, valid, a_hi, a_lo, parts_s);
        direct = false;
      }
    }
    if (direct) {
      if (valid == G::TPT) Body::template load_tile<true>(d, gin, valid, a_hi, a_lo, parts);
      else Body::template load_tile<false>(d, gin, valid, a_hi, a_lo, parts);
    }
    fence_smem_async();
    tc05_fence_before();
    __syncthreads();
    // every thread has read the staging buffer: the next tile's copy
    if (staged && tile + gridDim.x < d.tiles) {
      pending = true;
      if (tid == 0)
        tma_load(const_cast<cf*>(stg), Mem::at(in, (tile + gridDim.x) * G::TPT * G::L),
                 tile_bytes(tile + gridDim.x), lbar);
    }
    auto stage = [&](auto t_) {
      constexpr int t = decltype(t_)::value;
      if (failed) return;
      if (tid == 0) {
        tc05_fence_after();
        U::issue(tmem, a_hi, a_lo, b_hi, b_lo, bar);
      }
      const bool ok = mbar_wait(bar, parity, kWaitPolls);
      if (__syncthreads_or(!ok)) {
        if (tid == 0) {
          atomicExch(d.status, 1);
          mbar_wait(bar, parity, kWaitPolls);  // the UMMAs in flight finish before the free
        }
        failed = true;
        return;
      }
      parity ^= 1u;
      tc05_fence_after();
      U::template epilogue<t>(d, gout, valid, tmem, a_hi, a_lo, warp, lane);
      fence_smem_async();
      tc05_fence_before();
      __syncthreads();
    };
    stage(std::integral_constant<int, 0>());
    if constexpr (G::NTC > 1) stage(std::integral_constant<int, 1>());
    if constexpr (G::NTC > 2) stage(std::integral_constant<int, 2>());
  }
  // a copy still in flight (after a failure) lands before the CTA leaves
  if (pending && tid == 0) mbar_wait(lbar, lparity, kWaitPolls);
  tc05_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc05_fence_after();
    tmem_dealloc(tmem, G::TMEM_COLS);
  }
}

}  // namespace gbfft
