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
#include <cuda_runtime.h>

#include "fft_split.h"
#include "fft_stage.h"
#include "kernel_shapes.h"
#include "kernels.h"

namespace gbfft {

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
};

template <int R, int LMAP, int SMAP, class TR>
__global__ void __launch_bounds__(1024)
stockham_pass(const cf* __restrict__ in, cf* out, const __grid_constant__ PassDesc d) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cf* sm = reinterpret_cast<cf*>(smem_raw);
  using B = PassBody<R, LMAP, SMAP, DevMem, TR>;
  const int tid = threadIdx.x;
  for (int64_t tile = blockIdx.x; tile < d.tiles; tile += gridDim.x) {
    const typename B::Tile tl = B::tile_of(d, tile);
    if constexpr (TR::kContig) {
      // Persistent grids: pull this block's next tile into L2 while the
      // current one is computed (one 128-byte line per thread and pass of
      // this loop), so its stage-0 loads hit L2 instead of DRAM.
      if (d.l2_prefetch && tile + gridDim.x < d.tiles) {
        const int64_t L = int64_t(1) << TR::logL(d);
        const int64_t tile_elems = (int64_t)TR::G(d) * L;
        const int64_t valid = min(tile_elems, d.count_inner * L - (tile + gridDim.x) * tile_elems);
        const char* base = reinterpret_cast<const char*>(in + (tile + gridDim.x) * tile_elems);
        for (int64_t line = tid; line * 16 < valid; line += blockDim.x)
          asm volatile("prefetch.global.L2::evict_last [%0];" ::"l"(base + line * 128));
      }
    }
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

template <class SH, int S, bool FIRST_EXCHANGE>
__device__ __forceinline__ void split_exchange(cf (&v)[SH::kR], const PassDesc& d, cf* x, cf* st,
                                               uint64_t* bar, const cf* next_src, int tid) {
  using B = SplitBody<SH, DevMem>;
  B::template write_half<S, 0>(v, x, tid);
  __syncthreads();
  if (FIRST_EXCHANGE && tid == 0 && next_src)  // staging is free: every thread has read it
    tma_load(st, next_src, SH::kL * 8, bar);
  B::template read_half<S, 0>(v, x, tid);
  __syncthreads();
  B::template write_half<S, 1>(v, x, tid);
  __syncthreads();
  B::template read_half<S, 1>(v, x, tid);
  B::template compute<S>(v, d, tid);
  __syncthreads();
}

// One contiguous transform per block, persistent over tiles; the next
// transform streams into shared memory by TMA while this one is computed.
template <class SH, int MINB>
__global__ void __launch_bounds__(SH::kT, MINB)
stockham_staged(const cf* __restrict__ in, cf* out, const __grid_constant__ PassDesc d) {
  extern __shared__ __align__(128) unsigned char smem_staged[];
  cf* st = reinterpret_cast<cf*>(smem_staged);
  cf* x = st + SH::kL;
  uint64_t* bar = reinterpret_cast<uint64_t*>(x + SH::kHalfSlots);
  using B = SplitBody<SH, DevMem>;
  const int tid = threadIdx.x;
  const int64_t step = gridDim.x;
  int64_t tile = blockIdx.x;
  if (tid == 0) mbar_init(bar, 1);
  __syncthreads();
  if (tid == 0 && tile < d.tiles) tma_load(st, in + tile * SH::kL, SH::kL * 8, bar);
  uint32_t parity = 0;
  for (; tile < d.tiles; tile += step) {
    const bool ok = mbar_wait(bar, parity, kWaitPolls);
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        atomicExch(d.status, 1);
        mbar_wait(bar, parity, kWaitPolls);  // let the copy in flight land before leaving
      }
      return;
    }
    parity ^= 1u;
    const cf* next = tile + step < d.tiles ? in + (tile + step) * SH::kL : nullptr;
    cf v[SH::kR];
    if (d.conj_in) B::template first<true>(v, st, tid);
    else B::template first<false>(v, st, tid);
    split_exchange<SH, 0, true>(v, d, x, st, bar, next, tid);
    if constexpr (SH::kNst > 2) split_exchange<SH, 1, false>(v, d, x, st, bar, nullptr, tid);
    if constexpr (SH::kNst > 3) split_exchange<SH, 2, false>(v, d, x, st, bar, nullptr, tid);
    cf* o = out + tile * SH::kL;
    if (d.conj_out) B::template store<true>(v, o, tid);
    else B::template store<false>(v, o, tid);
  }
}

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

using KernelFn = void (*)(const cf*, cf*, PassDesc);

template <int R, int LMAP, int SMAP, class TR>
static KernelFn kfn() {
  return stockham_pass<R, LMAP, SMAP, TR>;
}

static KernelFn generic_kernel(int R, int lmap, int smap) {
#define GB_GEN(RR, A, B_) \
  if (R == RR && lmap == A && smap == B_) return kfn<RR, A, B_, RtTraits>();
  GB_GEN(2, 0, 0) GB_GEN(4, 0, 0) GB_GEN(8, 0, 0) GB_GEN(16, 0, 0)
  GB_GEN(2, 1, 1) GB_GEN(4, 1, 1) GB_GEN(8, 1, 1) GB_GEN(16, 1, 1)
  GB_GEN(2, 0, 1) GB_GEN(4, 0, 1) GB_GEN(8, 0, 1) GB_GEN(16, 0, 1)
#undef GB_GEN
  return nullptr;
}

const void* resolve_kernel(int R, int lmap, int smap, const PassDesc& d, bool generic_only,
                           bool* specialised) {
  if (specialised) *specialised = !generic_only;
  if (!generic_only) {
#define GB_TRY(LOGL, SCHED, NST, RR, G, LM, SM, CONTIG, EPI)                                 \
  if (shape_matches(d, R, lmap, smap, LOGL, SCHED, NST, RR, G, LM, SM, CONTIG, EPI))         \
    return (const void*)kfn<RR, LM, SM, CtTraits<LOGL, SCHED, NST, RR, G, CONTIG, EPI>>();
  GB_SHAPES(GB_TRY)
#undef GB_TRY
  }
  if (specialised) *specialised = false;
  return (const void*)generic_kernel(R, lmap, smap);
}

template <class SH, int MINB>
static KernelFn staged_fn() {
  return stockham_staged<SH, MINB>;
}

bool resolve_staged(const PassDesc& d, bool generic_only, StagedLaunch* s) {
  if (generic_only) return false;
#define GB_STAGED(LOGL, SCHED, NST, MINB)                                      \
  if (staged_shape_matches(d, LOGL, SCHED, NST)) {                            \
    using SH = SplitShape<LOGL, SCHED, NST>;                                   \
    s->fn = (const void*)staged_fn<SH, MINB>();                                \
    s->block = SH::kT;                                                         \
    s->smem = split_smem_bytes<SH>();                                          \
    return true;                                                               \
  }
  GB_STAGED_SHAPES(GB_STAGED)
#undef GB_STAGED
  return false;
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
  s.grid = (int)(g < tiles ? g : tiles);
  return cudaSuccess;
}

cudaError_t launch_staged(const StagedLaunch& s, const PassDesc& d, const void* in, void* out,
                          cudaStream_t st) {
  KernelFn k = reinterpret_cast<KernelFn>(const_cast<void*>(s.fn));
  if (!k || s.grid < 1) return cudaErrorInvalidValue;
  k<<<s.grid, s.block, s.smem, st>>>(static_cast<const cf*>(in), static_cast<cf*>(out), d);
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
