// See exec.h.
#include "exec.h"

#include <algorithm>

namespace gbfft {

cudaError_t bind_launches(const PlanSpec& s, const Caps& caps, const cf* tables, int* status,
                          PassLaunch* launches) {
  for (int i = 0; i < s.passes.size(); ++i) {
    const PassSpec& p = s.passes[i];
    PassLaunch l{};
    if (p.kind == PASS_TRANSPOSE) l.grid = caps.sm_count;  // SMs: the transpose sizes its grid
    if (p.kind == PASS_FFT) {
      l.d = pass_desc(p, 0, s.batch, s.batch);
      l.d.tw = tables;
      l.d.epi_hi = (p.epi == 1 || p.epi == 2) ? tables + p.epi_hi_off : nullptr;
      l.d.epi_lo = (p.epi == 1 || p.epi == 2) ? tables + p.epi_lo_off : nullptr;
      l.d.status = status;
      l.d.h = p.conv ? static_cast<const cf*>(s.filter[p.h_dim]) : nullptr;
      l.R = p.R;
      l.lmap = p.lmap;
      l.smap = p.smap;
      l.grid = p.grid;
      l.block = p.block;
      l.smem = p.smem;
      if (p.tc_prec) {
        l.fn = resolve_tc_pass(p.logL, p.tc_prec, p.variant, p.io16);
        if (!l.fn) return cudaErrorInvalidDeviceFunction;
        l.specialised = true;
      } else {
        l.fn = resolve_kernel(l.R, l.lmap, l.smap, l.d, s.generic_only, &l.specialised);
      }
      cudaError_t e = prepare_launch(l);
      if (e != cudaSuccess) return e;
      if (p.tc_prec) {
        // persistent grid: the DFT-matrix fragments a block builds once serve
        // many tiles
        int per_sm = 0;
        e = occupancy(l, &per_sm);
        if (e != cudaSuccess) return e;
        if (p.variant != 1) {
          // the occupancy query reports one block per SM for this kernel
          // where its registers and shared memory allow more (measured):
          // count from the kernel's attributes, within the SM's tensor memory
          int own = 0;
          e = resident_blocks(l.fn, l.block, l.smem, umma_tmem_cols(p.logL), &own);
          if (e != cudaSuccess) return e;
          per_sm = std::max(per_sm, own);
        }
        l.ctas_per_sm = per_sm;
        const int64_t g = (int64_t)std::max(per_sm, 1) * caps.sm_count;
        l.grid = (int)std::min<int64_t>(g, l.grid);
        l.persistent_grid = l.grid;
        launches[i] = l;
        continue;
      }
      // the library's choice for contiguous FP32 transforms of 2^12 is the
      // register kernel (0.320 against 0.335 ms per 2^27 elements for the
      // staged one, the choice the autotuner makes in every measured run);
      // variant 2 still asks for the staged kernel
      const bool reg4096 = p.variant == 0 && !p.conv && !p.tc_prec && p.logL == 12 &&
                           p.lmap == MAP_ROWS && p.smap == MAP_ROWS;
      const bool want_staged =
          (p.variant == 0 && !reg4096) || p.variant == 2 || p.variant == 4;
      l.has_staged = want_staged && resolve_staged(l.d, l.lmap, l.smap, s.generic_only, &l.staged);
      l.staged.tmap = p.variant != 4;
      if (l.has_staged) {
        e = prepare_staged(l.staged, l.d.tiles, caps.sm_count);
        if (e != cudaSuccess) return e;
      }
      if (p.variant == 3 && l.specialised) {
        int per_sm = 0;
        e = occupancy(l, &per_sm);
        if (e != cudaSuccess) return e;
        const int64_t g = (int64_t)std::max(per_sm, 1) * caps.sm_count;
        l.grid = (int)std::min<int64_t>(g, l.grid);
        l.persistent_grid = l.grid;
        l.d.l2_prefetch = 1;
      }
    }
    launches[i] = l;
  }
  return cudaSuccess;
}

cudaError_t enqueue_tables(const PlanSpec& s, cf* tables, cudaStream_t st) {
  for (const TwSegment& t : s.tables) {
    cudaError_t e = launch_twiddle_gen(tables + t.off, t.count, t.den, t.mode, t.r, t.mult, st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

static cudaError_t enqueue_range(const PlanSpec& s, const PassLaunch* launches, const void* in,
                                 void* out, void* work, int64_t b0, int64_t nb, cudaStream_t st,
                                 int64_t work2_off);

cudaError_t enqueue_passes(const PlanSpec& s, const PassLaunch* launches, const void* in,
                           void* out, void* work, int64_t b0, int64_t nb, cudaStream_t st,
                           int64_t work2_off) {
  if (work2_off < 0) work2_off = s.work2_off;
  if (nb <= 0) return cudaSuccess;
  if (s.chunk_batch <= 0 || nb <= s.chunk_batch)
    return enqueue_range(s, launches, in, out, work, b0, nb, st, work2_off);
  // sub-batches in stream order, each reusing the workspace from its start
  const int64_t E = s.dims == 1 ? s.n[0] : s.n[0] * s.n[1];
  const int64_t eb = elem_bytes(s.precision);
  for (int64_t c = 0; c < nb; c += s.chunk_batch) {
    const int64_t n = std::min(s.chunk_batch, nb - c);
    cudaError_t e = enqueue_range(s, launches, static_cast<const char*>(in) + c * E * eb,
                                  static_cast<char*>(out) + c * E * eb, work, b0 + c, n, st,
                                  work2_off);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

static cudaError_t enqueue_range(const PlanSpec& s, const PassLaunch* launches, const void* in,
                                 void* out, void* work, int64_t b0, int64_t nb, cudaStream_t st,
                                 int64_t work2_off) {
  if (nb <= 0) return cudaSuccess;
  const int64_t E = s.dims == 1 ? s.n[0] : s.n[0] * s.n[1];
  // the second workspace buffer of six-step plans
  void* work2 = work ? static_cast<char*>(work) + work2_off * elem_bytes(s.precision) : nullptr;
  auto buf = [&](int b) -> void* {
    return b == BUF_IN ? const_cast<void*>(in) : b == BUF_OUT ? out : b == BUF_WORK2 ? work2 : work;
  };
  for (int i = 0; i < s.passes.size(); ++i) {
    const PassSpec& p = s.passes[i];
    const void* src = buf(p.src);
    void* dst = buf(p.dst);
    cudaError_t e;
    if (p.kind == PASS_COPY) {
      e = launch_copy(src, dst, nb * E, 1, 1, st);
    } else if (p.kind == PASS_TRANSPOSE) {
      e = launch_transpose(src, dst, nb, p.tr_rows, p.tr_cols, p.tr_logN, p.tr_sign, p.io16,
                           launches[i].grid, st);
    } else {
      PassLaunch l = launches[i];
      if (b0 != 0 || nb != s.batch) {
        PassDesc d = pass_desc(p, b0, nb, s.batch);
        d.tw = l.d.tw;
        d.epi_hi = l.d.epi_hi;
        d.epi_lo = l.d.epi_lo;
        d.status = l.d.status;
        d.h = l.d.h;
        l.d = d;
        l.fn = p.tc_prec ? resolve_tc_pass(p.logL, p.tc_prec, p.variant, p.io16)
                         : resolve_kernel(l.R, l.lmap, l.smap, l.d, s.generic_only, &l.specialised);
        e = prepare_launch(l);
        if (e != cudaSuccess) return e;
        d.l2_prefetch = launches[i].d.l2_prefetch;
        l.d.l2_prefetch = d.l2_prefetch;
        l.grid = (int)std::min<int64_t>(d.tiles, l.persistent_grid ? l.persistent_grid : 0x7fffffff);
      }
      if (l.d.tiles == 0) continue;
      if (l.has_staged && ((uintptr_t)src & 15) == 0) {
        StagedLaunch sl = l.staged;
        sl.grid = (int)std::min<int64_t>(sl.max_grid > 0 ? sl.max_grid : sl.grid, l.d.tiles);
        e = launch_staged(sl, l.d, src, dst, st);
      } else {
        e = launch_pass(l, src, dst, st);
      }
    }
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace gbfft
