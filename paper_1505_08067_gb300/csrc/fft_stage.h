// Phases of one Stockham pass, per thread (see fft_core.h for the stage
// formulation).  A tile is processed as
//
//   first(tid)                               global -> registers, stage 0
//   for s = 1 .. nst-1:
//     barrier; read(s, tid)                   shared -> registers, twiddle, DFT
//     if s < nst-1: barrier; write(s, tid)    registers -> shared
//   (the last read phase stores straight to global memory)
//
// The GPU kernel runs each phase on all threads with __syncthreads() between
// them.  A CPU test harness runs the same phase functions thread by thread,
// with a memory policy that checks every index, so the pass's addressing is
// verified on the host.  `Mem` supplies the five memory operations.
#pragma once
#include "fft_core.h"

namespace gbfft {

template <int R, int LMAP, int SMAP, class Mem>
struct PassBody {
  static constexpr int LAYOUT = LMAP;  // shared layout follows the load map

  struct Tile {
    int64_t outer, inner;
  };

  GB_HD static Tile tile_of(const PassDesc& d, int64_t tile) {
    Tile tl;
    tl.outer = tile / d.tiles_inner;
    tl.inner = tile - tl.outer * d.tiles_inner;
    return tl;
  }

  GB_HD static bool valid(const PassDesc& d, const Tile& tl, int g) {
    return tl.inner * d.G + g < d.count_inner;
  }

  // ------------------------------------------------------------ stage 0 --
  template <int RR>
  GB_HD static void first_r(cf (&v)[R], const PassDesc& d, const cf* in, cf* out, cf* sm,
                            const Tile& tl, int tid) {
    constexpr int NB = R / RR;
    int g, t;
    thread_coords(LMAP, tid, d.T, d.G, g, t);
    const bool ok = valid(d, tl, g);
    const int stride = (1 << d.logL) / RR;
GB_UNROLL
    for (int q = 0; q < NB; ++q) {
      const int jb = q * d.T + t;
GB_UNROLL
      for (int i = 0; i < RR; ++i) {
        cf x = mk(0.f, 0.f);
        if (ok) x = Mem::ldg(in, elem_offset(d.in, tl.outer, tl.inner, g, jb + i * stride));
        if (d.conj_in) x.y = -x.y;
        v[q * RR + i] = x;
      }
      dft_radix<RR>(v + q * RR);
    }
    if (d.nst == 1) {
      store_r<RR>(v, d, out, tl, tid, 1, LMAP);
    } else {
      write_r<RR>(v, d, sm, tid, 1);
    }
  }

  // --------------------------------------------- shared -> registers -----
  template <int RR>
  GB_HD static void read_r(cf (&v)[R], const PassDesc& d, int s, int Ns, cf* out,
                           const cf* sm, const Tile& tl, int tid) {
    constexpr int NB = R / RR;
    const bool last = (s == d.nst - 1);
    const int map = last ? SMAP : LMAP;
    int g, t;
    thread_coords(map, tid, d.T, d.G, g, t);
    const int stride = (1 << d.logL) / RR;
GB_UNROLL
    for (int q = 0; q < NB; ++q) {
      const int jb = q * d.T + t;
      const int k = jb & (Ns - 1);
      const cf* w = d.tw + d.tw_off[s] + k * RR;
GB_UNROLL
      for (int i = 0; i < RR; ++i) {
        cf x = Mem::lds(sm, smem_slot(LAYOUT, g, jb + i * stride, d.G, d.pitch));
        if (i > 0) x = cmul(x, Mem::ldtw(w + i));
        v[q * RR + i] = x;
      }
      dft_radix<RR>(v + q * RR);
    }
    if (last) store_r<RR>(v, d, out, tl, tid, Ns, map);
  }

  // --------------------------------------------- registers -> shared -----
  template <int RR>
  GB_HD static void write_r(const cf (&v)[R], const PassDesc& d, cf* sm, int tid, int Ns) {
    constexpr int NB = R / RR;
    int g, t;
    thread_coords(LMAP, tid, d.T, d.G, g, t);
GB_UNROLL
    for (int q = 0; q < NB; ++q) {
      const int jb = q * d.T + t;
      const int k = jb & (Ns - 1);
      const int base = (jb - k) * RR + k;
GB_UNROLL
      for (int i = 0; i < RR; ++i)
        Mem::sts(sm, smem_slot(LAYOUT, g, base + i * Ns, d.G, d.pitch), v[q * RR + i]);
    }
  }

  // --------------------------------------------- registers -> global -----
  // In the last stage jb < Ns, so element i of butterfly jb is output jb + i*Ns.
  template <int RR>
  GB_HD static void store_r(const cf (&v)[R], const PassDesc& d, cf* out, const Tile& tl,
                            int tid, int Ns, int map) {
    constexpr int NB = R / RR;
    int g, t;
    thread_coords(map, tid, d.T, d.G, g, t);
    if (!valid(d, tl, g)) return;
    const int64_t col = tl.inner * d.G + g;  // column index n2 in a four-step pass
GB_UNROLL
    for (int q = 0; q < NB; ++q) {
      const int jb = q * d.T + t;
GB_UNROLL
      for (int i = 0; i < RR; ++i) {
        const int64_t a = jb + i * Ns;
        cf x = v[q * RR + i];
        if (d.epi) {
          const int64_t m = col * a;
          const cf w = cmul(Mem::ldtw(d.epi_hi + (m >> d.epi_lo_bits)),
                            Mem::ldtw(d.epi_lo + (m & ((1 << d.epi_lo_bits) - 1))));
          x = cmul(x, w);
        }
        if (d.conj_out) x.y = -x.y;
        Mem::stg(out, elem_offset(d.out, tl.outer, tl.inner, g, a), x);
      }
    }
  }

  // ---------------------------------------------------- dispatch on radix --
  GB_HD static void first(cf (&v)[R], const PassDesc& d, const cf* in, cf* out, cf* sm,
                          const Tile& tl, int tid) {
    switch (d.rlog[0]) {
      case 1: if (R >= 2) first_r<(R >= 2 ? 2 : R)>(v, d, in, out, sm, tl, tid); break;
      case 2: if (R >= 4) first_r<(R >= 4 ? 4 : R)>(v, d, in, out, sm, tl, tid); break;
      case 3: if (R >= 8) first_r<(R >= 8 ? 8 : R)>(v, d, in, out, sm, tl, tid); break;
      case 4: if (R >= 16) first_r<(R >= 16 ? 16 : R)>(v, d, in, out, sm, tl, tid); break;
      default: break;
    }
  }

  GB_HD static void read(cf (&v)[R], const PassDesc& d, int s, int Ns, cf* out, const cf* sm,
                         const Tile& tl, int tid) {
    switch (d.rlog[s]) {
      case 1: if (R >= 2) read_r<(R >= 2 ? 2 : R)>(v, d, s, Ns, out, sm, tl, tid); break;
      case 2: if (R >= 4) read_r<(R >= 4 ? 4 : R)>(v, d, s, Ns, out, sm, tl, tid); break;
      case 3: if (R >= 8) read_r<(R >= 8 ? 8 : R)>(v, d, s, Ns, out, sm, tl, tid); break;
      case 4: if (R >= 16) read_r<(R >= 16 ? 16 : R)>(v, d, s, Ns, out, sm, tl, tid); break;
      default: break;
    }
  }

  GB_HD static void write(const cf (&v)[R], const PassDesc& d, int s, int Ns, cf* sm, int tid) {
    switch (d.rlog[s]) {
      case 1: if (R >= 2) write_r<(R >= 2 ? 2 : R)>(v, d, sm, tid, Ns); break;
      case 2: if (R >= 4) write_r<(R >= 4 ? 4 : R)>(v, d, sm, tid, Ns); break;
      case 3: if (R >= 8) write_r<(R >= 8 ? 8 : R)>(v, d, sm, tid, Ns); break;
      case 4: if (R >= 16) write_r<(R >= 16 ? 16 : R)>(v, d, sm, tid, Ns); break;
      default: break;
    }
  }
};

}  // namespace gbfft
