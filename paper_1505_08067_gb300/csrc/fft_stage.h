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
//
// `TR` (traits) says which pass parameters are compile-time constants: the
// generic kernel reads everything from the descriptor; specialised kernels fix
// the length, radix schedule, tile and contiguous strides, so that every
// shared-memory, twiddle and global offset inside a butterfly becomes an
// immediate.
//
// Backward transforms use DFT^-1(x) = swap(DFT(swap(x))) with
// swap(a + ib) = b + ia, which is only a renaming of registers at the first
// load and the last store.
#pragma once
#include "fft_core.h"

namespace gbfft {

// Offset of slot(base + d) from slot(base) for slot(x) = x + (x >> 4), valid
// for every (base, d) pair the Stockham reads and writes produce: either d is
// a multiple of 16, or base and base + d stay inside one 16-element block
// apart from whole-block steps of d (see the derivation in fft_core.h).
GB_HD int pad_off(int d) { return d + (d >> 4); }

// All parameters from the descriptor.
struct RtTraits {
  static constexpr bool kContig = false;
  static constexpr int kMaxStages = 15;
  static constexpr int kEpi = -1;  // decided at run time
  GB_HD static int logL(const PassDesc& d) { return d.logL; }
  GB_HD static int nst(const PassDesc& d) { return d.nst; }
  GB_HD static int rlog(const PassDesc& d, int s) { return d.rlog[s]; }
  GB_HD static int G(const PassDesc& d) { return d.G; }
  GB_HD static int T(const PassDesc& d) { return d.T; }
  GB_HD static int pitch(const PassDesc& d) { return d.pitch; }
  GB_HD static int64_t in_e(const PassDesc& d) { return d.in.e; }
  GB_HD static int64_t in_g(const PassDesc& d) { return d.in.g; }
  GB_HD static int64_t out_e(const PassDesc& d) { return d.out.e; }
  GB_HD static int64_t out_g(const PassDesc& d) { return d.out.g; }
};

// Length 2^LOGL, schedule SCHED (log2 radices, 4 bits each, stage 0 in the
// low nibble), NST stages, R elements per thread, G transforms per tile.
// CONTIG: transforms contiguous (element stride 1, transform stride L) in and
// out.  EPI: four-step twiddle on store (0/1).
template <int LOGL, uint32_t SCHED, int NST, int R, int G_, bool CONTIG, int EPI>
struct CtTraits {
  static constexpr bool kContig = CONTIG;
  static constexpr int kMaxStages = NST;
  static constexpr int kEpi = EPI;
  static constexpr int kT = (1 << LOGL) / R;
  static constexpr int kPitch = (1 << LOGL) + ((1 << LOGL) >> 4) + (16 / G_ > 1 ? 16 / G_ : 1);
  GB_HD static int logL(const PassDesc&) { return LOGL; }
  GB_HD static int nst(const PassDesc&) { return NST; }
  GB_HD static int rlog(const PassDesc&, int s) { return (int)((SCHED >> (4 * s)) & 15u); }
  GB_HD static int G(const PassDesc&) { return G_; }
  GB_HD static int T(const PassDesc&) { return kT; }
  GB_HD static int pitch(const PassDesc&) { return kPitch; }
  GB_HD static int64_t in_e(const PassDesc& d) { return CONTIG ? 1 : d.in.e; }
  GB_HD static int64_t in_g(const PassDesc& d) { return CONTIG ? (1 << LOGL) : d.in.g; }
  GB_HD static int64_t out_e(const PassDesc& d) { return CONTIG ? 1 : d.out.e; }
  GB_HD static int64_t out_g(const PassDesc& d) { return CONTIG ? (1 << LOGL) : d.out.g; }
};

template <int R, int LMAP, int SMAP, class Mem, class TR = RtTraits>
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
    return tl.inner * TR::G(d) + g < d.count_inner;
  }

  // Shared slot of element a of transform g (before the in-butterfly offset).
  GB_HD static int slot(const PassDesc& d, int g, int a) {
    return smem_slot(LAYOUT, g, a, TR::G(d), TR::pitch(d));
  }
  // Slot of element base + delta, delta = i * (Ns or L/r).
  GB_HD static int slot_plus(const PassDesc& d, int g, int base, int sbase, int delta) {
    if (LAYOUT == MAP_ROWS) return sbase + pad_off(delta);
    return slot(d, g, base + delta);
  }

  // ------------------------------------------------------------ stage 0 --
  template <int RR, bool SWAP, bool STORE = true>
  GB_HD static void first_r(cf (&v)[R], const PassDesc& d, const cf* in, cf* out, cf* sm,
                            const Tile& tl, int tid) {
    constexpr int NB = R / RR;
    int g, t;
    thread_coords(LMAP, tid, TR::T(d), TR::G(d), g, t);
    const bool ok = valid(d, tl, g);
    const int stride = (1 << TR::logL(d)) / RR;
    const int64_t e = TR::in_e(d);
    const cf* tb = in + (tl.outer * d.in.o + tl.inner * d.in.t + (int64_t)g * TR::in_g(d));
GB_UNROLL
    for (int q = 0; q < NB; ++q) {
      const int jb = q * TR::T(d) + t;
      const cf* p = tb + (int64_t)jb * e;
GB_UNROLL
      for (int i = 0; i < RR; ++i) {
        cf x = mk(0.f, 0.f);
        if (ok) x = Mem::ldg(p, (int64_t)(i * stride) * e);
        v[q * RR + i] = SWAP ? mk(x.y, x.x) : x;
      }
      dft_radix<RR>(v + q * RR);
    }
    if (TR::nst(d) == 1) {
      if (!STORE) return;
      if (d.conj_out) store_r<RR, true>(v, d, out, tl, tid, 1, LMAP);
      else store_r<RR, false>(v, d, out, tl, tid, 1, LMAP);
    } else {
      write_r<RR>(v, d, sm, tid, 1);
    }
  }

  // --------------------------------------------- shared -> registers -----
  // Twiddles: one table load of w = w_{Ns*r}^k per butterfly, w^i formed as
  // products of lower powers (at most four roundings) instead of r-1 table
  // loads: the passes were bound by the load queue (2^9..2^12: 92-95% of
  // the HBM copy bandwidth with table loads, 99-102% with powers).
  template <int RR, bool SWAP, bool STORE = true>
  GB_HD static void read_r(cf (&v)[R], const PassDesc& d, int s, int Ns, cf* out,
                           const cf* sm, const Tile& tl, int tid) {
    constexpr int NB = R / RR;
    const bool last = STORE && (s == TR::nst(d) - 1);
    const int map = last ? SMAP : LMAP;
    int g, t;
    thread_coords(map, tid, TR::T(d), TR::G(d), g, t);
    const int stride = (1 << TR::logL(d)) / RR;
GB_UNROLL
    for (int q = 0; q < NB; ++q) {
      const int jb = q * TR::T(d) + t;
      const int k = jb & (Ns - 1);
      // twiddles w_{Ns*r}^{i*k}, stored i-major: consecutive k are adjacent
      const cf* w = d.tw + d.tw_off[s] + k;
      cf pw[RR];
      pw[1] = Mem::ldtw(w + Ns);
GB_UNROLL
      for (int i = 2; i < RR; ++i) pw[i] = cmul(pw[i / 2], pw[i - i / 2]);
      const int sb = slot(d, g, jb);
GB_UNROLL
      for (int i = 0; i < RR; ++i) {
        cf x = Mem::lds(sm, slot_plus(d, g, jb, sb, i * stride));
        if (i > 0) x = cmul(x, pw[i]);
        v[q * RR + i] = x;
      }
      dft_radix<RR>(v + q * RR);
    }
    if (last) store_r<RR, SWAP>(v, d, out, tl, tid, Ns, map);
  }

  // --------------------------------------------- registers -> shared -----
  template <int RR>
  GB_HD static void write_r(const cf (&v)[R], const PassDesc& d, cf* sm, int tid, int Ns) {
    constexpr int NB = R / RR;
    int g, t;
    thread_coords(LMAP, tid, TR::T(d), TR::G(d), g, t);
GB_UNROLL
    for (int q = 0; q < NB; ++q) {
      const int jb = q * TR::T(d) + t;
      const int k = jb & (Ns - 1);
      const int base = (jb - k) * RR + k;
      const int sb = slot(d, g, base);
GB_UNROLL
      for (int i = 0; i < RR; ++i)
        Mem::sts(sm, slot_plus(d, g, base, sb, i * Ns), v[q * RR + i]);
    }
  }

  // --------------------------------------------- registers -> global -----
  // In the last stage jb < Ns, so element i of butterfly jb is output jb + i*Ns.
  template <int RR, bool SWAP>
  GB_HD static void store_r(const cf (&v)[R], const PassDesc& d, cf* out, const Tile& tl,
                            int tid, int Ns, int map) {
    constexpr int NB = R / RR;
    int g, t;
    thread_coords(map, tid, TR::T(d), TR::G(d), g, t);
    if (!valid(d, tl, g)) return;
    const int64_t col = tl.inner * TR::G(d) + g;  // column index n2 in a four-step pass
    const int64_t e = TR::out_e(d);
    cf* tb = out + (tl.outer * d.out.o + tl.inner * d.out.t + (int64_t)g * TR::out_g(d));
    const int epi = TR::kEpi < 0 ? d.epi : TR::kEpi;
    // full-table mode: the twiddle of output (col, a) sits at col + a * columns
    const cf* tfull = d.epi_lo + col;
    // factored mode: powers of w_N^{col Ns}, each a product of two lower ones
    cf pw[RR];
    if (epi == 4) {
      pw[0] = mk(1.f, 0.f);
      if (RR > 1) pw[1] = Mem::rotor(col * (int64_t)Ns, d.epi_logN);  // col*Ns < N
GB_UNROLL
      for (int i = 2; i < RR; ++i) pw[i] = cmul(pw[i / 2], pw[i - i / 2]);
    }
GB_UNROLL
    for (int q = 0; q < NB; ++q) {
      const int jb = q * TR::T(d) + t;
      cf* p = tb + (int64_t)jb * e;
      const cf* pt = tfull + (int64_t)jb * d.count_inner;
      const cf base = epi == 4 ? Mem::rotor(col * (int64_t)jb, d.epi_logN) : mk(1.f, 0.f);
GB_UNROLL
      for (int i = 0; i < RR; ++i) {
        cf x = v[q * RR + i];
        if (epi == 4) {
          x = cmul(x, i == 0 ? base : cmul(base, pw[i]));
        } else if (epi == 1) {
          const int64_t m = col * (int64_t)(jb + i * Ns);
          const cf w = cmul(Mem::ldtw(d.epi_hi + (m >> d.epi_lo_bits)),
                            Mem::ldtw(d.epi_lo + (m & ((int64_t(1) << d.epi_lo_bits) - 1))));
          x = cmul(x, w);
        } else if (epi == 2) {
          x = cmul(x, Mem::ldtw(pt + (int64_t)(i * Ns) * d.count_inner));
        } else if (epi == 3) {
          const int64_t m = col * (int64_t)(jb + i * Ns);  // < N <= 2^24: exact in FP32
          x = cmul(x, Mem::rotor(m, d.epi_logN));
        }
        Mem::stg(p, (int64_t)(i * Ns) * e, SWAP ? mk(x.y, x.x) : x);
      }
    }
  }

  // --------------------------------------- fast convolution (two rounds) --
  // Round 1 runs the forward stages without the final store (STORE = false).
  // conv_mid then multiplies output a (a = jb + i*Ns of the last stage) by
  // h_scale * H_u[a], swaps re/im and writes it to shared memory in natural
  // order; round 2 reads it back like a stage-0 load (first_smem) and runs
  // the forward stages again, the last one storing with the swap undone:
  // swap(DFT(swap(Y))) is the unnormalised inverse DFT of Y.
  template <int RR>
  GB_HD static void conv_mid_r(const cf (&v)[R], const PassDesc& d, cf* sm, const Tile& tl,
                               int tid, int Ns) {
    constexpr int NB = R / RR;
    int g, t;
    thread_coords(LMAP, tid, TR::T(d), TR::G(d), g, t);
    const int64_t u = tl.inner * TR::G(d) + g;
    const cf* hb = d.h;
    int64_t he = 1;
    if (d.h_lines > 1) {
      hb += ((d.h_first + u) % d.h_lines) * TR::in_g(d);
      he = TR::in_e(d);
    }
    const float sc = d.h_scale;
GB_UNROLL
    for (int q = 0; q < NB; ++q) {
      const int jb = q * TR::T(d) + t;
GB_UNROLL
      for (int i = 0; i < RR; ++i) {
        const int a = jb + i * Ns;
        const cf x = cmul(v[q * RR + i], Mem::ldtw(hb + (int64_t)a * he));
        Mem::sts(sm, slot(d, g, a), mk(x.y * sc, x.x * sc));
      }
    }
  }

  // When the last stage and stage 0 both have radix R (one butterfly per
  // thread), the thread's round-1 outputs t + i*L/R are exactly the inputs of
  // its round-2 stage-0 butterfly: filter, swap and DFT in registers, no
  // exchange between the rounds.
  GB_HD static bool conv_in_regs(const PassDesc& d) {
    return (1 << TR::rlog(d, TR::nst(d) - 1)) == R && (1 << TR::rlog(d, 0)) == R;
  }
  GB_HD static void conv_regs(cf (&v)[R], const PassDesc& d, const Tile& tl, int tid) {
    int g, t;
    thread_coords(LMAP, tid, TR::T(d), TR::G(d), g, t);
    const int64_t u = tl.inner * TR::G(d) + g;
    const cf* hb = d.h;
    int64_t he = 1;
    if (d.h_lines > 1) {
      hb += ((d.h_first + u) % d.h_lines) * TR::in_g(d);
      he = TR::in_e(d);
    }
    const float sc = d.h_scale;
    const int stride = (1 << TR::logL(d)) / R;
GB_UNROLL
    for (int i = 0; i < R; ++i) {
      const cf x = cmul(v[i], Mem::ldtw(hb + (int64_t)(t + i * stride) * he));
      v[i] = mk(x.y * sc, x.x * sc);
    }
    dft_radix<R>(v);
  }

  // Stage 0 of round 2: the loads of first_r, from shared memory.  Results
  // stay in registers; the caller writes them after a barrier.
  template <int RR>
  GB_HD static void first_smem_r(cf (&v)[R], const PassDesc& d, const cf* sm, int tid) {
    constexpr int NB = R / RR;
    int g, t;
    thread_coords(LMAP, tid, TR::T(d), TR::G(d), g, t);
    const int stride = (1 << TR::logL(d)) / RR;
GB_UNROLL
    for (int q = 0; q < NB; ++q) {
      const int jb = q * TR::T(d) + t;
GB_UNROLL
      for (int i = 0; i < RR; ++i) v[q * RR + i] = Mem::lds(sm, slot(d, g, jb + i * stride));
      dft_radix<RR>(v + q * RR);
    }
  }

  GB_HD static void conv_mid(const cf (&v)[R], const PassDesc& d, cf* sm, const Tile& tl, int tid) {
    const int last = TR::nst(d) - 1;
    const int Ns = (1 << TR::logL(d)) >> TR::rlog(d, last);
    switch (TR::rlog(d, last)) {
      case 1: if (R >= 2) conv_mid_r<(R >= 2 ? 2 : R)>(v, d, sm, tl, tid, Ns); break;
      case 2: if (R >= 4) conv_mid_r<(R >= 4 ? 4 : R)>(v, d, sm, tl, tid, Ns); break;
      case 3: if (R >= 8) conv_mid_r<(R >= 8 ? 8 : R)>(v, d, sm, tl, tid, Ns); break;
      case 4: if (R >= 16) conv_mid_r<(R >= 16 ? 16 : R)>(v, d, sm, tl, tid, Ns); break;
      default: break;
    }
  }

  GB_HD static void first_smem(cf (&v)[R], const PassDesc& d, const cf* sm, int tid) {
    switch (TR::rlog(d, 0)) {
      case 1: if (R >= 2) first_smem_r<(R >= 2 ? 2 : R)>(v, d, sm, tid); break;
      case 2: if (R >= 4) first_smem_r<(R >= 4 ? 4 : R)>(v, d, sm, tid); break;
      case 3: if (R >= 8) first_smem_r<(R >= 8 ? 8 : R)>(v, d, sm, tid); break;
      case 4: if (R >= 16) first_smem_r<(R >= 16 ? 16 : R)>(v, d, sm, tid); break;
      default: break;
    }
  }

  // Round 1 stage 0: global -> registers, DFT, shared-memory write (no store
  // even for a single-stage pass).
  GB_HD static void first_nostore(cf (&v)[R], const PassDesc& d, const cf* in, cf* sm,
                                  const Tile& tl, int tid) {
    switch (TR::rlog(d, 0)) {
      case 1: if (R >= 2) first_r<(R >= 2 ? 2 : R), false, false>(v, d, in, nullptr, sm, tl, tid); break;
      case 2: if (R >= 4) first_r<(R >= 4 ? 4 : R), false, false>(v, d, in, nullptr, sm, tl, tid); break;
      case 3: if (R >= 8) first_r<(R >= 8 ? 8 : R), false, false>(v, d, in, nullptr, sm, tl, tid); break;
      case 4: if (R >= 16) first_r<(R >= 16 ? 16 : R), false, false>(v, d, in, nullptr, sm, tl, tid); break;
      default: break;
    }
  }

  // Round 1 stages s >= 1: no store after the last one.
  GB_HD static void read_nostore(cf (&v)[R], const PassDesc& d, int s, int Ns, const cf* sm,
                                 const Tile& tl, int tid) {
    switch (TR::rlog(d, s)) {
      case 1: if (R >= 2) read_r<(R >= 2 ? 2 : R), false, false>(v, d, s, Ns, nullptr, sm, tl, tid); break;
      case 2: if (R >= 4) read_r<(R >= 4 ? 4 : R), false, false>(v, d, s, Ns, nullptr, sm, tl, tid); break;
      case 3: if (R >= 8) read_r<(R >= 8 ? 8 : R), false, false>(v, d, s, Ns, nullptr, sm, tl, tid); break;
      case 4: if (R >= 16) read_r<(R >= 16 ? 16 : R), false, false>(v, d, s, Ns, nullptr, sm, tl, tid); break;
      default: break;
    }
  }

  // Single-stage round 2: store the registers (swap undone).
  GB_HD static void store_first(const cf (&v)[R], const PassDesc& d, cf* out, const Tile& tl,
                                int tid) {
    switch (TR::rlog(d, 0)) {
      case 1: if (R >= 2) store_r<(R >= 2 ? 2 : R), true>(v, d, out, tl, tid, 1, LMAP); break;
      case 2: if (R >= 4) store_r<(R >= 4 ? 4 : R), true>(v, d, out, tl, tid, 1, LMAP); break;
      case 3: if (R >= 8) store_r<(R >= 8 ? 8 : R), true>(v, d, out, tl, tid, 1, LMAP); break;
      case 4: if (R >= 16) store_r<(R >= 16 ? 16 : R), true>(v, d, out, tl, tid, 1, LMAP); break;
      default: break;
    }
  }

  // ---------------------------------------------------- dispatch on radix --
  template <bool SWAP>
  GB_HD static void first_s(cf (&v)[R], const PassDesc& d, const cf* in, cf* out, cf* sm,
                            const Tile& tl, int tid) {
    switch (TR::rlog(d, 0)) {
      case 1: if (R >= 2) first_r<(R >= 2 ? 2 : R), SWAP>(v, d, in, out, sm, tl, tid); break;
      case 2: if (R >= 4) first_r<(R >= 4 ? 4 : R), SWAP>(v, d, in, out, sm, tl, tid); break;
      case 3: if (R >= 8) first_r<(R >= 8 ? 8 : R), SWAP>(v, d, in, out, sm, tl, tid); break;
      case 4: if (R >= 16) first_r<(R >= 16 ? 16 : R), SWAP>(v, d, in, out, sm, tl, tid); break;
      default: break;
    }
  }

  template <bool SWAP>
  GB_HD static void read_s(cf (&v)[R], const PassDesc& d, int s, int Ns, cf* out,
                           const cf* sm, const Tile& tl, int tid) {
    switch (TR::rlog(d, s)) {
      case 1: if (R >= 2) read_r<(R >= 2 ? 2 : R), SWAP>(v, d, s, Ns, out, sm, tl, tid); break;
      case 2: if (R >= 4) read_r<(R >= 4 ? 4 : R), SWAP>(v, d, s, Ns, out, sm, tl, tid); break;
      case 3: if (R >= 8) read_r<(R >= 8 ? 8 : R), SWAP>(v, d, s, Ns, out, sm, tl, tid); break;
      case 4: if (R >= 16) read_r<(R >= 16 ? 16 : R), SWAP>(v, d, s, Ns, out, sm, tl, tid); break;
      default: break;
    }
  }

  GB_HD static void first(cf (&v)[R], const PassDesc& d, const cf* in, cf* out, cf* sm,
                          const Tile& tl, int tid) {
    if (d.conj_in) first_s<true>(v, d, in, out, sm, tl, tid);
    else first_s<false>(v, d, in, out, sm, tl, tid);
  }

  GB_HD static void read(cf (&v)[R], const PassDesc& d, int s, int Ns, cf* out, const cf* sm,
                         const Tile& tl, int tid) {
    if (s == TR::nst(d) - 1 && d.conj_out) read_s<true>(v, d, s, Ns, out, sm, tl, tid);
    else read_s<false>(v, d, s, Ns, out, sm, tl, tid);
  }

  GB_HD static void write(const cf (&v)[R], const PassDesc& d, int s, int Ns, cf* sm, int tid) {
    switch (TR::rlog(d, s)) {
      case 1: if (R >= 2) write_r<(R >= 2 ? 2 : R)>(v, d, sm, tid, Ns); break;
      case 2: if (R >= 4) write_r<(R >= 4 ? 4 : R)>(v, d, sm, tid, Ns); break;
      case 3: if (R >= 8) write_r<(R >= 8 ? 8 : R)>(v, d, sm, tid, Ns); break;
      case 4: if (R >= 16) write_r<(R >= 16 ? 16 : R)>(v, d, sm, tid, Ns); break;
      default: break;
    }
  }
};

}  // namespace gbfft
