// Phases of the staged Stockham pass for large contiguous transforms
// (L = 2^12 .. 2^14, one transform per thread block), per thread.
//
// Why a second body: with one 1024-thread block per SM holding a whole 2^14
// transform in a full-size shared exchange buffer, there is no room to fetch
// the next transform while this one is computed, so the SM alternates between
// waiting for HBM and computing.  Here each thread holds R = 2 * r elements
// (two radix-r butterflies per stage), which makes every exchange fit a buffer
// of HALF the transform:
//
//   In a write phase, butterfly jb = q*T + t (T = L/R threads) writes its r
//   outputs to (u*r*Ns) + k + i*Ns with u = jb / Ns, k = jb mod Ns.  Since
//   r*Ns divides L/2 for every stage but the last, the outputs of butterfly q
//   land in half [q >= NB/2] of the transform (NB = R/r butterflies per thread).
//   In a read phase, element i of butterfly jb' is jb' + i*L/r', in half
//   [i >= r'/2].
//
// So an exchange runs in two rounds: round h writes the butterflies whose
// outputs are in half h, then reads every element of half h that this thread
// needs into the registers that round h just freed.  The other half of shared
// memory holds the next transform, loaded by TMA (cp.async.bulk) while the
// current one is computed (Bergach et al. Sec. 3.4: a transform is read once
// and written once; here the read of transform t+1 overlaps the compute of t).
//
// Register slots: after round 0 slots [0, R/2) hold, for each next-stage
// butterfly q', its elements i < r'/2 at q'*(r'/2) + i; after round 1 slots
// [R/2, R) hold i >= r'/2 at R/2 + q'*(r'/2) + (i - r'/2).  The renaming to
// v[q'*r' + i] is static and costs nothing once unrolled.
//
// Column tiles (G > 1): the same body runs G adjacent columns of a strided
// pass side by side (transform g = thread id mod G), element a of column g at
// slot a*G + g.  The next tile's rows are copied by one bulk copy per row
// (G*8 bytes each), so the strided loads leave the per-thread load queue.
#pragma once
#include "fft_core.h"
#include "fft_stage.h"

namespace gbfft {

// Compile-time shape of a staged pass: R elements (R/16 radix-16
// butterflies) per thread; G transforms per tile (1: one contiguous
// transform; > 1: G adjacent columns of a strided pass); EPI the four-step
// twiddle applied on store (0, 2 full table, 3 computed; column tiles only).
//   ROWS_IN: the tile's input is G contiguous rows (the transposing pass of a
//   four-step plan), staged one row per bulk copy with a pitch of L + kRowPad;
//   otherwise G adjacent columns staged interleaved (element a of column g at
//   a*G + g).  The output side is the same for both: G columns.
template <int LOGL, uint32_t SCHED, int NST, int R_ = 32, int G_ = 1, int EPI_ = 0,
          bool ROWS_IN = false>
struct SplitShape {
  static constexpr int kL = 1 << LOGL;
  static constexpr int kR = R_;
  static constexpr int kG = G_;
  static constexpr int kEpi = EPI_;
  static constexpr bool kRowsIn = ROWS_IN;
  // row pitch padding of the staged rows: the stage-0 loads of a half warp
  // (G columns x 16/G threads) then hit distinct bank pairs (2-way for G = 16)
  static constexpr int kRowPad = ROWS_IN ? (16 / G_ > 2 ? 16 / G_ : 2) : 0;
  static constexpr int kStageElems = ROWS_IN ? G_ * ((1 << LOGL) + kRowPad) : (1 << LOGL) * G_;
  static constexpr int kTt = kL / kR;             // threads per transform
  static constexpr int kT = kTt * kG;             // threads per block
  static constexpr int kHalf = kL / 2;            // exchange buffer holds half of each transform
  static constexpr int kHalfSlots = kHalf * kG + ((kHalf * kG) >> 4) + 1;
  static constexpr int kNst = NST;
  GB_HDC static constexpr int rlog(int s) { return (int)((SCHED >> (4 * s)) & 15u); }
  GB_HDC static constexpr int radix(int s) { return 1 << rlog(s); }
  GB_HDC static constexpr int ns_before(int s) {
    return s == 0 ? 1 : ns_before(s - 1) * radix(s - 1);
  }
  // A final stage of radix NB = R/16 after a radix-16 one runs in registers:
  // stage nst-2 has Ns = L/(16 NB) = T, so thread t's butterflies
  // jb = q*T + t (q < NB) write outputs p + q*L/NB with p = t + i*T (i < 16)
  // -- exactly the NB inputs of the last stage's butterfly p (Ns = L/NB).
  // One shared-memory exchange fewer.
  static constexpr int kNB = R_ / 16;
  static constexpr bool kFuseLast = NST >= 2 && radix(NST - 1) == kNB && rlog(NST - 2) == 4;
  static constexpr int kExchanges = kFuseLast ? NST - 2 : NST - 1;
  // Stage twiddles as powers of one loaded root (SplitBody::compute) where a
  // block fills most of an SM (column tiles, 2^13 and 2^14): fewer loads whose
  // latency few warps cannot hide.  The contiguous 2^12 shape runs four
  // blocks per SM and is faster with one table load per twiddle (measured).
  static constexpr bool kPowTw = G_ > 1 || LOGL >= 13;
  // Load the fused last stage's roots during the last exchange (radix-2
  // last stage: measured faster) or inside the store loop (radix 4).
  static constexpr bool kPrefetchFused = kPowTw && kFuseLast && kNB == 2;
  // The roots depend on the thread and the stage only, not on the tile: a
  // kernel with registers to spare loads them once, before its first tile,
  // and keeps them -- those of the exchanged stages for column tiles and
  // 2^14 (the 2^13 shape, two blocks per SM at up to 128 registers, measured
  // 1% slower holding them), those of the fused last stage (16 per thread)
  // only for 2^14 (one 256-thread block per SM, up to 255 registers).
  static constexpr bool kHoldRoots = kPowTw && (G_ > 1 || LOGL == 14);
  static constexpr bool kHoldFused = kPowTw && kFuseLast && G_ == 1 && LOGL == 14;
};

template <class SH, class Mem>
struct SplitBody {
  static constexpr int R = SH::kR;
  static constexpr int T = SH::kTt;  // threads per transform
  static constexpr int L = SH::kL;
  static constexpr int G = SH::kG;

  // thread -> (transform g, thread t within it); G adjacent lanes share a row
  GB_HD static void coords(int tid, int& g, int& t) {
    if (G == 1) { g = 0; t = tid; }
    else { t = tid / G; g = tid - t * G; }
  }
  // Half-buffer slot of element a (rebased into [0, L/2)) of transform g.
  GB_HD static int hslot(int a, int g) {
    const int s = a * G + g;
    return s + (s >> 4);
  }
  // Slot of element base + d given the slot of base: for G = 1 the constant
  // offset of fft_core.h's derivation; for G > 1 constant when d*G is a
  // multiple of 16, else recomputed.
  template <int D>
  GB_HD static int hslot_plus(int sb, int base, int g, int i) {
    if constexpr (G == 1 || (D * G) % 16 == 0) return sb + pad_off(i * D * G);
    else return hslot(base + i * D, g);
  }

  // ---------------------------------------------- stage 0 from staging -----
  // `st` holds the tile: element a of transform g at st[a*G + g] (columns),
  // or at st[g*(L + kRowPad) + a] (rows).
  template <bool SWAP>
  GB_HD static void first(cf (&v)[R], const cf* st, int tid) {
    constexpr int RR = SH::radix(0);
    constexpr int NB = R / RR;
    constexpr int stride = L / RR;
    int g, t;
    coords(tid, g, t);
GB_UNROLL
    for (int q = 0; q < NB; ++q) {
      const int jb = q * T + t;
GB_UNROLL
      for (int i = 0; i < RR; ++i) {
        const int a = jb + i * stride;
        cf x = Mem::lds(st, SH::kRowsIn ? g * (L + SH::kRowPad) + a : a * G + g);
        v[q * RR + i] = SWAP ? mk(x.y, x.x) : x;
      }
      dft_radix<RR>(v + q * RR);
    }
  }

  // ---------------------------------- exchange after stage S, round H -----
  // Write the butterflies of stage S whose outputs lie in half H.
  template <int S, int H>
  GB_HD static void write_half(const cf (&v)[R], cf* x, int tid) {
    constexpr int RR = SH::radix(S);
    constexpr int NB = R / RR;
    constexpr int Ns = SH::ns_before(S);
    int g, t;
    coords(tid, g, t);
GB_UNROLL
    for (int q = H * (NB / 2); q < (H + 1) * (NB / 2); ++q) {
      const int jb = q * T + t;
      const int k = jb & (Ns - 1);
      const int base = (jb - k) * RR + k - H * (L / 2);  // rebased into the half buffer
      const int sb = hslot(base, g);
GB_UNROLL
      for (int i = 0; i < RR; ++i)
        Mem::sts(x, hslot_plus<Ns>(sb, base, g, i), v[q * RR + i]);
    }
  }

  // Read, for stage S+1, this thread's elements that lie in half H into the
  // register slots [H*R/2, (H+1)*R/2).
  template <int S, int H>
  GB_HD static void read_half(cf (&v)[R], const cf* x, int tid) {
    constexpr int RR = SH::radix(S + 1);
    constexpr int NB = R / RR;
    constexpr int stride = L / RR;
    constexpr int HR = RR / 2;
    int g, t;
    coords(tid, g, t);
GB_UNROLL
    for (int q = 0; q < NB; ++q) {
      const int jb = q * T + t;
      const int sb = hslot(jb, g);
GB_UNROLL
      for (int i = 0; i < HR; ++i)
        v[H * (R / 2) + q * HR + i] = Mem::lds(x, sb + pad_off(i * stride * G));
    }
  }

  // This thread's twiddle roots: for the stage after exchange S (S <
  // kExchanges) and for the fused last stage.
  template <int S>
  static constexpr int nb_after() { return S < SH::kExchanges ? R / SH::radix(S + 1) : 1; }
  struct Roots {
    cf r0[nb_after<0>()], r1[nb_after<1>()], r2[nb_after<2>()];
    cf fr[16];
  };
  template <int S>
  GB_HD static auto roots_of(Roots& x) -> cf (&)[nb_after<S>()] {
    if constexpr (S == 0) return x.r0;
    else if constexpr (S == 1) return x.r1;
    else return x.r2;
  }

  // Twiddle roots w_{RR*Ns}^k of this thread's butterflies in stage S+1
  // (SH::kPowTw), loaded before the exchange that precedes the stage so that
  // the exchange hides their latency (or once per kernel, SH::kHoldRoots).
  template <int S>
  GB_HD static void roots(cf (&r)[R / SH::radix(S + 1)], const PassDesc& d, int tid) {
    constexpr int s = S + 1;
    constexpr int NB = R / SH::radix(s);
    constexpr int Ns = SH::ns_before(s);
    int g, t;
    coords(tid, g, t);
GB_UNROLL
    for (int q = 0; q < NB; ++q)
      r[q] = Mem::ldtw(d.tw + d.tw_off[s] + ((q * T + t) & (Ns - 1)) + Ns);
  }

  // Stage S+1 after both rounds: undo the slot renaming, twiddle, DFT.
  // `r`: the roots<S>() of this thread (used when SH::kPowTw).
  template <int S>
  GB_HD static void compute(cf (&v)[R], const PassDesc& d, int tid,
                            const cf (&r)[R / SH::radix(S + 1)]) {
    constexpr int s = S + 1;
    constexpr int RR = SH::radix(s);
    constexpr int NB = R / RR;
    constexpr int HR = RR / 2;
    constexpr int Ns = SH::ns_before(s);
    int g, t;
    coords(tid, g, t);
    cf w[R];
GB_UNROLL
    for (int q = 0; q < NB; ++q)
GB_UNROLL
      for (int i = 0; i < RR; ++i)
        w[q * RR + i] = i < HR ? v[q * HR + i] : v[R / 2 + q * HR + (i - HR)];
GB_UNROLL
    for (int q = 0; q < NB; ++q) {
      const int jb = q * T + t;
      const int k = jb & (Ns - 1);
      const cf* tw = d.tw + d.tw_off[s] + k;
      // kPowTw: one table load of w_{RR*Ns}^k per butterfly (r[q]), its
      // powers by products (at most four roundings)
      cf pw[RR];
      if (SH::kPowTw) {
        pw[1] = r[q];
GB_UNROLL
        for (int i = 2; i < RR; ++i) pw[i] = cmul(pw[i / 2], pw[i - i / 2]);
      }
GB_UNROLL
      for (int i = 1; i < RR; ++i)
        w[q * RR + i] = cmul(w[q * RR + i], SH::kPowTw ? pw[i] : Mem::ldtw(tw + i * Ns));
      dft_radix<RR>(w + q * RR);
    }
GB_UNROLL
    for (int i = 0; i < R; ++i) v[i] = w[i];
  }

  // ------------------------------------------------ output of element pos --
  // Tile output base `o`; element pos of transform g at o + pos (G = 1) or
  // o + g*out.g + pos*out.e (column tiles), times the four-step twiddle
  // w_N^{col * pos} of column col = col0 + g when SH::kEpi != 0.
  // `og` = o for G = 1, else this thread's column o + g*out.g; offsets in
  // 32 bits (pos * out.e < 2^31 for every frame the planner emits).
  // (kEpi == 4 is applied by the caller, which knows the butterfly structure)
  template <bool SWAP>
  GB_HD static cf out_value(const PassDesc& d, int col, int pos, cf x) {
    if constexpr (SH::kEpi == 2) {
      x = cmul(x, Mem::ldtw(d.epi_lo + col + pos * (int)d.count_inner));  // < N <= 2^24
    } else if constexpr (SH::kEpi == 3) {
      x = cmul(x, Mem::rotor(col * pos, d.epi_logN));  // < N <= 2^24
    }
    return SWAP ? mk(x.y, x.x) : x;
  }
  template <bool SWAP>
  GB_HD static void put(const PassDesc& d, cf* og, int col, int pos, cf x) {
    x = out_value<SWAP>(d, col, pos, x);
    if constexpr (G == 1) Mem::stg(og, pos, x);
    else Mem::stg(og, pos * (int)d.out.e, x);
  }
  GB_HD static cf* column_out(const PassDesc& d, cf* o, int g) {
    return G == 1 ? o : o + g * d.out.g;
  }

  // ---------------------------- fast convolution: between the two rounds --
  // After round 1 (the forward stages; with SH::kFuseLast the last one is
  // computed here) this thread holds the spectrum at positions t + m*T,
  // m < R.  Each value is multiplied by h_scale * H[position] and swapped
  // (re <-> im), and round 2's stage 0 (radix 16), whose butterfly q reads
  // positions t + (q + i*NB)*T, runs on the registers: no exchange between
  // the rounds.  `line`: the tile (contiguous lines) or its first column
  // (column tiles: line line + g for transform g) selects the filter
  // (PassDesc::h_lines).  `fst` (column tiles whose filters are staged,
  // PassDesc::tmap_h_ok): the tile's filters in shared memory like the data
  // (position a of column g at a*G + g); else (null) the filter is read from
  // global memory.
  GB_HD static void conv_middle(cf (&v)[R], const PassDesc& d, int64_t line, int tid,
                                const cf* fst = nullptr) {
    constexpr int NB = SH::kNB;
    static_assert(SH::radix(0) == 16, "round 2 starts with a radix-16 stage");
    static_assert(G == 1 || !SH::kFuseLast, "column tiles end with a radix-16 stage");
    int g, t;
    coords(tid, g, t);
    cf y[R];  // y[m]: spectrum at position t + m*T
    if constexpr (SH::kFuseLast) {
      constexpr int s = SH::kNst - 1;
      constexpr int Ns = L / NB;
      const cf* tw = d.tw + d.tw_off[s];
GB_UNROLL
      for (int i = 0; i < 16; ++i) {
        const int p = t + i * T;
        cf x[NB];
        x[0] = v[i];
GB_UNROLL
        for (int q = 1; q < NB; ++q) x[q] = cmul(v[q * 16 + i], Mem::ldtw(tw + q * Ns + p));
        dft_radix<NB>(x);
GB_UNROLL
        for (int q = 0; q < NB; ++q) y[i + 16 * q] = x[q];  // position p + q*L/NB
      }
    } else {
      // last stage radix 16, Ns = L/16: output i of butterfly q*T + t is at
      // t + (q + i*NB)*T
GB_UNROLL
      for (int q = 0; q < NB; ++q)
GB_UNROLL
        for (int i = 0; i < 16; ++i) y[q + i * NB] = v[q * 16 + i];
    }
    const float sc = d.h_scale;
    if (fst) {
GB_UNROLL
      for (int m = 0; m < R; ++m) {
        const cf z = cmul(y[m], Mem::lds(fst, (t + m * T) * G + g));
        y[m] = mk(z.y * sc, z.x * sc);
      }
    } else {
      // contiguous lines: line u's filter at h + u * L; column tiles: column
      // u's at h + u * in.g, element a at a * in.e (a shared filter: h + a)
      const cf* h = d.h;
      int64_t he = 1;
      if (d.h_lines > 1) {
        h += ((d.h_first + line + g) % d.h_lines) * (G == 1 ? (int64_t)L : d.in.g);
        he = G == 1 ? 1 : d.in.e;
      }
GB_UNROLL
      for (int m = 0; m < R; ++m) {
        const cf z = cmul(y[m], Mem::ldtw(h + (int64_t)(t + m * T) * he));
        y[m] = mk(z.y * sc, z.x * sc);
      }
    }
GB_UNROLL
    for (int q = 0; q < NB; ++q) {
GB_UNROLL
      for (int i = 0; i < 16; ++i) v[q * 16 + i] = y[q + i * NB];
      dft_radix<16>(v + q * 16);
    }
  }

  // ------------ fused last stage (radix NB) + store (SH::kFuseLast) ------
  // v[q*16 + i] holds output i of butterfly q of stage nst-2, i.e. element
  // p + q*Ns with p = t + i*T and Ns = L/NB.  The last stage's butterfly p
  // multiplies input q by w_L^{q p} (row q of the i-major table), takes a
  // length-NB DFT and writes output q to p + q*Ns.
  // Roots w_L^p of the fused last stage's butterflies p = t + i*T (i < 16),
  // loaded before the last exchange like roots<S>() (SH::kPrefetchFused).
  GB_HD static void fused_roots(cf (&fr)[16], const PassDesc& d, int tid) {
    constexpr int Ns = L / SH::kNB;
    int g, t;
    coords(tid, g, t);
    const cf* tw = d.tw + d.tw_off[SH::kNst - 1] + Ns + t;
GB_UNROLL
    for (int i = 0; i < 16; ++i) fr[i] = Mem::ldtw(tw + i * T);
  }

  // FR_READY: fr holds the roots (fused_roots ran); else each is loaded here.
  template <bool SWAP, bool FR_READY = SH::kPrefetchFused>
  GB_HD static void store_fused(const cf (&v)[R], const PassDesc& d, cf* o, int64_t col0,
                                int tid, const cf (&fr)[16]) {
    static_assert(SH::kEpi != 4, "the factored twiddle needs the plain last stage");
    constexpr int s = SH::kNst - 1;
    constexpr int NB = SH::kNB;
    constexpr int Ns = L / NB;
    int g, t;
    coords(tid, g, t);
    cf* og = column_out(d, o, g);
    const cf* tw = d.tw + d.tw_off[s];
GB_UNROLL
    for (int i = 0; i < 16; ++i) {
      const int p = t + i * T;
      cf x[NB], pw[NB];
      x[0] = v[i];
      if (SH::kPowTw) {  // w_L^{q p} = (w_L^p)^q
        pw[1] = FR_READY ? fr[i] : Mem::ldtw(tw + Ns + p);
GB_UNROLL
        for (int q = 2; q < NB; ++q) pw[q] = cmul(pw[q / 2], pw[q - q / 2]);
      }
GB_UNROLL
      for (int q = 1; q < NB; ++q)
        x[q] = cmul(v[q * 16 + i], SH::kPowTw ? pw[q] : Mem::ldtw(tw + q * Ns + p));
      dft_radix<NB>(x);
GB_UNROLL
      for (int q = 0; q < NB; ++q) put<SWAP>(d, og, (int)col0 + g, p + q * Ns, x[q]);
    }
  }

  // ------------------------------------------------ last stage to global --
  // Outputs i in [I0, I1) of each of this thread's last-stage butterflies
  // (positions jb + i*Ns), passed as emit(g, pos, value) with the four-step
  // twiddle and the swap applied.
  template <bool SWAP, int I0, int I1, class Emit>
  GB_HD static void store_range(const cf (&v)[R], const PassDesc& d, int64_t col0, int tid,
                                Emit emit) {
    constexpr int s = SH::kNst - 1;
    constexpr int RR = SH::radix(s);
    constexpr int NB = R / RR;
    constexpr int Ns = SH::ns_before(s);
    int g, t;
    coords(tid, g, t);
    const int col = (int)col0 + g;
    // factored four-step twiddle: with jb = t + q T,
    //   w_N^{col (jb + i Ns)} = w_N^{col t} (w_N^{col T})^q (w_N^{col Ns})^i:
    // three sincospi per call (the first two and the step of the third), the
    // rest by products (a butterfly's base after at most NB - 1 of them)
    cf pw[RR], base = mk(1.f, 0.f), qstep = mk(1.f, 0.f);
    if constexpr (SH::kEpi == 4) {
      pw[0] = mk(1.f, 0.f);
      pw[1] = Mem::rotor(col * (int64_t)Ns, d.epi_logN);  // col*Ns < N
GB_UNROLL
      for (int i = 2; i < RR; ++i) pw[i] = cmul(pw[i / 2], pw[i - i / 2]);
      base = Mem::rotor(col * (int64_t)t, d.epi_logN);  // col*t < N
      if (NB > 1) qstep = Mem::rotor(col * (int64_t)T, d.epi_logN);  // col*T < N
    }
GB_UNROLL
    for (int q = 0; q < NB; ++q) {
      const int jb = q * T + t;
      if (SH::kEpi == 4 && q > 0) base = cmul(base, qstep);
GB_UNROLL
      for (int i = I0; i < I1; ++i) {
        cf x = v[q * RR + i];
        if constexpr (SH::kEpi == 4) x = cmul(x, i == 0 ? base : cmul(base, pw[i]));
        emit(g, jb + i * Ns, out_value<SWAP>(d, col, jb + i * Ns, x));
      }
    }
  }

  template <bool SWAP>
  GB_HD static void store(const cf (&v)[R], const PassDesc& d, cf* o, int64_t col0, int tid) {
    constexpr int RR = SH::radix(SH::kNst - 1);
    int g, t;
    coords(tid, g, t);
    cf* og = column_out(d, o, g);
    store_range<SWAP, 0, RR>(v, d, col0, tid, [&](int, int pos, cf x) {
      if constexpr (G == 1) Mem::stg(og, pos, x);
      else Mem::stg(og, pos * (int)d.out.e, x);
    });
  }

  // Column tiles, half H of the output rows, [H*L/2, (H+1)*L/2): outputs i
  // in [H*RR/2, (H+1)*RR/2) of every butterfly, since the last stage writes
  // jb + i*Ns with jb < Ns = L/RR.  store_half_smem puts them in xs in the
  // layout of a tensor-map box, row a of column g at (a - H*L/2)*G + g (a
  // warp's lanes -- adjacent columns, then adjacent rows -- write consecutive
  // slots: no bank conflicts); store_half writes them to global memory.
  template <bool SWAP, int H>
  GB_HD static void store_half_smem(const cf (&v)[R], const PassDesc& d, cf* xs, int64_t col0,
                                    int tid) {
    static_assert(G > 1, "column tiles only");
    constexpr int RR = SH::radix(SH::kNst - 1);
    store_range<SWAP, H * RR / 2, (H + 1) * RR / 2>(v, d, col0, tid, [&](int g, int pos, cf x) {
      Mem::sts(xs, (pos - H * (L / 2)) * G + g, x);
    });
  }
  template <bool SWAP, int H>
  GB_HD static void store_half(const cf (&v)[R], const PassDesc& d, cf* o, int64_t col0,
                               int tid) {
    static_assert(G > 1, "column tiles only");
    constexpr int RR = SH::radix(SH::kNst - 1);
    int g, t;
    coords(tid, g, t);
    cf* og = column_out(d, o, g);
    store_range<SWAP, H * RR / 2, (H + 1) * RR / 2>(v, d, col0, tid, [&](int, int pos, cf x) {
      Mem::stg(og, pos * (int)d.out.e, x);
    });
  }
};

// Shared-memory bytes of a staged pass: staging (whole tile) + half
// exchange buffer + one 8-byte mbarrier.
template <class SH>
constexpr int split_smem_bytes() {
  return SH::kStageElems * 8 + SH::kHalfSlots * 8 + 16;
}

}  // namespace gbfft
