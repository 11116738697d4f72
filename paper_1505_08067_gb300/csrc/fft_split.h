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
#pragma once
#include "fft_core.h"
#include "fft_stage.h"

namespace gbfft {

// Compile-time shape of a staged pass; R elements (R/16 radix-16
// butterflies) per thread.
template <int LOGL, uint32_t SCHED, int NST, int R_ = 32>
struct SplitShape {
  static constexpr int kL = 1 << LOGL;
  static constexpr int kR = R_;
  static constexpr int kT = kL / kR;              // threads per transform (= per block)
  static constexpr int kHalf = kL / 2;            // exchange buffer holds half a transform
  static constexpr int kHalfSlots = kHalf + (kHalf >> 4) + 1;
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
};

template <class SH, class Mem>
struct SplitBody {
  static constexpr int R = SH::kR;
  static constexpr int T = SH::kT;
  static constexpr int L = SH::kL;

  GB_HD static int hslot(int a) { return a + (a >> 4); }  // a in [0, L/2)

  // ---------------------------------------------- stage 0 from staging -----
  // `st` holds the whole transform, unpadded (element a at st[a]).
  template <bool SWAP>
  GB_HD static void first(cf (&v)[R], const cf* st, int t) {
    constexpr int RR = SH::radix(0);
    constexpr int NB = R / RR;
    constexpr int stride = L / RR;
GB_UNROLL
    for (int q = 0; q < NB; ++q) {
      const int jb = q * T + t;
GB_UNROLL
      for (int i = 0; i < RR; ++i) {
        cf x = Mem::lds(st, jb + i * stride);
        v[q * RR + i] = SWAP ? mk(x.y, x.x) : x;
      }
      dft_radix<RR>(v + q * RR);
    }
  }

  // ---------------------------------- exchange after stage S, round H -----
  // Write the butterflies of stage S whose outputs lie in half H.
  template <int S, int H>
  GB_HD static void write_half(const cf (&v)[R], cf* x, int t) {
    constexpr int RR = SH::radix(S);
    constexpr int NB = R / RR;
    constexpr int Ns = SH::ns_before(S);
GB_UNROLL
    for (int q = H * (NB / 2); q < (H + 1) * (NB / 2); ++q) {
      const int jb = q * T + t;
      const int k = jb & (Ns - 1);
      const int base = (jb - k) * RR + k - H * (L / 2);  // rebased into the half buffer
      const int sb = hslot(base);
GB_UNROLL
      for (int i = 0; i < RR; ++i) Mem::sts(x, sb + pad_off(i * Ns), v[q * RR + i]);
    }
  }

  // Read, for stage S+1, this thread's elements that lie in half H into the
  // register slots [H*R/2, (H+1)*R/2).
  template <int S, int H>
  GB_HD static void read_half(cf (&v)[R], const cf* x, int t) {
    constexpr int RR = SH::radix(S + 1);
    constexpr int NB = R / RR;
    constexpr int stride = L / RR;
    constexpr int HR = RR / 2;
GB_UNROLL
    for (int q = 0; q < NB; ++q) {
      const int jb = q * T + t;
      const int sb = hslot(jb);
GB_UNROLL
      for (int i = 0; i < HR; ++i)
        v[H * (R / 2) + q * HR + i] = Mem::lds(x, sb + pad_off(i * stride));
    }
  }

  // Stage S+1 after both rounds: undo the slot renaming, twiddle, DFT.
  template <int S>
  GB_HD static void compute(cf (&v)[R], const PassDesc& d, int t) {
    constexpr int s = S + 1;
    constexpr int RR = SH::radix(s);
    constexpr int NB = R / RR;
    constexpr int HR = RR / 2;
    constexpr int Ns = SH::ns_before(s);
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
GB_UNROLL
      for (int i = 1; i < RR; ++i) w[q * RR + i] = cmul(w[q * RR + i], Mem::ldtw(tw + i * Ns));
      dft_radix<RR>(w + q * RR);
    }
GB_UNROLL
    for (int i = 0; i < R; ++i) v[i] = w[i];
  }

  // ------------ fused last stage (radix NB) + store (SH::kFuseLast) ------
  // v[q*16 + i] holds output i of butterfly q of stage nst-2, i.e. element
  // p + q*Ns with p = t + i*T and Ns = L/NB.  The last stage's butterfly p
  // multiplies input q by w_L^{q p} (row q of the i-major table), takes a
  // length-NB DFT and writes output q to p + q*Ns.
  template <bool SWAP>
  GB_HD static void store_fused(const cf (&v)[R], const PassDesc& d, cf* out, int t) {
    constexpr int s = SH::kNst - 1;
    constexpr int NB = SH::kNB;
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
      for (int q = 0; q < NB; ++q) Mem::stg(out, p + q * Ns, SWAP ? mk(x[q].y, x[q].x) : x[q]);
    }
  }

  // ---------------------------- fast convolution: between the two rounds --
  // After round 1 (the forward stages; with SH::kFuseLast the last one is
  // computed here) this thread holds the spectrum at positions t + m*T,
  // m < R.  Each value is multiplied by h_scale * H[position] and swapped
  // (re <-> im), and round 2's stage 0 (radix 16), whose butterfly q reads
  // positions t + (q + i*NB)*T, runs on the registers: no exchange between
  // the rounds.  `line` selects the line's filter (PassDesc::h_lines).
  GB_HD static void conv_middle(cf (&v)[R], const PassDesc& d, int64_t line, int t) {
    constexpr int NB = SH::kNB;
    static_assert(SH::radix(0) == 16, "round 2 starts with a radix-16 stage");
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
    const cf* h = d.h;
    if (d.h_lines > 1) h += ((d.h_first + line) % d.h_lines) * (int64_t)L;
    const float sc = d.h_scale;
GB_UNROLL
    for (int m = 0; m < R; ++m) {
      const cf z = cmul(y[m], Mem::ldtw(h + t + m * T));
      y[m] = mk(z.y * sc, z.x * sc);
    }
GB_UNROLL
    for (int q = 0; q < NB; ++q) {
GB_UNROLL
      for (int i = 0; i < 16; ++i) v[q * 16 + i] = y[q + i * NB];
      dft_radix<16>(v + q * 16);
    }
  }

  // ------------------------------------------------ last stage to global --
  template <bool SWAP>
  GB_HD static void store(const cf (&v)[R], cf* out, int t) {
    constexpr int s = SH::kNst - 1;
    constexpr int RR = SH::radix(s);
    constexpr int NB = R / RR;
    constexpr int Ns = SH::ns_before(s);
GB_UNROLL
    for (int q = 0; q < NB; ++q) {
      const int jb = q * T + t;
GB_UNROLL
      for (int i = 0; i < RR; ++i) {
        const cf x = v[q * RR + i];
        Mem::stg(out, jb + i * Ns, SWAP ? mk(x.y, x.x) : x);
      }
    }
  }
};

// Shared-memory bytes of a staged pass: staging (whole transform) + half
// exchange buffer + one 8-byte mbarrier.
template <class SH>
constexpr int split_smem_bytes() {
  return SH::kL * 8 + SH::kHalfSlots * 8 + 16;
}

}  // namespace gbfft
