// Tensor-core class on the 5th-generation tensor cores (tcgen05): index
// arithmetic and operand layouts of the UMMA Stockham stages.  Host/device
// code, so the CPU replay checks every address the kernel computes.
//
// A transform of length L = r0 * 16^n (r0 in {1, 2, 4, 8}, 16 <= L <= 2^14)
// runs as an optional radix-r0 first stage in FP32 registers while the tile
// is loaded, then n radix-16 stages (Sec. 2.1 mixed radix; Sec. 3.2 radix
// clustering), each a dense 16-point DFT matmul on the tensor cores:
//
//   D[m][2o + c'] = sum_{i, c} A[m][2i + c] * B[2i + c][2o + c']
//
// A row m is the twiddled input of one butterfly as 16 complex values
// (re, im interleaved along K = 32, FP16 or BF16), B the real 32 x 32 block
// form of the 16-point DFT matrix, D the butterfly's 16 outputs (re, im
// interleaved along N = 32) accumulated in FP32 in tensor memory.  One UMMA
// instruction (M = 128, N = 32, K = 16) covers 128 butterflies and half of
// K; a tile of T = max(L, 4096) elements has T / 16 butterflies per stage, so
// T / 2048 row blocks of 128.
//
// Operands sit in shared memory in the K-major layout with the 64-byte
// swizzle: rows of 64 bytes (32 16-bit values), the 16-byte chunk c of row m
// stored at chunk c ^ ((m >> 1) & 3), eight-row groups 512 bytes apart.  The
// byte offset of complex input i of row m is then
//
//   aoff(m, i) = 64 m + 16 ((i >> 2) ^ ((m >> 1) & 3)) + 4 (i & 3),
//
// a linear map over GF(2) of the bits of (m, i): a thread computes its own
// part once and XORs a compile-time constant per element.
//
// Which butterfly each A row holds is a per-stage bit permutation of the row
// index (umma_perm_code).  Tensor memory hands row m of D to lane m % 32 of warp
// quadrant (m / 32) % 4, so the permutation decides which outputs the lanes of
// a warp hold together; the tables were chosen so that the 32 lanes' 4-byte
// stores of one output into the next stage's A operand fall into 32 (at worst
// 16) distinct shared-memory banks.  The last stage keeps the natural order so
// that lanes store consecutive output elements to global memory.
#pragma once
#include <stdint.h>
#include <string.h>

#include "fft_core.h"
#include "tc_stage.h"

namespace gbfft {

// umma_perm_code(L, t): bit k of the A row index of tensor-core stage t holds
// bit nibble_k of the butterfly index u = tr * (L/16) + jb (tr: transform
// within the tile, jb: butterfly within the transform).
GB_HD constexpr uint64_t umma_perm_code(int logL, int t) {
  // nibble k = butterfly-index bit held by row bit k
  if (logL == 4) return t == 0 ? 0x76543210ull : 0;
  if (logL == 5) return t == 0 ? 0x76543210ull : 0;
  if (logL == 6) return t == 0 ? 0x76543210ull : 0;
  if (logL == 7) return t == 0 ? 0x76543210ull : 0;
  if (logL == 8) return t == 0 ? 0x76543210ull : t == 1 ? 0x76543210ull : 0;
  if (logL == 9) return t == 0 ? 0x76543201ull : t == 1 ? 0x76543210ull : 0;
  if (logL == 10) return t == 0 ? 0x76451302ull : t == 1 ? 0x76543210ull : 0;
  if (logL == 11) return t == 0 ? 0x76542310ull : t == 1 ? 0x76543210ull : 0;
  if (logL == 12) return t == 0 ? 0x76354210ull : t == 1 ? 0x73120654ull : t == 2 ? 0x76543210ull : 0;
  if (logL == 13) return t == 0 ? 0x843276510ull : t == 1 ? 0x874362510ull : t == 2 ? 0x876543210ull : 0;
  if (logL == 14) return t == 0 ? 0x9854376210ull : t == 1 ? 0x9854372610ull : t == 2 ? 0x9876543210ull : 0;
  return 0;
}

// umma_load_lanes_code(L): nibble k is the bit of the loader's work item that
// lane bit k selects.  Work items are tile elements (r0 = 1) or first-stage
// butterflies (r0 > 1); bits 0 and 1 are always lane bits, so every 32-byte
// sector a warp load touches is used whole.
GB_HD constexpr uint32_t umma_load_lanes_code(int logL) {
  // nibble k = bit of the loader's work item selected by lane bit k
  if (logL == 4) return 0x43210u;
  if (logL == 5) return 0x43210u;
  if (logL == 6) return 0x43210u;
  if (logL == 7) return 0x43210u;
  if (logL == 8) return 0x54210u;
  if (logL == 9) return 0x65410u;
  if (logL == 10) return 0x65410u;
  if (logL == 11) return 0x65410u;
  if (logL == 12) return 0x98210u;
  if (logL == 13) return 0x98410u;
  if (logL == 14) return 0xa9810u;
  return 0;
}

// Warps of a tcgen05 block for length 2^logL: 8, and 16 at 2^14, whose 256
// tensor-memory columns per block leave room for two blocks per SM only (16
// warps there would leave an SM with half the warps of the shorter lengths).
GB_HD constexpr int umma_warps(int logL) { return logL == 14 ? 16 : 8; }

// Shared-memory bytes of the staging buffer of a tcgen05 CTA (elements of
// eb bytes): tiles of 4096 elements (L <= 2^12) are copied into shared memory
// by one bulk copy while the previous tile is computed, and the loader reads
// them from there; 128 bytes of alignment and the copy's mbarrier included.
// Longer transforms (tiles of L elements, 64 or 128 KB) and the split class
// (two A operands; with the buffer three CTAs fit an SM instead of four,
// measured slower) load from global memory.
GB_HD constexpr int umma_staging_bytes(int logL, int eb, bool split) {
  return logL <= 12 && !split ? 128 + 4096 * eb + 16 : 0;
}

template <int LOGL>
struct UmmaGeo {
  static_assert(LOGL >= 4 && LOGL <= 14, "tensor-core lengths are 2^4 .. 2^14");
  static constexpr int L = 1 << LOGL;
  static constexpr int R0B = LOGL % 4;               // log2 of the FP32 first-stage radix
  static constexpr int R0 = 1 << R0B;
  static constexpr int NTC = LOGL / 4;               // radix-16 tensor-core stages
  static constexpr int LOGT = LOGL > 12 ? LOGL : 12;  // tile of 2^LOGT elements
  static constexpr int T = 1 << LOGT;
  static constexpr int ROWB = LOGT - 4;              // log2 of butterflies per stage per tile
  static constexpr int ROWS = 1 << ROWB;
  static constexpr int RB = ROWS / 128;              // row blocks (one UMMA M = 128 each)
  static constexpr int BPSB = LOGL - 4;              // log2 butterflies per transform and stage
  static constexpr int TPT = T / L;                  // transforms per tile
  static constexpr int TMEM_COLS = 32 * RB;          // FP32 accumulator columns
  static constexpr int A_BYTES = ROWS * 64;          // one A operand (16-bit values)
  static constexpr int B_BYTES = 32 * 64;            // one 32 x 32 B operand
  // loader work items: tile elements, or first-stage butterflies
  static constexpr int ITEMS = R0B ? T / R0 : T;
  static constexpr int NWARP = umma_warps(LOGL);
  static constexpr int THREADS = 32 * NWARP;
  static constexpr int ITEMS_PER_THREAD = ITEMS / THREADS;
  // log2 of Ns before tensor-core stage t (the radices of earlier stages multiplied)
  GB_HD static constexpr int ns_log(int t) { return R0B + 4 * t; }
};

// Bit permutation of the A rows of stage t: row -> butterfly, butterfly -> row.
template <int LOGL>
GB_HD int umma_u_of_row(int t, int m) {
  int u = 0;
  const uint64_t c = umma_perm_code(LOGL, t);
GB_UNROLL
  for (int k = 0; k < UmmaGeo<LOGL>::ROWB; ++k) u |= ((m >> k) & 1) << ((c >> (4 * k)) & 15);
  return u;
}
template <int LOGL>
GB_HD int umma_row_of_u(int t, int u) {
  int m = 0;
  const uint64_t c = umma_perm_code(LOGL, t);
GB_UNROLL
  for (int k = 0; k < UmmaGeo<LOGL>::ROWB; ++k) m |= ((u >> ((c >> (4 * k)) & 15)) & 1) << k;
  return m;
}

GB_HD float u32_as_f32(uint32_t u) {
  float f;
  memcpy(&f, &u, 4);
  return f;
}

// Byte offset of complex element i (a pair of 16-bit values) of row m of an
// A operand, and of the 16-bit element (n, k) of a B operand stored N x K.
GB_HD uint32_t umma_aoff(int m, int i) {
  return (uint32_t)(64 * m + 16 * (((i >> 2) & 3) ^ ((m >> 1) & 3)) + 4 * (i & 3));
}
GB_HD uint32_t umma_boff(int n, int k) {
  return (uint32_t)(64 * n + 16 * (((k >> 3) & 3) ^ ((n >> 1) & 3)) + 2 * (k & 7));
}

// Value of the real 32 x 32 B matrix of the forward 16-point DFT at
// (k = 2i + c, n = 2o + c'): Y_o = sum_i x_i w16^{io}, w16 = exp(-2 pi i/16),
// with w16^{io} = cos(th) - i sin(th):
//   re Y_o += re x_i cos(th) + im x_i sin(th),  im Y_o += -re x_i sin(th) + im x_i cos(th).
// cos16 (tc_stage.h) gives the exact FP32 constants of the FP32 path.
GB_HD float umma_dft_entry(int k, int n) {
  const int i = k >> 1, o = n >> 1;
  const int m = (i * o) & 15;
  const float c = cos16(m), s = -cos16(m + 4);  // cos(th), sin(th)
  const bool kre = (k & 1) == 0, nre = (n & 1) == 0;
  if (kre && nre) return c;
  if (!kre && nre) return s;
  if (kre && !nre) return -s;
  return c;
}

// Position within its transform of output o of butterfly jb of a stage whose
// earlier radices multiply to Ns = 2^s (Stockham: (jb - k)*16 + k + o*Ns with
// k = jb mod Ns), written with disjoint bit fields.
GB_HD int umma_out_pos(int s, int jb, int o) {
  return ((jb >> s) << (s + 4)) | (o << s) | (jb & ((1 << s) - 1));
}

// Where output o of butterfly u of tensor-core stage t goes: butterfly u2 and
// input i2 of stage t + 1, and the index of its twiddle w_{16 Ns'}^{i2 k2} in
// that stage's table (entry i2 * Ns' + k2, k2 = jb2 mod Ns').  All three are
// linear in the bits of (u, o) with the parts of u and of o on disjoint bits.
template <int LOGL>
GB_HD void umma_next(int t, int u, int o, int& u2, int& i2, int& tw) {
  using G = UmmaGeo<LOGL>;
  const int tr = u >> G::BPSB, jb = u & ((1 << G::BPSB) - 1);
  const int p = umma_out_pos(G::ns_log(t), jb, o);
  const int jb2 = p & ((1 << G::BPSB) - 1);
  i2 = p >> G::BPSB;
  u2 = (tr << G::BPSB) | jb2;
  const int s2 = G::ns_log(t + 1);
  tw = (i2 << s2) | (jb2 & ((1 << s2) - 1));
}

// Work item e of the loader: the tile element (r0 = 1) or the first-stage
// butterfly (r0 > 1) that lane bits and (warp, iteration) bits select.
template <int LOGL>
GB_HD int umma_load_item(int lane, int rest) {
  int e = 0, r = rest;
  int pos = 0;
  constexpr uint32_t c = umma_load_lanes_code(LOGL);
GB_UNROLL
  for (int b = 0; (1 << b) < UmmaGeo<LOGL>::ITEMS; ++b) {
    int k = -1;
GB_UNROLL
    for (int j = 0; j < 5; ++j)
      if ((int)((c >> (4 * j)) & 15) == b) k = j;
    if (k >= 0) {
      e |= ((lane >> k) & 1) << b;
    } else {
      e |= ((r >> pos) & 1) << b;
      ++pos;
    }
  }
  return e;
}

// Stage-0 input of a loaded element (r0 = 1): tile element e -> butterfly u,
// input i (position pos = jb + i * L/16 of transform tr).
template <int LOGL>
GB_HD void umma_load_target(int e, int& u, int& i) {
  using G = UmmaGeo<LOGL>;
  const int tr = e >> LOGL, pos = e & (G::L - 1);
  u = (tr << G::BPSB) | (pos & ((1 << G::BPSB) - 1));
  i = pos >> G::BPSB;
}

// r0 > 1: output o of first-stage butterfly e (transform tr, jb0 < L/r0, which
// read elements jb0 + q * L/r0, q < r0) -> butterfly u, input i of
// tensor-core stage 0 and its twiddle index (entry i * r0 + (jb mod r0)).
template <int LOGL>
GB_HD void umma_first_target(int e, int o, int& u, int& i, int& tw) {
  using G = UmmaGeo<LOGL>;
  const int tr = e >> (LOGL - G::R0B), jb0 = e & ((1 << (LOGL - G::R0B)) - 1);
  const int p = (jb0 << G::R0B) | o;
  const int jb = p & ((1 << G::BPSB) - 1);
  i = p >> G::BPSB;
  u = (tr << G::BPSB) | jb;
  tw = (i << G::R0B) | (jb & (G::R0 - 1));
}

// ------------------------------------------------------- per-thread body --
// The kernel's per-thread steps, shared with the CPU replay through the memory
// policy Mem: at (a base pointer advanced by elements), ldg_sw / stg_sw (global
// element loads and stores, real and imaginary parts swapped when asked),
// ldtw (twiddle table), sts32 (a 32-bit store at a byte address of the A
// operands) and kHalfIO (complex32 storage).  a_hi / a_lo are the byte
// addresses of the two A operands (a_lo only for the split class).
template <int LOGL, int PREC, class Mem>
struct UmmaBody {
  using G = UmmaGeo<LOGL>;
  static constexpr int P = PREC == TC_BF16X3 ? TC_BF16 : PREC;
  static constexpr bool SPLIT = PREC == TC_BF16X3;
  // first twiddle table of the tensor-core stages in the pass schedule
  static constexpr int ST0 = G::R0B ? 1 : 0;
  // FP16: each tensor-core stage's input is scaled by the exact 1/16 so that
  // the 16-point sums stay in the FP16 range; the scales are undone at the
  // end.  The loader skips its scale for complex32 input without an FP32
  // first stage (the input is FP16 already); the later stages' scales ride on
  // their twiddles.
  static constexpr bool LOAD_SCALE = P == TC_FP16 && !(Mem::kHalfIO && G::R0B == 0);
  static constexpr int SCALED_STAGES = P == TC_FP16 ? G::NTC - 1 + (LOAD_SCALE ? 1 : 0) : 0;

  // Rounds the stage input v to 16 bits (scaled by 1/16 first when SCALE)
  // and stores it at byte offset `off` of the A operand; for the split class
  // the rounding error goes to a_lo.
  template <bool SCALE>
  GB_HD static void put_a(uint32_t a_hi, uint32_t a_lo, uint32_t off, cf v) {
    if (SCALE) v = mk(v.x * 0.0625f, v.y * 0.0625f);
    const uint32_t h = pack_rn<P>(v.x, v.y);
    Mem::sts32(a_hi + off, h);
    if (SPLIT) Mem::sts32(a_lo + off, pack_rn<P>(v.x - lo16_to_f32<P>(h), v.y - hi16_to_f32<P>(h)));
  }

  // The loader: every work item of thread (warp, lane) -- tile elements
  // (r0 = 1), or radix-r0 first-stage butterflies computed in FP32 -- into
  // the stage-0 A operand.  `valid` transforms of the tile are read; the rest
  // are zeros.  Item e = e_t | e_b | e_j: e_t from (lane, warp), e_b from the
  // block of CH items, e_j from the item within the block.  Every index below
  // (element, A row and offset, twiddle) is linear in the bits of e, so it is
  // the thread's part of the block (BlockPart) and a compile-time constant,
  // XORed (or added: element offsets have disjoint bits).
  static constexpr int CH = G::ITEMS_PER_THREAD < 8 ? G::ITEMS_PER_THREAD : 8;
  static constexpr int KB = G::ITEMS_PER_THREAD / CH;
  GB_HD static int elem_of(int e) {  // first element of first-stage butterfly e
    return G::R0B ? ((e >> (LOGL - G::R0B)) << LOGL) | (e & ((1 << (LOGL - G::R0B)) - 1)) : e;
  }
  GB_HD static int tr_of(int e) { return e >> (LOGL - G::R0B); }
  GB_HD static uint32_t off_of(int e) {  // r0 = 1: A-operand offset of tile element e
    int u, i;
    umma_load_target<LOGL>(e, u, i);
    return umma_aoff(umma_row_of_u<LOGL>(0, u), i);
  }
  GB_HD static void first_of(int e, int o, uint32_t& off, int& i, int& tw) {  // r0 > 1
    int u;
    umma_first_target<LOGL>(e, o, u, i, tw);
    off = umma_aoff(umma_row_of_u<LOGL>(0, u), i);
  }

  // The parts of block b of CH items of the thread whose item part is et
  // (umma_load_item(lane, warp)): first item, its first element, A offset
  // and (r0 > 1) stage-0 input and twiddle index.  They do not depend on the
  // tile, so a kernel may compute them once and keep them.
  struct BlockPart {
    int eb, xb;
    uint32_t offb;
    int ib, twb;
  };
  GB_HD static BlockPart block_part_of(int et, int b) {
    BlockPart p{};
    p.eb = et | umma_load_item<LOGL>(0, b * CH * G::NWARP);
    p.xb = elem_of(p.eb);
    if (G::R0B == 0) p.offb = off_of(p.eb);
    else first_of(p.eb, 0, p.offb, p.ib, p.twb);
    return p;
  }

  // FULL: every transform of the tile is valid (no per-item check).
  // parts(b) gives the thread's BlockPart of block b.
  template <bool FULL, class Parts>
  GB_HD static void load_tile(const PassDesc& d, const cf* gin, int valid, uint32_t a_hi,
                              uint32_t a_lo, const Parts& parts) {
    const bool swap = d.conj_in != 0;
#pragma unroll 1
    for (int b = 0; b < KB; ++b) {
      const BlockPart bp = parts(b);
      const cf* gb = Mem::at(gin, bp.xb);
      if constexpr (Mem::kHalfIO && !LOAD_SCALE && P == TC_FP16 && !SPLIT && G::R0B == 0) {
        // complex32 into an FP16 operand, unscaled: the loaded pair is the
        // operand's pair (swapped for the inverse), no conversion
        uint32_t h[CH];
GB_UNROLL
        for (int j = 0; j < CH; ++j) {
          const int ej = umma_load_item<LOGL>(0, j * G::NWARP);
          h[j] = FULL || tr_of(bp.eb | ej) < valid ? Mem::ldg_pair(gb, ej, swap) : 0u;
        }
GB_UNROLL
        for (int j = 0; j < CH; ++j)
          Mem::sts32(a_hi + (bp.offb ^ off_of(umma_load_item<LOGL>(0, j * G::NWARP))), h[j]);
      } else if (G::R0B == 0) {
        cf v[CH];
GB_UNROLL
        for (int j = 0; j < CH; ++j) {
          const int ej = umma_load_item<LOGL>(0, j * G::NWARP);
          v[j] = FULL || tr_of(bp.eb | ej) < valid ? Mem::ldg_sw(gb, ej, swap) : mk(0.f, 0.f);
        }
GB_UNROLL
        for (int j = 0; j < CH; ++j)
          put_a<LOAD_SCALE>(a_hi, a_lo, bp.offb ^ off_of(umma_load_item<LOGL>(0, j * G::NWARP)), v[j]);
      } else {
        const cf* tw = d.tw + d.tw_off[1];
GB_UNROLL
        for (int j = 0; j < CH; ++j) {
          const int ej = umma_load_item<LOGL>(0, j * G::NWARP);
          const bool ok = FULL || tr_of(bp.eb | ej) < valid;
          cf y[G::R0];
GB_UNROLL
          for (int q = 0; q < G::R0; ++q)
            y[q] = ok ? Mem::ldg_sw(gb, elem_of(ej) + q * (G::L / G::R0), swap) : mk(0.f, 0.f);
          if (G::R0 == 2) dft_small<2, 1>(y);
          else if (G::R0 == 4) dft_small<4, 1>(y);
          else dft_pq<2, 4>(y);
          uint32_t offj;
          int ij, twj;
          first_of(ej, 0, offj, ij, twj);
          // output o becomes input i of its stage-0 butterfly with k = o and
          // i the same for every o, so its twiddle is s^o with s = w^i: one
          // table load (entry i * r0 + 1), powers by a running product
          const int i = bp.ib ^ ij;
          const cf s1 = i > 0 ? Mem::ldtw(tw + ((bp.twb ^ twj) | 1)) : mk(1.f, 0.f);
          cf w = s1;
GB_UNROLL
          for (int o = 0; o < G::R0; ++o) {
            uint32_t offo;
            int io, two;
            first_of(0, o, offo, io, two);
            cf v = y[o];
            if (o > 0 && i > 0) {
              v = cmul(v, w);
              w = cmul(w, s1);
            }
            put_a<LOAD_SCALE>(a_hi, a_lo, bp.offb ^ offj ^ offo, v);
          }
        }
      }
    }
  }

  // The thread's part of the addressing of the butterfly in A row m of
  // tensor-core stage t (it does not depend on the tile): after the last
  // stage its output position (tr * L + the position bits that do not
  // depend on the output index); before, the next stage's A offset and
  // twiddles of its output 0.
  struct RowPart {
    int tr, pos;
    uint32_t off;
    int tw;
    cf step;  // next stages: the ratio of consecutive outputs' twiddles
    cf run;   // the twiddle of the next output to be stored (updated as outputs are)
  };
  //
  // Twiddles: output o of the butterfly becomes input i' of its next-stage
  // butterfly with k' = k + o*Ns (k = jb mod Ns) and i' independent of o
  // (the stage's outputs keep their block: (jb / Ns) * 16 Ns lies in one
  // multiple of L/16), so its twiddle w_{16 Ns'}^{i' k'} = c * s^o with
  // c = w^{i' k} and s = w^{i' Ns} = (c s) * conj(c): two table loads per
  // row, then a running product (at most 16 further roundings, ~1e-6).  For
  // FP16, c carries the next stage's exact 1/16.
  template <int t>
  GB_HD static RowPart row_part(const PassDesc& d, int m) {
    RowPart rp{};
    const int u = umma_u_of_row<LOGL>(t, m);
    if (t == G::NTC - 1) {
      rp.tr = u >> G::BPSB;
      rp.pos = (rp.tr << LOGL) | umma_out_pos(G::ns_log(t), u & ((1 << G::BPSB) - 1), 0);
    } else {
      int u2, i2;
      umma_next<LOGL>(t, u, 0, u2, i2, rp.tw);
      rp.off = umma_aoff(umma_row_of_u<LOGL>(t + 1, u2), i2);
      int u2o, i2o, two;
      umma_next<LOGL>(t, 0, 1, u2o, i2o, two);  // output 1's part of the table index
      const cf* tw = d.tw + d.tw_off[ST0 + t + 1];
      const cf c0 = Mem::ldtw(tw + rp.tw);
      const cf c1 = Mem::ldtw(tw + (rp.tw ^ two));
      rp.step = cmul(c1, cconj(c0));
      rp.run = P == TC_FP16 ? mk(c0.x * 0.0625f, c0.y * 0.0625f) : c0;
    }
    return rp;
  }

  // Outputs O0 .. O0 + NO - 1 of that butterfly (r holds their 2 NO FP32
  // values, so a thread can read its tensor-memory row in parts): stored to
  // global memory after the last stage, else twiddled, rounded and stored as
  // the next stage's A operand.  Each output's own part of the addressing is
  // a compile-time constant XORed (or added) to the row's part.
  template <int t, int O0 = 0, int NO = 16>
  GB_HD static void epilogue_part(const PassDesc& d, cf* gout, int valid, RowPart& rp,
                                  const uint32_t (&r)[2 * NO], uint32_t a_hi, uint32_t a_lo) {
    if (t == G::NTC - 1) {
      if (rp.tr >= valid) return;
      // the row's first output in the tile; output o is o << ns_log(t) further
      cf* o_base = Mem::at(gout, rp.pos);
      const bool swap = d.conj_out != 0;
GB_UNROLL
      for (int j = 0; j < NO; ++j) {
        const int o = O0 + j;
        cf v = mk(u32_as_f32(r[2 * j]), u32_as_f32(r[2 * j + 1]));
        if (SCALED_STAGES > 0) {  // undo the FP16 stages' 1/16: exact powers of two
          const float sc = (float)(1 << (4 * SCALED_STAGES));
          v = mk(v.x * sc, v.y * sc);
        }
        Mem::stg_sw(o_base, o << G::ns_log(t), v, swap);
      }
    } else {
GB_UNROLL
      for (int j = 0; j < NO; ++j) {
        const int o = O0 + j;
        int u2o, i2o, two;
        umma_next<LOGL>(t, 0, o, u2o, i2o, two);
        const uint32_t off = rp.off ^ umma_aoff(umma_row_of_u<LOGL>(t + 1, u2o), i2o);
        cf v = mk(u32_as_f32(r[2 * j]), u32_as_f32(r[2 * j + 1]));
        v = cmul(v, rp.run);               // c * s^o
        rp.run = cmul(rp.run, rp.step);
        put_a<false>(a_hi, a_lo, off, v);
      }
    }
  }
};

// UMMA shared-memory matrix descriptor (K-major, 64-byte swizzle): start
// address, leading-dimension byte offset (unused by swizzled K-major
// operands; 16), stride byte offset between eight-row groups (512), the
// descriptor version of this tensor-core generation, and the layout code.
GB_HD uint64_t umma_smem_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)(16u >> 4) << 16;
  d |= (uint64_t)(512u >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)4 << 61;
  return d;
}

// Instruction descriptor of kind::f16 with FP32 accumulation, K-major A and
// B, M = 128, N = 32; ab = 0 for FP16 operands, 1 for BF16.
GB_HD uint32_t umma_idesc(int ab) {
  return (1u << 4) | ((uint32_t)ab << 7) | ((uint32_t)ab << 10) | ((32u >> 3) << 17) |
         ((128u >> 4) << 24);
}

}  // namespace gbfft
