// Tensor-core class: radix-16 Stockham stages computed as small dense DFT
// matmuls on the tensor cores (warp-level MMA m16n8k16, FP16 or BF16 inputs,
// FP32 accumulation), plus a split-BF16x3 compensated variant.  The Stockham
// data movement, the twiddles (FP32, FP64-generated tables) and the exchanges
// are those of fft_stage.h; only the length-16 DFT of each butterfly changes.
//
// One MMA group = 16 butterflies.  With x = twiddled inputs of a butterfly and
// F[o][i] = w16^{o i}, the group computes, in real block form,
//   D[b][n] = sum_k A[b][k] B[k][n]
//   A = [ x_r(b, 0..15) | x_i(b, 0..15) ]            16 x 32  (K blocks: re, im)
//   B = [[ cos  , -sin ],                               32 x 32  (N blocks: Y_r 0..7,
//        [ sin  ,  cos ]]  with entries at (i, o)                 Y_r 8..15, Y_i 0..7, Y_i 8..15)
// so D[b] = [Y_r(b, 0..15) | Y_i(b, 0..15)]: 2 K blocks x 4 N blocks = 8 MMAs.
//
// Fragment ownership (m16n8k16): lane = 4 g + t.  A rows g and g+8 (the group's
// butterflies g, g+8), A columns 2t, 2t+1, 2t+8, 2t+9 (points); D rows g, g+8,
// D columns 2t, 2t+1 of each N block (outputs 2t, 2t+1, 2t+8, 2t+9).  Each lane
// therefore loads and stores the same 8 (butterfly, point) pairs:
//   butterflies {g, g+8} x points {2t, 2t+1, 2t+8, 2t+9}.
//
// FP16 keeps values in range by scaling each stage's input by 1/16 (exact) and
// the result by 16^stages at the end.  BF16x3 splits x = x_hi + x_lo and
// F = F_hi + F_lo (each BF16) and accumulates x_hi F_hi + x_hi F_lo + x_lo F_hi.
//
// The per-lane steps are host/device code; the warp-wide MMA is PTX on the GPU
// and an explicit fragment-level emulation in the CPU test harness.
#pragma once
#include <stdint.h>
#include <string.h>

#include "fft_core.h"

namespace gbfft {

enum { TC_FP16 = 1, TC_BF16 = 2, TC_BF16X3 = 3 };

// ------------------------------------------------ 16-bit conversions (RN) --
// Round-to-nearest-even FP32 -> FP16 / BF16 bit patterns, written from the
// IEEE formats (finite inputs; overflow saturates to infinity).
GB_HD uint16_t f32_to_bf16_bits(float f) {
  uint32_t u;
  memcpy(&u, &f, 4);
  const uint32_t lsb = (u >> 16) & 1u;
  u += 0x7fffu + lsb;
  return (uint16_t)(u >> 16);
}
GB_HD float bf16_bits_to_f32(uint16_t h) {
  uint32_t u = (uint32_t)h << 16;
  float f;
  memcpy(&f, &u, 4);
  return f;
}
GB_HD uint16_t f32_to_f16_bits(float f) {
  uint32_t u;
  memcpy(&u, &f, 4);
  const uint32_t sign = (u >> 16) & 0x8000u;
  int32_t exp = (int32_t)((u >> 23) & 0xff) - 127 + 15;
  uint32_t man = u & 0x7fffffu;
  if (((u >> 23) & 0xff) == 0) return (uint16_t)sign;  // FP32 zero / denormal -> 0
  if (exp >= 31) return (uint16_t)(sign | 0x7c00u);
  if (exp <= 0) {  // FP16 subnormal
    if (exp < -10) return (uint16_t)sign;
    man |= 0x800000u;
    const int shift = 14 - exp;
    uint32_t h = man >> shift;
    const uint32_t rem = man & ((1u << shift) - 1), half = 1u << (shift - 1);
    if (rem > half || (rem == half && (h & 1u))) ++h;
    return (uint16_t)(sign | h);
  }
  uint32_t h = ((uint32_t)exp << 10) | (man >> 13);
  const uint32_t rem = man & 0x1fffu;
  if (rem > 0x1000u || (rem == 0x1000u && (h & 1u))) ++h;  // may carry into the exponent
  return (uint16_t)(sign | h);
}
GB_HD float f16_bits_to_f32(uint16_t h) {
  const uint32_t sign = (uint32_t)(h & 0x8000u) << 16;
  int exp = (h >> 10) & 0x1f;
  uint32_t man = h & 0x3ffu;
  uint32_t u;
  if (exp == 0) {
    if (man == 0) {
      u = sign;
    } else {  // subnormal: normalise
      exp = 1;
      while (!(man & 0x400u)) {
        man <<= 1;
        --exp;
      }
      man &= 0x3ffu;
      u = sign | ((uint32_t)(exp - 15 + 127) << 23) | (man << 13);
    }
  } else if (exp == 31) {
    u = sign | 0x7f800000u | (man << 13);
  } else {
    u = sign | ((uint32_t)(exp - 15 + 127) << 23) | (man << 13);
  }
  float f;
  memcpy(&f, &u, 4);
  return f;
}

template <int PREC>
GB_HD uint16_t to16(float f) {
  return PREC == TC_FP16 ? f32_to_f16_bits(f) : f32_to_bf16_bits(f);
}
template <int PREC>
GB_HD float from16(uint16_t h) {
  return PREC == TC_FP16 ? f16_bits_to_f32(h) : bf16_bits_to_f32(h);
}
GB_HD uint32_t pack2(uint16_t lo, uint16_t hi) { return (uint32_t)lo | ((uint32_t)hi << 16); }

// Two FP32 values to a packed pair of 16-bit values (round to nearest even);
// the hardware conversion on the GPU, the bit-level one on the host.
template <int PREC>
GB_HD uint32_t pack_rn(float lo, float hi) {
#ifdef __CUDA_ARCH__
  uint32_t r;
  if (PREC == TC_FP16) asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  else asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  return r;
#else
  return pack2(to16<PREC>(lo), to16<PREC>(hi));
#endif
}
template <int PREC>
GB_HD float lo16_to_f32(uint32_t r) { return from16<PREC>((uint16_t)(r & 0xffffu)); }
template <int PREC>
GB_HD float hi16_to_f32(uint32_t r) { return from16<PREC>((uint16_t)(r >> 16)); }

// ----------------------------------------------------- fragment geometry --

// The 8 (butterfly-in-group, point) pairs a lane owns, in register order:
// slot s = 4*rowsel + j, rowsel 0 -> butterfly g, 1 -> g + 8; j -> point
// {2t, 2t+1, 2t+8, 2t+9}[j].
GB_HD int tc_row(int lane, int s) { return (lane >> 2) + 8 * (s >> 2); }
GB_HD int tc_point(int lane, int s) {
  const int t = lane & 3, j = s & 3;
  return 2 * t + (j & 1) + 8 * (j >> 1);
}

// Value of the real 32 x 32 B matrix at (k, n): k < 16 re(x_k), else im(x_{k-16});
// n < 16 re(Y_n), else im(Y_{n-16}); Y_o = sum_i x_i w16^{o i}.
// cos(2 pi m / 16) for m = 0..15, the constants mul_w16 uses; -sin(2 pi m / 16)
// is cos16(m + 4).  Branch-free, so the fragments build without divergence.
GB_HD float cos16(int m) {
  m &= 15;
  const int q = m & 7;                         // cos(2 pi (m + 8) / 16) = -cos(2 pi m / 16)
  const int a = q <= 4 ? q : 8 - q;            // cos is even: |angle| in eighths of a half turn
  const float mag = a == 0 ? 1.f : a == 1 ? GB_C8 : a == 2 ? GB_H2 : a == 3 ? GB_S8 : 0.f;
  const bool neg = (q > 4) != (m >= 8);
  return neg ? -mag : mag;
}

GB_HD float tc_dft_entry(int k, int n) {
  const int i = k & 15, o = n & 15;
  const int m = (i * o) & 15;
  const cf w = mk(cos16(m), cos16(m + 4));  // (cos, -sin)(2 pi o i / 16)
  const bool kre = k < 16, nre = n < 16;
  if (kre && nre) return w.x;    //  re(x) cos
  if (!kre && nre) return -w.y;  // -im(x) (-sin)
  if (kre && !nre) return w.y;   //  re(x) (-sin)
  return w.x;                    //  im(x) cos
}

// B fragment registers of N block nb and K block kb for this lane:
// reg0 = (k = 2t, 2t+1), reg1 = (k = 2t+8, 2t+9), n = g.  `part` selects the
// high (0) or low (1) half of a BF16 split.
template <int PREC>
GB_HD void tc_b_frag(int lane, int kb, int nb, int part, uint32_t& r0, uint32_t& r1) {
  const int g = lane >> 2, t = lane & 3;
  const int n = 8 * nb + g;
  float v[4];
  const int ks[4] = {2 * t, 2 * t + 1, 2 * t + 8, 2 * t + 9};
  for (int q = 0; q < 4; ++q) v[q] = tc_dft_entry(16 * kb + ks[q], n);
  r0 = pack_rn<PREC>(v[0], v[1]);
  r1 = pack_rn<PREC>(v[2], v[3]);
  if (part == 1) {
    r0 = pack_rn<PREC>(v[0] - lo16_to_f32<PREC>(r0), v[1] - hi16_to_f32<PREC>(r0));
    r1 = pack_rn<PREC>(v[2] - lo16_to_f32<PREC>(r1), v[3] - hi16_to_f32<PREC>(r1));
  }
}

// A fragment registers of K block kb from the lane's 8 complex inputs x[s]:
// reg0 = (row g, cols 2t, 2t+1), reg1 = (row g+8, cols 2t, 2t+1),
// reg2 = (row g, cols 2t+8, 2t+9), reg3 = (row g+8, cols 2t+8, 2t+9).
// With SPLIT, also the low parts x - hi(x) of the same registers (BF16x3).
template <int PREC, bool SPLIT>
GB_HD void tc_a_frag(const cf (&x)[8], int kb, uint32_t (&a)[4], uint32_t (&alo)[4]) {
  float v[8];
GB_UNROLL
  for (int s = 0; s < 8; ++s) v[s] = kb == 0 ? x[s].x : x[s].y;
  // slot s: rowsel = s >> 2, j = s & 3 with points {2t, 2t+1, 2t+8, 2t+9}
  const int lo_idx[4] = {0, 4, 2, 6};  // row g pts 2t,2t+1 | row g+8 | row g pts +8 | row g+8 +8
GB_UNROLL
  for (int r = 0; r < 4; ++r) {
    const float v0 = v[lo_idx[r]], v1 = v[lo_idx[r] + 1];
    a[r] = pack_rn<PREC>(v0, v1);
    if (SPLIT)
      alo[r] = pack_rn<PREC>(v0 - lo16_to_f32<PREC>(a[r]), v1 - hi16_to_f32<PREC>(a[r]));
  }
}

// The lane's 8 complex outputs from the 4 N-block accumulators d[nb][0..3]:
// d[nb][0,1] = (row g, cols 2t, 2t+1), d[nb][2,3] = (row g+8, ...); N blocks
// 0/1 = Y_r outputs 0..7 / 8..15, 2/3 = Y_i.
GB_HD void tc_outputs(const float (&d)[4][4], cf (&y)[8]) {
  for (int s = 0; s < 8; ++s) {
    const int rowsel = s >> 2, j = s & 3;
    const int hi8 = j >> 1, c = j & 1;  // output 2t + c + 8*hi8 -> N block hi8 (re), 2 + hi8 (im)
    y[s] = mk(d[hi8][2 * rowsel + c], d[2 + hi8][2 * rowsel + c]);
  }
}

// ------------------------------------------------------------- per lane --
// A tile of 4096 complex elements: 4096 / L contiguous transforms of length
// L = 16^NST.  8 warps; per stage each warp runs 2 MMA groups of 16
// butterflies (256 butterflies = 4096 / 16 per stage).  Butterfly u of the tile
// belongs to transform u / (L/16) and is butterfly jb = u mod (L/16) of it.
//
// Addressing.  A group is 16 consecutive butterflies u0 .. u0+15 (u0 a
// multiple of 16).  Every position the group touches -- stage inputs
// tr*L + jb + i*L/16, stage outputs tr*L + (jb - k)*16 + k + o*Ns, twiddle
// rows i*Ns + k -- splits into a group base and a per-lane offset with
// disjoint bits (so base + off = base ^ off), the offset depending only on the
// lane's fixed (row, point) pairs.  The shared-memory swizzle is linear over
// GF(2), slot(a ^ b) = slot(a) ^ slot(b), so a lane's slot is
// slot(base) ^ slot(off): one XOR per element, the offsets computed once.
template <int LOGL, int PREC, class Mem>
struct TcBody {
  static constexpr int L = 1 << LOGL;
  static constexpr int NST = LOGL / 4;
  static constexpr int BPS = L / 16;    // butterflies per transform and stage
  static constexpr int TPC = 4096 / L;  // transforms per tile

  // Shared-memory slot of tile element e: the low four bits (the bank pair
  // of an 8-byte access) XORed with a linear function of higher bits, so the
  // map is bijective and GF(2)-linear.  Within a half warp the fragment-shaped
  // accesses vary bits {0,1} and {9,10} (stage inputs i*L/16 + r), {1,2} and
  // {4,5} (stage-0 outputs 16 r + o) or {0,1} and {5,6} (stage-1 outputs
  // r + 16 o); the function sends bits 9,10 to 2,3, bits 4,5 to 0,3 and
  // bits 5,6 to 3,2, which makes every one of these patterns conflict-free
  // (for L = 256 the same three patterns appear).
  GB_HD static int slot(int e) {
    return e ^ (((e >> 4) & 5) ^ ((e >> 2) & 8) ^ ((e >> 7) & 12));
  }

  // Staging buffer (the next tile, copied in by bulk copies of kChunk
  // elements, each followed by a 2-slot gap): element e at pslot(e).  The gap
  // shifts the banks of the stage-0 loads, element u0 + r + i*L/16, by 2 per
  // chunk, which separates the 4 lanes that share r within a half warp.
  // Additive: pslot(base + off) = pslot(base) + pslot(off) for disjoint bits.
  static constexpr int kChunkLog = LOGL >= 12 ? 8 : 4;
  static constexpr int kChunk = 1 << kChunkLog;
  static constexpr int kStageSlots = 4096 + 2 * (4096 >> kChunkLog);
  GB_HD static int pslot(int e) { return e + 2 * (e >> kChunkLog); }

  // Group base and lane offset of input i of the lane's row r (0..15) of the
  // group starting at butterfly u0, for a stage with Ns = 16^S.
  GB_HD static void in_pos(int u0, int r, int i, int& base, int& off) {
    if (BPS == 1) {  // L = 16: one butterfly per transform
      base = u0 * 16;
      off = r * 16 + i;
    } else {
      const int tr = u0 / BPS, jb0 = u0 - tr * BPS;
      base = tr * L + jb0;
      off = r + i * (L / 16);
    }
  }
  // Output o of row r for a stage with Ns (position (jb - k)*16 + k + o*Ns).
  template <int Ns>
  GB_HD static void out_pos(int u0, int r, int o, int& base, int& off) {
    if (BPS == 1) {
      base = u0 * 16;
      off = r * 16 + o;
    } else {
      const int tr = u0 / BPS, jb0 = u0 - tr * BPS;
      if (Ns == 1) {
        base = tr * L + jb0 * 16;
        off = r * 16 + o;
      } else {  // Ns >= 16: k = jb0 mod Ns + r
        const int k0 = jb0 & (Ns - 1);
        base = tr * L + (jb0 - k0) * 16 + k0;
        off = r + o * Ns;
      }
    }
  }
  // First transform of the group and whether all its rows share it.
  GB_HD static int transform_of(int u0, int r) { return BPS == 1 ? u0 + r : u0 / BPS; }

  // Inputs of MMA group h of warp w for stage S: 8 complex values, twiddled.
  template <int S>
  GB_HD static void gather(cf (&x)[8], const PassDesc& d, const cf* gin, const cf* sm, int w,
                           int h, int lane, int valid, bool swap) {
    constexpr int Ns = 1 << (4 * S);
    const int u0 = w * 32 + h * 16;
    int base, off0;
    in_pos(u0, 0, 0, base, off0);
    const int sbase = slot(base);
    const cf* tw = nullptr;
    if (S > 0) {
      // twiddle row i*Ns + k with k = (jb0 mod Ns) + r (Ns >= 16 divides jb0's block)
      const int jb0 = BPS == 1 ? 0 : u0 - (u0 / BPS) * BPS;
      tw = d.tw + d.tw_off[S] + (jb0 & (Ns - 1));
    }
GB_UNROLL
    for (int s8 = 0; s8 < 8; ++s8) {
      const int r = tc_row(lane, s8), i = tc_point(lane, s8);
      int b_, off;
      in_pos(u0, r, i, b_, off);
      cf v;
      if (S == 0) {  // from the staging buffer `sm` (padded), or global memory if null
        if (transform_of(u0, r) < valid)
          v = sm ? Mem::lds(sm, pslot(base) + pslot(off)) : Mem::ldg(gin, base + off);
        else
          v = mk(0.f, 0.f);
        v = swap ? mk(v.y, v.x) : v;
      } else {
        v = Mem::lds(sm, sbase ^ slot(off));
        if (i > 0) v = cmul(v, Mem::ldtw(tw + i * Ns + r));
      }
      if (PREC == TC_FP16) v = mk(v.x * 0.0625f, v.y * 0.0625f);  // exact 1/16 per stage
      x[s8] = v;
    }
  }

  // Outputs of group h: to shared memory, or to global memory after the last stage.
  template <int S>
  GB_HD static void scatter(const cf (&y)[8], cf* gout, cf* sm, int w, int h, int lane,
                            int valid, bool swap) {
    constexpr int Ns = 1 << (4 * S);
    const int u0 = w * 32 + h * 16;
    int base, off0;
    out_pos<Ns>(u0, 0, 0, base, off0);
    const int sbase = slot(base);
GB_UNROLL
    for (int s8 = 0; s8 < 8; ++s8) {
      const int r = tc_row(lane, s8), o = tc_point(lane, s8);
      int b_, off;
      out_pos<Ns>(u0, r, o, b_, off);
      cf v = y[s8];
      if (S == NST - 1) {
        if (transform_of(u0, r) >= valid) continue;
        if (PREC == TC_FP16) {  // undo the 1/16 per stage: exact powers of two
          const float sc = (float)(1 << (4 * NST));
          v = mk(v.x * sc, v.y * sc);
        }
        Mem::stg(gout, base + off, swap ? mk(v.y, v.x) : v);
      } else {
        Mem::sts(sm, sbase ^ slot(off), v);
      }
    }
  }
};

}  // namespace gbfft
