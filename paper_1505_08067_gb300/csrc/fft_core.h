// Per-thread building blocks of the Stockham pass kernel.
//
// The method (Bergach et al.): each transform -- or each column/row of a
// multi-pass split -- is computed by one on-chip block that holds the whole
// sequence (Sec. 3.4: one FFT per compute unit, global memory touched only at
// the first read and the last write); inside the block the transform runs as a
// sequence of radix stages (Sec. 2.1, mixed radix; Sec. 3.2, radix clustering)
// separated by a barrier (Sec. 3.2 "FFT performance model").  Sizes that do
// not fit one block are split into passes joined by twiddle multiplies and a
// transpose (Sec. 3.3, Sec. 3.4).
//
// Stage formulation (Stockham autosort, natural order in and out): for a stage
// of radix r after stages whose radices multiply to Ns, butterfly jb
// (0 <= jb < L/r) reads elements jb + i*L/r (i < r), multiplies element i by
// w_{Ns*r}^{i*k} with k = jb mod Ns, takes a length-r DFT and writes element i
// to (jb - k)*r + k + i*Ns.
//
// Everything here compiles both for the GPU (nvcc) and for a host compiler,
// so the test harness can replay a pass's exact index arithmetic on the CPU
// and check every access against its buffer before a kernel runs.
#pragma once
#include <stdint.h>

#if defined(__CUDACC__)
#define GB_HD __host__ __device__ __forceinline__
#define GB_HDC __host__ __device__
#define GB_UNROLL _Pragma("unroll")
#else
#define GB_HD inline
#define GB_HDC
#define GB_UNROLL
#endif

namespace gbfft {

struct alignas(8) cf {
  float x, y;
};

GB_HD cf mk(float x, float y) { cf r; r.x = x; r.y = y; return r; }

// Complex add / subtract.  On sm_100 and later one paired-FP32 instruction
// does both halves (same IEEE round-to-nearest result per component; a - b
// is b * (-1) + a, whose single rounding equals the subtraction's).
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000
#define GB_PAIRED 1
__device__ __forceinline__ float2 f2(cf a) { return make_float2(a.x, a.y); }
__device__ __forceinline__ cf fc(float2 a) { cf r; r.x = a.x; r.y = a.y; return r; }
GB_HD cf cadd(cf a, cf b) { return fc(__fadd2_rn(f2(a), f2(b))); }
GB_HD cf csub(cf a, cf b) { return fc(__ffma2_rn(f2(b), make_float2(-1.f, -1.f), f2(a))); }
// a + s * (b.y, b.x) with s = (sx, sy) in {+1, -1}^2: adds a quarter-turn
// rotation of b without moving b's halves first.
GB_HD cf cadd_rot(cf a, cf b, float sx, float sy) {
  return fc(__ffma2_rn(make_float2(b.y, b.x), make_float2(sx, sy), f2(a)));
}
#else
GB_HD cf cadd(cf a, cf b) { return mk(a.x + b.x, a.y + b.y); }
GB_HD cf csub(cf a, cf b) { return mk(a.x - b.x, a.y - b.y); }
GB_HD cf cadd_rot(cf a, cf b, float sx, float sy) { return mk(a.x + sx * b.y, a.y + sy * b.x); }
#endif
GB_HD cf cmul(cf a, cf b) { return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
GB_HD cf cconj(cf a) { return mk(a.x, -a.y); }

// cos(pi/8), sin(pi/8), sqrt(2)/2 rounded to FP32.
#define GB_C8 0.92387953251128674f
#define GB_S8 0.38268343236508977f
#define GB_H2 0.70710678118654752f

// a * w16^m, w16 = exp(-2 pi i / 16).  Quarter turns are exact swaps and
// sign flips; odd multiples of an eighth turn cost two multiplies.
GB_HD cf mul_w16(cf a, int m) {
  switch (m & 15) {
    case 0: return a;
    case 4: return mk(a.y, -a.x);
    case 8: return mk(-a.x, -a.y);
    case 12: return mk(-a.y, a.x);
    case 2: return mk(GB_H2 * (a.x + a.y), GB_H2 * (a.y - a.x));
    case 6: return mk(GB_H2 * (a.y - a.x), -GB_H2 * (a.x + a.y));
    case 10: return mk(-GB_H2 * (a.x + a.y), GB_H2 * (a.x - a.y));
    case 14: return mk(GB_H2 * (a.x - a.y), GB_H2 * (a.x + a.y));
    case 1: return cmul(a, mk(GB_C8, -GB_S8));
    case 3: return cmul(a, mk(GB_S8, -GB_C8));
    case 5: return cmul(a, mk(-GB_S8, -GB_C8));
    case 7: return cmul(a, mk(-GB_C8, -GB_S8));
    case 9: return cmul(a, mk(-GB_C8, GB_S8));
    case 11: return cmul(a, mk(-GB_S8, GB_C8));
    case 13: return cmul(a, mk(GB_S8, GB_C8));
    default: return cmul(a, mk(GB_C8, GB_S8));  // 15
  }
}

// Forward DFT of length P in {1, 2, 4} on v[0], v[S], ..., natural order.
template <int P, int S>
GB_HD void dft_small(cf* v) {
  if (P == 2) {
    cf a = v[0], b = v[S];
    v[0] = cadd(a, b);
    v[S] = csub(a, b);
  } else if (P == 4) {
    cf a0 = v[0], a1 = v[S], a2 = v[2 * S], a3 = v[3 * S];
    cf t0 = cadd(a0, a2), t1 = csub(a0, a2);
    cf t2 = cadd(a1, a3), t3 = csub(a1, a3);
    v[0] = cadd(t0, t2);
    v[2 * S] = csub(t0, t2);
    v[S] = cadd_rot(t1, t3, 1.f, -1.f);      // t1 - i*t3
    v[3 * S] = cadd_rot(t1, t3, -1.f, 1.f);  // t1 + i*t3
  }
}

// Forward DFT of length N = P*Q in registers, natural order in and out.
// Index split n = Q*n1 + n2, k = k1 + P*k2: length-P DFTs over n1, twiddle
// w_N^{n2*k1}, length-Q DFTs over n2 (Cooley-Tukey), then the output
// permutation, which after unrolling is only a renaming of registers.
template <int P, int Q>
GB_HD void dft_pq(cf* v) {
  constexpr int N = P * Q;
GB_UNROLL
  for (int n2 = 0; n2 < Q; ++n2) dft_small<P, Q>(v + n2);
GB_UNROLL
  for (int k1 = 1; k1 < P; ++k1)
GB_UNROLL
    for (int n2 = 1; n2 < Q; ++n2)
      v[Q * k1 + n2] = mul_w16(v[Q * k1 + n2], (n2 * k1 * (16 / N)) & 15);
GB_UNROLL
  for (int k1 = 0; k1 < P; ++k1) dft_small<Q, 1>(v + Q * k1);
  cf t[N];
GB_UNROLL
  for (int k1 = 0; k1 < P; ++k1)
GB_UNROLL
    for (int k2 = 0; k2 < Q; ++k2) t[k1 + P * k2] = v[Q * k1 + k2];
GB_UNROLL
  for (int i = 0; i < N; ++i) v[i] = t[i];
}

template <int RR>
GB_HD void dft_radix(cf* v) {
  if (RR == 2) dft_small<2, 1>(v);
  else if (RR == 4) dft_small<4, 1>(v);
  else if (RR == 8) dft_pq<2, 4>(v);
  else if (RR == 16) dft_pq<4, 4>(v);
}

// ---------------------------------------------------------------- layout --

enum { MAP_ROWS = 0, MAP_COLS = 1 };

// One pass = a batch of length-L transforms grouped G to a thread block
// ("tile").  Element a of transform g of tile (outer, inner) lives at
//   outer*o + inner*t + g*gs + a*e        (separately for input and output).
struct Strides {
  int64_t o, t, g, e;
};

struct PassDesc {
  int32_t logL;        // L = 2^logL, 1 <= L <= 2^14
  int32_t nst;         // number of radix stages
  int32_t rlog[15];    // log2 of each stage's radix (1..4)
  int32_t tw_off[15];  // stage s twiddles start at tw + tw_off[s]: [k][i], Ns*r entries
  int32_t G;           // transforms per tile
  int32_t T;           // threads per transform = L / R
  int32_t pitch;       // shared-memory pitch per transform (row layout)
  int32_t smem_elems;  // shared-memory complex elements used
  int64_t tiles;       // tiles in the whole pass
  int64_t tiles_inner; // tiles per outer index
  int64_t count_inner; // valid transforms per outer index (ragged last tile)
  Strides in, out;
  int32_t conj_in, conj_out;  // backward transform = conj(forward(conj(x)))
  int32_t epi;                // multiply output (n2, k1) by w_N^{n2*k1}; how w is found:
                              //   1 two-level tables hi[m >> lo_bits] * lo[m & (2^lo_bits - 1)]
                              //   2 full table in the output's layout: epi_lo[n2 + k1 * N2]
                              //   3 computed: sincospi of the exact FP32 angle 2 m / N
                              //   4 factored: the last stage writes k1 = jb + i*Ns, so
                              //     w = w_N^{n2 jb} * (w_N^{n2 Ns})^i: two sincospi per
                              //     butterfly and step, powers of the step by products
  int32_t epi_lo_bits;
  int32_t epi_logN;
  int32_t l2_prefetch;        // contiguous passes on a persistent grid: prefetch next tile
  const cf* tw;
  const cf* epi_hi;
  const cf* epi_lo;
  int* status;  // device word set to nonzero if a bounded wait gives up
  // Fast convolution (conv = 1): forward stages, multiply output a of line u
  // (u = inner tile index * G + g) by h_scale * H_u[a], then the same
  // stages on swapped data (the unnormalised inverse transform), so that
  // out = h_scale * IDFT(H_u . DFT(x)).  h_lines = 1: one filter for every
  // line, H_u[a] = h[a].  Otherwise per-line filters laid out like one frame
  // of the input: H_u[a] = h[((h_first + u) mod h_lines) * in.g + a * in.e].
  int32_t conv;
  float h_scale;
  int64_t h_lines, h_first;
  const cf* h;
  // Column tiles of the staged kernel: when tmap_in_ok, the tile's input is
  // copied by tensor-map (TMA) box loads; when tmap_out_ok, its output (G
  // columns) is written by tensor-map box stores.  tmap_in / tmap_out are
  // CUtensorMaps encoded at launch over `in` / `out` viewed as rows of in.e /
  // out.e complex64 elements (dims {e, rows}, box {G, min(rows of a copy,
  // 256)}); tile coordinates from tma_tile_coords.
  int32_t tmap_in_ok, tmap_out_ok;
  alignas(64) unsigned char tmap_in[128];
  alignas(64) unsigned char tmap_out[128];
  // Fast convolution over column tiles with per-line filters
  // (cols_filter_staged): when tmap_h_ok, each tile's filters (G columns of
  // the filter frame, laid out like the input frame) are copied into shared
  // memory by tensor-map boxes over h (dims {in.e, L}, box {G, min(L, 256)}).
  int32_t tmap_h_ok;
  alignas(64) unsigned char tmap_h[128];
};

// Column tiles of a fast convolution whose filters can be staged by tile:
// one filter per column (h_lines = the row length in.e, adjacent columns
// adjacent: in.g = 1), starting at column 0 (h_first = 0), so that the
// filters of the tile's columns col0 .. col0 + G - 1 are the same columns of
// the filter frame.
GB_HD bool cols_filter_staged(const PassDesc& d) {
  return d.conv && d.G > 1 && d.h_lines > 1 && d.h_lines == d.in.e && d.in.g == 1 &&
         d.h_first == 0 && d.in.e % 2 == 0;
}

// Can the column tiles of `d` (G adjacent columns of L rows) be moved by
// tensor-map boxes over the buffer with strides `st` (d.in or d.out) viewed
// as rows of st.e elements?  Every tile offset outer*st.o + inner*st.t must
// split into a row y and a column x with x + G <= st.e (st.o a multiple of
// st.e, the inner tiles within one row), and x must be even (st.e and G
// even) so that each box starts on a 16-byte boundary.  `rows`: the rows
// the map spans.
GB_HD bool cols_map_rows(const PassDesc& d, const Strides& st, int64_t& rows) {
  const int64_t e = st.e, L = int64_t(1) << d.logL;
  if (d.G < 2 || d.G % 2 || st.g != 1 || st.t != d.G || e < d.G || e % 2 || st.o % e ||
      d.tiles_inner < 1 || d.tiles_inner * d.G > e || d.tiles < 1 || d.tiles % d.tiles_inner ||
      (L > 512 && L % 512))
    return false;
  rows = (d.tiles / d.tiles_inner - 1) * (st.o / e) + L;
  return rows <= (int64_t(1) << 31);
}

// Column tiles whose output goes half through tensor-map box stores: only
// 32-byte row segments (G = 4).  With 64- or 128-byte segments the register
// stores are already efficient and the extra pass through shared memory
// measured slower.
GB_HD bool cols_store_map(const PassDesc& d) { return d.G * 8 <= 32; }

// Tensor-map coordinates of column tile `tile`'s first element in the buffer
// with strides `st`: its offset outer*st.o + inner*st.t written as y*st.e + x
// (x the column, y the row).
GB_HD void tma_tile_coords(const PassDesc& d, const Strides& st, int64_t tile, int32_t& x,
                           int32_t& y) {
  const int64_t outer = tile / d.tiles_inner, inner = tile - outer * d.tiles_inner;
  const int64_t off = outer * st.o + inner * st.t;
  const int64_t row = off / st.e;
  y = (int32_t)row;
  x = (int32_t)(off - row * st.e);
}

GB_HD void thread_coords(int map, int tid, int T, int G, int& g, int& t) {
  if (map == MAP_ROWS) { g = tid / T; t = tid - g * T; }
  else { t = tid / G; g = tid - t * G; }
}

// Shared-memory slot of element a of transform g.  Row layout: a padding
// slot every 16 elements plus a per-transform offset (pitch); column layout:
// transforms interleaved, a padding slot every 16.  Both keep the Stockham
// reads and writes free of bank conflicts for the tile shapes the planner
// emits.
//
// In the row layout slot(x) = x + (x >> 4) inside a transform, and a
// butterfly touches x = base + i*D with D = L/r (reads) or D = Ns (writes).
// Then slot(base + i*D) = slot(base) + i*D + ((i*D) >> 4) exactly:
//   - if D is a multiple of 16 the low four bits of base are untouched;
//   - reads: base = jb < L/r = D, so when D < 16 (D divides 16) base + i*D
//     never carries into the next 16-block beyond what i*D itself does;
//   - writes: base = (jb - k)*r + k with k = jb mod Ns < Ns, and (jb - k)*r
//     is a multiple of Ns*r; if Ns*r <= 16 everything stays inside one
//     16-block, otherwise (jb - k)*r is a multiple of 16 and base mod 16 = k,
//     which again adds no carry to i*D.
// So the offsets of a butterfly's elements are constants whenever D is.
GB_HD int smem_slot(int layout, int g, int a, int G, int pitch) {
  if (layout == MAP_ROWS) return g * pitch + a + (a >> 4);
  int s = a * G + g;
  return s + (s >> 4);
}

GB_HD int64_t elem_offset(const Strides& s, int64_t outer, int64_t inner, int g, int64_t a) {
  return outer * s.o + inner * s.t + (int64_t)g * s.g + a * s.e;
}

}  // namespace gbfft
