// Test infrastructure: replays the GPU pass kernel's per-thread phases on the
// CPU, thread by thread, exactly as planned by the library's planner, with a
// memory policy that checks every access:
//   - global loads/stores and twiddle loads stay inside their buffers;
//   - shared-memory slots stay inside the tile's allocation;
//   - every shared read hits a slot written in the immediately preceding
//     write phase (no stale read), no slot is written twice in one phase
//     (no write collision);
//   - every output element of a pass is written exactly once.
// It never stands in for the GPU: the library has no CPU path, and the GPU
// parity tests compare the CUDA kernels with the FP64 oracle.  This harness
// only lets the index arithmetic be checked before a kernel runs.

#include <array>
#include <type_traits>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "fft_split.h"
#include "fft_stage.h"
#include "kernel_shapes.h"
#include "planner.h"
#include "tc_stage.h"
#include "umma_stage.h"
#include "queue_ring.h"

using namespace gbfft;

namespace {

struct Ctx {
  const cf* in = nullptr;
  int64_t in_len = 0;
  cf* out = nullptr;
  int64_t out_len = 0;
  std::vector<uint8_t>* out_hits = nullptr;
  const cf* tw = nullptr;
  int64_t tw_len = 0;
  const cf* h = nullptr;  // convolution filter of the pass being replayed
  int64_t h_len = 0;
  int smem_len = 0;
  std::vector<int64_t>* slot_epoch = nullptr;
  std::vector<int64_t>* slot_write = nullptr;
  int64_t epoch = 0;        // phase counter of the register / staged replays
  int64_t read_epoch = -2;  // TC replay: shared reads must see this write phase
  int64_t write_epoch = -2; // TC replay: shared writes belong to this phase
  bool split_epochs = false;
  int64_t errors = 0;
  int64_t special_passes = 0;
  int64_t staged_passes = 0;
  const cf* staging = nullptr;  // staged kernel: whole-transform buffer (TMA target)
  const cf* smem_base = nullptr;  // TC replay: base of the two shared buffers
  int staging_len = 0;
  std::string first_error;
};
Ctx g;

void err(const char* what, int64_t idx) {
  if (g.errors++ == 0) {
    char b[256];
    snprintf(b, sizeof b, "%s (index %lld)", what, (long long)idx);
    g.first_error = b;
  }
}

struct CheckMem {
  static cf ldg(const cf* p, int64_t off) {
    const int64_t idx = (p - g.in) + off;
    if (idx < 0 || idx >= g.in_len) { err("global load out of bounds", idx); return mk(0, 0); }
    return g.in[idx];
  }
  static void stg(cf* p, int64_t off, cf v) {
    const int64_t idx = (p - g.out) + off;
    if (idx < 0 || idx >= g.out_len) { err("global store out of bounds", idx); return; }
    if ((*g.out_hits)[idx]++) err("output element written twice", idx);
    g.out[idx] = v;
  }
  static cf ldtw(const cf* p) {
    if (g.h && !(p >= g.tw && p < g.tw + g.tw_len)) {  // not a twiddle: a filter load
      const int64_t off = p - g.h;
      if (off < 0 || off >= g.h_len) { err("filter load out of bounds", off); return mk(1, 0); }
      return *p;
    }
    int64_t off = p - g.tw;
    if (off < 0 || off >= g.tw_len) { err("twiddle load out of bounds", off); return mk(1, 0); }
    return *p;
  }
  static cf lds(const cf* s, int i) {
    if (g.staging && s == g.staging) {
      if (i < 0 || i >= g.staging_len) { err("staging load out of bounds", i); return mk(0, 0); }
      return s[i];
    }
    if (g.smem_base && s != g.smem_base) {  // second TC buffer
      i += (int)(s - g.smem_base);
      s = g.smem_base;
    }
    if (i < 0 || i >= g.smem_len) { err("shared load out of bounds", i); return mk(0, 0); }
    const int64_t want = g.split_epochs ? g.read_epoch : g.epoch;
    if ((*g.slot_epoch)[i] != want) err("shared load of a slot not written in the last phase", i);
    return s[i];
  }
  static cf rotor(int64_t m, int logN) {
    const int64_t N = int64_t(1) << logN;
    if (m < 0 || m >= N) err("rotor exponent out of range", m);
    const double a = -2.0 * M_PI * (double)m / (double)N;
    return mk((float)cos(a), (float)sin(a));
  }
  static void sts(cf* s, int i, cf v) {
    if (g.smem_base && s != g.smem_base) {
      i += (int)(s - g.smem_base);
      s = const_cast<cf*>(g.smem_base);
    }
    if (i < 0 || i >= g.smem_len) { err("shared store out of bounds", i); return; }
    const int64_t ph = g.split_epochs ? g.write_epoch : g.epoch;
    if ((*g.slot_write)[i] == ph) err("two writes to one shared slot in one phase", i);
    (*g.slot_write)[i] = ph;
    (*g.slot_epoch)[i] = ph;
    s[i] = v;
  }
};

// Host twiddles for the harness only (FP64, rounded to FP32).
cf root(int64_t e, int64_t den) {
  e %= den;
  double a = -2.0 * M_PI * (double)e / (double)den;
  return mk((float)cos(a), (float)sin(a));
}

template <int R, int LM, int SM, class TR = RtTraits>
void run_pass_t(const PassDesc& d, const cf* in, cf* out) {
  using B = PassBody<R, LM, SM, CheckMem, TR>;
  const int nthr = d.G * d.T;
  std::vector<cf> smem(std::max(1, d.smem_elems));
  std::vector<int64_t> ep(smem.size(), -1), wr(smem.size(), -1);
  g.slot_epoch = &ep;
  g.slot_write = &wr;
  g.smem_len = d.smem_elems;
  std::vector<std::array<cf, R>> V(nthr);
  for (int64_t tile = 0; tile < d.tiles; ++tile) {
    typename B::Tile tl = B::tile_of(d, tile);
    ++g.epoch;
    for (int tid = 0; tid < nthr; ++tid) {
      cf (&v)[R] = *reinterpret_cast<cf(*)[R]>(V[tid].data());
      B::first(v, d, in, out, smem.data(), tl, tid);
    }
    int Ns = 1 << d.rlog[0];
    for (int s = 1; s < d.nst; ++s) {
      for (int tid = 0; tid < nthr; ++tid) {
        cf (&v)[R] = *reinterpret_cast<cf(*)[R]>(V[tid].data());
        B::read(v, d, s, Ns, out, smem.data(), tl, tid);
      }
      if (s < d.nst - 1) {
        ++g.epoch;
        for (int tid = 0; tid < nthr; ++tid) {
          cf (&v)[R] = *reinterpret_cast<cf(*)[R]>(V[tid].data());
          B::write(v, d, s, Ns, smem.data(), tid);
        }
      }
      Ns <<= d.rlog[s];
    }
  }
}

// Fast-convolution tile (conv_tile in the library): round 1 without the final
// store, the filter phase writing natural order, round 2 with the store.
template <int R, int MAP, class TR = RtTraits>
void run_conv_t(const PassDesc& d, const cf* in, cf* out) {
  using B = PassBody<R, MAP, MAP, CheckMem, TR>;
  const int nthr = d.G * d.T;
  std::vector<cf> smem(std::max(1, d.smem_elems));
  std::vector<int64_t> ep(smem.size(), -1), wr(smem.size(), -1);
  g.slot_epoch = &ep;
  g.slot_write = &wr;
  g.smem_len = d.smem_elems;
  std::vector<std::array<cf, R>> V(nthr);
  auto reg = [&](int t) -> cf (&)[R] { return *reinterpret_cast<cf(*)[R]>(V[t].data()); };
  for (int64_t tile = 0; tile < d.tiles; ++tile) {
    typename B::Tile tl = B::tile_of(d, tile);
    ++g.epoch;
    for (int t = 0; t < nthr; ++t) B::first_nostore(reg(t), d, in, smem.data(), tl, t);
    auto stages = [&](bool round1) {
      int Ns = 1 << d.rlog[0];
      for (int s = 1; s < d.nst; ++s) {
        for (int t = 0; t < nthr; ++t) {
          if (round1) B::read_nostore(reg(t), d, s, Ns, smem.data(), tl, t);
          else B::template read_s<true>(reg(t), d, s, Ns, out, smem.data(), tl, t);
        }
        if (s < d.nst - 1) {
          ++g.epoch;
          for (int t = 0; t < nthr; ++t) B::write(reg(t), d, s, Ns, smem.data(), t);
        }
        Ns <<= d.rlog[s];
      }
    };
    stages(true);
    if (B::conv_in_regs(d)) {
      for (int t = 0; t < nthr; ++t) B::conv_regs(reg(t), d, tl, t);
    } else {
      ++g.epoch;
      for (int t = 0; t < nthr; ++t) B::conv_mid(reg(t), d, smem.data(), tl, t);
      for (int t = 0; t < nthr; ++t) B::first_smem(reg(t), d, smem.data(), t);
    }
    if (d.nst == 1) {
      for (int t = 0; t < nthr; ++t) B::store_first(reg(t), d, out, tl, t);
    } else {
      ++g.epoch;
      for (int t = 0; t < nthr; ++t) B::write(reg(t), d, 0, 1, smem.data(), t);
      stages(false);
    }
  }
}

template <int MAP>
void run_conv_maps(int R, const PassDesc& d, const cf* in, cf* out) {
  switch (R) {
    case 2: run_conv_t<2, MAP>(d, in, out); break;
    case 4: run_conv_t<4, MAP>(d, in, out); break;
    case 8: run_conv_t<8, MAP>(d, in, out); break;
    case 16: run_conv_t<16, MAP>(d, in, out); break;
    default: err("bad R", R);
  }
}

bool run_conv_staged(const PassDesc& d, const cf* in, cf* out);

bool run_conv_special(int R, int map, const PassDesc& d, const cf* in, cf* out) {
#define GB_TRY(LOGL, SCHED, NST, RR, G, LMAP_, SMAP_, CONTIG, EPI)                          \
  if (shape_matches(d, R, map, map, LOGL, SCHED, NST, RR, G, LMAP_, SMAP_, CONTIG, EPI)) {   \
    run_conv_t<RR, LMAP_, CtTraits<LOGL, SCHED, NST, RR, G, CONTIG, EPI>>(d, in, out);      \
    return true;                                                                         \
  }
  GB_SHAPES_CONV(GB_TRY)
#undef GB_TRY
  return false;
}

// The same compile-time shapes the GPU library instantiates.
template <int R, int LM, int SM, class TR>
void run_ct(const PassDesc& d, const cf* in, cf* out);

bool run_special(int R, int lmap, int smap, const PassDesc& d, const cf* in, cf* out) {
#define GB_TRY(LOGL, SCHED, NST, RR, G, LMAP_, SMAP_, CONTIG, EPI)                          \
  if (shape_matches(d, R, lmap, smap, LOGL, SCHED, NST, RR, G, LMAP_, SMAP_, CONTIG, EPI)) { \
    run_ct<RR, LMAP_, SMAP_, CtTraits<LOGL, SCHED, NST, RR, G, CONTIG, EPI>>(d, in, out);   \
    return true;                                                                         \
  }
  GB_SHAPES(GB_TRY)
#undef GB_TRY
  return false;
}

// Staged kernel (fft_split.h): the TMA copy of a tile into the staging buffer
// becomes a memcpy; the phase order and barriers follow the kernel.
template <class SH, bool CONV = false>
void run_staged_t(const PassDesc& d, const cf* in, cf* out) {
  using B = SplitBody<SH, CheckMem>;
  constexpr int R = SH::kR;
  constexpr int TILE = SH::kStageElems;
  std::vector<cf> st(TILE), x(SH::kHalfSlots);
  std::vector<int64_t> ep(x.size(), -1), wr(x.size(), -1);
  g.slot_epoch = &ep;
  g.slot_write = &wr;
  g.smem_len = SH::kHalfSlots;
  g.staging = st.data();
  g.staging_len = TILE;
  std::vector<std::array<cf, R>> V(SH::kT);
  auto reg = [&](int t) -> cf (&)[R] { return *reinterpret_cast<cf(*)[R]>(V[t].data()); };
  for (int64_t tile = 0; tile < d.tiles; ++tile) {
    // the bulk copies: one contiguous transform, or one G-column segment per row
    int64_t src, dst, col0;
    if constexpr (SH::kG == 1) {
      src = dst = tile * SH::kL;
      col0 = tile;
    } else {
      const int64_t outer = tile / d.tiles_inner, inner = tile - outer * d.tiles_inner;
      src = outer * d.in.o + inner * d.in.t;
      dst = outer * d.out.o + inner * d.out.t;
      col0 = inner * SH::kG;
    }
    // column tiles the GPU copies by tensor-map boxes: element (y + a, x + c)
    // of the map, which must lie inside its {in.e, rows} extent (TMA would
    // fill zeros outside it) and be the element the row copy reads
    int64_t map_rows = 0;
    const bool use_map = SH::kG > 1 && !SH::kRowsIn && cols_map_rows(d, d.in, map_rows);
    int32_t mx = 0, my = 0;
    if (use_map) tma_tile_coords(d, d.in, tile, mx, my);
    for (int a = 0; a < SH::kL; ++a)
      for (int c = 0; c < SH::kG; ++c) {
        if constexpr (SH::kRowsIn) {  // one bulk copy per row, pitched
          st[c * (SH::kL + SH::kRowPad) + a] = CheckMem::ldg(in, src + c * SH::kL + a);
        } else if (use_map) {
          const int64_t row = (int64_t)my + a, col = (int64_t)mx + c;
          if (row >= map_rows || col >= d.in.e || mx % 2 ||
              row * d.in.e + col != src + c + a * d.in.e)
            err("tensor-map box outside the map or off the row copy", row * d.in.e + col);
          st[a * SH::kG + c] = CheckMem::ldg(in, row * d.in.e + col);
        } else {
          st[a * SH::kG + c] = CheckMem::ldg(in, src + (SH::kG == 1 ? a : c + a * d.in.e));
        }
      }
    for (int t = 0; t < SH::kT; ++t) {
      if (d.conj_in) B::template first<true>(reg(t), st.data(), t);
      else B::template first<false>(reg(t), st.data(), t);
    }
    auto exchange = [&](auto S_) {
      constexpr int S = decltype(S_)::value;
      ++g.epoch;
      for (int t = 0; t < SH::kT; ++t) B::template write_half<S, 0>(reg(t), x.data(), t);
      for (int t = 0; t < SH::kT; ++t) B::template read_half<S, 0>(reg(t), x.data(), t);
      ++g.epoch;
      for (int t = 0; t < SH::kT; ++t) B::template write_half<S, 1>(reg(t), x.data(), t);
      for (int t = 0; t < SH::kT; ++t) {
        B::template read_half<S, 1>(reg(t), x.data(), t);
        cf r[SH::kR / SH::radix(S + 1)];
        if constexpr (SH::kPowTw) B::template roots<S>(r, d, t);
        B::template compute<S>(reg(t), d, t, r);
      }
    };
    auto round = [&]() {
      exchange(std::integral_constant<int, 0>());
      if constexpr (SH::kExchanges > 1) exchange(std::integral_constant<int, 1>());
      if constexpr (SH::kExchanges > 2) exchange(std::integral_constant<int, 2>());
    };
    round();
    cf* o = out + dst;
    bool conv_swap = false;
    if constexpr (CONV) {
      // column tiles with per-column filters: the tile's filters are copied
      // into the staging buffer by tensor-map boxes over h (element (a, g) at
      // row a, column col0 + g of the filter frame, inside its {in.e, L}
      // extent), as the kernel does when its filter map encodes
      const bool fstage = SH::kG > 1 && cols_filter_staged(d) && use_map;
      if (fstage) {
        for (int a = 0; a < SH::kL; ++a)
          for (int c = 0; c < SH::kG; ++c) {
            const int64_t col = col0 + c;
            if (col >= d.in.e || col0 % 2) err("filter box outside the filter frame", col);
            const int64_t hi = (int64_t)a * d.in.e + col;
            if (hi < 0 || hi >= g.h_len) { err("filter load out of bounds", hi); continue; }
            st[a * SH::kG + c] = g.h[hi];
          }
      }
      for (int t = 0; t < SH::kT; ++t) B::conv_middle(reg(t), d, col0, t, fstage ? st.data() : nullptr);
      round();
      if constexpr (SH::kG == 1 || SH::kFuseLast) {
        for (int t = 0; t < SH::kT; ++t) {
          if constexpr (SH::kFuseLast) { cf fr[16]; B::fused_roots(fr, d, t); B::template store_fused<true, true>(reg(t), d, o, col0, t, fr); }
          else B::template store<true>(reg(t), d, o, col0, t);
        }
        continue;
      }
      conv_swap = true;
    }
    const bool swap_out = conv_swap || d.conj_out;
    // column tiles the GPU writes half by tensor-map box stores: rows
    // [0, L/2) go to the exchange buffer in the box layout (every slot
    // written once), then box element (a, c) to row y + a, column x + c of the
    // output map, which must be the element the register store writes; rows
    // [L/2, L) by register stores
    int64_t out_rows = 0;
    if constexpr (SH::kG > 1 && !SH::kFuseLast) {
      if (cols_store_map(d) && cols_map_rows(d, d.out, out_rows)) {
        int32_t ox = 0, oy = 0;
        tma_tile_coords(d, d.out, tile, ox, oy);
        ++g.epoch;
        for (int t = 0; t < SH::kT; ++t) {
          if (swap_out) B::template store_half_smem<true, 0>(reg(t), d, x.data(), col0, t);
          else B::template store_half_smem<false, 0>(reg(t), d, x.data(), col0, t);
        }
        for (int a = 0; a < SH::kL / 2; ++a)
          for (int c = 0; c < SH::kG; ++c) {
            const int slot = a * SH::kG + c;
            if (wr[slot] != g.epoch) err("box-store slot not written in this half", slot);
            const int64_t row = (int64_t)oy + a, col = (int64_t)ox + c;
            if (row >= out_rows || col >= d.out.e || ox % 2 ||
                row * d.out.e + col != dst + c + a * d.out.e)
              err("tensor-map box store outside the map or off the column", row * d.out.e + col);
            CheckMem::stg(out, row * d.out.e + col, x[slot]);
          }
        for (int t = 0; t < SH::kT; ++t) {
          if (swap_out) B::template store_half<true, 1>(reg(t), d, o, col0, t);
          else B::template store_half<false, 1>(reg(t), d, o, col0, t);
        }
        continue;
      }
    }
    for (int t = 0; t < SH::kT; ++t) {
      if constexpr (SH::kFuseLast) {
        if (swap_out) { cf fr[16]; B::fused_roots(fr, d, t); B::template store_fused<true, true>(reg(t), d, o, col0, t, fr); }
        else { cf fr[16]; B::fused_roots(fr, d, t); B::template store_fused<false, true>(reg(t), d, o, col0, t, fr); }
      } else {
        if (swap_out) B::template store<true>(reg(t), d, o, col0, t);
        else B::template store<false>(reg(t), d, o, col0, t);
      }
    }
  }
  g.staging = nullptr;
}

// Transposing passes (GB_STAGED_TRANS_SHAPES).
bool run_staged_trans(int lmap, int smap, const PassDesc& d, const cf* in, cf* out) {
#define GB_STAGED_TRANS(LOGL, SCHED, NST, RR, G)                                  \
  if (staged_trans_matches(d, lmap, smap, LOGL, SCHED, NST, G)) {                 \
    run_staged_t<SplitShape<LOGL, SCHED, NST, RR, G, 0, true>>(d, in, out);       \
    return true;                                                                 \
  }
  GB_STAGED_TRANS_SHAPES(GB_STAGED_TRANS)
#undef GB_STAGED_TRANS
  return false;
}

// Column tiles of strided passes (GB_STAGED_COLS_SHAPES).
bool run_staged_cols(int lmap, int smap, const PassDesc& d, const cf* in, cf* out) {
#define GB_STAGED_COLS(LOGL, SCHED, NST, RR, G, EPI, CONV)                                  \
  if (staged_cols_matches(d, lmap, smap, LOGL, SCHED, NST, G, EPI, CONV)) {                  \
    run_staged_t<SplitShape<LOGL, SCHED, NST, RR, G, EPI>, CONV != 0>(d, in, out);           \
    return true;                                                                          \
  }
  GB_STAGED_COLS_SHAPES(GB_STAGED_COLS)
#undef GB_STAGED_COLS
  return false;
}

bool run_conv_staged(const PassDesc& d, const cf* in, cf* out) {
#define GB_TRY_STAGED(LOGL, SCHED, NST, MINB, RR)                     \
  if (staged_shape_matches(d, LOGL, SCHED, NST, true)) {              \
    run_staged_t<SplitShape<LOGL, SCHED, NST, RR>, true>(d, in, out); \
    return true;                                                      \
  }
  GB_STAGED_SHAPES(GB_TRY_STAGED)
#undef GB_TRY_STAGED
  return false;
}

bool run_staged(const PassDesc& d, const cf* in, cf* out) {
#define GB_TRY_STAGED(LOGL, SCHED, NST, MINB, RR)             \
  if (staged_shape_matches(d, LOGL, SCHED, NST)) {            \
    run_staged_t<SplitShape<LOGL, SCHED, NST, RR>>(d, in, out); \
    return true;                                              \
  }
  GB_STAGED_SHAPES(GB_TRY_STAGED)
#undef GB_TRY_STAGED
  return false;
}

// Tensor-core class: the kernel's per-lane gather / scatter with the warp-wide
// m16n8k16 MMA emulated from the 32 lanes' fragments (PTX fragment layouts).
template <int P>
void mma_emulate(float (&d)[32][4], const uint32_t (&a)[32][4], const uint32_t (&b)[32][2]) {
  double A[16][16], Bm[16][8];
  for (int lane = 0; lane < 32; ++lane) {
    const int gq = lane >> 2, t = lane & 3;
    auto lo = [](uint32_t r) { return (double)from16<P>((uint16_t)(r & 0xffffu)); };
    auto hi = [](uint32_t r) { return (double)from16<P>((uint16_t)(r >> 16)); };
    A[gq][2 * t] = lo(a[lane][0]);      A[gq][2 * t + 1] = hi(a[lane][0]);
    A[gq + 8][2 * t] = lo(a[lane][1]);  A[gq + 8][2 * t + 1] = hi(a[lane][1]);
    A[gq][2 * t + 8] = lo(a[lane][2]);  A[gq][2 * t + 9] = hi(a[lane][2]);
    A[gq + 8][2 * t + 8] = lo(a[lane][3]); A[gq + 8][2 * t + 9] = hi(a[lane][3]);
    Bm[2 * t][gq] = lo(b[lane][0]);     Bm[2 * t + 1][gq] = hi(b[lane][0]);
    Bm[2 * t + 8][gq] = lo(b[lane][1]); Bm[2 * t + 9][gq] = hi(b[lane][1]);
  }
  for (int lane = 0; lane < 32; ++lane) {
    const int gq = lane >> 2, t = lane & 3;
    const int rows[4] = {gq, gq, gq + 8, gq + 8}, cols[4] = {2 * t, 2 * t + 1, 2 * t, 2 * t + 1};
    for (int q = 0; q < 4; ++q) {
      double s = 0;
      for (int k = 0; k < 16; ++k) s += A[rows[q]][k] * Bm[k][cols[q]];
      d[lane][q] = (float)((double)d[lane][q] + s);
    }
  }
}

template <int LOGL, int PREC>
void run_tc_t(const PassDesc& d, const cf* in, cf* out) {
  constexpr int P = PREC == TC_BF16X3 ? TC_BF16 : PREC;
  constexpr bool SPLIT = PREC == TC_BF16X3;
  using B = TcBody<LOGL, P, CheckMem>;
  constexpr int TPC = 4096 >> LOGL, NST = LOGL / 4;
  std::vector<cf> sm(8192);
  std::vector<int64_t> ep(sm.size(), -100), wr(sm.size(), -100);
  g.slot_epoch = &ep;
  g.slot_write = &wr;
  g.smem_len = 8192;
  g.smem_base = sm.data();
  g.split_epochs = true;
  uint32_t bh[32][2][4][2], bl[32][2][4][2];
  for (int lane = 0; lane < 32; ++lane)
    for (int kb = 0; kb < 2; ++kb)
      for (int nb = 0; nb < 4; ++nb) {
        tc_b_frag<P>(lane, kb, nb, 0, bh[lane][kb][nb][0], bh[lane][kb][nb][1]);
        tc_b_frag<P>(lane, kb, nb, 1, bl[lane][kb][nb][0], bl[lane][kb][nb][1]);
      }
  // the kernel's staging buffer: the tile's valid transforms in chunks of
  // kChunk elements, each followed by a 2-slot gap (the bulk copies)
  std::vector<cf> stg(B::kStageSlots);
  int64_t phase = 0;
  for (int64_t tile = 0; tile < d.tiles; ++tile) {
    const int64_t first = tile * TPC;
    const int valid = (int)std::min<int64_t>(TPC, d.count_inner - first);
    const cf* gin = in + first * (1 << LOGL);
    cf* gout = out + first * (1 << LOGL);
    for (int e = 0; e < valid * (1 << LOGL); ++e)
      stg[B::pslot(e)] = CheckMem::ldg(in, first * (1 << LOGL) + e);
    g.staging = stg.data();
    g.staging_len = B::kStageSlots;
    auto stage = [&](auto S_) {
      constexpr int S = decltype(S_)::value;
      g.read_epoch = phase;
      g.write_epoch = ++phase;
      const cf* src = S == 0 ? stg.data() : sm.data() + ((S + 1) & 1) * 4096;
      cf* dst = sm.data() + (S & 1) * 4096;
      for (int w = 0; w < 8; ++w)
        for (int h = 0; h < 2; ++h) {
          cf x[32][8], y[32][8];
          for (int lane = 0; lane < 32; ++lane)
            B::template gather<S>(x[lane], d, gin, src, w, h, lane, valid, d.conj_in != 0);
          float acc[4][32][4] = {};
          for (int kb = 0; kb < 2; ++kb) {
            uint32_t a[32][4], alo[32][4];
            for (int lane = 0; lane < 32; ++lane) tc_a_frag<P, SPLIT>(x[lane], kb, a[lane], alo[lane]);
            for (int nb = 0; nb < 4; ++nb) {
              uint32_t b0[32][2], b1[32][2];
              for (int lane = 0; lane < 32; ++lane) {
                b0[lane][0] = bh[lane][kb][nb][0]; b0[lane][1] = bh[lane][kb][nb][1];
                b1[lane][0] = bl[lane][kb][nb][0]; b1[lane][1] = bl[lane][kb][nb][1];
              }
              mma_emulate<P>(acc[nb], a, b0);
              if (SPLIT) {
                mma_emulate<P>(acc[nb], a, b1);
                mma_emulate<P>(acc[nb], alo, b0);
              }
            }
          }
          for (int lane = 0; lane < 32; ++lane) {
            float dl[4][4];
            for (int nb = 0; nb < 4; ++nb)
              for (int q = 0; q < 4; ++q) dl[nb][q] = acc[nb][lane][q];
            tc_outputs(dl, y[lane]);
            B::template scatter<S>(y[lane], gout, dst, w, h, lane, valid, d.conj_out != 0);
          }
        }
    };
    stage(std::integral_constant<int, 0>());
    if constexpr (NST > 1) stage(std::integral_constant<int, 1>());
    if constexpr (NST > 2) stage(std::integral_constant<int, 2>());
  }
  g.smem_base = nullptr;
  g.staging = nullptr;
  g.split_epochs = false;
}

bool run_tc(int logL, int prec, const PassDesc& d, const cf* in, cf* out) {
#define GB_TC(LG, PR)                  \
  if (logL == LG && prec == PR) {      \
    run_tc_t<LG, PR>(d, in, out);      \
    return true;                       \
  }
  GB_TC(4, 1) GB_TC(4, 2) GB_TC(4, 3)
  GB_TC(8, 1) GB_TC(8, 2) GB_TC(8, 3)
  GB_TC(12, 1) GB_TC(12, 2) GB_TC(12, 3)
#undef GB_TC
  return false;
}

// ------------------------------------------------ tcgen05 class replay --
// The UMMA kernel's per-thread body (umma_stage.h) on the CPU.  Shared
// memory is a byte array holding the A operand(s); every 32-bit store must
// land inside it and no word may be written twice in one phase, and after each
// phase every word of the operand must have been written.  The UMMA itself is
// emulated from the operand layout the hardware reads (K-major, 64-byte
// swizzle: element (m, k) at (m / 8) * 512 + (m % 8) * 64 + ((k / 8) ^
// ((m % 8) / 2)) * 16 + (k % 8) * 2), written here independently of the
// kernel's per-pair offsets; tensor memory is a row-major FP32 array whose
// rows the replay hands to the same (warp, lane, row block) that reads them
// on the GPU, each exactly once per stage.
struct UmmaReplay {
  std::vector<uint8_t> bytes;
  std::vector<int64_t> word_phase;
  int64_t phase = 0;
};
UmmaReplay g_umma;

struct UmmaCheckMem : CheckMem {
  static constexpr bool kHalfIO = false;
  static const cf* at(const cf* p, int64_t e) { return p + e; }
  static cf* at(cf* p, int64_t e) { return p + e; }
  static cf ldg_sw(const cf* p, int64_t off, bool swap) {
    const cf v = ldg(p, off);
    return swap ? mk(v.y, v.x) : v;
  }
  static void stg_sw(cf* p, int64_t off, cf v, bool swap) { stg(p, off, swap ? mk(v.y, v.x) : v); }
  static void sts32(uint32_t addr, uint32_t v) {
    if (addr % 4 || addr + 4 > g_umma.bytes.size()) { err("A-operand store out of bounds", addr); return; }
    if (g_umma.word_phase[addr / 4] == g_umma.phase) err("two writes to one A word in one phase", addr);
    g_umma.word_phase[addr / 4] = g_umma.phase;
    memcpy(&g_umma.bytes[addr], &v, 4);
  }
};

GB_HD uint32_t umma_hw_offset(int m, int k) {
  return (uint32_t)((m / 8) * 512 + (m % 8) * 64 + (((k / 8) ^ ((m % 8) / 2)) & 3) * 16 + (k % 8) * 2);
}

template <int LOGL, int PREC>
void run_umma_t(const PassDesc& d, const cf* in, cf* out) {
  using Body = UmmaBody<LOGL, PREC, UmmaCheckMem>;
  using G = UmmaGeo<LOGL>;
  constexpr int P = Body::P;
  constexpr bool SPLIT = Body::SPLIT;
  const uint32_t a_hi = 0, a_lo = G::A_BYTES;
  g_umma.bytes.assign((SPLIT ? 2 : 1) * G::A_BYTES, 0);
  g_umma.word_phase.assign(g_umma.bytes.size() / 4, -1);
  // the DFT matrix as the kernel builds it, read back through the B layout
  double Bh[32][32], Bl[32][32];
  for (int n = 0; n < 32; ++n)
    for (int k = 0; k < 32; ++k) {
      const float v = umma_dft_entry(k, n);
      const uint16_t h = P == TC_FP16 ? f32_to_f16_bits(v) : f32_to_bf16_bits(v);
      Bh[k][n] = from16<P>(h);
      Bl[k][n] = SPLIT ? bf16_bits_to_f32(f32_to_bf16_bits(v - bf16_bits_to_f32(h))) : 0.0;
      if (umma_boff(n, k) != umma_hw_offset(n, k)) err("B offset differs from the UMMA layout", n * 32 + k);
    }
  auto a_val = [&](uint32_t base, int m, int k) {
    uint16_t h;
    memcpy(&h, &g_umma.bytes[base + umma_hw_offset(m, k)], 2);
    return (double)from16<P>(h);
  };
  auto check_written = [&](const char* what) {
    for (size_t w = 0; w < g_umma.word_phase.size(); ++w)
      if (g_umma.word_phase[w] != g_umma.phase) { err(what, (int64_t)w); break; }
  };
  std::vector<float> D((size_t)G::ROWS * 32);
  std::vector<int> row_reads(G::ROWS);
  for (int64_t tile = 0; tile < d.tiles; ++tile) {
    const int64_t first = tile * G::TPT;
    const int valid = (int)std::min<int64_t>(G::TPT, d.count_inner - first);
    const cf* gin = in + first * G::L;
    cf* gout = out + first * G::L;
    ++g_umma.phase;
    for (int warp = 0; warp < G::NWARP; ++warp)
      for (int lane = 0; lane < 32; ++lane) {
        const int et = umma_load_item<LOGL>(lane, warp);
        auto parts = [&](int b) { return Body::block_part_of(et, b); };
        if (valid == G::TPT) Body::template load_tile<true>(d, gin, valid, a_hi, a_lo, parts);
        else Body::template load_tile<false>(d, gin, valid, a_hi, a_lo, parts);
      }
    check_written("A-operand word not written by the loader");
    auto stage = [&](auto t_) {
      constexpr int t = decltype(t_)::value;
      for (int m = 0; m < G::ROWS; ++m)
        for (int n = 0; n < 32; ++n) {
          double acc = 0;
          for (int k = 0; k < 32; ++k) {
            const double ah = a_val(a_hi, m, k);
            acc += ah * Bh[k][n];
            if (SPLIT) acc += ah * Bl[k][n] + a_val(a_lo, m, k) * Bh[k][n];
          }
          D[(size_t)m * 32 + n] = (float)acc;
        }
      ++g_umma.phase;
      std::fill(row_reads.begin(), row_reads.end(), 0);
      for (int warp = 0; warp < G::NWARP; ++warp)
        for (int lane = 0; lane < 32; ++lane)
          for (int rb = warp >> 2; rb < G::RB; rb += G::NWARP / 4) {
            const int m = rb * 128 + (warp & 3) * 32 + lane;
            ++row_reads[m];
            // as the kernel: one row part, the row read in two halves
            typename Body::RowPart rp = Body::template row_part<t>(d, m);
            uint32_t r[16];
            memcpy(r, &D[(size_t)m * 32], sizeof r);
            Body::template epilogue_part<t, 0, 8>(d, gout, valid, rp, r, a_hi, a_lo);
            memcpy(r, &D[(size_t)m * 32 + 16], sizeof r);
            Body::template epilogue_part<t, 8, 8>(d, gout, valid, rp, r, a_hi, a_lo);
          }
      for (int m = 0; m < G::ROWS; ++m)
        if (row_reads[m] != 1) { err("tensor-memory row not read exactly once", m); break; }
      if (t < G::NTC - 1) check_written("A-operand word not written by the epilogue");
    };
    stage(std::integral_constant<int, 0>());
    if constexpr (G::NTC > 1) stage(std::integral_constant<int, 1>());
    if constexpr (G::NTC > 2) stage(std::integral_constant<int, 2>());
  }
}

bool run_umma(int logL, int prec, const PassDesc& d, const cf* in, cf* out) {
#define GB_UM(LG)                                                        \
  if (logL == LG) {                                                      \
    if (prec == 1) run_umma_t<LG, 1>(d, in, out);                        \
    else if (prec == 2) run_umma_t<LG, 2>(d, in, out);                   \
    else run_umma_t<LG, 3>(d, in, out);                                  \
    return true;                                                         \
  }
  GB_UM(4) GB_UM(5) GB_UM(6) GB_UM(7) GB_UM(8) GB_UM(9) GB_UM(10) GB_UM(11) GB_UM(12)
  GB_UM(13) GB_UM(14)
#undef GB_UM
  return false;
}

template <int LM, int SM>
void run_maps(int R, const PassDesc& d, const cf* in, cf* out) {
  switch (R) {
    case 2: run_pass_t<2, LM, SM>(d, in, out); break;
    case 4: run_pass_t<4, LM, SM>(d, in, out); break;
    case 8: run_pass_t<8, LM, SM>(d, in, out); break;
    case 16: run_pass_t<16, LM, SM>(d, in, out); break;
    default: err("bad R", R);
  }
}

template <int R, int LM, int SM, class TR>
void run_ct(const PassDesc& d, const cf* in, cf* out) {
  run_pass_t<R, LM, SM, TR>(d, in, out);
}

int64_t replay(const int64_t* n, int dims, int64_t batch, int direction, int precision,
               const fft_plan_options_t* opt, int smem_optin, int specialised,
               const float* in_f, float* out_f, char* msg, size_t msg_len,
               int64_t* special_passes, const ConvSpec* conv, const float* const* filters,
               const int64_t* filter_len) {
  Caps caps;
  caps.smem_optin = smem_optin;
  static PlanSpec s;
  make_plan(s, n, dims, batch, direction, precision, opt, caps, conv);
  g = Ctx{};
  if (s.status != FFT_OK) {
    snprintf(msg, msg_len, "plan failed: %s", s.error);
    return -1;
  }
  const int64_t E = (dims == 1 ? n[0] : n[0] * n[1]) * batch;
  std::vector<cf> tables(std::max<int64_t>(1, s.table_elems));
  for (const TwSegment& t : s.tables)
    for (int64_t j = 0; j < t.count; ++j) {
      int64_t e = t.mode == 0 ? (j / t.r) * (j % t.r) : j * t.mult;
      tables[t.off + j] = root(e, t.den);
    }
  std::vector<cf> work(std::max<int64_t>(1, s.work_elems));
  const cf* in = reinterpret_cast<const cf*>(in_f);
  cf* out = reinterpret_cast<cf*>(out_f);
  for (const PassSpec& p : s.passes) {
    // the second workspace buffer of six-step plans starts work2_off in
    auto buf = [&](int b) -> cf* {
      return b == BUF_IN ? const_cast<cf*>(in) : b == BUF_OUT ? out
             : b == BUF_WORK2 ? work.data() + s.work2_off : work.data();
    };
    const cf* src = buf(p.src);
    cf* dst = buf(p.dst);
    if (p.kind == PASS_COPY) {
      for (int64_t i = 0; i < E; ++i) dst[i] = src[i];
      continue;
    }
    if (p.kind == PASS_TRANSPOSE) {
      // written out from the definition: dst[b][c][r] = src[b][r][c], times
      // exp(sign 2 pi i r c / 2^logN) when a twiddle is asked for
      const int64_t R = p.tr_rows, C = p.tr_cols;
      if (R * C * batch != E) err("transpose does not cover the batch", R * C);
      if (src == dst) err("transpose in place", 0);
      for (int64_t b = 0; b < batch; ++b)
        for (int64_t r = 0; r < R; ++r)
          for (int64_t c = 0; c < C; ++c) {
            cf v = src[b * R * C + r * C + c];
            if (p.tr_logN > 0) {
              cf w = root(r * c, int64_t(1) << p.tr_logN);
              if (p.tr_sign > 0) w = mk(w.x, -w.y);
              v = mk(v.x * w.x - v.y * w.y, v.x * w.y + v.y * w.x);
            }
            dst[b * R * C + c * R + r] = v;
          }
      continue;
    }
    PassDesc d = pass_desc(p, 0, batch, batch);
    d.tw = tables.data();
    d.epi_hi = (p.epi == 1 || p.epi == 2) ? tables.data() + p.epi_hi_off : nullptr;
    d.epi_lo = (p.epi == 1 || p.epi == 2) ? tables.data() + p.epi_lo_off : nullptr;
    // In-place passes read and write the same buffer: copy the source so the
    // checker can tell loads from stores.
    std::vector<cf> src_copy;
    if (src == dst) {
      src_copy.assign(src, src + E);
      src = src_copy.data();
    }
    g.in = src;
    g.in_len = E;  // every buffer of a replayed plan holds the whole batch
    g.out = dst;
    g.out_len = E;
    std::vector<uint8_t> hits(g.out_len, 0);
    g.out_hits = &hits;
    g.tw = tables.data();
    g.tw_len = s.table_elems;
    g.h = nullptr;
    g.h_len = 0;
    if (p.conv) {
      d.h = reinterpret_cast<const cf*>(filters[p.h_dim]);
      g.h = d.h;
      g.h_len = filter_len[p.h_dim];
      const bool want_staged = p.variant == 0 || p.variant == 2;
      if (specialised && !s.generic_only && want_staged && p.lmap == MAP_ROWS &&
          run_conv_staged(d, src, dst))
        ++g.staged_passes;
      else if (specialised && !s.generic_only && want_staged && p.lmap == MAP_COLS &&
               cols_filter_staged(d) && run_staged_cols(p.lmap, p.smap, d, src, dst))
        ++g.staged_passes;
      else if (specialised && !s.generic_only && run_conv_special(p.R, p.lmap, d, src, dst)) ++g.special_passes;
      else if (p.lmap == MAP_ROWS) run_conv_maps<0>(p.R, d, src, dst);
      else run_conv_maps<1>(p.R, d, src, dst);
    } else if (p.tc_prec) {
      if (!(p.variant == 1 ? run_tc(p.logL, p.tc_prec, d, src, dst)
                           : run_umma(p.logL, p.tc_prec, d, src, dst)))
        err("no replay for this tensor-core pass", p.logL);
    }
    else if (specialised && !s.generic_only &&
             ((p.variant == 0 && !(p.logL == 12 && p.lmap == MAP_ROWS && p.smap == MAP_ROWS)) ||
              p.variant == 2) &&  // contiguous 2^12: the library's choice is the register kernel
             (p.lmap == MAP_COLS ? run_staged_cols(p.lmap, p.smap, d, src, dst)
              : p.smap == MAP_COLS ? run_staged_trans(p.lmap, p.smap, d, src, dst)
                                   : run_staged(d, src, dst)))
      ++g.staged_passes;
    else if (specialised && !s.generic_only && run_special(p.R, p.lmap, p.smap, d, src, dst)) ++g.special_passes;
    else if (p.lmap == MAP_ROWS && p.smap == MAP_ROWS) run_maps<0, 0>(p.R, d, src, dst);
    else if (p.lmap == MAP_COLS && p.smap == MAP_COLS) run_maps<1, 1>(p.R, d, src, dst);
    else run_maps<0, 1>(p.R, d, src, dst);
    for (int64_t i = 0; i < g.out_len; ++i)
      if (hits[i] != 1) { err("output element not written exactly once", i); break; }
  }
  snprintf(msg, msg_len, "%s", g.first_error.c_str());
  if (special_passes) *special_passes = g.special_passes + 1000 * g.staged_passes;
  return g.errors;
}

}  // namespace

extern "C" {

// Plans (n, dims, batch, direction, options) for a device with the given
// limits, replays every pass on the CPU and writes the result to `out`
// (complex64, same size as `in`).  Returns the number of access violations;
// the first one is described in msg.
int64_t emu_run(const int64_t* n, int dims, int64_t batch, int direction, int precision,
                const fft_plan_options_t* opt, int smem_optin, int specialised,
                const float* in_f, float* out_f, char* msg, size_t msg_len,
                int64_t* special_passes) {
  return replay(n, dims, batch, direction, precision, opt, smem_optin, specialised, in_f, out_f,
                msg, msg_len, special_passes, nullptr, nullptr, nullptr);
}

// The same for a fast-convolution plan: filters[d] (complex64, filter_len[d]
// elements) with lines[d] and scale[d] as in fft_filter_t.
int64_t emu_conv_run(const int64_t* n, int dims, int64_t batch, const int64_t* lines,
                     const float* scale, const float* const* filters, const int64_t* filter_len,
                     const fft_plan_options_t* opt, int smem_optin, int specialised,
                     const float* in_f, float* out_f, char* msg, size_t msg_len,
                     int64_t* special_passes) {
  ConvSpec cs;
  for (int d = 0; d < dims && d < 2; ++d) {
    cs.lines[d] = lines[d];
    cs.scale[d] = scale[d];
  }
  return replay(n, dims, batch, -1, 0, opt, smem_optin, specialised, in_f, out_f, msg, msg_len,
                special_passes, &cs, filters, filter_len);
}

// The work queue's host bookkeeping (queue_ring.h) against a model of the
// ring: a worker completing tickets in order at random moments, a host
// submitting (only into free slots) and scanning for completions at random
// moments, sometimes after a slot has been reused and completed again.
// Checks that a scan never reports an incomplete ticket, always reports every
// complete one, and that a slot is only rewritten after its previous ticket
// is complete.  exact = 1 scans with an equality test on the done word
// instead (the form that loses completions once a slot is reused), so a
// caller can check that the replay catches it.  Returns 0, or 1 with a message.
int emu_ring_replay(uint64_t seed, int slots, int jobs, int exact, char* msg, size_t msg_len) {
  std::vector<uint64_t> done(slots, 0);
  uint64_t issued = 0, worker_next = 1, completed = 0, x = seed * 2654435761u + 1;
  auto rnd = [&](int m) {
    x ^= x << 13;
    x ^= x >> 7;
    x ^= x << 17;
    return (int)(x % (uint64_t)m);
  };
  auto done_at = [&](int s) { return done[s]; };
  auto scan = [&]() {
    if (!exact) return ring_completed(completed, issued, slots, done_at);
    uint64_t c = completed;
    while (c < issued && done[(c) % slots] == c + 1) ++c;
    return c;
  };
  for (long step = 0; worker_next <= (uint64_t)jobs || completed < (uint64_t)jobs; ++step) {
    if (step > 100L * jobs + 1000) {
      snprintf(msg, msg_len, "no progress: issued %llu, worker at %llu, host saw %llu",
               (unsigned long long)issued, (unsigned long long)worker_next - 1,
               (unsigned long long)completed);
      return 1;
    }
    const int a = rnd(16);
    if (a < 6 && issued < (uint64_t)jobs) {  // host submits if the slot is free
      const uint64_t t = issued + 1;
      const int s = (int)((t - 1) % slots);
      if (ring_slot_free(t, slots, done[s])) {
        if (t > (uint64_t)slots && worker_next <= t - slots) {
          snprintf(msg, msg_len, "slot %d rewritten before ticket %llu completed", s,
                   (unsigned long long)(t - slots));
          return 1;
        }
        issued = t;
      }
    } else if (a < 13) {  // the worker completes the next ticket, if issued
      if (worker_next <= issued) {
        done[(worker_next - 1) % slots] = worker_next;
        ++worker_next;
      }
    } else {  // the host looks (rarely: slots get reused in between)
      const uint64_t c = scan();
      if (c > worker_next - 1) {
        snprintf(msg, msg_len, "ticket %llu reported complete, worker at %llu",
                 (unsigned long long)c, (unsigned long long)worker_next - 1);
        return 1;
      }
      if (c != std::min<uint64_t>(issued, worker_next - 1)) {
        snprintf(msg, msg_len, "scan stopped at %llu, %llu complete", (unsigned long long)c,
                 (unsigned long long)std::min<uint64_t>(issued, worker_next - 1));
        return 1;
      }
      completed = c;
    }
  }
  return 0;
}

}  // extern "C"
