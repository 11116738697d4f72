// Pass shapes compiled with every parameter fixed at compile time (see
// CtTraits in fft_stage.h).  Each entry:
//   GB_SHAPE(log2 L, schedule, stages, R, G, load map, store map, contiguous, epilogue)
// schedule = log2 radices, stage 0 in the low nibble.  A pass whose shape
// matches an entry runs that instantiation; every other pass runs the generic
// kernel, which computes the same transform with run-time parameters.
#pragma once

#define GB_SHAPES(GB_SHAPE) GB_SHAPES_CONTIG(GB_SHAPE) GB_SHAPES_FOURSTEP(GB_SHAPE)

/* batched contiguous transforms, radix-16 stages, remainder last */
#define GB_SHAPES_CONTIG(GB_SHAPE)                            \
  GB_SHAPE(8, 0x44, 2, 16, 16, 0, 0, true, 0)                 \
  GB_SHAPE(9, 0x144, 3, 16, 8, 0, 0, true, 0)                 \
  GB_SHAPE(10, 0x244, 3, 16, 4, 0, 0, true, 0)                \
  GB_SHAPE(11, 0x344, 3, 16, 2, 0, 0, true, 0)                \
  GB_SHAPE(12, 0x444, 3, 16, 1, 0, 0, true, 0)                \
  GB_SHAPE(13, 0x1444, 4, 16, 1, 0, 0, true, 0)               \
  GB_SHAPE(14, 0x2444, 4, 16, 1, 0, 0, true, 0)

/* four-step N = 2^20, 2^22, 2^24: column pass (twiddle on store: full table, */
/* computed or factored) and row pass (transposed store); 2D column pass of */
/* 4096 rows */
#define GB_SHAPES_FOURSTEP(GB_SHAPE)                          \
  GB_SHAPE(10, 0x244, 3, 16, 16, 1, 1, false, 2)              \
  GB_SHAPE(10, 0x244, 3, 16, 16, 1, 1, false, 3)              \
  GB_SHAPE(10, 0x244, 3, 16, 16, 0, 1, false, 0)              \
  GB_SHAPE(11, 0x344, 3, 16, 8, 1, 1, false, 2)               \
  GB_SHAPE(11, 0x344, 3, 16, 8, 1, 1, false, 3)               \
  GB_SHAPE(11, 0x344, 3, 16, 8, 0, 1, false, 0)               \
  GB_SHAPE(12, 0x444, 3, 16, 4, 1, 1, false, 2)               \
  GB_SHAPE(12, 0x444, 3, 16, 4, 1, 1, false, 3)               \
  GB_SHAPE(12, 0x444, 3, 16, 4, 0, 1, false, 0)               \
  GB_SHAPE(12, 0x444, 3, 16, 4, 1, 1, false, 0)              \
  GB_SHAPE(10, 0x244, 3, 16, 16, 1, 1, false, 4)             \
  GB_SHAPE(11, 0x344, 3, 16, 8, 1, 1, false, 4)              \
  GB_SHAPE(12, 0x444, 3, 16, 4, 1, 1, false, 4)              \
  GB_SHAPES_FOURSTEP_MID(GB_SHAPE)

/* four-step N = 2^15..2^19 (passes of 128..512 points, 16 transforms per */
/* tile): column passes with the factored twiddle, transposing row passes */
#define GB_SHAPES_FOURSTEP_MID(GB_SHAPE)                      \
  GB_SHAPE(7, 0x34, 2, 16, 16, 1, 1, false, 4)                \
  GB_SHAPE(8, 0x44, 2, 16, 16, 1, 1, false, 4)                \
  GB_SHAPE(9, 0x144, 3, 16, 16, 1, 1, false, 4)               \
  GB_SHAPE(8, 0x44, 2, 16, 16, 0, 1, false, 0)                \
  GB_SHAPE(9, 0x144, 3, 16, 16, 0, 1, false, 0)

/* fast convolution: range lines of 4096 / 8192 / 16384, azimuth columns */
/* of 4096 (the 2D frame's column pass) */
#define GB_SHAPES_CONV(GB_SHAPE)                              \
  GB_SHAPE(12, 0x444, 3, 16, 1, 0, 0, true, 0)                \
  GB_SHAPE(13, 0x1444, 4, 16, 1, 0, 0, true, 0)               \
  GB_SHAPE(14, 0x2444, 4, 16, 1, 0, 0, true, 0)               \
  GB_SHAPE(12, 0x444, 3, 16, 4, 1, 1, false, 0)

// Contiguous transforms that run the staged kernel (fft_split.h): whole
// transform per block, TMA prefetch of the next one, half-size exchanges.
//   GB_STAGED(log2 L, schedule, stages, blocks per SM, elements per thread)
// 2^13 and 2^14 end with a stage of radix R/16, run in registers.
#define GB_STAGED_SHAPES(GB_STAGED) \
  GB_STAGED(12, 0x444, 3, 4, 32)    \
  GB_STAGED(13, 0x1444, 4, 2, 32)   \
  GB_STAGED(14, 0x2444, 4, 1, 64)

// Column tiles of strided passes that run the staged kernel (G adjacent
// columns per block, rows copied by 16-byte asynchronous copies while the
// previous tile is computed, half-size exchanges):
//   GB_STAGED_COLS(log2 L, schedule, stages, R, G, epilogue, conv)
// four-step first passes (epilogue 2, 3 or 4), the 2D column pass and the
// azimuth convolution of 4096-row frames (conv 1: per-column filters staged
// by tile, cols_filter_staged).
#define GB_STAGED_COLS_SHAPES(GB_STAGED_COLS)      \
  GB_STAGED_COLS(12, 0x444, 3, 32, 4, 0, 1)        \
  GB_STAGED_COLS(10, 0x244, 3, 32, 16, 2, 0)       \
  GB_STAGED_COLS(10, 0x244, 3, 32, 16, 3, 0)       \
  GB_STAGED_COLS(11, 0x344, 3, 32, 8, 2, 0)        \
  GB_STAGED_COLS(11, 0x344, 3, 32, 8, 3, 0)        \
  GB_STAGED_COLS(12, 0x444, 3, 32, 4, 2, 0)        \
  GB_STAGED_COLS(12, 0x444, 3, 32, 4, 3, 0)        \
  GB_STAGED_COLS(12, 0x444, 3, 32, 4, 0, 0)        \
  GB_STAGED_COLS(10, 0x244, 3, 32, 16, 4, 0)       \
  GB_STAGED_COLS(11, 0x344, 3, 32, 8, 4, 0)        \
  GB_STAGED_COLS(12, 0x444, 3, 32, 4, 4, 0)       \
  GB_STAGED_COLS(10, 0x244, 3, 32, 8, 2, 0)       \
  GB_STAGED_COLS(10, 0x244, 3, 32, 8, 3, 0)       \
  GB_STAGED_COLS(10, 0x244, 3, 32, 8, 4, 0)       \
  GB_STAGED_COLS(11, 0x344, 3, 32, 4, 2, 0)       \
  GB_STAGED_COLS(11, 0x344, 3, 32, 4, 3, 0)       \
  GB_STAGED_COLS(11, 0x344, 3, 32, 4, 4, 0)

// Transposing passes (G contiguous rows in, G columns out: the second pass of
// a four-step plan) that run the staged kernel:
//   GB_STAGED_TRANS(log2 L, schedule, stages, R, G)
#define GB_STAGED_TRANS_SHAPES(GB_STAGED_TRANS) \
  GB_STAGED_TRANS(10, 0x244, 3, 32, 16)         \
  GB_STAGED_TRANS(11, 0x344, 3, 32, 8)          \
  GB_STAGED_TRANS(12, 0x444, 3, 32, 4)          \
  GB_STAGED_TRANS(10, 0x244, 3, 32, 8)          \
  GB_STAGED_TRANS(11, 0x344, 3, 32, 4)

namespace gbfft {

// Does pass descriptor `d` (run with R elements per thread and these maps)
// have exactly this compile-time shape?
GB_HD bool shape_matches(const PassDesc& d, int R, int lmap, int smap, int logL, uint32_t sched,
                         int nst, int sR, int G, int slmap, int ssmap, bool contig, int epi) {
  uint32_t s = 0;
  for (int i = 0; i < d.nst && i < 8; ++i) s |= (uint32_t)d.rlog[i] << (4 * i);
  if (d.nst > 8) return false;
  const int64_t L = int64_t(1) << d.logL;
  const bool is_contig = d.in.e == 1 && d.out.e == 1 && d.in.g == L && d.out.g == L &&
                         d.in.t == d.G * L && d.out.t == d.G * L;
  return d.logL == logL && s == sched && d.nst == nst && R == sR && d.G == G && lmap == slmap &&
         smap == ssmap && d.epi == epi && (!contig || is_contig);
}

// Is `d` a pass the staged kernel of this (log2 L, schedule, stages) runs?
// One whole contiguous transform per tile, no four-step epilogue; `conv`
// selects the fast-convolution form.
GB_HD bool staged_shape_matches(const PassDesc& d, int logL, uint32_t sched, int nst,
                                bool conv = false) {
  uint32_t s = 0;
  for (int i = 0; i < d.nst && i < 8; ++i) s |= (uint32_t)d.rlog[i] << (4 * i);
  if (d.nst > 8) return false;
  const int64_t L = int64_t(1) << d.logL;
  return d.G == 1 && d.epi == 0 && d.conv == (conv ? 1 : 0) && d.in.e == 1 && d.out.e == 1 && d.in.t == L && d.out.t == L &&
         d.logL == logL && s == sched && d.nst == nst;
}

// Is `d` (with these thread maps) a column pass the staged column kernel of
// this shape runs?  G adjacent columns per tile, columns contiguous, row
// strides that keep every row copy 16-byte aligned.
GB_HD bool staged_cols_matches(const PassDesc& d, int lmap, int smap, int logL, uint32_t sched,
                               int nst, int G, int epi, int conv) {
  uint32_t s = 0;
  for (int i = 0; i < d.nst && i < 8; ++i) s |= (uint32_t)d.rlog[i] << (4 * i);
  if (d.nst > 8) return false;
  return lmap == MAP_COLS && smap == MAP_COLS && d.G == G && d.logL == logL && s == sched &&
         d.nst == nst && d.epi == epi && d.conv == conv && d.in.g == 1 && d.out.g == 1 &&
         d.in.t == G && d.out.t == G && d.in.e % 2 == 0 && d.in.o % 2 == 0 && G % 2 == 0;
}

// Is `d` a transposing pass (G contiguous rows of L in, written as G columns)
// the staged kernel of this shape runs?
GB_HD bool staged_trans_matches(const PassDesc& d, int lmap, int smap, int logL, uint32_t sched,
                                int nst, int G) {
  uint32_t s = 0;
  for (int i = 0; i < d.nst && i < 8; ++i) s |= (uint32_t)d.rlog[i] << (4 * i);
  if (d.nst > 8) return false;
  const int64_t L = int64_t(1) << logL;
  return lmap == MAP_ROWS && smap == MAP_COLS && d.G == G && d.logL == logL && s == sched &&
         d.nst == nst && d.epi == 0 && d.conv == 0 && d.in.e == 1 && d.in.g == L &&
         d.in.t == G * L && d.out.g == 1 && d.out.t == G && d.in.o % 2 == 0 && G % 2 == 0;
}

}  // namespace gbfft
