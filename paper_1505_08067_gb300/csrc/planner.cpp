// Host-side planner (no CUDA calls).  See planner.h.
#include "planner.h"
#include "umma_stage.h"

#include <math.h>
#include <stdio.h>

#include <algorithm>
#include <limits>
#include <sstream>

namespace gbfft {

static int ilog2(int64_t v) {
  int l = 0;
  while ((int64_t(1) << l) < v) ++l;
  return l;
}
static bool is_pow2(int64_t v) { return v >= 1 && (v & (v - 1)) == 0; }

// Shared-memory complex elements a pass with G transforms of length L uses.
static int row_pitch(int L, int G) { return L + (L >> 4) + std::max(1, 16 / std::max(G, 1)); }
static int smem_elems_for(int L, int G, int lmap) {
  if (L <= 1) return 0;
  if (lmap == MAP_ROWS) return G * row_pitch(L, G);
  int s = L * G;
  return s + (s >> 4) + 1;
}

int block_log2_limit(const Caps& caps) {
  int best = 1;
  for (int k = 1; k <= 20; ++k) {
    int L = 1 << k;
    size_t bytes = (size_t)smem_elems_for(L, 1, MAP_ROWS) * 8;
    if (bytes > (size_t)caps.smem_optin) break;
    if (L / 16 > caps.max_block) break;
    best = k;
  }
  return best;
}

Sched default_schedule(int logL, int logR) {
  Sched s;
  if (logL <= 0) return s;
  if (logR > logL) logR = logL;
  int full = logL / logR, rem = logL % logR;
  for (int i = 0; i < full; ++i) s.push_back(logR);
  if (rem) s.push_back(rem);
  return s;
}

static bool fill_launch(PassSpec& p, const Caps& caps, const char*& err) {
  const int L = 1 << p.logL;
  if (p.kind == PASS_COPY || p.kind == PASS_TRANSPOSE) {
    p.block = 256;
    p.grid = 0;
    return true;
  }
  if (p.tc_prec && p.variant == 1) {
    // warp-level MMA kernel: 8 warps, two shared buffers of 4096 complex, a
    // staging buffer for the next tile (chunks of 2^8 or 2^4 elements each
    // followed by a 2-slot gap) and its mbarrier
    const int chunk_log = p.logL >= 12 ? 8 : 4;
    p.block = 256;
    p.pitch = 0;
    p.smem_elems = 2 * 4096 + 4096 + 2 * (4096 >> chunk_log);
    p.smem = (size_t)p.smem_elems * 8 + 16;
    if (p.smem > (size_t)caps.smem_optin) {
      err = "tensor-core tile does not fit in shared memory";
      return false;
    }
    return true;
  }
  if (p.tc_prec) {
    // tcgen05 kernel: 8 warps; the A operand of a tile (T/16 rows of 64
    // bytes; twice for the split class), the DFT matrix and its low part
    // (2 KB each), an mbarrier and the tensor-memory address, 1 KB of
    // alignment slack, and for tiles of 4096 elements the staging buffer.  Each CTA holds 32 tensor-memory columns per 128
    // rows; the shared-memory request keeps the CTAs an SM can hold within
    // its 512 columns.
    const int logT = p.logL > 12 ? p.logL : 12;
    const int rows = 1 << (logT - 4);
    const size_t a = (size_t)rows * 64;
    p.block = 32 * umma_warps(p.logL);
    p.pitch = 0;
    p.smem = (p.tc_prec == FFT_PREC_TC_BF16X3 ? 2 : 1) * a + 2 * 2048 + 16 + 1024 +
             umma_staging_bytes(p.logL, p.io16 ? 4 : 8, p.tc_prec == FFT_PREC_TC_BF16X3);
    const int cols = 32 * (rows / 128);
    const size_t per_sm = (size_t)caps.smem_optin + 1024;  // the runtime keeps 1 KB per CTA
    const size_t floor_smem = per_sm / (size_t)(512 / cols + 1) + 1 - 1024;
    if (p.smem < floor_smem) p.smem = floor_smem;
    p.smem_elems = (int)(p.smem / 8);
    if (p.smem > (size_t)caps.smem_optin) {
      err = "tensor-core tile does not fit in shared memory";
      return false;
    }
    return true;
  }
  if (p.R < 2 || p.R > 16 || !is_pow2(p.R) || p.R > L) {
    err = "radix (elements per thread) must be 2, 4, 8 or 16 and at most the pass length";
    return false;
  }
  int sum = 0;
  for (int r : p.rlogs) {
    if (r < 1 || (1 << r) > p.R) {
      err = "every stage radix must be between 2 and the elements per thread";
      return false;
    }
    sum += r;
  }
  if (sum != p.logL || p.rlogs.empty() || p.rlogs.size() > 15) {
    err = "radix schedule must multiply to the pass length";
    return false;
  }
  const int T = L / p.R;
  if (p.G < 1) p.G = 1;
  if ((int64_t)p.G * T > caps.max_block) {
    err = "tile too large for one thread block";
    return false;
  }
  if (p.lmap != p.smap && p.rlogs.size() < 2) {
    err = "a transposing pass needs at least two stages";
    return false;
  }
  p.block = p.G * T;
  p.pitch = row_pitch(L, p.G);
  p.smem_elems = smem_elems_for(L, p.G, p.lmap);
  if (p.rlogs.size() == 1 && !p.conv) p.smem_elems = 0;  // single stage: registers only
  p.smem = (size_t)p.smem_elems * 8;
  if (p.smem > (size_t)caps.smem_optin) {
    err = "tile does not fit in shared memory";
    return false;
  }
  return true;
}

bool reshape_pass(PassSpec& p, int R, const Sched& rlogs, int G, const Caps& caps) {
  PassSpec q = p;
  q.R = R;
  q.rlogs = rlogs;
  if (G > 0 && q.batch_is_tiles) q.G = G;
  if (G > 0 && !q.batch_is_tiles) {
    // strided passes: tile must divide the number of transforms per outer index
    if (q.count_inner % G) return false;
    q.G = G;
    q.tiles_inner = q.count_inner / G;
    // strides of the tile index follow G
    if (q.lmap == MAP_COLS) q.in.t = G;             // column tiles: adjacent columns
    else q.in.t = q.in.g * G;                       // row tiles: G rows
    if (q.smap == MAP_COLS) q.out.t = G;
    else q.out.t = q.out.g * G;
  }
  const char* err = nullptr;
  if (!fill_launch(q, caps, err)) return false;
  p = q;
  return true;
}

static PassSpec fft_pass(int logL, int R, const Sched& sched) {
  PassSpec p;
  p.kind = PASS_FFT;
  p.logL = logL;
  p.R = R;
  p.rlogs = sched;
  return p;
}

static int choose_R(int logL, int req) {
  int L = 1 << logL;
  int R = req > 0 ? req : 16;
  if (R > L) R = L;
  while (L / R > 1024) R *= 2;
  return R;
}

static Sched sched_for(int logL, int R, uint32_t forced) {
  if (forced) {
    Sched s;
    for (int i = 0; i < 8 && ((forced >> (4 * i)) & 15); ++i) s.push_back((forced >> (4 * i)) & 15);
    return s;
  }
  return default_schedule(logL, ilog2(R));
}

// Batched contiguous transforms: `units` transforms of length 2^logL per
// batch entry, consecutive in memory.
static PassSpec contiguous_pass(int logL, int64_t batch, int64_t units_per_batch, int R,
                                uint32_t forced, int tile, const Caps& caps) {
  const int64_t units_total = batch * units_per_batch;
  PassSpec p = fft_pass(logL, R, sched_for(logL, R, forced));
  const int L = 1 << logL;
  const int T = L / R;
  int G = tile > 0 ? tile : std::max(1, 256 / T);
  while ((int64_t)G > 1 && (int64_t)G / 2 >= units_total) G /= 2;  // no idle tile slots
  while ((int64_t)G * T > caps.max_block) G /= 2;
  if (G < 1) G = 1;
  p.G = G;
  p.lmap = p.smap = MAP_ROWS;
  p.batch_is_tiles = true;
  p.units_per_batch = units_per_batch;
  p.count_inner = units_total;
  p.tiles_inner = (units_total + G - 1) / G;
  p.tiles = p.tiles_inner;
  p.outer = 1;
  p.in = Strides{0, (int64_t)G * L, L, 1};
  p.out = p.in;
  return p;
}

void make_plan(PlanSpec& s, const int64_t* n, int dims, int64_t batch, int direction,
               int precision, const fft_plan_options_t* opt, const Caps& caps,
               const ConvSpec* conv) {
  s = PlanSpec();
  fft_plan_options_t o{};
  if (opt) o = *opt;
  auto fail = [&](fft_status_t st, const char* msg) {
    s.status = st;
    snprintf(s.error, sizeof s.error, "%s", msg);
    s.passes.clear();
  };
  if (!n) { fail(FFT_ERR_INVALID_ARG, "n is null"); return; }
  if (dims != 1 && dims != 2) { fail(FFT_ERR_INVALID_ARG, "dims must be 1 or 2"); return; }
  if (batch < 0) { fail(FFT_ERR_INVALID_ARG, "batch must be >= 0"); return; }
  if (direction != FFT_FORWARD && direction != FFT_INVERSE)
    { fail(FFT_ERR_INVALID_ARG, "direction must be FFT_FORWARD (-1) or FFT_INVERSE (+1)"); return; }
  if (precision < FFT_PREC_FP32 || precision > FFT_PREC_TC_FP16_C32)
    { fail(FFT_ERR_INVALID_ARG, "unknown precision"); return; }
  if (precision != FFT_PREC_FP32) {
    // tensor-core classes: batched 1D lengths 2^4 .. 2^14 on the tcgen05
    // kernel; the warp-level MMA kernel (variant 1) covers 16, 256 and 4096
    const int64_t l = (dims == 1 && n) ? n[0] : 0;
    if (o.variant != 0 && o.variant != 1) {
      fail(FFT_ERR_INVALID_ARG, "tensor-core plans take variant 0 (tcgen05) or 1 (warp MMA)");
      return;
    }
    const bool ok = o.variant == 1 ? (l == 16 || l == 256 || l == 4096)
                                   : (l >= 16 && l <= (int64_t(1) << 24) && is_pow2(l));
    if (precision == FFT_PREC_TC_FP16_C32 && o.variant == 1) {
      fail(FFT_ERR_NOT_IMPLEMENTED, "complex32 storage runs on the tcgen05 kernel (variant 0)");
      return;
    }
    if (!ok) {
      fail(FFT_ERR_NOT_IMPLEMENTED,
           o.variant == 1
               ? "the warp-level tensor-core kernel covers batched 1D lengths 16, 256, 4096"
               : "the tensor-core classes cover batched 1D transforms of length 2^4 .. 2^24");
      return;
    }
  }
  if (o.radix && (o.radix < 2 || o.radix > 16 || !is_pow2(o.radix)))
    { fail(FFT_ERR_INVALID_ARG, "radix option must be 2, 4, 8 or 16"); return; }
  if (o.variant < 0 || o.variant > 4) { fail(FFT_ERR_INVALID_ARG, "variant must be 0..4"); return; }
  if (o.epilogue < 0 || o.epilogue > 4) { fail(FFT_ERR_INVALID_ARG, "epilogue must be 0..4"); return; }
  if (o.tile < 0 || o.tile > 1024 || (o.tile && !is_pow2(o.tile)))
    { fail(FFT_ERR_INVALID_ARG, "tile option must be a power of two <= 1024"); return; }
  s.dims = dims;
  s.batch = batch;
  s.direction = direction;
  s.precision = precision;
  for (int d = 0; d < dims; ++d) {
    if (!is_pow2(n[d])) { fail(FFT_ERR_UNSUPPORTED_SIZE, "each length must be a power of two >= 1"); return; }
    s.n[d] = n[d];
  }
  int bmax = block_log2_limit(caps);
  if (o.max_block_log2 > 0) {
    if (o.max_block_log2 < 2) { fail(FFT_ERR_INVALID_ARG, "max_block_log2 must be >= 2"); return; }
    bmax = std::min(bmax, o.max_block_log2);
  }
  s.max_block_log2 = bmax;
  s.generic_only = o.generic != 0;
  const int inv = direction == FFT_INVERSE;

  if (conv) {
    // Fast convolution: every line on one SM, forward stages, filter, forward
    // stages on swapped data, one pass per dimension.
    s.conv = true;
    s.direction = FFT_FORWARD;
    if (precision != FFT_PREC_FP32)
      { fail(FFT_ERR_NOT_IMPLEMENTED, "fast convolution runs in FP32 only"); return; }
    for (int d = 0; d < dims; ++d) {
      if (n[d] < 2) { fail(FFT_ERR_UNSUPPORTED_SIZE, "convolution lengths must be >= 2"); return; }
      if (ilog2(n[d]) > bmax)
        { fail(FFT_ERR_NOT_IMPLEMENTED, "convolution lines must fit one on-chip block (<= 2^14)"); return; }
    }
    // lines along dimension d per frame: the other lengths (1D: the batch)
    const int64_t lines_of[2] = {dims == 1 ? batch : n[1], dims == 1 ? 0 : n[0]};
    for (int d = 0; d < dims; ++d) {
      const int64_t l = conv->lines[d];
      if (l != 1 && l != lines_of[d]) {
        fail(FFT_ERR_INVALID_ARG, dims == 1 ? "filter lines must be 1 or the batch"
                                            : "filter lines must be 1 or the lines of a frame along that dimension");
        return;
      }
    }
    const int dl = dims == 1 ? 0 : 1;  // contiguous dimension
    const int lc = ilog2(n[dl]);
    const int64_t units = dims == 1 ? 1 : n[0];
    // at least two stages where possible: the shared buffer is there anyway
    int R = std::min(choose_R(lc, o.radix), std::max(2, 1 << (lc - 1)));
    PassSpec p = contiguous_pass(lc, batch, units, R, o.schedule, o.tile, caps);
    p.conv = 1;
    p.conj_out = 1;
    p.h_dim = dl;
    p.h_lines = conv->lines[dl];
    p.h_scale = conv->scale[dl];
    s.passes.push_back(p);
    if (dims == 2) {
      const int64_t rows = n[0], cols = n[1];
      const int lr = ilog2(rows);
      int Rr = std::min(choose_R(lr, o.radix), std::max(2, 1 << (lr - 1)));
      PassSpec q = fft_pass(lr, Rr, default_schedule(lr, ilog2(Rr)));
      const int64_t B = int64_t(1) << bmax;
      int G = (int)std::min<int64_t>({16, B / rows, cols});
      q.G = G;
      q.lmap = q.smap = MAP_COLS;
      q.count_inner = cols;
      q.tiles_inner = cols / G;
      q.outer = batch;
      q.tiles = batch * q.tiles_inner;
      q.in = Strides{rows * cols, G, 1, cols};
      q.out = q.in;
      q.src = BUF_OUT;
      q.dst = BUF_OUT;
      q.conv = 1;
      q.conj_out = 1;
      q.h_dim = 0;
      q.h_lines = conv->lines[0];
      q.h_scale = conv->scale[0];
      s.passes.push_back(q);
    }
  } else if (dims == 1) {
    const int64_t N = n[0];
    const int logN = ilog2(N);
    if (logN > 24) { fail(FFT_ERR_UNSUPPORTED_SIZE, "1D length must be <= 2^24"); return; }
    if (N == 1) {
      PassSpec p;
      p.kind = PASS_COPY;
      p.copy_count = batch;
      s.passes.push_back(p);
    } else if (precision != FFT_PREC_FP32) {
      // radix-16 stages as DFT matmuls, after a radix-2/4/8 FP32 stage when L
      // is not a power of 16; tiles of max(L, 4096) elements; `units`
      // contiguous transforms of length L per batch entry
      const int tcp = precision == FFT_PREC_TC_FP16_C32 ? FFT_PREC_TC_FP16 : precision;
      const int h16 = precision == FFT_PREC_TC_FP16_C32;
      auto tc_pass = [&](int logL, int64_t units) {
        Sched sch;
        if (logL % 4) sch.push_back(logL % 4);
        for (int i = 0; i < logL / 4; ++i) sch.push_back(4);
        const int logT = logL > 12 ? logL : 12;
        PassSpec p = contiguous_pass(logL, batch, units, 16, 0, 1 << (logT - logL), caps);
        p.rlogs = sch;
        p.G = 1 << (logT - logL);
        p.tiles_inner = (batch * units + p.G - 1) / p.G;
        p.tiles = p.tiles_inner;
        p.in = Strides{0, (int64_t)p.G << logL, int64_t(1) << logL, 1};
        p.out = p.in;
        p.tc_prec = tcp;
        p.io16 = h16;
        p.conj_in = p.conj_out = inv;
        return p;
      };
      if (logN <= 14) {
        s.passes.push_back(tc_pass(logN, 1));
      } else {
        // Six-step (Sec. 3.3 split into passes, with explicit transposes):
        // x viewed as A[n1][n2] (N1 x N2, N = N1 N2, N1 <= N2);
        //   T1  B = A^T                       (N2 rows of N1)
        //   F1  C[n2][.] = DFT_N1(B[n2][.])   (tensor-core rows)
        //   T2  D[k1][n2] = C[n2][k1] w_N^{n2 k1}
        //   F2  E[k1][.] = DFT_N2(D[k1][.])
        //   T3  X[k2 N1 + k1] = E[k1][k2]
        // through two workspace buffers (so in == out is allowed), in
        // sub-batches like the FP32 two-pass plans.
        const int l1 = logN / 2, l2 = logN - l1;
        const int64_t N1 = int64_t(1) << l1, N2 = int64_t(1) << l2;
        const int64_t chunk = two_pass_chunk(N);
        const int64_t cb = std::min(batch, chunk);
        s.chunk_batch = batch > chunk ? chunk : 0;
        s.work_elems = 2 * cb * N;
        s.work2_off = cb * N;
        auto transpose = [&](int64_t rows, int64_t cols, int twiddle_logN, int src, int dst) {
          PassSpec t;
          t.kind = PASS_TRANSPOSE;
          t.tr_rows = rows;
          t.tr_cols = cols;
          t.tr_logN = twiddle_logN;
          t.tr_sign = inv ? 1 : -1;
          t.io16 = h16;
          t.src = src;
          t.dst = dst;
          return t;
        };
        PassSpec f1 = tc_pass(l1, N2), f2 = tc_pass(l2, N1);
        f1.src = f1.dst = BUF_WORK;
        f2.src = f2.dst = BUF_WORK2;
        s.passes.push_back(transpose(N1, N2, 0, BUF_IN, BUF_WORK));
        s.passes.push_back(f1);
        s.passes.push_back(transpose(N2, N1, logN, BUF_WORK, BUF_WORK2));
        s.passes.push_back(f2);
        s.passes.push_back(transpose(N1, N2, 0, BUF_WORK2, BUF_OUT));
      }
    } else if (logN <= bmax) {
      int R = choose_R(logN, o.radix);
      PassSpec p = contiguous_pass(logN, batch, 1, R, o.schedule, o.tile, caps);
      p.conj_in = p.conj_out = inv;
      s.passes.push_back(p);
    } else {
      // Four-step split N = N1 * N2 (Sec. 3.3): columns of length N1, then
      // rows of length N2 written transposed.  N1 <= N2 keeps the strided
      // column tiles wide.
      const int l1 = o.split_log2 ? o.split_log2 : logN / 2, l2 = logN - l1;
      if (l1 < 1 || l2 < 2 || l1 > bmax) {
        fail(FFT_ERR_INVALID_ARG, "split_log2 must leave both passes between 2 and the block limit");
        return;
      }
      if (l2 > bmax) { fail(FFT_ERR_UNSUPPORTED_SIZE, "length needs more than two passes"); return; }
      const int64_t N1 = int64_t(1) << l1, N2 = int64_t(1) << l2;
      const int64_t B = int64_t(1) << bmax;
      // pass 1: column FFTs of length N1 over N2 columns, twiddle on store
      int R1 = choose_R(l1, o.radix);
      PassSpec p1 = fft_pass(l1, R1, sched_for(l1, R1, o.schedule));
      // transforms per tile of the four-step passes: 8 for 1024 points and 4
      // for 2048 (256-thread blocks, two per SM, so one block's stores overlap
      // the other's exchanges) measured faster than 16 / 8 in one 512-thread
      // block (2^20: 84% against 77% of the HBM bandwidth; 2^22: 79% against
      // 78%); 4096-point passes keep 4 (two columns would leave 16-byte rows)
      const auto tile_cap = [](int l) { return l == 10 ? 8 : l == 11 ? 4 : 16; };
      int G1 = (int)std::min<int64_t>({tile_cap(l1), B / N1, N2});
      if (o.tile) G1 = std::min(G1, o.tile);  // columns per tile (tuning)
      p1.G = G1;
      p1.lmap = p1.smap = MAP_COLS;
      p1.count_inner = N2;
      p1.tiles_inner = N2 / G1;
      p1.outer = batch;
      p1.tiles = batch * p1.tiles_inner;
      p1.in = Strides{N, G1, 1, N2};
      p1.out = p1.in;
      p1.src = BUF_IN;
      p1.dst = BUF_WORK;
      p1.conj_in = inv;
      // four-step twiddle source: factored (a sincospi per butterfly and step,
      // powers of the step by products; no table), measured fastest at
      // N = 2^20..2^24; the autotuner also tries the tables and sincospi
      p1.epi = o.epilogue ? o.epilogue : 4;
      p1.epi_logN = logN;
      p1.epi_lo_bits = (logN + 1) / 2;
      // pass 2: row FFTs of length N2 over N1 rows, transposed store
      // the transposed store needs a shared-memory exchange: at least two stages
      int R2 = std::min(choose_R(l2, o.radix), 1 << (l2 - 1));
      PassSpec p2 = fft_pass(l2, R2, default_schedule(l2, ilog2(R2)));
      int G2 = (int)std::min<int64_t>({tile_cap(l2), B / N2, N1});
      if (o.tile) G2 = std::min(G2, o.tile);  // rows per tile (tuning)
      p2.G = G2;
      p2.lmap = MAP_ROWS;
      p2.smap = MAP_COLS;
      p2.count_inner = N1;
      p2.tiles_inner = N1 / G2;
      p2.outer = batch;
      p2.tiles = batch * p2.tiles_inner;
      p2.in = Strides{N, (int64_t)G2 * N2, N2, 1};
      p2.out = Strides{N, G2, 1, N1};
      p2.src = BUF_WORK;
      p2.dst = BUF_OUT;
      p2.conj_out = inv;
      s.passes.push_back(p1);
      s.passes.push_back(p2);
      // sub-batches keep the strided passes' working set bounded; the
      // workspace holds one sub-batch
      const int64_t chunk = two_pass_chunk(N);
      s.chunk_batch = batch > chunk ? chunk : 0;
      s.work_elems = std::min(batch, chunk) * N;
    }
  } else {
    const int64_t rows = n[0], cols = n[1];
    const int lr = ilog2(rows), lc = ilog2(cols);
    if (lr > bmax || lc > bmax)
      { fail(FFT_ERR_UNSUPPORTED_SIZE, "2D lengths must each fit one on-chip block (<= 2^14)"); return; }
    if (rows == 1 && cols == 1) {
      PassSpec p;
      p.kind = PASS_COPY;
      p.copy_count = batch;
      s.passes.push_back(p);
    }
    if (cols > 1) {  // range (row) FFTs: contiguous
      int R = choose_R(lc, o.radix);
      PassSpec p = contiguous_pass(lc, batch, rows, R, o.schedule, 0, caps);
      p.conj_in = inv;
      p.conj_out = inv && rows == 1;
      s.passes.push_back(p);
    }
    if (rows > 1) {  // azimuth (column) FFTs: strided tiles = fused transpose
      int R = choose_R(lr, o.radix);
      PassSpec p = fft_pass(lr, R, default_schedule(lr, ilog2(R)));
      const int64_t B = int64_t(1) << bmax;
      int G = (int)std::min<int64_t>({16, B / rows, cols});
      if (o.tile) G = std::min(G, o.tile);  // columns per tile (tuning)
      p.G = G;
      p.lmap = p.smap = MAP_COLS;
      p.count_inner = cols;
      p.tiles_inner = cols / G;
      p.outer = batch;
      p.tiles = batch * p.tiles_inner;
      p.in = Strides{rows * cols, G, 1, cols};
      p.out = p.in;
      p.src = cols > 1 ? BUF_OUT : BUF_IN;
      p.dst = BUF_OUT;
      p.conj_in = inv && cols == 1;
      p.conj_out = inv;
      s.passes.push_back(p);
    }
  }

  // launch shapes and twiddle tables
  int64_t off = 0;
  for (auto& p : s.passes) {
    p.variant = o.variant;  // kernels without a staged / prefetching form ignore it
    const char* err = nullptr;
    if (!fill_launch(p, caps, err)) { fail(FFT_ERR_INVALID_ARG, err); return; }
    if (p.kind != PASS_FFT) continue;
    p.tw_off.assign(p.rlogs.size(), 0);
    int64_t Ns = int64_t(1) << p.rlogs[0];
    for (size_t st = 1; st < p.rlogs.size(); ++st) {
      const int r = 1 << p.rlogs[st];
      p.tw_off[st] = (int32_t)off;
      // i-major: entry i*Ns + k = w_{Ns*r}^{i*k}
      s.tables.push_back(TwSegment{off, Ns * r, Ns * r, 1, 0, (int)Ns});
      off += Ns * r;
      off = (off + 1) & ~int64_t(1);  // keep 16-byte alignment of segments
      Ns *= r;
    }
    if (p.epi == 1) {
      const int64_t N = int64_t(1) << p.epi_logN;
      const int64_t lo = int64_t(1) << p.epi_lo_bits;
      p.epi_lo_off = off;
      s.tables.push_back(TwSegment{off, lo, N, 1, 1, 1});
      off += lo;
      p.epi_hi_off = off;
      s.tables.push_back(TwSegment{off, N / lo, N, lo, 1, 1});
      off += N / lo;
      off = (off + 1) & ~int64_t(1);
    } else if (p.epi == 2) {
      // entry n2 + k1 * N2 = w_N^{k1 n2}: a stage-style table with r = N2
      const int64_t N = int64_t(1) << p.epi_logN;
      p.epi_lo_off = off;
      p.epi_hi_off = off;
      s.tables.push_back(TwSegment{off, N, N, 1, 0, (int)p.count_inner});
      off += N;
      off = (off + 1) & ~int64_t(1);
    }
  }
  s.table_elems = off;
  for (auto& p : s.passes) {
    if (p.kind == PASS_FFT) {
      int64_t g = p.tiles;
      if (g > 0x7fffffff) g = 0x7fffffff;
      p.grid = (int)g;
    }
  }
}

PassDesc pass_desc(const PassSpec& p, int64_t b0, int64_t nb, int64_t n_total) {
  (void)n_total;
  PassDesc d{};
  d.logL = p.logL;
  d.nst = (int)p.rlogs.size();
  for (size_t i = 0; i < p.rlogs.size() && i < 15; ++i) {
    d.rlog[i] = p.rlogs[i];
    d.tw_off[i] = i < p.tw_off.size() ? p.tw_off[i] : 0;
  }
  d.G = p.G;
  d.T = (1 << p.logL) / p.R;
  d.pitch = p.pitch;
  d.smem_elems = p.smem_elems;
  if (p.batch_is_tiles) {
    const int64_t units = nb * p.units_per_batch;
    d.count_inner = units;
    d.tiles_inner = (units + p.G - 1) / p.G;
    d.tiles = d.tiles_inner;
  } else {
    d.count_inner = p.count_inner;
    d.tiles_inner = p.tiles_inner;
    d.tiles = nb * p.tiles_inner;
  }
  d.in = p.in;
  d.out = p.out;
  d.conj_in = p.conj_in;
  d.conj_out = p.conj_out;
  d.epi = p.epi;
  d.epi_lo_bits = p.epi_lo_bits;
  d.epi_logN = p.epi_logN;
  d.conv = p.conv;
  d.h_scale = p.h_scale;
  d.h_lines = p.h_lines > 0 ? p.h_lines : 1;
  // line u of a sub-batch starting at entry b0 is line b0 * units + u overall
  d.h_first = p.batch_is_tiles ? (b0 * p.units_per_batch) % d.h_lines : 0;
  return d;
}

std::string describe(const PlanSpec& s) {
  std::ostringstream o;
  o << "{\"dims\":" << s.dims << ",\"n\":[" << s.n[0];
  if (s.dims == 2) o << "," << s.n[1];
  o << "],\"batch\":" << s.batch << ",\"direction\":" << s.direction
    << ",\"precision\":" << s.precision << ",\"max_block_log2\":" << s.max_block_log2
    << ",\"generic\":" << (s.generic_only ? 1 : 0) << ",\"conv\":" << (s.conv ? 1 : 0)
    << ",\"workspace_bytes\":" << s.work_elems * 8 << ",\"table_elems\":" << s.table_elems
    << ",\"chunk_batch\":" << s.chunk_batch
    << ",\"passes\":[";
  for (size_t i = 0; i < s.passes.size(); ++i) {
    const PassSpec& p = s.passes[i];
    if (i) o << ",";
    o << "{\"kind\":\""
      << (p.kind == PASS_FFT ? "fft" : p.kind == PASS_COPY ? "copy" : "transpose") << "\"";
    if (p.kind == PASS_TRANSPOSE)
      o << ",\"rows\":" << p.tr_rows << ",\"cols\":" << p.tr_cols << ",\"twiddle_logN\":"
        << p.tr_logN << ",\"io16\":" << p.io16;
    if (p.kind == PASS_FFT) {
      o << ",\"L\":" << (1 << p.logL) << ",\"R\":" << p.R << ",\"G\":" << p.G
        << ",\"lmap\":\"" << (p.lmap ? "cols" : "rows") << "\",\"smap\":\""
        << (p.smap ? "cols" : "rows") << "\",\"radices\":[";
      for (size_t j = 0; j < p.rlogs.size(); ++j) o << (j ? "," : "") << (1 << p.rlogs[j]);
      o << "],\"tiles\":" << p.tiles << ",\"tiles_inner\":" << p.tiles_inner
        << ",\"count_inner\":" << p.count_inner << ",\"outer\":" << p.outer
        << ",\"in\":[" << p.in.o << "," << p.in.t << "," << p.in.g << "," << p.in.e << "]"
        << ",\"out\":[" << p.out.o << "," << p.out.t << "," << p.out.g << "," << p.out.e << "]"
        << ",\"block\":" << p.block << ",\"grid\":" << p.grid << ",\"smem\":" << p.smem
        << ",\"pitch\":" << p.pitch << ",\"epi\":" << p.epi << ",\"epi_logN\":" << p.epi_logN
        << ",\"conj_in\":" << p.conj_in << ",\"conj_out\":" << p.conj_out
        << ",\"variant\":" << p.variant << ",\"tc_prec\":" << p.tc_prec
        << ",\"io16\":" << p.io16;
      if (p.conv)
        o << ",\"conv\":1,\"h_dim\":" << p.h_dim << ",\"h_lines\":" << p.h_lines
          << ",\"h_scale\":" << p.h_scale;
    } else {
      o << ",\"count\":" << p.copy_count;
    }
    o << ",\"src\":" << p.src << ",\"dst\":" << p.dst << "}";
  }
  o << "]";
  if (s.tuning[0]) o << ",\"tuning\":" << s.tuning;
  o << "}";
  return o.str();
}

// ------------------------------------------------- schedule digraph --------

static bool edge_cost(int log2n, const int* radix_logs, int j, const double* cost, int s,
                      double& c) {
  if (s + radix_logs[j] > log2n) return false;
  c = cost[(size_t)j * log2n + s];
  return !(c < 0) && c == c;
}

uint64_t count_schedules(int log2n, const int* radix_logs, int n_radix) {
  std::vector<uint64_t> ways(log2n + 1, 0);
  ways[0] = 1;
  for (int s = 0; s < log2n; ++s)
    for (int j = 0; j < n_radix; ++j) {
      int t = s + radix_logs[j];
      if (radix_logs[j] >= 1 && t <= log2n) ways[t] += ways[s];
    }
  return ways[log2n];
}

bool shortest_schedule(int log2n, const int* radix_logs, int n_radix, const double* cost,
                       std::vector<int>& path, double& total) {
  const double INF = std::numeric_limits<double>::infinity();
  std::vector<double> dist(log2n + 1, INF);
  std::vector<int> prev(log2n + 1, -1), via(log2n + 1, -1);
  std::vector<char> done(log2n + 1, 0);
  dist[0] = 0;
  // Dijkstra over the stage nodes (Sec. 3.2); the graph is tiny, so a linear
  // scan for the closest unsettled node is enough.
  for (int it = 0; it <= log2n; ++it) {
    int u = -1;
    for (int v = 0; v <= log2n; ++v)
      if (!done[v] && dist[v] < INF && (u < 0 || dist[v] < dist[u])) u = v;
    if (u < 0) break;
    done[u] = 1;
    for (int j = 0; j < n_radix; ++j) {
      double c;
      if (radix_logs[j] < 1 || !edge_cost(log2n, radix_logs, j, cost, u, c)) continue;
      int v = u + radix_logs[j];
      if (dist[u] + c < dist[v]) {
        dist[v] = dist[u] + c;
        prev[v] = u;
        via[v] = radix_logs[j];
      }
    }
  }
  if (!(dist[log2n] < INF)) return false;
  path.clear();
  for (int v = log2n; v > 0; v = prev[v]) path.push_back(via[v]);
  std::reverse(path.begin(), path.end());
  total = dist[log2n];
  return true;
}

bool schedule_cost(int log2n, const int* radix_logs, int n_radix, const double* cost,
                   const int* path, int len, double& total) {
  int s = 0;
  total = 0;
  for (int i = 0; i < len; ++i) {
    int j = -1;
    for (int k = 0; k < n_radix; ++k)
      if (radix_logs[k] == path[i]) j = k;
    double c;
    if (j < 0 || !edge_cost(log2n, radix_logs, j, cost, s, c)) return false;
    total += c;
    s += path[i];
  }
  return s == log2n;
}

}  // namespace gbfft
