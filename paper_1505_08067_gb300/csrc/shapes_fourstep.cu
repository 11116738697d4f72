// Compile-time instantiations of the four-step column/row passes and the 2D
// column pass; see kernel_shapes.h.
#include "kernels_impl.cuh"

namespace gbfft {

const void* resolve_fourstep_shape(int R, int lmap, int smap, const PassDesc& d) {
#define GB_TRY(LOGL, SCHED, NST, RR, G, LM, SM, CONTIG, EPI)                                 \
  if (shape_matches(d, R, lmap, smap, LOGL, SCHED, NST, RR, G, LM, SM, CONTIG, EPI))         \
    return (const void*)kfn<RR, LM, SM, CtTraits<LOGL, SCHED, NST, RR, G, CONTIG, EPI>>();
  GB_SHAPES_FOURSTEP(GB_TRY)
#undef GB_TRY
  return nullptr;
}

// Staged column tiles (see GB_STAGED_COLS_SHAPES).
bool resolve_staged_cols_shape(const PassDesc& d, int lmap, int smap, StagedLaunch* s) {
#define GB_STAGED_COLS(LOGL, SCHED, NST, RR, G, EPI, CONV)                         \
  if (staged_cols_matches(d, lmap, smap, LOGL, SCHED, NST, G, EPI, CONV)) {         \
    using SH = SplitShape<LOGL, SCHED, NST, RR, G, EPI>;                           \
    s->fn = (const void*)staged_fn<SH, (SH::kT <= 256 ? 2 : 1), CONV != 0>();                           \
    s->block = SH::kT;                                                             \
    s->smem = split_smem_bytes<SH>();                                              \
    return true;                                                                   \
  }
  GB_STAGED_COLS_SHAPES(GB_STAGED_COLS)
#undef GB_STAGED_COLS
  return false;
}

// Staged transposing passes (see GB_STAGED_TRANS_SHAPES).
bool resolve_staged_trans_shape(const PassDesc& d, int lmap, int smap, StagedLaunch* s) {
#define GB_STAGED_TRANS(LOGL, SCHED, NST, RR, G)                                     \
  if (staged_trans_matches(d, lmap, smap, LOGL, SCHED, NST, G)) {                    \
    using SH = SplitShape<LOGL, SCHED, NST, RR, G, 0, true>;                         \
    s->fn = (const void*)staged_fn<SH, (SH::kT <= 256 ? 2 : 1), false>();                                  \
    s->block = SH::kT;                                                               \
    s->smem = split_smem_bytes<SH>();                                                \
    return true;                                                                     \
  }
  GB_STAGED_TRANS_SHAPES(GB_STAGED_TRANS)
#undef GB_STAGED_TRANS
  return false;
}

}  // namespace gbfft
