// Fast-convolution passes (matched filtering, e.g. SAR range and azimuth
// compression): generic kernels for every (R, map) and the compile-time
// shapes of GB_SHAPES_CONV.  See conv_tile in kernels_impl.cuh.
#include "kernels_impl.cuh"

namespace gbfft {

template <int R, int MAP, class TR>
static const void* conv_fn() {
  return (const void*)stockham_conv<R, MAP, TR>;
}

static const void* generic_conv(int R, int map) {
#define GB_GEN(RR)                                                           \
  if (R == RR) return map == MAP_ROWS ? conv_fn<RR, MAP_ROWS, RtTraits>()    \
                                      : conv_fn<RR, MAP_COLS, RtTraits>();
  GB_GEN(2) GB_GEN(4) GB_GEN(8) GB_GEN(16)
#undef GB_GEN
  return nullptr;
}

const void* resolve_conv_kernel(int R, int map, const PassDesc& d, bool generic_only,
                                bool* specialised) {
  if (specialised) *specialised = false;
  if (map != MAP_ROWS && map != MAP_COLS) return nullptr;
  if (!generic_only) {
#define GB_TRY(LOGL, SCHED, NST, RR, G, LM, SM, CONTIG, EPI)                                  \
  if (shape_matches(d, R, map, map, LOGL, SCHED, NST, RR, G, LM, SM, CONTIG, EPI)) {          \
    if (specialised) *specialised = true;                                                    \
    return conv_fn<RR, LM, CtTraits<LOGL, SCHED, NST, RR, G, CONTIG, EPI>>();                 \
  }
    GB_SHAPES_CONV(GB_TRY)
#undef GB_TRY
  }
  return generic_conv(R, map);
}

// Staged convolution kernels: one contiguous line per block, the next line
// copied into shared memory by TMA, the filter applied in registers between
// the two rounds.
bool resolve_conv_staged_shape(const PassDesc& d, StagedLaunch* s) {
#define GB_STAGED(LOGL, SCHED, NST, MINB, RR)                  \
  if (staged_shape_matches(d, LOGL, SCHED, NST, true)) {       \
    using SH = SplitShape<LOGL, SCHED, NST, RR>;               \
    s->fn = (const void*)staged_fn<SH, MINB, true>();          \
    s->block = SH::kT;                                         \
    s->smem = split_smem_bytes<SH>();                          \
    return true;                                               \
  }
  GB_STAGED_SHAPES(GB_STAGED)
#undef GB_STAGED
  return false;
}

}  // namespace gbfft
