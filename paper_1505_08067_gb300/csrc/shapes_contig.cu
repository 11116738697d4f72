// Compile-time instantiations of the batched contiguous shapes (register and
// TMA-staged kernels); see kernel_shapes.h.
#include "kernels_impl.cuh"

namespace gbfft {

const void* resolve_contig_shape(int R, int lmap, int smap, const PassDesc& d) {
#define GB_TRY(LOGL, SCHED, NST, RR, G, LM, SM, CONTIG, EPI)                                 \
  if (shape_matches(d, R, lmap, smap, LOGL, SCHED, NST, RR, G, LM, SM, CONTIG, EPI))         \
    return (const void*)kfn<RR, LM, SM, CtTraits<LOGL, SCHED, NST, RR, G, CONTIG, EPI>>();
  GB_SHAPES_CONTIG(GB_TRY)
#undef GB_TRY
  return nullptr;
}

bool resolve_staged_shape(const PassDesc& d, StagedLaunch* s) {
#define GB_STAGED(LOGL, SCHED, NST, MINB, RR)                \
  if (staged_shape_matches(d, LOGL, SCHED, NST)) {           \
    using SH = SplitShape<LOGL, SCHED, NST, RR>;             \
    s->fn = (const void*)staged_fn<SH, MINB>();              \
    s->block = SH::kT;                                       \
    s->smem = split_smem_bytes<SH>();                        \
    return true;                                             \
  }
  GB_STAGED_SHAPES(GB_STAGED)
#undef GB_STAGED
  return false;
}

}  // namespace gbfft
