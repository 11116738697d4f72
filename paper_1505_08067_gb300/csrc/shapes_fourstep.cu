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

}  // namespace gbfft
