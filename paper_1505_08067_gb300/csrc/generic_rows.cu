// Generic stockham_pass instantiations (every parameter from the
// descriptor) for load map 0 / store map 0; see kernels.cu.
#include "kernels_impl.cuh"

namespace gbfft {

const void* generic_kernel_rows(int R) {
  switch (R) {
    case 2: return (const void*)kfn<2, 0, 0, RtTraits>();
    case 4: return (const void*)kfn<4, 0, 0, RtTraits>();
    case 8: return (const void*)kfn<8, 0, 0, RtTraits>();
    case 16: return (const void*)kfn<16, 0, 0, RtTraits>();
    default: return nullptr;
  }
}

}  // namespace gbfft
