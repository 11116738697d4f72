// Kernels of the FP16 tensor-core class on tcgen05 with complex32 input and
// output (FP16 real and imaginary parts, 4 bytes per element; the kernel body
// and its design: umma_kernel.cuh).
#include "umma_kernel.cuh"

namespace gbfft {

const void* resolve_umma_c32(int logL, size_t* smem) {
#define GB_UMMA(LG)                                                              \
  if (logL == LG) {                                                              \
    *smem = Umma<LG, TC_FP16, true>::SMEM + 1024 + umma_staging_bytes(LG, 4, false); \
    return (const void*)stockham_umma<LG, TC_FP16, true>;                        \
  }
  GB_UMMA(4) GB_UMMA(5) GB_UMMA(6) GB_UMMA(7) GB_UMMA(8) GB_UMMA(9) GB_UMMA(10) GB_UMMA(11)
  GB_UMMA(12) GB_UMMA(13) GB_UMMA(14)
#undef GB_UMMA
  return nullptr;
}

}  // namespace gbfft
