// Kernels of the tensor-core class on tcgen05 with complex64 input and output
// (the kernel body and its design: umma_kernel.cuh).
#include "umma_kernel.cuh"

namespace gbfft {

const void* resolve_umma(int logL, int prec, size_t* smem) {
#define GB_UMMA(LG)                                                              \
  if (logL == LG) {                                                              \
    if (prec == TC_FP16) {                                                       \
      *smem = Umma<LG, TC_FP16>::SMEM + 1024 + umma_staging_bytes(LG, 8, false); \
      return (const void*)stockham_umma<LG, TC_FP16, false>;                     \
    }                                                                            \
    if (prec == TC_BF16) {                                                       \
      *smem = Umma<LG, TC_BF16>::SMEM + 1024 + umma_staging_bytes(LG, 8, false); \
      return (const void*)stockham_umma<LG, TC_BF16, false>;                     \
    }                                                                            \
    if (prec == TC_BF16X3) {                                                     \
      *smem = Umma<LG, TC_BF16X3>::SMEM + 1024 + umma_staging_bytes(LG, 8, true); \
      return (const void*)stockham_umma<LG, TC_BF16X3, false>;                   \
    }                                                                            \
  }
  GB_UMMA(4) GB_UMMA(5) GB_UMMA(6) GB_UMMA(7) GB_UMMA(8) GB_UMMA(9) GB_UMMA(10) GB_UMMA(11)
  GB_UMMA(12) GB_UMMA(13) GB_UMMA(14)
#undef GB_UMMA
  return nullptr;
}

// Tensor-memory columns one CTA of this length allocates.
int umma_tmem_cols(int logL) {
  const int logT = logL > 12 ? logL : 12;
  return 32 * ((1 << (logT - 4)) / 128);
}

}  // namespace gbfft
