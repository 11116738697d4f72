// Host-side launch interface of the device kernels in kernels.cu.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

#include "fft_core.h"

namespace gbfft {

// Everything needed to launch one stockham_pass.
struct PassLaunch {
  PassDesc d;
  int R;            // elements per thread (register radix): 2, 4, 8 or 16
  int lmap, smap;   // thread maps of the load (and middle) stages and of the store
  int grid, block;  // grid size (tiles are grid-strided) and threads per block
  size_t smem;      // dynamic shared memory in bytes
};

cudaError_t launch_pass(const PassLaunch& p, const void* in, void* out, cudaStream_t st);
cudaError_t kernel_attributes(int R, int lmap, int smap, cudaFuncAttributes* attr);
cudaError_t occupancy(int R, int lmap, int smap, int block, size_t smem, int* ctas_per_sm);
cudaError_t launch_copy(const void* in, void* out, int64_t count, int64_t in_stride,
                        int64_t out_stride, cudaStream_t st);
cudaError_t launch_twiddle_gen(void* out, int64_t count, int64_t den, int mode, int r,
                               int64_t mult, cudaStream_t st);

}  // namespace gbfft
