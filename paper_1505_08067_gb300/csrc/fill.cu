// Seeded synthetic inputs generated on the device: complex64 values with real
// and imaginary parts uniform in [-1, 1), from a counter-based hash, so a
// workload of any size is produced in place at memory speed and any slice of
// it can be regenerated independently (on the host too: synth.uniform_hash
// implements the same generator).
//
// Generator: SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom
// number generators", OOPSLA 2014) evaluated at a counter: for stream index k
// the state is seed + (k + 1) * 0x9E3779B97F4A7C15, mixed by
//   z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9
//   z = (z ^ (z >> 27)) * 0x94D049BB133111EB
//   z =  z ^ (z >> 31)
// (64-bit wrap-around arithmetic).  The top 24 bits give u = (z >> 40) * 2^-24
// in [0, 1) and the value 2u - 1, exact in FP32.  Element j uses stream
// indices 2j (real part) and 2j + 1 (imaginary part).
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/gbfft.h"

namespace gbfft {
fft_status_t set_error(fft_status_t st, const char* msg);
}

namespace {

__device__ __forceinline__ float hash_uniform(uint64_t seed, uint64_t k) {
  uint64_t z = seed + (k + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return 2.0f * ((float)(uint32_t)(z >> 40) * 5.9604644775390625e-08f) - 1.0f;  // 2^-24
}

__global__ void fill_uniform_kernel(float2* out, int64_t count, uint64_t seed, uint64_t first) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < count;
       j += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t k = 2 * (first + (uint64_t)j);
    out[j] = make_float2(hash_uniform(seed, k), hash_uniform(seed, k + 1));
  }
}

}  // namespace

extern "C" fft_status_t fft_fill_uniform(void* out, int64_t count, uint64_t seed, uint64_t first,
                                         void* stream) {
  if (count < 0) return gbfft::set_error(FFT_ERR_INVALID_ARG, "count must be >= 0");
  if (count == 0) return FFT_OK;
  if (!out || ((uintptr_t)out & 7))
    return gbfft::set_error(FFT_ERR_INVALID_ARG, "out must be an 8-byte aligned device pointer");
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return gbfft::set_error(FFT_ERR_CUDA, "no usable CUDA device");
  }
  int64_t blocks = (count + 255) / 256;
  if (blocks > (int64_t)sms * 32) blocks = (int64_t)sms * 32;
  fill_uniform_kernel<<<(int)blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(
      static_cast<float2*>(out), count, seed, first);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return gbfft::set_error(FFT_ERR_CUDA, cudaGetErrorString(e));
  return FFT_OK;
}
