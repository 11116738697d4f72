// fft_wait_selftest (include/gbfft.h): the library's bounded mbarrier wait,
// run where it must give up.
#include <cuda_runtime.h>

#include "../../include/gbfft.h"
#include "kernels_impl.cuh"

namespace gbfft {

fft_status_t set_error(fft_status_t st, const char* msg);

// One block: thread 0 initialises an mbarrier expecting one arrival that
// never comes; every thread waits on its first phase with the kernels' wait
// loop (mbar_wait), limited to `polls`; a give-up on any thread sets *status.
__global__ void wait_selftest_kernel(int* status, uint32_t polls) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) mbar_init(&bar, 1);
  __syncthreads();
  const bool ok = mbar_wait(&bar, 0, polls);
  if (__syncthreads_or(!ok) && threadIdx.x == 0) atomicExch(status, 1);
}

}  // namespace gbfft

extern "C" fft_status_t fft_wait_selftest(uint32_t polls, int* gave_up) {
  using namespace gbfft;
  if (!gave_up || polls < 1 || polls > kWaitPolls)
    return set_error(FFT_ERR_INVALID_ARG, "fft_wait_selftest: polls must be 1 .. 2^22");
  int* status = nullptr;
  cudaError_t e = cudaMalloc(&status, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(status, 0, sizeof(int));
  if (e == cudaSuccess) {
    wait_selftest_kernel<<<1, 128>>>(status, polls);
    e = cudaGetLastError();
  }
  int h = 0;
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(&h, status, sizeof(int), cudaMemcpyDeviceToHost);
  if (status) cudaFree(status);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_error(FFT_ERR_CUDA, cudaGetErrorString(e));
  }
  *gave_up = h;
  return FFT_OK;
}
