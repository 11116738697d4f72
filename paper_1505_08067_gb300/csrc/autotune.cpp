#include "autotune.h"

namespace gbfft {

fft_status_t autotune_plan(PlanSpec& spec, const Caps& caps, void* tables, void* work) {
  (void)spec;
  (void)caps;
  (void)tables;
  (void)work;
  return set_error(FFT_ERR_NOT_IMPLEMENTED, "autotuning is not built yet");
}

}  // namespace gbfft
