// Plan-time autotuner (Sec. 3.2 model + runtime validation); see autotune.cpp.
#pragma once
#include <stddef.h>

#include "../../include/gbfft.h"
#include "planner.h"

namespace gbfft {

// Chooses plan options for (n, dims, batch, direction) on the current device
// (`device`), starting from the caller's options `base` (fields the caller set
// are kept).  Times candidate plans on trial buffers; may allocate device
// memory while it runs.  Writes a JSON report of what it measured.
fft_status_t autotune_options(const int64_t* n, int dims, int64_t batch, int direction,
                              const fft_plan_options_t& base, const Caps& caps, int device,
                              fft_plan_options_t* chosen, char* report, size_t report_len);

fft_status_t set_error(fft_status_t st, const char* msg);

}  // namespace gbfft
