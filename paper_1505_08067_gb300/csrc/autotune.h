// Plan-time autotuner (Sec. 3.2): per-(radix, start stage) stage costs are
// benchmarked on this GPU, the shortest path over the schedule digraph gives
// the model's best radix schedule, and the model's choice is checked against
// timings of whole passes before it is kept.
#pragma once
#include "../../include/gbfft.h"
#include "planner.h"

namespace gbfft {

// Retunes the passes of `spec` in place (radix schedule, elements per thread,
// tile) using the plan's device tables and workspace for trial launches.
fft_status_t autotune_plan(PlanSpec& spec, const Caps& caps, void* tables, void* work);

fft_status_t set_error(fft_status_t st, const char* msg);

}  // namespace gbfft
