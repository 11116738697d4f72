// Binding a plan's passes to device pointers and enqueueing them; shared by the
// plan objects of the C ABI and by entry points that keep their tables and
// workspace elsewhere.
#pragma once
#include <cuda_runtime.h>

#include "kernels.h"
#include "planner.h"

namespace gbfft {

// Fills launches[i] for every pass of `s` (tables = device twiddle tables of
// s.table_elems entries).  Resolves and prepares each kernel.
// `status` is a device int the staged kernels set if a bounded wait gives up.
cudaError_t bind_launches(const PlanSpec& s, const Caps& caps, const cf* tables, int* status,
                          PassLaunch* launches);

// Enqueues the twiddle-table generation of `s` into `tables` on `st`.
cudaError_t enqueue_tables(const PlanSpec& s, cf* tables, cudaStream_t st);

// Enqueues every pass for batch entries [b0, b0 + nb); `in` and `out` already
// point at entry b0, `work` holds min(nb, s.chunk_batch) entries (all nb when
// the plan has no sub-batches) starting with entry b0.  Two-pass plans with
// chunk_batch > 0 run in sub-batches of chunk_batch entries, in stream order.
// work2_off: offset (elements) of a six-step plan's second workspace buffer
// when the workspace was sized for fewer transforms than the plan's (a
// server job's own workspace); -1 = the plan's.
cudaError_t enqueue_passes(const PlanSpec& s, const PassLaunch* launches, const void* in,
                           void* out, void* work, int64_t b0, int64_t nb, cudaStream_t st,
                           int64_t work2_off = -1);

}  // namespace gbfft
