// Host-side bookkeeping of the work queue's ring (no CUDA; see queue.cu).
// Ticket t (1, 2, ...) lives in slot (t - 1) mod slots.  The worker completes
// tickets in order and writes each completed ticket into its slot's done
// word, so a slot's done word only grows.
#pragma once
#include <stdint.h>

namespace gbfft {

// Highest ticket c with every ticket up to c complete, starting from the
// known `completed` (< issued possible) and reading slot done words through
// done_at(slot).  Ticket t is complete once its slot shows t or a later
// ticket: the slot may already have been reused and completed again before
// the host looks.
template <class DoneAt>
uint64_t ring_completed(uint64_t completed, uint64_t issued, int slots, DoneAt done_at) {
  while (completed < issued) {
    const uint64_t t = completed + 1;
    if (done_at((int)((t - 1) % (uint64_t)slots)) < t) break;
    completed = t;
  }
  return completed;
}

// May ticket t be written into its slot, whose done word is `done`?  Only
// once the slot's previous ticket (t - slots) is complete.
inline bool ring_slot_free(uint64_t t, int slots, uint64_t done) {
  return t <= (uint64_t)slots || done >= t - (uint64_t)slots;
}

}  // namespace gbfft
