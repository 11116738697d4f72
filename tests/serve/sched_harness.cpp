// Test infrastructure: drives the serving scheduler (csrc/scheduler.h) with a
// simulated device in discrete time steps.  Jobs arrive at given steps and run
// for given numbers of steps once launched (the scheduler's cost estimate is
// that exact duration); a group runs its jobs one after another.  Reports
// when each job launched, which group it joined, when it finished, the peak
// bytes in flight and which jobs were rejected.
#include <stdint.h>

#include <vector>

#include "scheduler.h"

using namespace gbfft;

extern "C" int sched_simulate(int n, const int* key, const uint64_t* bytes, const int* arrive,
                              const int* dur, const int* groupable, uint64_t budget, int max_group,
                              int backfill, int* launch_step, int* group_id, int* done_step,
                              uint64_t* peak_in_flight, int* rejected) {
  Scheduler s(budget, max_group, budget, backfill != 0);
  struct Run {
    SchedGroup g;
    int end;
  };
  std::vector<Run> running;
  int next_job = 0, finished = 0, gid = 0, step = 0;
  for (int i = 0; i < n; ++i) {
    launch_step[i] = -1;
    group_id[i] = -1;
    done_step[i] = -1;
    rejected[i] = 0;
  }
  while (finished < n && step < 1000000) {
    // completions
    for (size_t r = 0; r < running.size();) {
      if (running[r].end <= step) {
        for (auto& j : running[r].g.jobs) {
          done_step[j.id] = step;
          ++finished;
        }
        s.finished(running[r].g);
        running.erase(running.begin() + r);
      } else {
        ++r;
      }
    }
    // arrivals
    while (next_job < n && arrive[next_job] <= step) {
      SchedJob j;
      j.id = (uint64_t)next_job;
      j.key.n0 = key[next_job];
      j.bytes = (size_t)bytes[next_job];
      j.groupable = groupable[next_job] != 0;
      j.cost = dur[next_job];
      if (!s.submit(j)) {
        rejected[next_job] = 1;
        ++finished;
      }
      ++next_job;
    }
    // launches
    SchedGroup g;
    while (s.next(g, step)) {
      int end = step;
      for (auto& j : g.jobs) {
        launch_step[j.id] = step;
        group_id[j.id] = gid;
        end += dur[j.id];
      }
      if (s.in_flight() > budget) return -1;  // accounting broke the budget
      running.push_back(Run{g, end});
      ++gid;
    }
    ++step;
  }
  *peak_in_flight = s.peak_in_flight();
  return step;
}
