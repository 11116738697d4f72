// Serving scheduler: admission by device-memory budget and coalescing of
// same-shape jobs, independent of CUDA so that its policy can be exercised on
// a host without a GPU.  The server (server.cpp) owns one and drives it with
// CUDA streams and events; the test harness drives it with a fake device.
//
// Policy (continuous batching): jobs queue in arrival order.  Whenever the
// device side can take work, the oldest waiting job is launched together with
// every later waiting job of the same key (shape, direction, precision) that
// fits the group limits -- one coalesced launch.  A group is admitted only if
// the bytes it holds while running (inputs, outputs, workspace) fit in the
// budget next to everything already running; otherwise it waits for running
// groups to finish and release their bytes.  Admission is strictly in order of
// the oldest job, so no job is starved by smaller ones behind it.  A job larger
// than the whole budget is rejected.  Finished groups free their bytes at once,
// so jobs that arrive while others run are admitted as memory frees up.
#pragma once
#include <stddef.h>
#include <stdint.h>

#include <algorithm>
#include <deque>
#include <vector>

namespace gbfft {

struct JobKey {
  int dims = 1;
  int64_t n0 = 1, n1 = 1;
  int direction = -1;
  int precision = 0;
  bool operator==(const JobKey& o) const {
    return dims == o.dims && n0 == o.n0 && n1 == o.n1 && direction == o.direction &&
           precision == o.precision;
  }
};

struct SchedJob {
  uint64_t id = 0;
  JobKey key;
  int64_t batch = 0;
  size_t bytes = 0;        // held while running: in + out + workspace
  bool groupable = true;   // may share a launch with other jobs of its key
  double t_submit = 0;
};

struct SchedGroup {
  std::vector<SchedJob> jobs;
  size_t bytes = 0;
};

class Scheduler {
 public:
  Scheduler(size_t budget, int max_group, size_t max_group_bytes)
      : budget_(budget), max_group_(max_group), max_group_bytes_(max_group_bytes) {}

  // False if the job can never run (larger than the budget).
  bool submit(const SchedJob& j) {
    if (j.bytes > budget_) return false;
    pending_.push_back(j);
    return true;
  }

  // The next group to launch, if the oldest waiting job's group fits now.
  bool next(SchedGroup& g) {
    g.jobs.clear();
    g.bytes = 0;
    if (pending_.empty()) return false;
    const SchedJob head = pending_.front();
    if (in_flight_ + head.bytes > budget_) return false;
    g.jobs.push_back(head);
    g.bytes = head.bytes;
    pending_.pop_front();
    if (head.groupable) {
      for (auto it = pending_.begin(); it != pending_.end() && (int)g.jobs.size() < max_group_;) {
        if (it->groupable && it->key == head.key && g.bytes + it->bytes <= max_group_bytes_ &&
            in_flight_ + g.bytes + it->bytes <= budget_) {
          g.jobs.push_back(*it);
          g.bytes += it->bytes;
          it = pending_.erase(it);
        } else {
          ++it;
        }
      }
    }
    in_flight_ += g.bytes;
    peak_in_flight_ = std::max(peak_in_flight_, in_flight_);
    ++groups_;
    jobs_launched_ += g.jobs.size();
    return true;
  }

  void finished(const SchedGroup& g) { in_flight_ -= std::min(in_flight_, g.bytes); }

  size_t in_flight() const { return in_flight_; }
  size_t peak_in_flight() const { return peak_in_flight_; }
  size_t budget() const { return budget_; }
  size_t waiting() const { return pending_.size(); }
  uint64_t groups() const { return groups_; }
  uint64_t jobs_launched() const { return jobs_launched_; }

 private:
  size_t budget_;
  int max_group_;
  size_t max_group_bytes_;
  std::deque<SchedJob> pending_;
  size_t in_flight_ = 0, peak_in_flight_ = 0;
  uint64_t groups_ = 0, jobs_launched_ = 0;
};

}  // namespace gbfft
