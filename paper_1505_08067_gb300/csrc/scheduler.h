// Serving scheduler: admission by device-memory budget and coalescing of
// same-shape jobs, independent of CUDA so that its policy can be exercised on
// a host without a GPU.  The server (server.cpp) owns one and drives it with
// CUDA streams and events; the test harness drives it with a fake device.
//
// Policy (continuous batching): jobs queue in arrival order.  Whenever the
// device side can take work, the oldest waiting job (the head) is launched
// together with every later waiting job of the same key (shape, direction,
// precision) that fits the group limits -- one coalesced launch.  A group is
// admitted only if the bytes it holds while running (inputs, outputs,
// workspace) fit in the budget next to everything already running.  A job
// larger than the whole budget is rejected.  Finished groups free their bytes
// at once, so jobs that arrive while others run are admitted as memory frees
// up.
//
// Backfilling (unless strict arrival order is asked for): when the head does
// not fit, it gets a reservation -- the estimated time at which enough running
// groups will have finished (each job carries an estimated run time, `cost`)
// and the bytes left over next to it then.  A later job may start at once if
// it fits now and either ends before the reservation or fits in the bytes
// left over next to the head: with exact estimates a backfilled job never
// delays the head (the EASY backfilling rule of batch schedulers, with memory
// in place of processors).  Small jobs then stop queueing behind a large one
// that waits for memory.
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
  double cost = 0;         // estimated run time (the unit of `now` in next())
};

struct SchedGroup {
  std::vector<SchedJob> jobs;
  size_t bytes = 0;
  double cost = 0;         // sum of the jobs' costs: they run one after another
  uint64_t seq = 0;        // admission number (matches finished() to next())
};

class Scheduler {
 public:
  Scheduler(size_t budget, int max_group, size_t max_group_bytes, bool backfill = true)
      : budget_(budget), max_group_(max_group), max_group_bytes_(max_group_bytes),
        backfill_(backfill) {}

  // False if the job can never run (larger than the budget).
  bool submit(const SchedJob& j) {
    if (j.bytes > budget_) return false;
    pending_.push_back(j);
    return true;
  }

  // The next group to launch at time `now`: the head's group if it fits,
  // else (backfilling) a later job that cannot delay the head.
  bool next(SchedGroup& g, double now = 0) {
    g.jobs.clear();
    g.bytes = 0;
    g.cost = 0;
    if (pending_.empty()) return false;
    const SchedJob head = pending_.front();
    if (in_flight_ + head.bytes <= budget_) {
      take(g, pending_.begin(), now, nullptr);
    } else {
      if (!backfill_) return false;
      double shadow;
      size_t extra;
      reservation(head.bytes, now, shadow, extra);
      auto pick = pending_.end();
      int scanned = 0;
      for (auto it = pending_.begin() + 1; it != pending_.end() && scanned < kScan; ++it, ++scanned)
        if (can_backfill(*it, now, shadow, extra)) {
          pick = it;
          break;
        }
      if (pick == pending_.end()) return false;
      Limits lim{now, shadow, extra};
      take(g, pick, now, &lim);
    }
    in_flight_ += g.bytes;
    peak_in_flight_ = std::max(peak_in_flight_, in_flight_);
    g.seq = ++groups_;
    jobs_launched_ += g.jobs.size();
    running_.push_back(Run{g.seq, g.bytes, now + g.cost});
    return true;
  }

  void finished(const SchedGroup& g) {
    in_flight_ -= std::min(in_flight_, g.bytes);
    for (size_t i = 0; i < running_.size(); ++i)
      if (running_[i].seq == g.seq) {
        running_.erase(running_.begin() + i);
        break;
      }
  }

  size_t in_flight() const { return in_flight_; }
  size_t peak_in_flight() const { return peak_in_flight_; }
  size_t budget() const { return budget_; }
  size_t waiting() const { return pending_.size(); }
  uint64_t groups() const { return groups_; }
  uint64_t jobs_launched() const { return jobs_launched_; }
  uint64_t backfilled() const { return backfilled_; }

 private:
  static constexpr int kScan = 4096;  // waiting jobs examined per backfill attempt
  struct Run {
    uint64_t seq;
    size_t bytes;
    double end;  // estimated
  };
  struct Limits {
    double now, shadow;
    size_t extra;
  };

  // When the head (needing `need` bytes) can start if running groups end as
  // estimated (`shadow`; an overdue group is taken to end now), and the bytes
  // left over next to it then (`extra`).
  void reservation(size_t need, double now, double& shadow, size_t& extra) const {
    std::vector<Run> r = running_;
    std::sort(r.begin(), r.end(), [](const Run& a, const Run& b) { return a.end < b.end; });
    size_t avail = budget_ - std::min(budget_, in_flight_);
    shadow = now;
    extra = 0;
    for (const Run& x : r) {
      avail += x.bytes;
      shadow = std::max(shadow, x.end);
      if (avail >= need) {
        extra = avail - need;
        return;
      }
    }
  }

  // A backfilled job fits now and ends before the reservation or fits in the
  // bytes left over next to the head (which it then uses up).
  bool can_backfill(const SchedJob& j, double now, double shadow, size_t extra) const {
    if (in_flight_ + j.bytes > budget_) return false;
    return now + j.cost <= shadow || j.bytes <= extra;
  }

  // Admits *first and later same-key groupable jobs within the group limits
  // (and, when backfilling, `lim`'s rule for the group as a whole).
  void take(SchedGroup& g, std::deque<SchedJob>::iterator first, double now, Limits* lim) {
    const SchedJob j0 = *first;
    g.jobs.push_back(j0);
    g.bytes = j0.bytes;
    g.cost = j0.cost;
    auto it = pending_.erase(first);
    if (lim) ++backfilled_;
    if (!j0.groupable) return;
    for (; it != pending_.end() && (int)g.jobs.size() < max_group_;) {
      bool ok = it->groupable && it->key == j0.key && g.bytes + it->bytes <= max_group_bytes_ &&
                in_flight_ + g.bytes + it->bytes <= budget_;
      if (ok && lim)  // the whole group must still satisfy the backfill rule
        ok = now + g.cost + it->cost <= lim->shadow || g.bytes + it->bytes <= lim->extra;
      if (ok) {
        g.jobs.push_back(*it);
        g.bytes += it->bytes;
        g.cost += it->cost;
        if (lim) ++backfilled_;
        it = pending_.erase(it);
      } else {
        ++it;
      }
    }
  }

  size_t budget_;
  int max_group_;
  size_t max_group_bytes_;
  bool backfill_;
  std::deque<SchedJob> pending_;
  std::vector<Run> running_;
  size_t in_flight_ = 0, peak_in_flight_ = 0;
  uint64_t groups_ = 0, jobs_launched_ = 0, backfilled_ = 0;
};

}  // namespace gbfft
