// prof.h -- per-phase CUDA-event timing and a kernel-launch counter.
// Off by default; when on, each build records an event pair around each
// phase on its own stream and adds the elapsed times to a process-wide table
// once the build's work is complete.
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

namespace vr {

extern std::atomic<int64_t> g_launches;
extern std::atomic<int> g_profile_on;
inline void count_launch(int k = 1) { g_launches.fetch_add(k, std::memory_order_relaxed); }

// Event records of finished builds wait in a process-wide list and are read
// (their elapsed times added to the phase table) only when the table is
// queried, so a profiled build costs event records, not a synchronisation.
// Events come from a pool and go back to it once read.
struct ProfRec {
  const char *name;
  cudaEvent_t a, b;
  int64_t launches;
};
cudaEvent_t profile_event();
void profile_defer(std::vector<ProfRec> &recs);
// Phase-name filter (empty: every phase); a copy is taken per build.
std::vector<std::string> profile_filter();

class Prof {
 public:
  explicit Prof(cudaStream_t s) : s_(s), on_(g_profile_on.load() != 0) {
    if (on_) filter_ = profile_filter();
  }
  ~Prof() { finish(); }
  // Open a timed region; returns a token for end() (-1: not timed).  Regions
  // may nest; a region the filter leaves out still takes its place on the
  // stack of open regions, so end() without a token stays balanced.
  int begin(const char *name) {
    if (!on_) return -1;
    if (!selected(name)) {
      open_.push_back(-1);
      return -1;
    }
    ProfRec r{name, profile_event(), profile_event(), g_launches.load()};
    cudaEventRecord(r.a, s_);
    recs_.push_back(r);
    open_.push_back((int)recs_.size() - 1);
    return (int)recs_.size() - 1;
  }
  void end(int tok) {
    if (!on_) return;
    if (tok < 0) {  // an untimed region: drop its placeholder
      for (size_t i = open_.size(); i-- > 0;)
        if (open_[i] == -1) { open_.erase(open_.begin() + i); break; }
      return;
    }
    cudaEventRecord(recs_[tok].b, s_);
    recs_[tok].launches = g_launches.load() - recs_[tok].launches;
    for (size_t i = open_.size(); i-- > 0;)
      if (open_[i] == tok) { open_.erase(open_.begin() + i); break; }
  }
  // Close the innermost region still open.
  void end() {
    if (!on_ || open_.empty()) return;
    const int tok = open_.back();
    if (tok < 0) open_.pop_back();
    else end(tok);
  }
  void finish() {
    if (!on_) return;
    profile_defer(recs_);
    recs_.clear();
    open_.clear();
  }

 private:
  bool selected(const char *name) const {
    if (filter_.empty()) return true;
    for (auto &f : filter_)
      if (f == name) return true;
    return false;
  }
  cudaStream_t s_;
  bool on_;
  std::vector<std::string> filter_;
  std::vector<ProfRec> recs_;
  std::vector<int> open_;
};

}  // namespace vr
