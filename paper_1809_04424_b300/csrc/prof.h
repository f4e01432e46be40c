// prof.h -- per-phase CUDA-event timing and a kernel-launch counter.
// Off by default; when on, each build records an event pair around each
// phase on its own stream and adds the elapsed times to a process-wide table
// once the build's work is complete.
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <vector>

namespace vr {

extern std::atomic<int64_t> g_launches;
extern std::atomic<int> g_profile_on;
inline void count_launch(int k = 1) { g_launches.fetch_add(k, std::memory_order_relaxed); }

void profile_add(const char *name, double ms, int64_t launches);

class Prof {
 public:
  explicit Prof(cudaStream_t s) : s_(s), on_(g_profile_on.load() != 0) {}
  ~Prof() { finish(); }
  // Open a timed region; returns a token for end().  Regions may nest.
  int begin(const char *name) {
    if (!on_) return -1;
    Rec r{name, nullptr, nullptr, g_launches.load()};
    cudaEventCreate(&r.a);
    cudaEventCreate(&r.b);
    cudaEventRecord(r.a, s_);
    recs_.push_back(r);
    open_.push_back((int)recs_.size() - 1);
    return (int)recs_.size() - 1;
  }
  void end(int tok) {
    if (!on_ || tok < 0) return;
    cudaEventRecord(recs_[tok].b, s_);
    recs_[tok].launches = g_launches.load() - recs_[tok].launches;
    for (size_t i = open_.size(); i-- > 0;)
      if (open_[i] == tok) { open_.erase(open_.begin() + i); break; }
  }
  // Close the innermost region still open.
  void end() { end(open_.empty() ? -1 : open_.back()); }
  void finish() {
    if (!on_) return;
    for (auto &r : recs_) {
      float ms = 0.f;
      if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess)
        profile_add(r.name, ms, r.launches);
      cudaEventDestroy(r.a);
      cudaEventDestroy(r.b);
    }
    cudaGetLastError();
    recs_.clear();
    open_.clear();
  }

 private:
  struct Rec {
    const char *name;
    cudaEvent_t a, b;
    int64_t launches;
  };
  cudaStream_t s_;
  bool on_;
  std::vector<Rec> recs_;
  std::vector<int> open_;
};

}  // namespace vr
