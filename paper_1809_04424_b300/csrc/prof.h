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
  void begin(const char *name) {
    cur_ = name;
    l0_ = g_launches.load();
    if (!on_) return;
    Rec r{name, nullptr, nullptr, 0};
    cudaEventCreate(&r.a);
    cudaEventCreate(&r.b);
    cudaEventRecord(r.a, s_);
    recs_.push_back(r);
  }
  void end() {
    if (!on_ || recs_.empty()) return;
    cudaEventRecord(recs_.back().b, s_);
    recs_.back().launches = g_launches.load() - l0_;
  }
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
  }

 private:
  struct Rec {
    const char *name;
    cudaEvent_t a, b;
    int64_t launches;
  };
  cudaStream_t s_;
  bool on_;
  const char *cur_ = nullptr;
  int64_t l0_ = 0;
  std::vector<Rec> recs_;
};

}  // namespace vr
