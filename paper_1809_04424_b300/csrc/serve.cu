// serve.cu -- continuous-batching request server.
//
// vr_serve_submit copies a request's points to host memory and queues it;
// vr_serve_poll waits (bounded) for its result.  Two worker threads:
//   * the batch worker keeps up to n_streams micro-batches in flight, one per
//     stream.  Whenever a stream is free it takes the waiting requests of one
//     (dtype, d) class (oldest first, up to max_batch_clouds), packs their
//     points into the stream's pinned buffer, copies them in and launches the
//     sizing kernel; when sizes are back it admits clouds by their exact
//     output bytes against the memory budget left by the other in-flight
//     batches (deferred clouds go back to the front of the queue) and
//     launches the build; when that completes it hands each request its own
//     result.  Requests that arrive while batches run join the next batch,
//     so their work overlaps on the device with the batches in flight.
//   * n_large_workers threads build requests too large for the batch kernels
//     through vr_build, each on a stream of its own, so they overlap too.
// Results are vr_complex objects owned by the caller after poll (free with
// vr_complex_free); a batch's shared output arenas are released with the last
// of its results.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "complex.h"
#include "jobs.h"
#include "prims.cuh"

namespace {


struct Req {
  uint64_t ticket;
  int32_t n, d, maxdim;
  vr_dtype dtype;
  double maxrad;
  std::vector<unsigned char> pts;  // host copy of the points
};

struct Done {
  vr_status st;
  vr_complex *c;
};

struct Slot {
  cudaStream_t s = nullptr;
  unsigned char *hbuf = nullptr;   // pinned staging of a batch's points
  size_t hcap = 0;
  void *dbuf = nullptr;            // device copy of the points
  size_t dcap = 0;
  unsigned char *pdesc = nullptr;  // pinned per-cloud descriptors of the job
  size_t pcap = 0;
  vr::Job *job = nullptr;
  int state = 0;                   // 0 idle, 1 sizing, 2 building
  std::vector<Req> members;
  int64_t bytes = 0;
};

}  // namespace

struct vr_server {
  vr_server_opts opts{};
  int device = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_big, cv_done;
  std::map<std::pair<int, int>, std::deque<Req>> small_q;  // (dtype, d) -> requests
  std::deque<Req> big_q;
  std::unordered_map<uint64_t, Done> done;
  uint64_t next_ticket = 1;
  int64_t queued = 0;
  bool stop = false;
  std::vector<Slot> slots;
  std::vector<cudaStream_t> big_streams;
  std::thread batch_thr;
  std::vector<std::thread> big_thr;
  vr_server_stats stats{};  // under mu
};

namespace {

using namespace vr;

void deliver(vr_server *S, uint64_t ticket, vr_status st, vr_complex *c) {
  std::lock_guard<std::mutex> lk(S->mu);
  if (st == VR_OK) ++S->stats.completed;
  else ++S->stats.failed;
  S->done[ticket] = Done{st, c};
  S->cv_done.notify_all();
}

bool grow_pinned(unsigned char **p, size_t *cap, size_t need) {
  if (*cap >= need) return true;
  if (*p) cudaFreeHost(*p);
  size_t c = std::max(need, *cap * 2);
  if (cudaMallocHost((void **)p, c) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    *cap = 0;
    return false;
  }
  *cap = c;
  return true;
}

// Take one micro-batch (same dtype and d) from the small queues: the class
// whose head waited longest, up to max_batch_clouds requests.
bool take_batch(vr_server *S, std::vector<Req> &out) {
  std::lock_guard<std::mutex> lk(S->mu);
  std::deque<Req> *best = nullptr;
  for (auto &kv : S->small_q)
    if (!kv.second.empty() && (!best || kv.second.front().ticket < best->front().ticket)) best = &kv.second;
  if (!best) return false;
  const int lim = std::max(1, S->opts.max_batch_clouds);
  while (!best->empty() && (int)out.size() < lim) {
    out.push_back(std::move(best->front()));
    best->pop_front();
    --S->queued;
  }
  return true;
}

void fail_members(vr_server *S, Slot &sl, vr_status st) {
  for (auto &r : sl.members) deliver(S, r.ticket, st, nullptr);
  sl.members.clear();
}

void launch_slot(vr_server *S, Slot &sl, std::vector<Req> &batch) {
  const int d = batch[0].d;
  const vr_dtype dt = batch[0].dtype;
  const size_t es = dt == VR_I8 ? 1 : 4;
  size_t bytes = 0;
  std::vector<JobCloud> jc;
  for (auto &r : batch) {
    jc.push_back(JobCloud{(int64_t)(bytes / (es * d)), r.n, r.maxdim, r.maxrad});
    bytes += r.pts.size();
  }
  sl.members = std::move(batch);
  if (!grow_pinned(&sl.hbuf, &sl.hcap, bytes)) return fail_members(S, sl, VR_ERR_OOM);
  size_t off = 0;
  for (auto &r : sl.members) {
    memcpy(sl.hbuf + off, r.pts.data(), r.pts.size());
    off += r.pts.size();
  }
  if (sl.dcap < bytes) {
    if (sl.dbuf) cudaFreeAsync(sl.dbuf, sl.s);
    sl.dbuf = nullptr;
    sl.dcap = 0;
    if (dev_malloc(&sl.dbuf, std::max(bytes, (size_t)1 << 20), sl.s) != cudaSuccess) {
      cudaGetLastError();
      return fail_members(S, sl, VR_ERR_OOM);
    }
    sl.dcap = std::max(bytes, (size_t)1 << 20);
  }
  cudaMemcpyAsync(sl.dbuf, sl.hbuf, bytes, cudaMemcpyHostToDevice, sl.s);
  vr_status st;
  if (!grow_pinned(&sl.pdesc, &sl.pcap, job_pinned_bytes(jc.size()))) return fail_members(S, sl, VR_ERR_OOM);
  sl.job = job_create(sl.s, sl.dbuf, d, dt, jc, sl.pdesc, &st);
  if (!sl.job) return fail_members(S, sl, st);
  st = job_size_async(sl.job);
  if (st != VR_OK) {
    job_destroy(sl.job);
    sl.job = nullptr;
    return fail_members(S, sl, st);
  }
  sl.state = 1;
}

void batch_worker(vr_server *S) {
  cudaSetDevice(S->device);
  keep_pool_warm();
  for (;;) {
    bool progressed = false;
    int64_t inflight = 0;
    for (auto &sl : S->slots) inflight += sl.bytes;
    for (auto &sl : S->slots) {
      if (sl.state == 1 && job_ready(sl.job)) {
        std::vector<int> deferred;
        const int64_t budget = std::max<int64_t>(S->opts.mem_budget_bytes - inflight, 0);
        vr_status st = job_build_async(sl.job, budget, &deferred);
        if (st != VR_OK) {
          job_destroy(sl.job);
          sl.job = nullptr;
          sl.state = 0;
          fail_members(S, sl, st);
        } else {
          sl.bytes = job_out_bytes(sl.job);
          inflight += sl.bytes;
          if (!deferred.empty()) {  // back to the front of their queue
            std::lock_guard<std::mutex> lk(S->mu);
            S->stats.deferred += (int64_t)deferred.size();
            auto &q = S->small_q[{(int)sl.members[0].dtype, sl.members[0].d}];
            for (auto it = deferred.rbegin(); it != deferred.rend(); ++it) {
              q.push_front(std::move(sl.members[*it]));
              ++S->queued;
            }
          }
          sl.state = 2;
        }
        progressed = true;
      } else if (sl.state == 2 && job_ready(sl.job)) {
        std::vector<vr_complex *> res;
        std::vector<vr_status> st;
        job_finish(sl.job, res, st, true);
        for (size_t i = 0; i < sl.members.size(); ++i) {
          if (!res[i] && st[i] == VR_OK) continue;  // deferred: back in the queue
          deliver(S, sl.members[i].ticket, st[i], res[i]);
        }
        job_destroy(sl.job);
        sl.job = nullptr;
        sl.members.clear();
        inflight -= sl.bytes;
        sl.bytes = 0;
        sl.state = 0;
        progressed = true;
      }
    }
    for (auto &sl : S->slots) {
      if (sl.state != 0) continue;
      std::vector<Req> batch;
      if (!take_batch(S, batch)) break;
      {
        std::lock_guard<std::mutex> lk(S->mu);
        ++S->stats.batches;
      }
      launch_slot(S, sl, batch);
      progressed = true;
    }
    if (!progressed) {
      std::unique_lock<std::mutex> lk(S->mu);
      if (S->stop) {
        bool busy = false;
        for (auto &sl : S->slots) busy |= sl.state != 0;
        if (!busy) return;
      }
      bool any_q = false;
      for (auto &kv : S->small_q) any_q |= !kv.second.empty();
      bool inflight_any = false;
      for (auto &sl : S->slots) inflight_any |= sl.state != 0;
      if (!any_q && !inflight_any && !S->stop) S->cv_work.wait_for(lk, std::chrono::milliseconds(5));
      else if (inflight_any) {
        lk.unlock();
        std::this_thread::sleep_for(std::chrono::microseconds(20));
      }
    }
  }
}

void big_worker(vr_server *S, int k) {
  cudaSetDevice(S->device);
  cudaStream_t bs = S->big_streams[k];
  for (;;) {
    Req r;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv_big.wait(lk, [&] { return S->stop || !S->big_q.empty(); });
      if (S->big_q.empty()) return;
      r = std::move(S->big_q.front());
      S->big_q.pop_front();
      --S->queued;
      ++S->stats.large_builds;
    }
    vr_complex *c = nullptr;
    const vr_status st = vr_build(r.pts.data(), r.n, r.d, r.dtype, r.maxdim, r.maxrad, bs, &c);
    if (c) {  // outlive the server's stream: later copies and frees use the legacy stream
      cudaStreamSynchronize(bs);
      c->stream = nullptr;
    }
    deliver(S, r.ticket, st, c);
  }
}

}  // namespace

extern "C" {

vr_status vr_server_create(const vr_server_opts *opts, vr_server **out) {
  if (!out) { set_error("out is NULL"); return VR_ERR_ARG; }
  *out = nullptr;
  vr_server *S = new (std::nothrow) vr_server();
  if (!S) { set_error("host allocation failed"); return VR_ERR_OOM; }
  vr_server_opts o{};
  o.mem_budget_bytes = 8ll << 30;
  o.max_queue = 65536;
  o.n_streams = 3;
  o.max_batch_clouds = 512;
  o.n_large_workers = 4;
  o.device = -1;
  if (opts) {
    if (opts->mem_budget_bytes > 0) o.mem_budget_bytes = opts->mem_budget_bytes;
    if (opts->max_queue > 0) o.max_queue = opts->max_queue;
    if (opts->n_streams > 0) o.n_streams = opts->n_streams;
    if (opts->max_batch_clouds > 0) o.max_batch_clouds = opts->max_batch_clouds;
    if (opts->n_large_workers > 0) o.n_large_workers = opts->n_large_workers;
    o.device = opts->device;
  }
  S->opts = o;
  if (o.device >= 0) {
    if (cudaSetDevice(o.device) != cudaSuccess) {
      delete S;
      return cuda_status(cudaGetLastError(), "cudaSetDevice", __FILE__, __LINE__);
    }
  }
  cudaGetDevice(&S->device);
  S->slots.resize(o.n_streams);
  for (auto &sl : S->slots)
    if (cudaStreamCreateWithFlags(&sl.s, cudaStreamNonBlocking) != cudaSuccess) {
      delete S;
      return cuda_status(cudaGetLastError(), "cudaStreamCreate", __FILE__, __LINE__);
    }
  S->big_streams.resize(o.n_large_workers);
  for (auto &bs : S->big_streams)
    if (cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking) != cudaSuccess) {
      delete S;
      return cuda_status(cudaGetLastError(), "cudaStreamCreate", __FILE__, __LINE__);
    }
  S->batch_thr = std::thread(batch_worker, S);
  for (int k = 0; k < o.n_large_workers; ++k) S->big_thr.emplace_back(big_worker, S, k);
  *out = S;
  return VR_OK;
}

vr_status vr_serve_submit(vr_server *S, const void *points, int32_t n, int32_t d, vr_dtype dtype, int32_t maxdim,
                          double maxrad, uint64_t *ticket) {
  if (!S || !points || !ticket) { set_error("NULL argument"); return VR_ERR_ARG; }
  VR_TRY(check_cloud_args(n, d, dtype, maxdim, maxrad));
  Req r;
  r.n = n;
  r.d = d;
  r.dtype = dtype;
  r.maxdim = maxdim;
  r.maxrad = maxrad;
  const size_t bytes = (size_t)n * d * (dtype == VR_I8 ? 1 : 4);
  r.pts.resize(bytes);
  cudaPointerAttributes pa;
  const bool on_dev = cudaPointerGetAttributes(&pa, points) == cudaSuccess &&
                      (pa.type == cudaMemoryTypeDevice || pa.type == cudaMemoryTypeManaged);
  cudaGetLastError();
  if (on_dev) VR_CUDA(cudaMemcpy(r.pts.data(), points, bytes, cudaMemcpyDeviceToHost));
  else memcpy(r.pts.data(), points, bytes);
  std::lock_guard<std::mutex> lk(S->mu);
  if (S->stop) { set_error("server is shutting down"); return VR_ERR_BUSY; }
  if (S->queued >= S->opts.max_queue) { set_error("queue full (%lld requests)", (long long)S->queued); return VR_ERR_BUSY; }
  r.ticket = S->next_ticket++;
  *ticket = r.ticket;
  ++S->queued;
  ++S->stats.submitted;
  if (fused_fits(n, d)) {
    S->small_q[{(int)dtype, d}].push_back(std::move(r));
    S->cv_work.notify_one();
  } else {
    S->big_q.push_back(std::move(r));
    S->cv_big.notify_one();
  }
  return VR_OK;
}

vr_status vr_serve_poll(vr_server *S, uint64_t ticket, int64_t timeout_us, vr_complex **out) {
  if (!S || !out) { set_error("NULL argument"); return VR_ERR_ARG; }
  *out = nullptr;
  std::unique_lock<std::mutex> lk(S->mu);
  if (ticket == 0 || ticket >= S->next_ticket) { set_error("unknown ticket %llu", (unsigned long long)ticket); return VR_ERR_ARG; }
  auto ready = [&] { return S->done.count(ticket) != 0; };
  if (!ready()) {
    if (timeout_us <= 0 ||
        !S->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), ready)) {
      set_error("ticket %llu not ready", (unsigned long long)ticket);
      return VR_ERR_TIMEOUT;
    }
  }
  Done dn = S->done[ticket];
  S->done.erase(ticket);
  if (dn.st != VR_OK) {
    set_error("request %llu failed: %s", (unsigned long long)ticket, vr_status_string(dn.st));
    return dn.st;
  }
  *out = dn.c;
  return VR_OK;
}

vr_status vr_server_get_stats(vr_server *S, vr_server_stats *out) {
  if (!S || !out) { set_error("NULL argument"); return VR_ERR_ARG; }
  std::lock_guard<std::mutex> lk(S->mu);
  *out = S->stats;
  out->queued = S->queued;
  return VR_OK;
}

vr_status vr_server_destroy(vr_server *S) {
  if (!S) return VR_OK;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  S->cv_big.notify_all();
  if (S->batch_thr.joinable()) S->batch_thr.join();
  for (auto &t : S->big_thr)
    if (t.joinable()) t.join();
  for (auto &kv : S->done)
    if (kv.second.c) vr_complex_free(kv.second.c);
  S->done.clear();
  for (auto &sl : S->slots) {
    if (sl.dbuf) cudaFreeAsync(sl.dbuf, sl.s);
    if (sl.s) cudaStreamSynchronize(sl.s);
    if (sl.hbuf) cudaFreeHost(sl.hbuf);
    if (sl.pdesc) cudaFreeHost(sl.pdesc);
  }
  cudaDeviceSynchronize();
  for (auto &sl : S->slots)
    if (sl.s) cudaStreamDestroy(sl.s);
  for (auto bs : S->big_streams)
    if (bs) cudaStreamDestroy(bs);
  cudaGetLastError();
  delete S;
  return VR_OK;
}

}  // extern "C"
