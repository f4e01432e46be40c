// api.cu -- the extern "C" entry points of vr.h: argument checks, host/device
// input detection, result access and error reporting.
#include <atomic>
#include <mutex>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include "../../include/vr_inject.h"
#include "complex.h"
#include "jobs.h"
#include "prims.cuh"

namespace vr {

static thread_local char g_err[512] = "";

void set_error(const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

static std::atomic<int64_t> g_inj_alloc_nth{0};  // 0: off; k: the k-th allocation from now fails

cudaError_t dev_malloc(void **p, size_t bytes, cudaStream_t s) {
  int64_t k = g_inj_alloc_nth.load(std::memory_order_relaxed);
  while (k > 0) {
    if (g_inj_alloc_nth.compare_exchange_weak(k, k - 1, std::memory_order_relaxed)) {
      if (k == 1) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
      }
      break;
    }
  }
  return cudaMallocAsync(p, bytes, s);
}

// ---- one-shot stall hooks (armed by vr_inject_*; taken by the next launch
// that can honour them)
static std::mutex g_inj_mu;
static bool g_rs_armed = false, g_gram_armed = false;
static int64_t g_rs_tile = 0, g_gram_tile = 0;
static long g_rs_limit = 0, g_gram_limit = 0;

bool take_rs_stall(int64_t tiles, RsStall *out) {
  std::lock_guard<std::mutex> lk(g_inj_mu);
  if (!g_rs_armed || g_rs_tile >= tiles) return false;
  g_rs_armed = false;
  out->tile = g_rs_tile;
  out->limit = g_rs_limit;
  return true;
}

bool take_gram_stall(int tiles, int *tile, long *limit) {
  std::lock_guard<std::mutex> lk(g_inj_mu);
  if (!g_gram_armed || g_gram_tile >= tiles) return false;
  g_gram_armed = false;
  *tile = (int)g_gram_tile;
  *limit = g_gram_limit;
  return true;
}

int num_sms() {
  static std::atomic<int> cache[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  if (dev < 0 || dev >= 64) dev = 63;
  int v = cache[dev].load(std::memory_order_relaxed);
  if (v > 0) return v;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) {
    cudaGetLastError();
    return 1;
  }
  cache[dev].store(v, std::memory_order_relaxed);
  return v;
}

vr_status cuda_status(cudaError_t e, const char *what, const char *file, int line) {
  cudaGetLastError();
  set_error("%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
  return e == cudaErrorMemoryAllocation ? VR_ERR_OOM : VR_ERR_CUDA;
}

// Pool memory stays reserved between builds, so repeated calls do not go
// back to the driver for every workspace.
void keep_pool_warm() {
  static thread_local int done_dev = -1;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return; }
  if (done_dev == dev) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t thr = ~0ull;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  cudaGetLastError();
  done_dev = dev;
}

static bool is_device_pointer(const void *p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

static size_t elem_size(vr_dtype t) { return t == VR_I8 ? 1 : 4; }

}  // namespace vr

using namespace vr;

extern "C" {

const char *vr_last_error(void) { return g_err; }

const char *vr_status_string(vr_status s) {
  switch (s) {
    case VR_OK: return "VR_OK";
    case VR_ERR_ARG: return "VR_ERR_ARG";
    case VR_ERR_RANGE: return "VR_ERR_RANGE";
    case VR_ERR_UNSUPPORTED: return "VR_ERR_UNSUPPORTED";
    case VR_ERR_OOM: return "VR_ERR_OOM";
    case VR_ERR_CUDA: return "VR_ERR_CUDA";
    case VR_ERR_TIMEOUT: return "VR_ERR_TIMEOUT";
    case VR_ERR_BUSY: return "VR_ERR_BUSY";
    case VR_ERR_INTERNAL: return "VR_ERR_INTERNAL";
  }
  return "VR_ERR_UNKNOWN";
}

vr_status vr_build(const void *points, int32_t n, int32_t d, vr_dtype dtype, int32_t maxdim, double maxrad,
                   vr_stream_t stream, vr_complex **out) {
  g_err[0] = 0;
  if (!out) { set_error("out is NULL"); return VR_ERR_ARG; }
  *out = nullptr;
  if (!points) { set_error("points is NULL"); return VR_ERR_ARG; }
  if (dtype != VR_I8 && dtype != VR_I32 && dtype != VR_F32) { set_error("unknown dtype %d", (int)dtype); return VR_ERR_ARG; }
  if (d < 1) { set_error("d = %d must be >= 1", d); return VR_ERR_ARG; }
  if (n < 1 || n > VR_MAX_POINTS) { set_error("n = %d outside [1, %d]", n, VR_MAX_POINTS); return VR_ERR_RANGE; }
  if (maxdim < 0) { set_error("maxdim = %d is negative", maxdim); return VR_ERR_ARG; }
  if (maxdim > VR_MAX_DIM_SIMPLEX) { set_error("maxdim = %d above %d is not offered", maxdim, VR_MAX_DIM_SIMPLEX); return VR_ERR_UNSUPPORTED; }
  if (std::isnan(maxrad) || maxrad < 0.0) { set_error("maxrad must be >= 0 and not NaN"); return VR_ERR_ARG; }
  keep_pool_warm();
  cudaStream_t s = (cudaStream_t)stream;
  vr_complex *res = new (std::nothrow) vr_complex();
  if (!res) { set_error("host allocation failed"); return VR_ERR_OOM; }
  cudaGetDevice(&res->device);
  const void *dpts = points;
  void *staged = nullptr;
  const size_t bytes = (size_t)n * d * elem_size(dtype);
  if (!is_device_pointer(points)) {
    if (dev_malloc(&staged, bytes, s) != cudaSuccess) {
      cudaGetLastError();
      delete res;
      set_error("device allocation for the input copy failed");
      return VR_ERR_OOM;
    }
    cudaMemcpyAsync(staged, points, bytes, cudaMemcpyHostToDevice, s);
    dpts = staged;
  }
  vr_status st = build_cloud(dpts, n, d, dtype, maxdim, maxrad, s, res);
  if (staged) cudaFreeAsync(staged, s);
  if (st != VR_OK) {
    for (void *p : res->allocs) cudaFreeAsync(p, s);
    delete res;
    return st;
  }
  *out = res;
  return VR_OK;
}

vr_status vr_build_dmat(const void *D, int32_t n, vr_dtype dtype, int32_t maxdim, double maxrad,
                        vr_stream_t stream, vr_complex **out) {
  g_err[0] = 0;
  if (!out) { set_error("out is NULL"); return VR_ERR_ARG; }
  *out = nullptr;
  if (!D) { set_error("D is NULL"); return VR_ERR_ARG; }
  if (dtype != VR_I32 && dtype != VR_F32) { set_error("matrix dtype %d: VR_I32 or VR_F32", (int)dtype); return VR_ERR_ARG; }
  if (n < 1 || n > VR_MAX_POINTS) { set_error("n = %d outside [1, %d]", n, VR_MAX_POINTS); return VR_ERR_RANGE; }
  if (maxdim < 0) { set_error("maxdim = %d is negative", maxdim); return VR_ERR_ARG; }
  if (maxdim > VR_MAX_DIM_SIMPLEX) { set_error("maxdim = %d above %d is not offered", maxdim, VR_MAX_DIM_SIMPLEX); return VR_ERR_UNSUPPORTED; }
  if (std::isnan(maxrad) || maxrad < 0.0) { set_error("maxrad must be >= 0 and not NaN"); return VR_ERR_ARG; }
  keep_pool_warm();
  cudaStream_t s = (cudaStream_t)stream;
  vr_complex *res = new (std::nothrow) vr_complex();
  if (!res) { set_error("host allocation failed"); return VR_ERR_OOM; }
  cudaGetDevice(&res->device);
  const void *dm = D;
  void *staged = nullptr;
  const size_t bytes = (size_t)n * n * 4;
  if (!is_device_pointer(D)) {
    if (dev_malloc(&staged, bytes, s) != cudaSuccess) {
      cudaGetLastError();
      delete res;
      set_error("device allocation for the matrix copy failed");
      return VR_ERR_OOM;
    }
    cudaMemcpyAsync(staged, D, bytes, cudaMemcpyHostToDevice, s);
    dm = staged;
  }
  vr_status st = build_dmat(dm, n, dtype, maxdim, maxrad, s, res);
  if (staged) cudaFreeAsync(staged, s);
  if (st != VR_OK) {
    for (void *p : res->allocs) cudaFreeAsync(p, s);
    delete res;
    return st;
  }
  *out = res;
  return VR_OK;
}

vr_status vr_complex_dim(const vr_complex *c, int32_t k, vr_dim_view *v) {
  if (!c || !v) { set_error("NULL argument"); return VR_ERR_ARG; }
  if (k < 0 || k > c->maxdim) { set_error("dimension %d outside [0, %d]", k, c->maxdim); return VR_ERR_ARG; }
  v->k = k;
  v->count = c->count[k];
  v->verts = c->verts[k];
  v->grade = c->grade[k];
  v->colptr = k >= 1 ? c->colptr[k] : nullptr;
  v->rowidx = k >= 1 ? c->rowidx[k] : nullptr;
  return VR_OK;
}

vr_status vr_complex_grade_values(const vr_complex *c, const double **values, int64_t *ngrades) {
  if (!c || !values || !ngrades) { set_error("NULL argument"); return VR_ERR_ARG; }
  *values = c->grade_value;
  *ngrades = c->ngrades;
  return VR_OK;
}

vr_status vr_complex_counts(const vr_complex *c, int64_t counts[VR_MAX_DIM_SIMPLEX + 1], int32_t *maxdim) {
  if (!c || !counts) { set_error("NULL argument"); return VR_ERR_ARG; }
  for (int k = 0; k <= VR_MAX_DIM_SIMPLEX; ++k) counts[k] = c->count[k];
  if (maxdim) *maxdim = c->maxdim;
  return VR_OK;
}

vr_status vr_complex_stats(const vr_complex *c, vr_build_stats *s) {
  if (!c || !s) { set_error("NULL argument"); return VR_ERR_ARG; }
  *s = c->stats;
  return VR_OK;
}

vr_status vr_complex_status(const vr_complex *c) {
  if (!c) { set_error("NULL complex"); return VR_ERR_ARG; }
  VR_CUDA(cudaStreamSynchronize(c->stream));
  if (!c->late_flags) return VR_OK;
  int32_t f = 0;
  VR_CUDA(cudaMemcpy(&f, c->late_flags, sizeof(int32_t), cudaMemcpyDeviceToHost));
  return flags_to_status(f);
}

vr_status vr_complex_to_host(const vr_complex *c, int32_t k, int32_t *verts, int32_t *grade, int64_t *colptr,
                             int32_t *rowidx) {
  if (!c) { set_error("NULL complex"); return VR_ERR_ARG; }
  if (k < 0 || k > c->maxdim) { set_error("dimension %d outside [0, %d]", k, c->maxdim); return VR_ERR_ARG; }
  const int64_t m = c->count[k];
  cudaStream_t s = c->stream;
  int32_t late = 0;
  if (c->late_flags) VR_CUDA(cudaMemcpyAsync(&late, c->late_flags, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  if (verts && m) VR_CUDA(cudaMemcpyAsync(verts, c->verts[k], sizeof(int32_t) * m * (k + 1), cudaMemcpyDeviceToHost, s));
  if (grade && m) VR_CUDA(cudaMemcpyAsync(grade, c->grade[k], sizeof(int32_t) * m, cudaMemcpyDeviceToHost, s));
  if (k >= 1 && colptr) VR_CUDA(cudaMemcpyAsync(colptr, c->colptr[k], sizeof(int64_t) * (m + 1), cudaMemcpyDeviceToHost, s));
  if (k >= 1 && rowidx && m) VR_CUDA(cudaMemcpyAsync(rowidx, c->rowidx[k], sizeof(int32_t) * m * (k + 1), cudaMemcpyDeviceToHost, s));
  VR_CUDA(cudaStreamSynchronize(s));
  return late ? flags_to_status(late) : VR_OK;
}

vr_status vr_complex_grade_values_to_host(const vr_complex *c, double *values) {
  if (!c || !values) { set_error("NULL argument"); return VR_ERR_ARG; }
  VR_CUDA(cudaMemcpyAsync(values, c->grade_value, sizeof(double) * c->ngrades, cudaMemcpyDeviceToHost, c->stream));
  VR_CUDA(cudaStreamSynchronize(c->stream));
  return VR_OK;
}

vr_status vr_complex_barcode(vr_complex *c, int32_t dim, vr_stream_t stream, int64_t *nbars) {
  g_err[0] = 0;
  if (!c || !nbars) { set_error("NULL argument"); return VR_ERR_ARG; }
  if (dim < 0 || dim > c->maxdim) { set_error("dimension %d outside [0, %d]", dim, c->maxdim); return VR_ERR_ARG; }
  if (c->in_batch || !c->owned) {
    set_error("barcodes are computed on results of vr_build / vr_build_dmat / vr_serve_poll");
    return VR_ERR_UNSUPPORTED;
  }
  // A build the device reported as failed holds no valid complex to reduce.
  if (c->late_flags) VR_TRY(vr_complex_status(c));
  cudaStream_t s = stream ? (cudaStream_t)stream : c->stream;
  return vr::complex_barcode(c, dim, s, nbars);
}

vr_status vr_complex_bars(const vr_complex *c, int32_t dim, const int32_t **birth, const int32_t **death,
                          int64_t *nbars) {
  if (!c || !birth || !death || !nbars) { set_error("NULL argument"); return VR_ERR_ARG; }
  if (dim < 0 || dim > 3 || c->nbars[dim] < 0) { set_error("no barcode of dimension %d computed", dim); return VR_ERR_ARG; }
  *birth = c->bar_birth[dim];
  *death = c->bar_death[dim];
  *nbars = c->nbars[dim];
  return VR_OK;
}

vr_status vr_complex_bars_to_host(const vr_complex *c, int32_t dim, int32_t *birth, int32_t *death) {
  if (!c || !birth || !death) { set_error("NULL argument"); return VR_ERR_ARG; }
  if (dim < 0 || dim > 3 || c->nbars[dim] < 0) { set_error("no barcode of dimension %d computed", dim); return VR_ERR_ARG; }
  const int64_t m = c->nbars[dim];
  if (m) {
    VR_CUDA(cudaMemcpyAsync(birth, c->bar_birth[dim], sizeof(int32_t) * m, cudaMemcpyDeviceToHost, c->stream));
    VR_CUDA(cudaMemcpyAsync(death, c->bar_death[dim], sizeof(int32_t) * m, cudaMemcpyDeviceToHost, c->stream));
  }
  VR_CUDA(cudaStreamSynchronize(c->stream));
  return VR_OK;
}

void vr_complex_free(vr_complex *c) {
  if (!c || c->in_batch) return;
  for (void *p : c->bar_allocs) cudaFreeAsync(p, c->stream);
  if (c->owned)
    for (void *p : c->allocs) cudaFreeAsync(p, c->stream);
  cudaGetLastError();
  delete c;
}

}  // extern "C"

// ------------------------------------------------------------- profiling
#include <mutex>
#include <string>
#include <vector>

#include "prof.h"

namespace vr {
std::atomic<int64_t> g_launches{0};
std::atomic<int> g_profile_on{0};
struct PhaseTotal {
  std::string name;
  double ms;
  int64_t calls;
  int64_t launches;
};
static std::mutex g_prof_mu;
static std::vector<PhaseTotal> g_prof;

static void profile_add(const char *name, double ms, int64_t launches) {
  for (auto &p : g_prof)
    if (p.name == name) {
      p.ms += ms;
      p.calls += 1;
      p.launches += launches;
      return;
    }
  g_prof.push_back({name, ms, 1, launches});
}

static std::vector<std::string> g_filter;
std::vector<std::string> profile_filter() {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  return g_filter;
}

static std::vector<cudaEvent_t> g_event_pool;
static std::vector<ProfRec> g_pending;

cudaEvent_t profile_event() {
  {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (!g_event_pool.empty()) {
      cudaEvent_t e = g_event_pool.back();
      g_event_pool.pop_back();
      return e;
    }
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    e = nullptr;
  }
  return e;
}

// Read every pending record into the table (waits for its events); with
// g_prof_mu held.
static void resolve_pending_locked() {
  for (auto &r : g_pending) {
    float ms = 0.f;
    if (r.a && r.b && cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess)
      profile_add(r.name, ms, r.launches);
    if (r.a) g_event_pool.push_back(r.a);
    if (r.b) g_event_pool.push_back(r.b);
  }
  cudaGetLastError();
  g_pending.clear();
}

void profile_defer(std::vector<ProfRec> &recs) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  g_pending.insert(g_pending.end(), recs.begin(), recs.end());
  if (g_pending.size() > 16384) resolve_pending_locked();  // bound the list
}
}  // namespace vr

extern "C" {
void vr_profile_enable(int32_t on) { vr::g_profile_on.store(on ? 1 : 0); }

void vr_profile_select(const char *names) {
  std::vector<std::string> f;
  if (names) {
    std::string cur;
    for (const char *c = names;; ++c) {
      if (*c == ',' || *c == 0) {
        if (!cur.empty()) f.push_back(cur);
        cur.clear();
        if (!*c) break;
      } else {
        cur.push_back(*c);
      }
    }
  }
  std::lock_guard<std::mutex> lk(vr::g_prof_mu);
  vr::g_filter = f;
}

void vr_profile_reset(void) {
  std::lock_guard<std::mutex> lk(vr::g_prof_mu);
  vr::resolve_pending_locked();
  vr::g_prof.clear();
}

int32_t vr_profile_phases(void) {
  std::lock_guard<std::mutex> lk(vr::g_prof_mu);
  vr::resolve_pending_locked();
  return (int32_t)vr::g_prof.size();
}

vr_status vr_profile_phase(int32_t i, const char **name, double *total_ms, int64_t *calls, int64_t *launches) {
  std::lock_guard<std::mutex> lk(vr::g_prof_mu);
  vr::resolve_pending_locked();
  if (i < 0 || i >= (int32_t)vr::g_prof.size() || !name || !total_ms || !calls || !launches) {
    vr::set_error("profile phase index out of range or NULL argument");
    return VR_ERR_ARG;
  }
  *name = vr::g_prof[i].name.c_str();
  *total_ms = vr::g_prof[i].ms;
  *calls = vr::g_prof[i].calls;
  *launches = vr::g_prof[i].launches;
  return VR_OK;
}

int64_t vr_launch_count(void) { return vr::g_launches.load(); }
}  // extern "C"

// ------------------------------------------------------- fault injection
extern "C" {

vr_status vr_inject_alloc_failure(int64_t nth) {
  if (nth < 0) { vr::set_error("nth = %lld must be >= 0", (long long)nth); return VR_ERR_ARG; }
  vr::g_inj_alloc_nth.store(nth, std::memory_order_relaxed);
  return VR_OK;
}

vr_status vr_inject_lookback_stall(int64_t tile, int64_t wait_limit) {
  if (tile < 0 || wait_limit < 1) { vr::set_error("tile >= 0 and wait_limit >= 1 required"); return VR_ERR_ARG; }
  std::lock_guard<std::mutex> lk(vr::g_inj_mu);
  vr::g_rs_armed = true;
  vr::g_rs_tile = tile;
  vr::g_rs_limit = (long)wait_limit;
  return VR_OK;
}

vr_status vr_inject_gram_stall(int32_t tile, int64_t wait_limit) {
  if (tile < 0 || wait_limit < 1) { vr::set_error("tile >= 0 and wait_limit >= 1 required"); return VR_ERR_ARG; }
  std::lock_guard<std::mutex> lk(vr::g_inj_mu);
  vr::g_gram_armed = true;
  vr::g_gram_tile = tile;
  vr::g_gram_limit = (long)wait_limit;
  return VR_OK;
}

vr_status vr_inject_clear(void) {
  vr::g_inj_alloc_nth.store(0, std::memory_order_relaxed);
  vr::inject_admission_refusals(0);
  std::lock_guard<std::mutex> lk(vr::g_inj_mu);
  vr::g_rs_armed = vr::g_gram_armed = false;
  return VR_OK;
}

vr_status vr_inject_admission_refusals(int64_t k) {
  if (k < 0) { vr::set_error("k = %lld must be >= 0", (long long)k); return VR_ERR_ARG; }
  vr::inject_admission_refusals(k);
  return VR_OK;
}

vr_status vr_pool_used_bytes(int64_t *bytes) {
  if (!bytes) { vr::set_error("bytes is NULL"); return VR_ERR_ARG; }
  int dev = 0;
  VR_CUDA(cudaGetDevice(&dev));
  cudaMemPool_t pool;
  VR_CUDA(cudaDeviceGetDefaultMemPool(&pool, dev));
  uint64_t v = 0;
  VR_CUDA(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &v));
  *bytes = (int64_t)v;
  return VR_OK;
}

}  // extern "C"
