// build.cu -- host orchestration of one Vietoris-Rips build on one stream.
//
// Kernels in launch order (kernels.cuh): stage -> distance/bitmap -> row
// counts -> scans -> [sync 1: kept-edge count, value errors] -> edge keys in
// lexicographic order -> stable LSD radix sort on the distance bits -> (float:
// FP64 values + repair groups) -> dense-rank scan -> edge outputs and the
// neighbour CSR -> triangle counts -> scan -> tie groups -> [sync 2: triangle
// count] -> triangle emission -> tie-group merge.  Only sizes cross to the host.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <vector>

#include "complex.h"
#include "kernels.cuh"
#include "prof.h"

namespace vr {

// Stream-ordered allocations that are released together (on scope exit for
// workspaces; handed over to the result for outputs).  Between begin() and
// commit() alloc() only records the request; commit() makes one allocation
// and carves it (256-byte aligned pieces), so a group of arrays costs one
// allocator call.
struct Arena {
  cudaStream_t s;
  std::vector<void *> ptrs;
  bool grouping = false;
  std::vector<std::pair<void **, size_t>> pend;
  explicit Arena(cudaStream_t st) : s(st) {}
  ~Arena() {
    for (void *p : ptrs) cudaFreeAsync(p, s);
  }
  void begin() { grouping = true; }
  vr_status commit() {
    grouping = false;
    if (pend.empty()) return VR_OK;
    size_t total = 0;
    for (auto &q : pend) total += (q.second + 255) & ~(size_t)255;
    char *base = nullptr;
    VR_TRY(alloc(&base, (int64_t)total));
    size_t at = 0;
    for (auto &q : pend) {
      *q.first = base + at;
      at += (q.second + 255) & ~(size_t)255;
    }
    pend.clear();
    return VR_OK;
  }
  template <typename T>
  vr_status alloc(T **p, int64_t count) {
    size_t bytes = sizeof(T) * (size_t)std::max<int64_t>(count, 1);
    if (grouping) {
      *p = nullptr;
      pend.push_back({(void **)p, bytes});
      return VR_OK;
    }
    cudaError_t e = dev_malloc((void **)p, bytes, s);
    if (e != cudaSuccess) {
      cudaGetLastError();
      set_error("device allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
      return e == cudaErrorMemoryAllocation ? VR_ERR_OOM : VR_ERR_CUDA;
    }
    ptrs.push_back(*p);
    return VR_OK;
  }
  void release_to(std::vector<void *> &dst) {
    dst.insert(dst.end(), ptrs.begin(), ptrs.end());
    ptrs.clear();
  }
};

// per_sm: the grid is capped at this many CTAs per SM of the device.
static unsigned grid_for(int64_t work, int threads, int per_sm = 16) {
  const int64_t cap_ctas = (int64_t)num_sms() * per_sm;
  int64_t g = (work + threads - 1) / threads;
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(g, cap_ctas));
}

static int bitlen(uint64_t v) { return v ? 64 - __builtin_clzll(v) : 0; }

// Host mirror of the status word in mapped pinned memory.  At a sync point
// k_publish (one warp, launched behind the segment's last kernel) copies the
// status into it and then writes a fresh sequence number, which the host
// polls: no copy-engine transfer and no stream synchronisation between the
// segment's end and the host's next launch.
struct HostStatus {
  DevStatus st;
  uint64_t seq;
};
struct StatusMirror {
  HostStatus *h, *d;  // host and device addresses of one mapped buffer
  uint64_t next;      // last sequence number handed out
};

static StatusMirror *status_mirror() {
  thread_local StatusMirror m{nullptr, nullptr, 0};
  if (!m.h) {
    HostStatus *h = nullptr;
    if (cudaHostAlloc((void **)&h, sizeof(HostStatus), cudaHostAllocMapped | cudaHostAllocPortable) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    if (cudaHostGetDevicePointer((void **)&m.d, h, 0) != cudaSuccess) {
      cudaGetLastError();
      cudaFreeHost(h);
      return nullptr;
    }
    memset(h, 0, sizeof(HostStatus));
    m.h = h;
  }
  return &m;
}

// Copy the status word (and, if t_src is set, *t_src into its T field) to the
// host mirror, then publish seq.
static __global__ void k_keep_flags(const DevStatus *st, int32_t *late) {
  pdl_entry();
  if (threadIdx.x == 0) *late = __ldcg(&st->flags);
}

static __global__ void k_publish(const DevStatus *st, const int64_t *t_src, HostStatus *h, uint64_t seq) {
  pdl_entry();
  constexpr int NW = (int)(sizeof(DevStatus) / 4);
  static_assert(sizeof(DevStatus) % 4 == 0 && NW <= 32, "one warp copies the status word");
  const uint32_t *src = (const uint32_t *)st;
  if (threadIdx.x < NW) ((volatile uint32_t *)&h->st)[threadIdx.x] = __ldcg(src + threadIdx.x);
  __syncwarp();
  if (threadIdx.x == 0 && t_src) *(volatile int64_t *)&h->st.T = __ldcg(t_src);
  __threadfence_system();
  __syncwarp();
  if (threadIdx.x == 0) {
    __threadfence_system();
    *(volatile uint64_t *)&h->seq = seq;
  }
}

// Sync point, in two halves: publish_status enqueues the copy (work
// enqueued after it overlaps the host's wait); wait_status polls for it.  The
// wait asks the stream for errors every 1024 polls, so a failed kernel ends it.
static vr_status publish_status(const DevStatus *dst, StatusMirror *m, cudaStream_t s,
                                const int64_t *t_src = nullptr) {
  launch_dep(k_publish, 1, 32, 0, s, dst, t_src, m->d, ++m->next);
  count_launch();
  VR_CUDA(cudaGetLastError());
  return VR_OK;
}

static vr_status wait_status(StatusMirror *m, cudaStream_t s) {
  const uint64_t seq = m->next;
  const volatile uint64_t *p = &m->h->seq;
  for (uint64_t k = 1; *p != seq; ++k) {
    if ((k & 1023) == 0) {
      const cudaError_t e = cudaStreamQuery(s);
      if (e == cudaSuccess && *p != seq) {
        set_error("the status word was not published");
        return VR_ERR_INTERNAL;
      }
      if (e != cudaSuccess && e != cudaErrorNotReady) return cuda_status(e, "status wait", __FILE__, __LINE__);
    }
#if defined(__x86_64__)
    __builtin_ia32_pause();
#endif
  }
  std::atomic_thread_fence(std::memory_order_acquire);
  return flags_to_status(m->h->st.flags);
}

static vr_status read_status(const DevStatus *dst, StatusMirror *m, cudaStream_t s, const int64_t *t_src = nullptr) {
  VR_TRY(publish_status(dst, m, s, t_src));
  return wait_status(m, s);
}

// fp32 thresholds of the cap test: a_keep = largest float a with
// a (1 + crel) + 2^-100 <= r2 (certainly kept), a_drop = smallest float a with
// a (1 - crel) - 2^-100 > r2 (certainly dropped); both bounds are monotone in a.
static void f32_thresholds(double r2, double crel, float *a_keep, float *a_drop) {
  auto hi = [&](float a) { return (double)a * (1.0 + crel) + F32_ABS_SLACK; };
  auto lo = [&](float a) { return (double)a * (1.0 - crel) - F32_ABS_SLACK; };
  // Start from the solutions of the two linear bounds; a few ulp steps fix
  // the rounding of the estimate.
  float k = (float)((r2 - F32_ABS_SLACK) / (1.0 + crel));
  if (k < 0.f) k = 0.f;
  while (k > 0.f && hi(k) > r2) k = std::nextafter(k, -INFINITY);
  while (hi(std::nextafter(k, INFINITY)) <= r2) k = std::nextafter(k, INFINITY);
  if (hi(k) > r2) k = -1.f;  // nothing is certainly kept
  float dr = (float)((r2 + F32_ABS_SLACK) / (1.0 - crel));
  while (lo(dr) <= r2) dr = std::nextafter(dr, INFINITY);
  while (dr > 0.f && lo(std::nextafter(dr, -INFINITY)) > r2) dr = std::nextafter(dr, -INFINITY);
  *a_keep = k;
  *a_drop = dr;
}

template <bool F, int DR>
static void launch_dist(const void *X, int n, int d, int W, const Cap &cap, uint32_t *adj, DevStatus *st,
                        cudaStream_t s) {
  const int B = (n + 31) / 32;
  dim3 grid(B, (B + 7) / 8);
  launch_dep(k_dist_bitmap<F, DR>, grid, 256, 0, s, X, n, d, W, cap, adj, st, (int32_t *)nullptr);
}

bool gram_tc_eligible(vr_dtype dtype, int n, int d);
struct GramAcc;
vr_status gram_bitmap_tc(const void *X, int n, int d, bool F, const Cap &cap, uint32_t *adj, DevStatus *st,
                         cudaStream_t s, GramAcc *acc, int split = 0);

// Time-sliced adjacency of the max-edge triangle enumeration: at most this
// many bytes of snapshots (kept well inside L2), at most SNAP_MAX_S slices.
constexpr int64_t SNAP_BUDGET = int64_t(32) << 20;
// Below this many kept edges the lex order is taken (see force_lex).
constexpr int64_t SNAP_MIN_E = int64_t(1) << 15;
static int snap_slices(int n, int W, int64_t E) {
  const int64_t per = (int64_t)n * snap_stride(W) * 4;
  int64_t S = 1 + SNAP_BUDGET / std::max<int64_t>(per, 1);
  S = std::min<int64_t>(S, SNAP_MAX_S);
  S = std::min<int64_t>(S, std::max<int64_t>(E, 1));
  return (int)std::max<int64_t>(S, 1);
}

// Largest size of the tetrahedron stage's per-edge prefix table (E * W
// 16-bit counts); beyond it the face positions come from bisections.
constexpr int64_t TET_PRE_MAX_BYTES = int64_t(1) << 28;

// Largest kept-edge count for which the lexicographic triangle keys are
// generated before the host knows T (their buffer then holds the bound
// (sqrt 2 / 3) E^(3/2): at most 22M keys).
constexpr int64_t EARLY_TRI_MAX_E = int64_t(1) << 17;

// Max-edge key width: 0 = automatic (32-bit keys whenever the edge indices
// fit), 8 = always (e << 32) | z.  Set by vr_set_tri_key_width.
static std::atomic<int> g_tri_key_width{0};

// Max-edge key space: 0 = automatic (claimed by the generator, no triangle
// count before it, whenever the wedge-bound buffer is taken), 1 = counted
// (count, scan, then the generator at the scanned offsets), 2 = claimed with
// sub-buffers of CLAIM_TEST_SLOTS slots, so that claims run out and the
// counted generator takes over (tests).  Set by vr_set_tri_claim.
static std::atomic<int> g_tri_claim{0};
constexpr int64_t CLAIM_TEST_SLOTS = 64;

// Max-edge order: the key generator is enqueued before the host reads T when
// its buffer, sized by the wedge bound T <= sum_v C(deg v, 2) / 3, stays
// under this many bytes (4000-point float cloud: 33.0M keys for 19.8M
// triangles); the host's wait then overlaps the generator.
constexpr int64_t EARLY_GEN_MAX_BYTES = int64_t(1) << 30;

// Largest all-pairs count for which the edge keys are generated before the
// host knows the kept-edge count (the key buffers then hold every pair: at
// most 8M keys, n <= 4096, 160 MB of float keys, lex list and FP64 values).
// The 4000-point float cloud: 0.817 -> 0.808 ms against a limit of 1M pairs.
constexpr int64_t EARLY_KEYS_MAX = int64_t(1) << 23;

template <bool F>
static void dist_dispatch(const void *X, int n, int d, int W, const Cap &cap, uint32_t *adj, DevStatus *st,
                          cudaStream_t s) {
  if (d <= 4) launch_dist<F, 4>(X, n, d, W, cap, adj, st, s);
  else if (d <= 16) launch_dist<F, 16>(X, n, d, W, cap, adj, st, s);
  else if (d <= 32) launch_dist<F, 32>(X, n, d, W, cap, adj, st, s);
  else launch_dist<F, 0>(X, n, d, W, cap, adj, st, s);
}

template <bool F>
// `dmat` non-null: the edge values come from that n x n device matrix
// (dtype VR_I32 or VR_F32 = its element type; d and dpts unused, F false).
static vr_status build_impl(const void *dpts, int32_t n, int32_t d, vr_dtype dtype, int32_t maxdim, double maxrad,
                            cudaStream_t s, vr_complex *res, const void *dmat = nullptr) {
  StatusMirror *sm = status_mirror();
  if (!sm) {
    set_error("mapped host status buffer allocation failed");
    return VR_ERR_OOM;
  }
  const DevStatus *hst = &sm->h->st;
  Arena ws(s), out(s);
  Prof prof(s);
  const int W = (n + 31) / 32;
  const int64_t nd = (int64_t)n * d;

  // Cap parameters (integer: floor(fl(maxrad^2)); float: fl(maxrad^2)).
  Cap cap{};
  const double r2 = maxrad * maxrad;
  cap.keep_all = std::isinf(r2) ? 1 : 0;
  cap.r2 = r2;
  cap.crel = (d + 5) * std::ldexp(1.0, -24);
  if (!F && !cap.keep_all) {
    double f = std::floor(r2);
    cap.r2i = f >= 18446744073709551615.0 ? ~0ull : (uint64_t)f;
  }
  if (F && !cap.keep_all) {
    if (r2 >= 1e38) cap.keep_all = 1;  // beyond any fp32 first-pass value of valid input
    else {
      f32_thresholds(r2, cap.crel, &cap.a_keep, &cap.a_drop);
      cap.r2f_dn = (float)r2;
      if ((double)cap.r2f_dn > r2) cap.r2f_dn = std::nextafter(cap.r2f_dn, -INFINITY);
      cap.r2f_up = (float)r2;
      if ((double)cap.r2f_up < r2) cap.r2f_up = std::nextafter(cap.r2f_up, INFINITY);
    }
  }

  // Matrix input: keep iff key <= capkey (int: floor(maxrad); float: the
  // bits of the largest float <= maxrad).
  const bool dmf = dmat && dtype == VR_F32;
  int dm_keep_all = std::isinf(maxrad) ? 1 : 0;
  uint32_t capkey = 0;
  if (dmat && !dm_keep_all) {
    if (dmf) {
      if (maxrad >= 3.4028234663852886e38) dm_keep_all = 1;
      else {
        float f = (float)maxrad;
        if ((double)f > maxrad) f = std::nextafter(f, -INFINITY);
        memcpy(&capkey, &f, 4);
      }
    } else {
      const double f = std::floor(maxrad);
      capkey = f >= 2147483647.0 ? 0x7fffffffu : (uint32_t)f;
    }
  }

  DevStatus *st;
  void *X;
  uint32_t *adj;
  int32_t *adjpre, *deg, *up, *nbr_ptr;
  int2 *adjx;  // {row word, prefix count} pairs for the max-edge final write
  int64_t *lex_ptr;
  // The edge sort's scratch (digit histogram, tile status) and the edge-grade
  // look-back words, sized for every possible edge, follow the status word
  // in one block, so that a single memset clears all three up front.
  const int64_t E_ub = (int64_t)n * (n - 1) / 2;
  const int64_t eg_words = (E_ub + EG_TILE - 1) / EG_TILE + 1;
  RadixScratch rs{};
  uint64_t *eg_lb;  // look-back status of the edge-grade tiles + their ticket
  ws.begin();
  uint32_t *claim_ctr;  // the claiming generator's counters (zeroed with the status word)
  VR_TRY(ws.alloc(&st, 1));
  VR_TRY(ws.alloc(&claim_ctr, (CLAIM_CTRS + 1) * 32));  // + the final write's group ticket
  VR_TRY(ws.alloc(&rs.meta, rs_meta_bytes(E_ub)));
  VR_TRY(ws.alloc(&eg_lb, eg_words));
  // Staged points: int32 input is used in place (the build only reads it
  // before it returns); int8 and float are converted (and floats checked).
  const bool in_place = !dmat && dtype == VR_I32;
  if (!in_place) VR_TRY(F ? ws.alloc((float **)&X, nd) : ws.alloc((int32_t **)&X, nd));
  VR_TRY(ws.alloc(&adj, (int64_t)n * W));
  VR_TRY(ws.alloc(&adjpre, (int64_t)n * W));
  VR_TRY(ws.alloc(&adjx, (int64_t)n * W));
  VR_TRY(ws.alloc(&deg, n));
  VR_TRY(ws.alloc(&up, n));
  VR_TRY(ws.alloc(&nbr_ptr, n + 1));
  VR_TRY(ws.alloc(&lex_ptr, n + 1));
  // Clouds whose every possible edge fits EARLY_KEYS_MAX: the edge-key
  // buffers are sized for all pairs, so the key generator runs between the
  // status publish and the host's wait (the GPU works while the host reads
  // the edge count and allocates).
  const bool early_keys = E_ub <= EARLY_KEYS_MAX;
  uint64_t *keys = nullptr;
  uint32_t *lexe = nullptr;  // kept edges in lexicographic order, (i << 13) | j
  double *d64_lex = nullptr;
  int32_t *elp = nullptr;    // dense (i, j) -> lexicographic position (tetrahedra)
  const bool want_elp = n <= DENSE_MAX_N && maxdim >= 3;
  if (early_keys) {
    VR_TRY(ws.alloc(&keys, E_ub));
    VR_TRY(ws.alloc(&lexe, E_ub));
    if (F) VR_TRY(ws.alloc(&d64_lex, E_ub));
    if (want_elp) VR_TRY(ws.alloc(&elp, (int64_t)n * n));
  }
  VR_TRY(ws.commit());
  VR_CUDA(cudaMemsetAsync(st, 0, (size_t)((char *)(eg_lb + eg_words) - (char *)st), s));

  // Edge keys in (i, j) order: a stable sort on the distance bits alone then
  // yields (distance, i, j).  The generator also counts the sort's digit
  // histogram (into rs.meta, cleared above).
  int kbits;
  if (F) kbits = 31;
  else if (dmat) kbits = dm_keep_all ? 31 : std::max(1, bitlen(capkey));
  else {
    uint64_t bound = dtype == VR_I8 ? (uint64_t)d * 255ull * 255ull : INT_KEY_LIMIT - 1;
    if (!cap.keep_all) bound = std::min(bound, cap.r2i);
    kbits = std::max(1, bitlen(bound));
  }
  // Float keys: the lexicographic edge list first, then the keys over it (the
  // sort's histogram then comes from its own pass).
  KeyHist ekh{};
  auto edge_keys = [&](int64_t ecap) -> vr_status {
    if (!F) VR_TRY(radix_prepare(ecap, KEY_SHIFT, kbits, rs, s, &ekh, true));
    prof.begin("edge_keys");
    if constexpr (F) {
      launch_dep(k_lex_edges, (n + 7) / 8, 256, 0, s, n, W, adj, lex_ptr, lexe, elp, st);
      launch_dep(k_edge_keys_f32, grid_for((ecap + 31) / 32, EKF_WARPS, 16), EKF_WARPS * 32, 0, s,
                 (const float *)X, d, lexe, keys, d64_lex, st);
      count_launch();
    } else if (dmat) {
      if (dmf) launch_dep(k_dmat_keys<true>, (n + 7) / 8, 256, 0, s, dmat, n, W, adj, lex_ptr, keys, lexe, elp, ekh, st);
      else launch_dep(k_dmat_keys<false>, (n + 7) / 8, 256, 0, s, dmat, n, W, adj, lex_ptr, keys, lexe, elp, ekh, st);
    } else {
      launch_dep(k_edge_keys<F>, (n + 7) / 8, 256, 0, s, X, n, d, W, adj, lex_ptr, keys, lexe, elp, ekh, st);
    }
    count_launch();
    VR_CUDA(cudaGetLastError());
    prof.end();
    return VR_OK;
  };

  // Stage: convert to the working element type and check values (int8
  // with d <= 4 on the CUDA-core path: the distance kernel stages as it
  // loads; int32: in place).
  const bool tc = !dmat && gram_tc_eligible(dtype, n, d);
  const bool fused8 = !dmat && !tc && dtype == VR_I8 && d <= 4;
  if (in_place) X = (void *)dpts;
  prof.begin("stage");
  const unsigned gs = grid_for(nd, 256, 8);
  if (dmat) {
    const int nb = (n + 31) / 32;
    if (dmf) launch_dep(k_dmat_check<true>, nb * nb, 256, 0, s, dmat, n, st);
    else launch_dep(k_dmat_check<false>, nb * nb, 256, 0, s, dmat, n, st);
    count_launch();
  } else if (dtype == VR_I8 && !fused8) {
    launch_dep(k_stage<int8_t, false>, gs, 256, 0, s, (const int8_t *)dpts, nd, (int32_t *)X, st);
    count_launch();
  } else if (F) {
    launch_dep(k_stage<float, true>, gs, 256, 0, s, (const float *)dpts, nd, (float *)X, st);
    count_launch();
  }
  VR_CUDA(cudaGetLastError());
  prof.end();

  prof.begin("distance");
  if (dmat) {
    if (dmf) launch_dep(k_dmat_bitmap<true>, (n + 7) / 8, 256, 0, s, dmat, n, W, dm_keep_all, capkey, adj);
    else launch_dep(k_dmat_bitmap<false>, (n + 7) / 8, 256, 0, s, dmat, n, W, dm_keep_all, capkey, adj);
    count_launch();
  } else if (tc) {
    VR_TRY(gram_bitmap_tc(X, n, d, F, cap, adj, st, s, nullptr));  // tensor-core Gram tiles
  } else if (fused8) {
    const int B = (n + 31) / 32;
    launch_dep(k_dist_bitmap<false, 4, true>, dim3(B, (B + 7) / 8), 256, 0, s, dpts, n, d, W, cap, adj, st,
               (int32_t *)X);
    count_launch();
  } else {
    dist_dispatch<F>(X, n, d, W, cap, adj, st, s);
    count_launch();
  }
  VR_CUDA(cudaGetLastError());
  prof.end();
  prof.begin("row_counts");
  launch_dep(k_rows_scan, (n + 7) / 8, 256, 0, s, adj, n, W, adjpre, deg, up, nbr_ptr, lex_ptr, st, adjx);
  count_launch();
  VR_CUDA(cudaGetLastError());
  prof.end();

  // ---- sync 1: kept-edge count and value errors.
  VR_TRY(publish_status(st, sm, s));
  if (early_keys) VR_TRY(edge_keys(E_ub));
  VR_TRY(wait_status(sm, s));
  if (tc && (hst->flags & F_OVERFLOW)) {
    // The Gram tiles' near-cap list overflowed (pathological clustering at
    // the cap): rebuild the bitmap exactly on the CUDA cores (and the early
    // keys, after clearing the histogram they added to; unreachable while
    // the list holds at least EARLY_KEYS_MAX pairs, kept for safety).
    VR_CUDA(cudaMemsetAsync(&st->flags, 0, sizeof(int32_t), s));
    dist_dispatch<F>(X, n, d, W, cap, adj, st, s);
    count_launch();
    launch_dep(k_rows_scan, (n + 7) / 8, 256, 0, s, adj, n, W, adjpre, deg, up, nbr_ptr, lex_ptr, st, adjx);
    count_launch();
    VR_TRY(publish_status(st, sm, s));
    if (early_keys) {
      VR_CUDA(cudaMemsetAsync(rs.meta, 0, (size_t)RS_META_HEAD, s));
      VR_TRY(edge_keys(E_ub));
    }
    VR_TRY(wait_status(sm, s));
  }
  const int64_t E = hst->E;
  const int64_t wedges = hst->wedges;
  if (E > INT32_MAX) {
    set_error("%lld edges exceed the 2^31-1 limit of one dimension", (long long)E);
    return VR_ERR_RANGE;
  }

  int32_t *nbr_ord, *gstart;
  int32_t *everts, *egrade, *erow;
  int64_t *ecol, *bs_e;
  double *gval, *d64 = nullptr;
  // Every E-sized array of the rest of the build: one workspace block and one
  // output block.
  ws.begin();
  out.begin();
  if (!early_keys) {
    VR_TRY(ws.alloc(&keys, E));
    VR_TRY(ws.alloc(&lexe, E));
    if (F && E > 0) VR_TRY(ws.alloc(&d64_lex, E));
    if (want_elp) VR_TRY(ws.alloc(&elp, (int64_t)n * n));
  }
  VR_TRY(ws.alloc(&rs.tkeys, E));
  VR_TRY(ws.alloc(&bs_e, scan_tmp_slots(E)));
  VR_TRY(ws.alloc(&nbr_ord, 2 * E));
  int32_t *eidx = nullptr, *egd = nullptr;  // dense (i, j) -> order index / grade tables (allocated below)
  VR_TRY(ws.alloc(&gstart, E + 2));
  VR_TRY(out.alloc(&everts, 2 * E));
  VR_TRY(out.alloc(&egrade, E));
  VR_TRY(out.alloc(&ecol, E + 1));
  VR_TRY(out.alloc(&erow, 2 * E));
  VR_TRY(out.alloc(&gval, E + 1));
  int32_t *late_flags = nullptr;
  VR_TRY(out.alloc(&late_flags, 1));
  int32_t *midq = nullptr, *bigq = nullptr;
  uint64_t *k1 = nullptr, *k2 = nullptr, *gk = nullptr;
  uint32_t *v1 = nullptr, *v2 = nullptr;
  double *gd = nullptr;
  if (F && E > 0) {
    VR_TRY(ws.alloc(&d64, E));
    VR_TRY(ws.alloc(&midq, E));
    VR_TRY(ws.alloc(&bigq, E));
    VR_TRY(ws.alloc(&k1, E));
    VR_TRY(ws.alloc(&k2, E));
    VR_TRY(ws.alloc(&gk, E));
    VR_TRY(ws.alloc(&v1, E));
    VR_TRY(ws.alloc(&v2, E));
    VR_TRY(ws.alloc(&gd, E));
  }
  int32_t *tcnt = nullptr, *tsmallq = nullptr, *tmidq = nullptr, *tbigq = nullptr;
  int64_t *toff = nullptr;
  // Triangle order: lex mode is forced for tetrahedra and for clouds whose
  // rows are sparse (fewer neighbours on average than bitmap words): there
  // the lex walk takes each edge's candidates from the lexicographic edge
  // list, one bit test each, cheaper than the max-edge enumeration's
  // time-sliced rows (the 7322-point WorldMap-shaped cloud: 77 neighbours
  // per point, 229 words per row).  Otherwise lex_mode decides on the device
  // by the share of tied grades.
  const int sparse_rows = 2 * E < (int64_t)n * W ? 1 : 0;
  // Lex order is also certain, before the grades are known, when the keys'
  // distance field cannot hold enough distinct values for 95 % of the edges
  // (integer data: at most 2^kbits distinct squared distances), and it is
  // taken for small edge counts, where the time-sliced adjacency's fixed
  // cost exceeds the triangle sort's.
  const bool ties_certain = !F && kbits < 62 && (E - ((int64_t)1 << kbits)) * 20 > E;
  const int force_lex = (maxdim >= 3 || sparse_rows || ties_certain || E < SNAP_MIN_E) ? 1 : 0;
  SnapIdx sx{nullptr, nullptr, nullptr, 1, 1, snap_stride(W)};
  uint32_t *snap = nullptr;
  uint64_t *sbl = nullptr;
  int32_t *sboff = nullptr;
  const bool want_snap = maxdim == 2 && E > 0 && !force_lex;
  if (want_snap) {
    sx.S = snap_slices(n, W, E);
    sx.B = (E + sx.S - 1) / sx.S;
    VR_TRY(ws.alloc(&sbl, 2 * E));
    VR_TRY(ws.alloc(&sboff, (int64_t)n * (sx.S + 1)));
    if (sx.S > 1) VR_TRY(ws.alloc(&snap, (int64_t)(sx.S - 1) * n * sx.Wp));
  }
  // Small complexes (maxdim 2, E <= EARLY_TRI_MAX_E): the lexicographic
  // triangle keys get a buffer sized by the bound on the triangles of a graph
  // with E edges, T <= (sqrt 2 / 3) E^(3/2), so the generator can be enqueued
  // before the host reads T (it returns at once in max-edge mode).
  const bool early_tri = maxdim == 2 && E > 0 && E <= EARLY_TRI_MAX_E;
  const int64_t T_cap = early_tri ? (int64_t)std::ceil(std::sqrt(2.0) / 3.0 * std::pow((double)E, 1.5)) + 1 : 0;
  uint64_t *tk = nullptr;
  if (early_tri) VR_TRY(ws.alloc(&tk, T_cap));
  // Max-edge keys take 32 bits, (e << zbits) | z, when the edge indices fit
  // the bits n leaves (E <= 2^20 at n = 4000), else (e << 32) | z.
  const int me_zbits = std::max(1, bitlen((uint64_t)(n - 1)));
  const bool me_key32 = g_tri_key_width.load() != 8 && E <= (int64_t(1) << (32 - me_zbits));
  const int64_t T_wedge = wedges / 3 + 1;
  const bool early_gen = want_snap && (double)T_wedge * (me_key32 ? 4 : 8) <= (double)EARLY_GEN_MAX_BYTES;
  uint64_t *tk_me = nullptr;  // max-edge keys
  // Claimed key space (early_gen, unless counted keys are asked for): the
  // generator runs before any triangle count, taking room for each edge's
  // third vertices (16 bits each) from a buffer of 2 T_wedge slots (kpos[e]
  // locates them), and the final write reads them directly; the key buffer
  // is then needed only if a claim runs out, and is allocated after the
  // host's wait.  Otherwise the keys go to the bound-sized buffer.
  const int claim_mode = g_tri_claim.load();
  const bool claim = early_gen && claim_mode != 1;
  const int64_t tz_slots = 2 * T_wedge;
  int32_t *kpos = nullptr;
  uint16_t *tz = nullptr;
  if (early_gen && !claim) VR_TRY(ws.alloc(&tk_me, me_key32 ? (T_wedge + 1) / 2 : T_wedge));
  if (claim) {
    VR_TRY(ws.alloc(&kpos, E));
    VR_TRY(ws.alloc(&tz, tz_slots));
  }
  // The dense order-index and grade tables serve the lex-order kernels and
  // the counted max-edge count; on the claimed path nothing reads them, so
  // the edge-grade kernel skips their two scattered writes per edge (if the
  // device then takes lex order after all, its kernels look faces up
  // through the neighbour CSR instead).
  if (n <= DENSE_MAX_N && maxdim >= 2 && !claim) {
    VR_TRY(ws.alloc(&eidx, (int64_t)n * n));
    VR_TRY(ws.alloc(&egd, (int64_t)n * n));
  }
  if (maxdim >= 2 && E > 0) {
    VR_TRY(ws.alloc(&tcnt, E));
    VR_TRY(ws.alloc(&toff, E + 1));
    VR_TRY(ws.alloc(&tsmallq, E + 1));
    VR_TRY(ws.alloc(&tmidq, E + 1));
    VR_TRY(ws.alloc(&tbigq, E + 1));
  }
  VR_TRY(ws.commit());
  VR_TRY(out.commit());
  rs.err = &st->flags;
  sx.snap = snap;
  sx.bl = sbl;
  sx.boff = sboff;

  const unsigned ge = grid_for(E, 256);
  if (E > 0) {
    if (!early_keys) VR_TRY(edge_keys(E));
    prof.begin("edge_sort");
    static const char *const etag[2] = {"edge_sort.hist", "edge_sort.pass"};
    VR_TRY(radix_sort(keys, E, KEY_SHIFT, kbits, rs, s, &prof, etag, F ? RS_PREP_ZEROED : RS_PREP_HIST));
    prof.end();

    if (F) {
      prof.begin("fp64_repair");
      count_launch(3);
      const F64Src fsrc{d64_lex, adj, adjpre, W, deg, up, lex_ptr};
      launch_dep(k_f64_repair_small, ge, 256, 0, s, keys, E, fsrc, d64, midq, bigq, st);
      VR_CUDA(cudaGetLastError());
      launch_dep(k_repair_mid, (unsigned)num_sms() * 2, 256, 0, s, midq, fsrc, st, keys, d64);
      launch_dep(k_repair_big, 1, RS_THREADS, 0, s, bigq, fsrc, st, keys, d64, k1, v1, k2, v2, gk, gd);
      VR_CUDA(cudaGetLastError());
      prof.end();
    }
    prof.begin("edge_grades");
    const int64_t egt = (E + EG_TILE - 1) / EG_TILE;
    launch_dep(k_edge_grades<F>, (unsigned)egt, 256, 0, s, (const uint64_t *)keys, (const double *)d64, E,
               (const int2 *)adjx, W, (const int32_t *)nbr_ptr, everts, egrade, ecol, erow, gval, gstart, nbr_ord,
               eidx, egd, n, dmf ? 1 : 0, eg_lb, egt, st);
    count_launch();
    VR_CUDA(cudaGetLastError());
    prof.end();
  } else {
    const double zero = 0.0;
    const int64_t zero64 = 0;
    VR_CUDA(cudaMemcpyAsync(gval, &zero, sizeof(double), cudaMemcpyHostToDevice, s));
    VR_CUDA(cudaMemcpyAsync(ecol, &zero64, sizeof(int64_t), cudaMemcpyHostToDevice, s));
  }

  // Max-edge key generation (returns at once if the device chose lex order):
  // claimed (cl: before the triangle count, which then skips max-edge
  // edges), or at the counted offsets into the bound-sized buffer before the
  // host's wait, or after it.
  const EdgeIndex exm{adjx, adj, adjpre, nbr_ptr, nbr_ord, eidx, egd, egrade, W, n};
  const int64_t claim_sub = claim_mode == 2 ? CLAIM_TEST_SLOTS : tz_slots / CLAIM_CTRS;
  // The claiming generator runs one wave (five CTAs of 8 warps per SM at its
  // register count); each warp claims slots in chunks whose total over all
  // warps stays within the T_wedge slots of headroom (tz_slots >= T + T_wedge).
  const unsigned g_claim = grid_for(E, 16, 5);
  const int32_t claim_chunk = (int32_t)std::min<int64_t>(1024, T_wedge / ((int64_t)g_claim * 8));
  const ClaimBuf cb{tz, kpos, tcnt, claim_ctr, claim_sub, claim_chunk};
  auto me_gen = [&](int64_t cap, bool cl) -> vr_status {
    prof.begin("tri_gen");
    // 16-byte chunks per lane and row: Wp / 16 words rounded up to whole
    // chunks (a compile-time count per kernel).
    const int k4 = ((((sx.Wp + 15) >> 4) + 3) & ~3) >> 2;
    const unsigned g = cl ? g_claim : grid_for(E, 8, 32);
    auto go = [&](auto key, auto clt) {
      using KT = decltype(key);
      constexpr bool CL = decltype(clt)::value;
      KT *tkk = (KT *)tk_me;
      const int zb = sizeof(KT) == 4 ? me_zbits : 32;
      if (k4 <= 1)
        launch_dep(k_tri_gen_me<KT, 1, CL>, g, 256, 0, s, everts, E, W, n, nbr_ptr, toff, cap, tkk, zb, sx, st,
                   force_lex, cb);
      else if (k4 == 2)
        launch_dep(k_tri_gen_me<KT, 2, CL>, g, 256, 0, s, everts, E, W, n, nbr_ptr, toff, cap, tkk, zb, sx, st,
                   force_lex, cb);
      else if (k4 == 3)
        launch_dep(k_tri_gen_me<KT, 3, CL>, g, 256, 0, s, everts, E, W, n, nbr_ptr, toff, cap, tkk, zb, sx, st,
                   force_lex, cb);
      else
        launch_dep(k_tri_gen_me<KT, 4, CL>, g, 256, 0, s, everts, E, W, n, nbr_ptr, toff, cap, tkk, zb, sx, st,
                   force_lex, cb);
    };
    if (cl) go(uint32_t{0}, std::true_type{});
    else if (me_key32) go(uint32_t{0}, std::false_type{});
    else go(uint64_t{0}, std::false_type{});
    count_launch();
    VR_CUDA(cudaGetLastError());
    prof.end();
    return VR_OK;
  };
  if (maxdim >= 2 && E > 0) {
    if (want_snap) {
      // Time-sliced adjacency for the max-edge enumeration (returns at once
      // when the device finds lex mode).
      prof.begin("tri_snap");
      const int snap_threads = 32 * ((sx.Wp + 31) / 32);  // a warp per 32-word round of a row
      const size_t snap_smem = snap_build_smem(snap_threads / 32, sx.S);
      launch_dep(k_snap_build, (unsigned)std::min<int64_t>(n, (int64_t)num_sms() * 32), snap_threads, snap_smem, s,
                 adj, adjpre, W, n, nbr_ptr, nbr_ord, st, force_lex, sx.S, sx.B, snap, sbl, sboff);
      count_launch();
      VR_CUDA(cudaGetLastError());
      prof.end();
    }
    if (claim) VR_TRY(me_gen(0, true));
    prof.begin("tri_count");
    const EdgeIndex exc{adjx, adj, adjpre, nbr_ptr, nbr_ord, eidx, egd, egrade, W, n};
    const int me_claimed = claim ? 1 : 0;
    // After the claiming generator the count only has work in lex order (a
    // device decision, rare there): two CTAs per SM, grid-stride, instead of
    // a CTA per 64 edges that would mostly launch to return.
    const unsigned gcnt = claim ? grid_for(E, 8, 2) : grid_for(E, 8, 32);
    if (eidx)
      launch_dep(k_tri_count<true>, gcnt, 256, 0, s, everts, lexe, E, adj, adjpre, W, nbr_ptr,
                 nbr_ord, st, tcnt, force_lex, exc, (const int64_t *)lex_ptr, sparse_rows, sx, me_claimed);
    else
      launch_dep(k_tri_count<false>, gcnt, 256, 0, s, everts, lexe, E, adj, adjpre, W, nbr_ptr,
                 nbr_ord, st, tcnt, force_lex, exc, (const int64_t *)lex_ptr, sparse_rows, sx, me_claimed);
    count_launch(2);
    VR_TRY((scan_exclusive<int32_t, int64_t>(tcnt, toff, E, bs_e, s)));
    launch_dep(k_tri_groups, grid_for(E + 1, 256), 256, 0, s, gstart, tcnt, toff, tsmallq, tmidq, tbigq, st,
               force_lex);
    VR_CUDA(cudaGetLastError());
    prof.end();
  }

  // ---- sync 2: grade count, triangle count, tie-group sizes.
  VR_TRY(publish_status(st, sm, s));
  auto lex_tri_gen = [&](int64_t tcap) -> vr_status {
    prof.begin("tri_lex_gen");
    const EdgeIndex ex{adjx, adj, adjpre, nbr_ptr, nbr_ord, eidx, egd, egrade, W, n};
    if (eidx)
      launch_dep(k_lex_tri_gen<true>, grid_for(E, 8, 32), 256, 0, s, lexe, egrade, E, adj, adjpre, W, nbr_ptr,
                 nbr_ord, toff, tcap, tk, ex, st, force_lex, (const int64_t *)lex_ptr, sparse_rows);
    else
      launch_dep(k_lex_tri_gen<false>, grid_for(E, 8, 32), 256, 0, s, lexe, egrade, E, adj, adjpre, W, nbr_ptr,
                 nbr_ord, toff, tcap, tk, ex, st, force_lex, (const int64_t *)lex_ptr, sparse_rows);
    count_launch();
    VR_CUDA(cudaGetLastError());
    prof.end();
    return VR_OK;
  };
  if (early_tri) VR_TRY(lex_tri_gen(T_cap));
  if (early_gen && !claim) VR_TRY(me_gen(T_wedge, false));
  VR_TRY(wait_status(sm, s));
  const int64_t ngrades = E > 0 ? hst->ngrades : 1;
  const int64_t T = (maxdim >= 2 && E > 0) ? hst->T : 0;
  if (T > INT32_MAX) {
    set_error("%lld triangles exceed the 2^31-1 limit of one dimension", (long long)T);
    return VR_ERR_RANGE;
  }

  // Vertex and triangle outputs (one block) and the T-sized workspace.
  const bool lexm = T > 0 && lex_mode(E, ngrades, force_lex);
  const bool tets = maxdim >= 3 && T > 0;
  const bool bigfix = T > 0 && !lexm && hst->big_seg_count > 0;
  int32_t *vverts, *vgrade;
  int32_t *tverts = nullptr, *tgrade = nullptr, *trow = nullptr;
  int64_t *tcol = nullptr;
  uint64_t *tk1 = nullptr, *tk2 = nullptr;
  uint32_t *tv1 = nullptr, *tv2 = nullptr;
  int32_t *rtmp = nullptr;
  RadixScratch trs{};
  out.begin();
  ws.begin();
  VR_TRY(out.alloc(&vverts, n));
  VR_TRY(out.alloc(&vgrade, n));
  if (maxdim >= 2) {
    VR_TRY(out.alloc(&tverts, 3 * T));
    VR_TRY(out.alloc(&tgrade, T));
    VR_TRY(out.alloc(&tcol, T + 1));
    VR_TRY(out.alloc(&trow, 3 * T));
  }
  uint64_t *tk_lex = nullptr;  // tetrahedra: the triangles' keys in lexicographic order
  int32_t *ordidx = nullptr, *cnt4 = nullptr;
  int64_t *off4 = nullptr, *bs_t = nullptr;
  if (T > 0 && lexm && !early_tri) VR_TRY(ws.alloc(&tk, T));  // lex keys
  const bool claimed = claim && !(hst->flags & F_CLAIM);  // third vertices in claimed space
  if (T > 0 && !lexm && (!early_gen || (claim && !claimed))) VR_TRY(ws.alloc(&tk_me, me_key32 ? (T + 1) / 2 : T));
  if (early_gen && T > T_wedge) {
    set_error("%lld triangles exceed their bound %lld", (long long)T, (long long)T_wedge);
    return VR_ERR_INTERNAL;
  }
  if (lexm) {
    VR_TRY(ws.alloc(&trs.tkeys, T));
    VR_TRY(ws.alloc(&trs.meta, rs_meta_bytes(T)));
  }
  // Tetrahedra: per lexicographic edge, word-wise prefix counts of the common
  // neighbours (face positions by popcount instead of bisection) while the
  // table stays under TET_PRE_MAX_BYTES.
  uint16_t *tpre = nullptr;
  const bool use_tpre = tets && (double)E * W * 2 <= (double)TET_PRE_MAX_BYTES;
  if (use_tpre) VR_TRY(ws.alloc(&tpre, E * W));
  if (tets) {
    VR_TRY(ws.alloc(&tk_lex, T));
    VR_TRY(ws.alloc(&ordidx, T));
    VR_TRY(ws.alloc(&cnt4, T));
    VR_TRY(ws.alloc(&off4, T + 1));
    VR_TRY(ws.alloc(&bs_t, scan_tmp_slots(T)));
  }
  if (bigfix) {
    VR_TRY(ws.alloc(&tk1, T));
    VR_TRY(ws.alloc(&tk2, T));
    VR_TRY(ws.alloc(&tv1, T));
    VR_TRY(ws.alloc(&tv2, T));
    VR_TRY(ws.alloc(&rtmp, 3 * T));
  }
  VR_TRY(out.commit());
  VR_TRY(ws.commit());
  trs.err = &st->flags;
  // Vertices (and the triangles' closing colptr entry 3T); the same launch
  // clears the triangle sort's scratch.
  const int64_t tz_words = lexm ? rs_meta_bytes(T) / 8 : 0;
  launch_dep(k_vertices, grid_for(std::max<int64_t>(n, tz_words), 256), 256, 0, s, n, vverts, vgrade, tcol, T,
             (uint64_t *)trs.meta, tz_words);
  count_launch();
  VR_CUDA(cudaGetLastError());

  if (maxdim >= 2) {
    if (lexm) {
      // Lex-order generation, stable sort on the grade bits, final write.
      const int gbits = std::max(1, bitlen((uint64_t)(ngrades - 1)));
      // (The triangle generator is latency-bound: counting the sort's
      // histogram inside it cost more than the sort's own histogram pass.)
      if (!early_tri) VR_TRY(lex_tri_gen(T));
      const EdgeIndex ex{adjx, adj, adjpre, nbr_ptr, nbr_ord, eidx, egd, egrade, W, n};
      if (tets) VR_CUDA(cudaMemcpyAsync(tk_lex, tk, sizeof(uint64_t) * T, cudaMemcpyDeviceToDevice, s));
      prof.begin("tri_grade_sort");
      static const char *const ttag[2] = {"tri_sort.hist", "tri_sort.pass"};
      uint64_t *tks = tk;  // the sorted keys: tk or the sort's other buffer
      VR_TRY(radix_sort(tk, T, LEX_SHIFT, gbits, trs, s, &prof, ttag, RS_PREP_ZEROED, &tks));
      tk = tks;  // (the tetrahedron stage reads the sorted keys through tk)
      prof.end();
      prof.begin("tri_final");
      if (eidx)
        launch_dep(k_tri_final<true>, grid_for((T + 3) / 4, 256), 256, 0, s, tk, T, ex, tverts, tgrade, tcol, trow, st);
      else
        launch_dep(k_tri_final<false>, grid_for((T + 3) / 4, 256), 256, 0, s, tk, T, ex, tverts, tgrade, tcol, trow, st);
      count_launch();
      VR_CUDA(cudaGetLastError());
      prof.end();
    } else if (T > 0) {
      // Max-edge order: keys in final order from the time-sliced adjacency
      // (generated above when the bound-sized buffer was taken), then the
      // final write; tie groups merged after.
      // Claimed third vertices go straight to the final write; if a claim
      // ran out, the counted generator writes keys at the scanned offsets
      // (the claiming run's counts are exact either way).
      if (!early_gen || (claim && !claimed)) VR_TRY(me_gen(T, false));
      prof.begin("tri_final");
      if (claimed)
        launch_dep(k_tri_final_grp, grid_for((E + 31) / 32, 8, 4), 256, 0, s, (const uint16_t *)tz,
                   (const int32_t *)kpos, (const int32_t *)tcnt, (const int64_t *)toff, E, everts, egrade, exm,
                   tverts, tgrade, tcol, trow, claim_ctr + CLAIM_CTRS * 32, st);
      else if (me_key32)
        launch_dep(k_tri_final_me<uint32_t>, grid_for((T + 3) / 4, 256), 256, 0, s, (const uint32_t *)tk_me, me_zbits,
                   T, everts, egrade, exm, tverts, tgrade, tcol, trow, st);
      else
        launch_dep(k_tri_final_me<uint64_t>, grid_for((T + 3) / 4, 256), 256, 0, s, (const uint64_t *)tk_me, 32, T,
                   everts, egrade, exm, tverts, tgrade, tcol, trow, st);
      count_launch();
      VR_CUDA(cudaGetLastError());
      prof.end();
      prof.begin("tri_tie_merge");
      if (hst->small_seg_count > 0) {
        const size_t smem = (size_t)TRI_SMALL * (8 + 4 + 12);
        launch_dep(k_tri_fix_smem<TRI_SMALL>, std::min(hst->small_seg_count, num_sms() * 8), 256, smem, s, gstart, toff,
                   tsmallq, &st->small_seg_count, tverts, trow, st);
        count_launch();
        VR_CUDA(cudaGetLastError());
      }
      if (hst->mid_seg_count > 0) {
        const size_t smem = (size_t)TRI_MID * (8 + 4 + 12);
        VR_CUDA(cudaFuncSetAttribute(k_tri_fix_smem<TRI_MID>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
        launch_dep(k_tri_fix_smem<TRI_MID>, std::min(hst->mid_seg_count, num_sms()), 512, smem, s, gstart, toff, tmidq,
                   &st->mid_seg_count, tverts, trow, st);
        count_launch();
        VR_CUDA(cudaGetLastError());
      }
      if (bigfix) {
        launch_dep(k_tri_fix_big, (unsigned)std::min<int64_t>(hst->big_seg_count, (int64_t)num_sms() * 2), RS_THREADS, 0, s, gstart,
                   toff, tbigq, st, tverts, trow, tk1, tv1, tk2, tv2, rtmp);
        count_launch();
        VR_CUDA(cudaGetLastError());
      }
      prof.end();
    }
  }

  // Tetrahedra (maxdim 3): lexicographic generation from the lexicographic
  // triangle list, stable sort on the grade bits, final write.
  int64_t T4 = 0;
  int32_t *qverts = nullptr, *qgrade = nullptr, *qrow = nullptr;
  int64_t *qcol = nullptr;
  if (maxdim >= 3) {
    if (tets) {
      prof.begin("tet_count");
      if (tpre) {
        launch_dep(k_lex_pre, grid_for(E, 8, 32), 256, 0, s, lexe, E, adj, W, tpre, st);
        count_launch();
      }
      launch_dep(k_tri_ordidx, grid_for(T, 256), 256, 0, s, tk, T, tk_lex, ordidx, toff, adj, adjpre, W, deg, up,
                 lex_ptr, elp, n, tpre, st);
      launch_dep(k_tet_count, grid_for(T, 8, 32), 256, 0, s, tk_lex, T, adj, W, cnt4, st);
      count_launch(2);
      VR_TRY((scan_exclusive<int32_t, int64_t>(cnt4, off4, T, bs_t, s)));
      VR_CUDA(cudaGetLastError());
      prof.end();
      // ---- sync 3: tetrahedron count.
      VR_TRY(read_status(st, sm, s, off4 + T));
      T4 = hst->T;
      if (T4 > INT32_MAX) {
        set_error("%lld tetrahedra exceed the 2^31-1 limit of one dimension", (long long)T4);
        return VR_ERR_RANGE;
      }
    }
    uint64_t *keys4 = nullptr, *lex4 = nullptr;
    RadixScratch qrs{};
    const int qbits = std::max(1, bitlen((uint64_t)(ngrades - 1)));
    const bool packed = qbits <= 64 - TET_PACK_SHIFT;  // the sorted keys carry the vertices
    out.begin();
    ws.begin();
    VR_TRY(out.alloc(&qverts, 4 * T4));
    VR_TRY(out.alloc(&qgrade, T4));
    VR_TRY(out.alloc(&qcol, T4 + 1));
    VR_TRY(out.alloc(&qrow, 4 * T4));
    if (T4 > 0) {
      VR_TRY(ws.alloc(&keys4, T4));
      if (!packed) VR_TRY(ws.alloc(&lex4, T4));
      VR_TRY(ws.alloc(&qrs.tkeys, T4));
      VR_TRY(ws.alloc(&qrs.meta, rs_meta_bytes(T4)));
    }
    VR_TRY(out.commit());
    VR_TRY(ws.commit());
    qrs.err = &st->flags;
    if (T4 == 0) {
      VR_CUDA(cudaMemsetAsync(qcol, 0, sizeof(int64_t), s));
    } else {
      prof.begin("tet_gen");
      const EdgeIndex ex{adjx, adj, adjpre, nbr_ptr, nbr_ord, eidx, egd, egrade, W, n};
      if (eidx)
        launch_dep(k_tet_gen<true>, grid_for(T, 8, 32), 256, 0, s, tk_lex, T, adj, W, tgrade, ordidx, egrade, ex,
                   off4, T4, keys4, lex4, packed ? 1 : 0, st);
      else
        launch_dep(k_tet_gen<false>, grid_for(T, 8, 32), 256, 0, s, tk_lex, T, adj, W, tgrade, ordidx, egrade, ex,
                   off4, T4, keys4, lex4, packed ? 1 : 0, st);
      count_launch();
      VR_CUDA(cudaGetLastError());
      prof.end();
      prof.begin("tet_grade_sort");
      VR_TRY(radix_sort(keys4, T4, packed ? TET_PACK_SHIFT : 32, qbits, qrs, s));
      prof.end();
      prof.begin("tet_final");
      launch_dep(k_tet_final, grid_for(T4, 256), 256, 0, s, keys4, T4, lex4, tk_lex, toff, adj, adjpre, W, deg, up,
                 lex_ptr, ordidx, elp, n, packed ? 1 : 0, tpre, qverts, qgrade, qcol, qrow, st);
      count_launch();
      VR_CUDA(cudaGetLastError());
      prof.end();
    }
    // Value errors raised by the tetrahedron kernels (internal checks).
    VR_TRY(read_status(st, sm, s));
  }

  // The flags as the last kernel left them, for vr_complex_status (a
  // one-warp dependent launch: a copy-engine copy would break the chain of
  // dependent launches).
  launch_dep(k_keep_flags, 1, 32, 0, s, (const DevStatus *)st, late_flags);
  count_launch();
  VR_CUDA(cudaGetLastError());
  res->late_flags = late_flags;

  // Hand the outputs to the result.
  res->n = n;
  res->d = d;
  res->maxdim = maxdim;
  res->stream = s;
  res->count[0] = n;
  res->count[1] = maxdim >= 1 ? E : 0;
  res->count[2] = maxdim >= 2 ? T : 0;
  res->verts[0] = vverts;
  res->grade[0] = vgrade;
  res->verts[1] = everts;
  res->grade[1] = egrade;
  res->colptr[1] = ecol;
  res->rowidx[1] = erow;
  res->verts[2] = tverts;
  res->grade[2] = tgrade;
  res->colptr[2] = tcol;
  res->rowidx[2] = trow;
  res->count[3] = maxdim >= 3 ? T4 : 0;
  res->verts[3] = qverts;
  res->grade[3] = qgrade;
  res->colptr[3] = qcol;
  res->rowidx[3] = qrow;
  res->grade_value = gval;
  res->ngrades = ngrades;
  res->stats.kept_edges = E;
  res->stats.triangles = T;
  res->stats.ngrades = ngrades;
  // The float repair counters are final once the stream passes the repair
  // kernels, which precede sync 2.
  res->stats.near_tie_edges = F ? hst->near_tie : 0;
  double mre = 0.0;
  memcpy(&mre, &hst->max_rel_err_bits, sizeof(double));
  res->stats.max_rel_dist_err = F ? mre : 0.0;
  res->stats.tri_order = T == 0 ? 0 : lexm ? 1 : claimed ? 3 : 2;
  out.release_to(res->allocs);
  return VR_OK;
}

vr_status build_dmat(const void *D, int32_t n, vr_dtype dtype, int32_t maxdim, double maxrad, cudaStream_t s,
                     vr_complex *res) {
  return build_impl<false>(nullptr, n, 0, dtype, maxdim, maxrad, s, res, D);
}

vr_status build_cloud(const void *dpts, int32_t n, int32_t d, vr_dtype dtype, int32_t maxdim, double maxrad,
                      cudaStream_t s, vr_complex *res) {
  if (dtype == VR_F32) return build_impl<true>(dpts, n, d, dtype, maxdim, maxrad, s, res);
  return build_impl<false>(dpts, n, d, dtype, maxdim, maxrad, s, res);
}

}  // namespace vr

extern "C" vr_status vr_set_tri_claim(int32_t mode) {
  if (mode < 0 || mode > 2) {
    vr::set_error("triangle key space mode %d: 0 (automatic), 1 (counted) or 2 (claimed, test sub-buffers)", mode);
    return VR_ERR_ARG;
  }
  vr::g_tri_claim.store(mode);
  return VR_OK;
}

extern "C" vr_status vr_set_tri_key_width(int32_t bytes) {
  if (bytes != 0 && bytes != 8) {
    vr::set_error("triangle key width %d: 0 (automatic) or 8", bytes);
    return VR_ERR_ARG;
  }
  vr::g_tri_key_width.store(bytes);
  return VR_OK;
}
