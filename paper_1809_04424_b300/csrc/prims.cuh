// prims.cuh -- device primitives of the VR builder: error plumbing, the
// device status word, exclusive scans and a stable LSD radix sort.  All are
// written here (no CUB, no Thrust).  sm_103a, 32-wide warps.
#pragma once
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <utility>

#include "../../include/vr.h"
#include "prof.h"

namespace vr {

// ---------------------------------------------------------------- errors

void set_error(const char *fmt, ...);   // thread-local message (api.cu)
vr_status cuda_status(cudaError_t e, const char *what, const char *file, int line);

// cudaMallocAsync behind a test hook: vr_inject_alloc_failure(k) makes the
// k-th call from then on fail with cudaErrorMemoryAllocation (a host-side
// fault: nothing is allocated and nothing runs on the device).  Every device
// allocation of the library goes through it.
cudaError_t dev_malloc(void **p, size_t bytes, cudaStream_t s);

// Streaming multiprocessors of the current device (cudaDevAttrMultiProcessorCount,
// read once per device and cached; 1 if the query fails).  Grid caps and path
// thresholds are multiples of it.
int num_sms();

#define VR_TRY(x)                                                     \
  do {                                                                \
    vr_status s_ = (x);                                               \
    if (s_ != VR_OK) return s_;                                       \
  } while (0)
#define VR_CUDA(x)                                                    \
  do {                                                                \
    cudaError_t e_ = (x);                                             \
    if (e_ != cudaSuccess)                                            \
      return ::vr::cuda_status(e_, #x, __FILE__, __LINE__);           \
  } while (0)

// Flags a kernel can raise in the device status word.
enum : int32_t {
  F_NONFINITE = 1,   // non-finite float coordinate           -> VR_ERR_ARG
  F_F32_RANGE = 2,   // |float coordinate| > VR_MAX_F32_ABS   -> VR_ERR_RANGE
  F_INT_KEY = 4,     // kept integer d^2 >= 2^38              -> VR_ERR_RANGE
  F_INTERNAL = 8,    // invariant violated                    -> VR_ERR_INTERNAL
  F_TIMEOUT = 16,    // a bounded wait gave up                -> VR_ERR_TIMEOUT
  F_OVERFLOW = 32,   // an output arena was too small         -> retried by host
  F_DMAT = 64,       // distance matrix asymmetric or negative -> VR_ERR_ARG
  F_CLAIM = 128,     // claimed triangle key space ran out    -> keys regenerated by host
};

// Device-resident status and counters of one build (read back at sync points).
struct DevStatus {
  int32_t flags;
  int32_t mid_grp_count;     // float: repair groups queued for the CTA sort
  int32_t mid_seg_count;     // triangle segments queued for the large-smem CTA sort
  int32_t small_seg_count;   // triangle segments queued for the small-smem CTA sort
  int64_t E;                 // kept edges
  int64_t T;                 // triangles
  int64_t ngrades;
  int64_t near_tie;          // float: edges inside multi-edge repair groups
  uint64_t max_rel_err_bits; // float: max relative distance error (double bits)
  int64_t big_seg_max;       // largest triangle segment needing a global sort
  int64_t big_seg_count;
  int64_t big_seg_total;     // triangles inside the segments needing a global sort
  int64_t big_grp_max;       // float: largest repair group needing a global sort
  int64_t big_grp_count;
  uint64_t band_count;       // float Gram tiles: pairs left for the exact decision
  unsigned int rows_done;    // k_rows_scan: CTAs finished (the last one scans)
  int64_t wedges;            // sum over vertices of C(deg, 2): at least three times the triangle count
};

__device__ __forceinline__ void raise_flag(DevStatus *st, int32_t f) { atomicOr(&st->flags, f); }

// Flags after which the build's data can no longer be trusted: a bounded
// wait gave up (its tile's output positions, or a whole tile's output, are
// wrong) or an internal check failed.  Every kernel that consumes such data
// checks at entry (after griddepcontrol.wait, so the earlier kernels of the
// build have finished) and writes nothing: garbage indices never reach a
// load or a store.  The host reports the flag at its next status read.
constexpr int32_t F_FATAL = F_TIMEOUT | F_INTERNAL;
__device__ __forceinline__ bool build_failed(const DevStatus *st) {
  return (__ldcg(&st->flags) & F_FATAL) != 0;
}

inline vr_status flags_to_status(int32_t f) {
  if (f & F_INTERNAL) { set_error("internal invariant violated on the device"); return VR_ERR_INTERNAL; }
  if (f & F_NONFINITE) { set_error("non-finite float value"); return VR_ERR_ARG; }
  if (f & F_DMAT) { set_error("distance matrix is not symmetric or has a negative entry"); return VR_ERR_ARG; }
  if (f & F_F32_RANGE) { set_error("float coordinate magnitude above 2^50"); return VR_ERR_RANGE; }
  if (f & F_INT_KEY) { set_error("integer squared distance of a kept edge is >= 2^38"); return VR_ERR_RANGE; }
  if (f & F_TIMEOUT) { set_error("a bounded device wait timed out"); return VR_ERR_TIMEOUT; }
  return VR_OK;
}

// ------------------------------------------------------------- warp level

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}
__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

// ------------------------------------------------- dependent launches
// The build's kernels run back to back on one stream.  Each is launched with
// programmatic stream serialization and starts with pdl_entry(): it waits
// until the previous kernel has completed and its writes are visible, then
// lets the next kernel's CTAs be scheduled.  The next kernel's launch latency
// thus overlaps this kernel's run, and only one kernel ahead is ever resident
// and waiting (triggering before the wait let a chain of waiting kernels
// crowd the SMs: measured 4% slower on a 4000-point build).  A kernel
// launched the ordinary way passes pdl_entry() at once.
__device__ __forceinline__ void pdl_entry() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... P, typename... A>
inline cudaError_t launch_dep(void (*kernel)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              A &&...args) {
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<A>(args)...);
}

template <typename T>
__device__ __forceinline__ T warp_incl_scan(T v) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T u = __shfl_up_sync(0xffffffffu, v, o);
    if (lane_id() >= o) v += u;
  }
  return v;
}
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide exclusive scan of one value per thread (blockDim.x <= 1024,
// a multiple of 32).  `sh` holds >= 33 elements.  Returns the exclusive
// prefix; *total gets the block sum.
template <typename T>
__device__ T block_excl_scan(T v, T *sh, T *total) {
  const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  T inc = warp_incl_scan(v);
  if (lane_id() == 31) sh[w] = inc;
  __syncthreads();
  if (w == 0) {
    T x = lane_id() < nw ? sh[lane_id()] : T(0);
    T xi = warp_incl_scan(x);
    if (lane_id() < nw) sh[lane_id()] = xi - x;
    if (lane_id() == nw - 1) sh[32] = xi;
  }
  __syncthreads();
  T r = sh[w] + inc - v;
  if (total) *total = sh[32];
  __syncthreads();
  return r;
}

// ------------------------------------------------------------------ scans
// out[i] = sum_{j<i} in[j] for i in [0, L]; out[L] = total.  L is known on the
// host.  One launch for one chunk; two for up to SCAN_SELF_MAX chunks (chunk
// sums, then chunk scans that add up the sums before them themselves); three
// beyond (a one-CTA scan of the chunk sums in between).

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 16;
constexpr int SCAN_CHUNK = SCAN_THREADS * SCAN_ITEMS;

template <typename TI>
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_reduce(const TI *in, int64_t L, int64_t *bs) {
  pdl_entry();
  __shared__ int64_t sh[33];
  const int64_t base = (int64_t)blockIdx.x * SCAN_CHUNK;
  int64_t s = 0;
#pragma unroll  // all SCAN_ITEMS loads in flight
  for (int t = threadIdx.x; t < SCAN_CHUNK; t += SCAN_THREADS) {
    int64_t i = base + t;
    if (i < L) s += (int64_t)in[i];
  }
  int64_t tot;
  block_excl_scan<int64_t>(s, sh, &tot);
  if (threadIdx.x == 0) bs[blockIdx.x] = tot;
}

// One CTA: exclusive scan of bs[0..nb) in place, bs[nb] = total.
static __global__ void __launch_bounds__(1024) k_scan_sums(int64_t *bs, int64_t nb) {
  pdl_entry();
  __shared__ int64_t sh[33];
  int64_t carry = 0;
  for (int64_t b0 = 0; b0 < nb; b0 += 1024) {
    int64_t i = b0 + threadIdx.x;
    int64_t v = i < nb ? bs[i] : 0;
    int64_t tot;
    int64_t e = block_excl_scan<int64_t>(v, sh, &tot);
    if (i < nb) bs[i] = carry + e;
    carry += tot;
  }
  if (threadIdx.x == 0) bs[nb] = carry;
}

constexpr int64_t SCAN_SELF_MAX = 2048;

// self_off: bs holds raw chunk sums; the CTA adds up those before its chunk.
// Shared-memory slot of chunk element t: one pad word per SCAN_ITEMS so that a
// thread's run of SCAN_ITEMS consecutive elements does not sit in one bank.
__device__ __forceinline__ int scan_slot(int t) { return t + t / SCAN_ITEMS; }

template <typename TI, typename TO>
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_final(const TI *in, int64_t L, const int64_t *bs, TO *out,
                                                             int self_off) {
  pdl_entry();
  __shared__ int64_t buf[SCAN_CHUNK + SCAN_CHUNK / SCAN_ITEMS];
  __shared__ int64_t sh[33];
  __shared__ int64_t off_sh;
  const int64_t base = (int64_t)blockIdx.x * SCAN_CHUNK;
  if (self_off) {
    int64_t a = 0;
    for (int64_t q = threadIdx.x; q < (int64_t)blockIdx.x; q += SCAN_THREADS) a += bs[q];
    int64_t tot;
    block_excl_scan<int64_t>(a, sh, &tot);
    if (threadIdx.x == 0) off_sh = tot;
    __syncthreads();
  }
#pragma unroll  // all SCAN_ITEMS loads in flight
  for (int t = threadIdx.x; t < SCAN_CHUNK; t += SCAN_THREADS) {
    int64_t i = base + t;
    buf[scan_slot(t)] = i < L ? (int64_t)in[i] : 0;
  }
  __syncthreads();
  int64_t loc[SCAN_ITEMS];
  int64_t s = 0;
#pragma unroll
  for (int q = 0; q < SCAN_ITEMS; ++q) {
    loc[q] = s;
    s += buf[scan_slot(threadIdx.x * SCAN_ITEMS + q)];
  }
  __syncthreads();
  int64_t tot;
  const int64_t off = !bs ? 0 : self_off ? off_sh : bs[blockIdx.x];
  int64_t pre = block_excl_scan<int64_t>(s, sh, &tot) + off;
#pragma unroll
  for (int q = 0; q < SCAN_ITEMS; ++q) buf[scan_slot(threadIdx.x * SCAN_ITEMS + q)] = pre + loc[q];
  __syncthreads();
#pragma unroll
  for (int t = threadIdx.x; t < SCAN_CHUNK; t += SCAN_THREADS) {
    int64_t i = base + t;
    if (i < L) out[i] = (TO)buf[scan_slot(t)];
  }
  if (threadIdx.x == 0 && base + SCAN_CHUNK >= L) out[L] = (TO)(off + tot);
}

// `bs` needs scan_tmp_slots(L) slots.  out has L + 1 slots.
inline int64_t scan_tmp_slots(int64_t L) { return (L + SCAN_CHUNK - 1) / SCAN_CHUNK + 1; }

template <typename TI, typename TO>
inline vr_status scan_exclusive(const TI *in, TO *out, int64_t L, int64_t *bs, cudaStream_t s) {
  int64_t nb = (L + SCAN_CHUNK - 1) / SCAN_CHUNK;
  if (nb <= 1) {
    launch_dep(k_scan_final<TI, TO>, 1, SCAN_THREADS, 0, s, in, L, nullptr, out, 0);
    count_launch(1);
  } else if (nb <= SCAN_SELF_MAX) {
    count_launch(2);
    launch_dep(k_scan_reduce<TI>, (unsigned)nb, SCAN_THREADS, 0, s, in, L, bs);
    launch_dep(k_scan_final<TI, TO>, (unsigned)nb, SCAN_THREADS, 0, s, in, L, bs, out, 1);
  } else {
    count_launch(3);
    launch_dep(k_scan_reduce<TI>, (unsigned)nb, SCAN_THREADS, 0, s, in, L, bs);
    launch_dep(k_scan_sums, 1, 1024, 0, s, bs, nb);
    launch_dep(k_scan_final<TI, TO>, (unsigned)nb, SCAN_THREADS, 0, s, in, L, bs, out, 0);
  }
  VR_CUDA(cudaGetLastError());
  return VR_OK;
}

// ------------------------------------------------------------ radix sort
// Stable LSD radix sort of u64 keys (optional u32 payload) on bits
// [bit_lo, bit_lo + nbits), 8-bit digits.  Stability comes from ranking each
// 4096-key tile in order: a warp ranks 32 consecutive keys per round with
// __match_any_sync, warps cover consecutive 512-key slices, and the digit
// offsets of earlier warps/tiles are added.

constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_ITEMS = 16;                    // keys per lane
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;  // 4096 keys per tile
constexpr int RS_BINS = 256;

__device__ __forceinline__ uint32_t digit_of(uint64_t k, int shift, uint32_t mask) {
  return (uint32_t)(k >> shift) & mask;
}
// Mask of digit p of a sort on nbits bits: the last digit may be narrower, so
// bits above the sorted range never take part.
__host__ __device__ inline uint32_t digit_mask(int nbits, int p) {
  const int b = nbits - 8 * p;
  return b >= 8 ? 0xffu : (1u << b) - 1u;
}

// Rank the keys of one tile (positions [t0, t0 + cnt) of src).  On return
// rank[q] holds, for the lane's q-th key, its position among equal digits in
// the tile, and sh_cnt[d] the tile's count of digit d.  Keys are read by warp
// w at t0 + w*512 + q*32 + lane.
__device__ __forceinline__ void tile_rank(const uint64_t *src, int64_t t0, int64_t cnt, int shift, uint32_t mask,
                                          uint64_t (&key)[RS_ITEMS], uint32_t (&rank)[RS_ITEMS],
                                          uint32_t (*sh_wcnt)[RS_BINS], uint32_t *sh_cnt) {
  const int w = threadIdx.x >> 5, l = lane_id();
  for (int b = threadIdx.x; b < RS_WARPS * RS_BINS; b += RS_THREADS) (&sh_wcnt[0][0])[b] = 0;
  __syncthreads();
  const uint32_t lt = lanemask_lt();
  // All loads first (16 in flight per lane), then the ranking rounds.
#pragma unroll
  for (int q = 0; q < RS_ITEMS; ++q) {
    const int64_t idx = (int64_t)w * (32 * RS_ITEMS) + q * 32 + l;
    key[q] = idx < cnt ? src[t0 + idx] : ~0ull;
  }
#pragma unroll
  for (int q = 0; q < RS_ITEMS; ++q) {
    int64_t idx = (int64_t)w * (32 * RS_ITEMS) + q * 32 + l;
    bool ok = idx < cnt;
    uint32_t dg = ok ? digit_of(key[q], shift, mask) : RS_BINS;  // sentinel for empty lanes
    uint32_t peers = __match_any_sync(0xffffffffu, dg);
    uint32_t before = ok ? sh_wcnt[w][dg] : 0;
    rank[q] = before + __popc(peers & lt);
    __syncwarp();
    if (ok && (peers & lt) == 0) sh_wcnt[w][dg] = before + __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  // Exclusive prefix over warps for each digit, and tile totals.
  for (int d = threadIdx.x; d < RS_BINS; d += RS_THREADS) {
    uint32_t s = 0;
#pragma unroll
    for (int ww = 0; ww < RS_WARPS; ++ww) {
      uint32_t c = sh_wcnt[ww][d];
      sh_wcnt[ww][d] = s;
      s += c;
    }
    sh_cnt[d] = s;
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < RS_ITEMS; ++q) {
    int64_t idx = (int64_t)w * (32 * RS_ITEMS) + q * 32 + l;
    if (idx < cnt) rank[q] += sh_wcnt[w][digit_of(key[q], shift, mask)];
  }
}

// Multi-CTA sort ("onesweep" shape: one digit histogram pass over all
// digits, then one launch per digit pass).
//
// k_rs_hist_all: hist[p][d] = number of keys whose pass-p digit is d, for all
// passes in one read of the keys (shared atomics, one per key and digit).
constexpr int RS_MAX_PASSES = 8;
static __global__ void __launch_bounds__(RS_THREADS) k_rs_hist_all(const uint64_t *src, int64_t n, int bit_lo,
                                                                   int nbits, uint32_t *hist) {
  pdl_entry();
  const int passes = (nbits + 7) / 8;
  __shared__ uint32_t h[RS_MAX_PASSES][RS_BINS];
  for (int b = threadIdx.x; b < RS_MAX_PASSES * RS_BINS; b += RS_THREADS) (&h[0][0])[b] = 0;
  __syncthreads();
  // One tile per CTA and pass through the grid; a lane loads its 16 keys
  // (coalesced, all in flight) before counting them.
  for (int64_t t0 = (int64_t)blockIdx.x * RS_TILE; t0 < n; t0 += (int64_t)gridDim.x * RS_TILE) {
    uint64_t k[RS_ITEMS];
#pragma unroll
    for (int q = 0; q < RS_ITEMS; ++q) {
      const int64_t i = t0 + q * RS_THREADS + threadIdx.x;
      k[q] = i < n ? src[i] : 0;
    }
    for (int p = 0; p < passes; ++p) {
      const int shift = bit_lo + 8 * p;
      const uint32_t mask = digit_mask(nbits, p);
#pragma unroll
      for (int q = 0; q < RS_ITEMS; ++q) {
        const bool ok = t0 + q * RS_THREADS + threadIdx.x < n;
        const uint32_t dg = ok ? digit_of(k[q], shift, mask) : RS_BINS;
        if (ok) atomicAdd(&h[p][dg], 1u);
      }
    }
  }
  __syncthreads();
  for (int b = threadIdx.x; b < passes * RS_BINS; b += RS_THREADS) {
    const uint32_t v = (&h[0][0])[b];
    if (v) atomicAdd(&hist[b], v);
  }
}

// Per-(tile, digit) status word of a pass: tag in the top byte (2p + 1: the
// tile's own count is published; 2p + 2: the inclusive count over tiles
// 0..t is published; anything else: not yet), value below.  Tags are
// pass-specific, so one clearing serves every pass of a sort.
constexpr long RS_WAIT_LIMIT = 1l << 24;

// Test hook (vr_inject_lookback_stall): in one digit pass, tile `tile`
// publishes no status at all, so later tiles' look-back waits run out after
// `limit` polls.  Launched as a separate instantiation (INJ) only when armed.
struct RsStall {
  int64_t tile;
  long limit;
};
// Takes (and disarms) an armed stall for a pass of `tiles` tiles.
bool take_rs_stall(int64_t tiles, RsStall *out);
__device__ __forceinline__ void rs_publish(uint64_t *w, uint32_t tag, uint64_t v) {
  *(volatile uint64_t *)w = ((uint64_t)tag << 56) | v;
}

// Digit of key k in one pass: bits [sh, sh + 8) of the key under mask.  HI:
// the digit lies in the upper word and sh counts from bit 32; otherwise a
// funnel shift of the two words (a digit may straddle bit 32).
template <bool HI>
__device__ __forceinline__ uint32_t pass_digit(uint64_t k, int sh, uint32_t mask) {
  const uint32_t lo = (uint32_t)k, hi = (uint32_t)(k >> 32);
  return (HI ? hi >> sh : __funnelshift_r(lo, hi, sh)) & mask;
}

// One digit pass.  CTAs claim tiles in order (atomic ticket), so every
// earlier tile belongs to a CTA that is already running.  A CTA ranks its
// tile (stable: match.any peers and per-warp digit counters), publishes its
// per-digit counts, places the keys digit run by digit run in shared memory,
// adds up earlier tiles' counts by looking back until an inclusive count is
// found (bounded spin: a timeout raises F_TIMEOUT in *err), publishes its own
// inclusive counts and writes the runs out.  A ragged last tile is padded
// with all-ones keys: they take the largest digit, rank after every real key
// of it and are neither counted nor written.
// Tiles: OS_ITEMS keys per lane (4096 per tile, four CTAs per SM); sorts of
// at most OS_SMALL_N keys take OS_SMALL_ITEMS per lane (1024 per tile, eight
// CTAs per SM), so that a small sort spreads over more SMs.
constexpr int OS_ITEMS = 16;
constexpr int OS_TILE = RS_THREADS * OS_ITEMS;
constexpr int OS_SMALL_ITEMS = 4;
constexpr int OS_SMALL_TILE = RS_THREADS * OS_SMALL_ITEMS;
constexpr int64_t OS_SMALL_N = 1 << 18;
template <bool HI, int OS_ITEMS, int OS_MIN_BLOCKS, bool INJ>
__global__ void __launch_bounds__(RS_THREADS, OS_MIN_BLOCKS) k_rs_onesweep(const uint64_t *src, uint64_t *dst, int64_t n,
                                                               int sh, uint32_t mask, int pass,
                                                               const uint32_t *hist, uint64_t *status,
                                                               uint32_t *ticket, int32_t *err, RsStall stall,
                                                               uint32_t *tmask) {
  pdl_entry();
  // An earlier pass of this sort timed out: its output is not a permutation
  // of the keys, so this pass's digit counts would not match the histogram
  // (positions could leave the array).  Write nothing.  (A timeout in this
  // same pass only sets bit `pass`, so sibling tiles never skip.)
  if (pass > 0 && (*(volatile uint32_t *)tmask & ((1u << pass) - 1u))) return;
  __shared__ uint32_t wcnt[RS_WARPS][RS_BINS];  // per-warp digit counts, then each warp's run starts
  __shared__ int64_t gofs[RS_BINS];             // global position of a run's slot 0 in skey
  constexpr int OS_TILE = RS_THREADS * OS_ITEMS;
  __shared__ uint64_t skey[OS_TILE];
  __shared__ uint64_t scan_sh[33];
  __shared__ int64_t tile_sh;
  const int w = threadIdx.x >> 5, l = lane_id();
  for (int i = threadIdx.x; i < RS_WARPS * RS_BINS; i += RS_THREADS) (&wcnt[0][0])[i] = 0;
  if (threadIdx.x == 0) tile_sh = atomicAdd(ticket, 1u);
  __syncthreads();
  const int64_t t = tile_sh;
  const int64_t t0 = t * OS_TILE;
  const int c = n - t0 < OS_TILE ? (int)(n - t0) : OS_TILE;

  // Rank: lane l of warp w holds keys w*32*OS_ITEMS + q*32 + l of the tile.
  uint64_t key[OS_ITEMS];
  uint32_t pk[OS_ITEMS];  // rank among the warp's keys of the digit | digit << 16
  {
    const uint64_t *p = src + t0 + w * (32 * OS_ITEMS) + l;
    const int lim = c - (w * (32 * OS_ITEMS) + l);
#pragma unroll
    for (int q = 0; q < OS_ITEMS; ++q) key[q] = q * 32 < lim ? p[q * 32] : ~0ull;
    const uint32_t lt = lanemask_lt();
    uint32_t *wc = wcnt[w];
#pragma unroll
    for (int q = 0; q < OS_ITEMS; ++q) {
      const uint32_t dg = pass_digit<HI>(key[q], sh, mask);
      const uint32_t peers = __match_any_sync(0xffffffffu, dg);
      const uint32_t below = peers & lt;
      const uint32_t before = wc[dg];
      pk[q] = (before + __popc(below)) | (dg << 16);
      __syncwarp();
      if (below == 0) wc[dg] = before + __popc(peers);
      __syncwarp();
    }
  }
  __syncthreads();

  // Per digit b (one per thread): the tile's count, published at once; the
  // tile-local start of each warp's run of b.
  const int b = threadIdx.x;  // RS_THREADS == RS_BINS
  uint32_t v = 0;
#pragma unroll
  for (int ww = 0; ww < RS_WARPS; ++ww) v += wcnt[ww][b];
  if (b == (int)mask) v -= OS_TILE - c;  // the padding
  const uint32_t tag_agg = 2 * pass + 1, tag_inc = 2 * pass + 2;
  uint64_t *my = status + t * RS_BINS + b;
  const bool withhold = INJ && t == stall.tile;  // test hook: this tile never publishes
  const long wait_limit = INJ ? stall.limit : RS_WAIT_LIMIT;
  if (!withhold) rs_publish(my, t == 0 ? tag_inc : tag_agg, v);
  // One scan for both starts: the digit's start over all keys (from the
  // histogram) in the high bits, its start inside the tile in the low 16.
  const uint64_t both = block_excl_scan<uint64_t>(((uint64_t)hist[b] << 16) | v, scan_sh, (uint64_t *)nullptr);
  const uint32_t lp = (uint32_t)(both & 0xffffu);
  {
    uint32_t run = lp;
#pragma unroll
    for (int ww = 0; ww < RS_WARPS; ++ww) {
      const uint32_t x = wcnt[ww][b];
      wcnt[ww][b] = run;
      run += x;
    }
  }
  __syncthreads();
  {
    const uint32_t *wc = wcnt[w];
#pragma unroll
    for (int q = 0; q < OS_ITEMS; ++q) skey[wc[pk[q] >> 16] + (pk[q] & 0xffffu)] = key[q];
  }

  // Look back in windows of LB_WIN predecessors (loads issued together),
  // consumed in order until an inclusive count; a word not yet published
  // restarts the window there.
  uint64_t excl = 0;
  if (t > 0) {
    constexpr int LB_WIN = 4;
    const uint64_t *pk0 = my - RS_BINS;  // tile t - 1
    int64_t k = t - 1;
    long spins = 0;
    bool done = false;
    while (!done && k >= 0) {
      uint64_t wv[LB_WIN];
#pragma unroll
      for (int q = 0; q < LB_WIN; ++q)
        wv[q] = q <= k ? *(volatile const uint64_t *)(pk0 - q * RS_BINS) : 0;
      int used = 0;
#pragma unroll
      for (int q = 0; q < LB_WIN; ++q) {
        if (done || used != q || q > k) continue;
        const uint32_t tag = (uint32_t)(wv[q] >> 56);
        if (tag == tag_inc || tag == tag_agg) {
          excl += wv[q] & ((1ull << 56) - 1);
          ++used;
          if (tag == tag_inc) done = true;
        }
      }
      k -= used;
      pk0 -= used * RS_BINS;
      if (!done && used == 0) {
        if (++spins > wait_limit) {
          // Gave up: excl holds only some earlier tiles' counts, so every
          // position below stays inside the digit's range (in bounds, but
          // the result is wrong and the flag reports it).
          atomicOr(err, F_TIMEOUT);
          atomicOr(tmask, 1u << pass);
          break;
        }
        __nanosleep(64);  // yield issue slots to the warps still ranking
      }
    }
    if (!withhold) rs_publish(my, tag_inc, excl + v);
  }
  gofs[b] = (int64_t)(both >> 16) + (int64_t)excl - (int64_t)lp;
  __syncthreads();
  uint64_t *out = dst;
  for (int i = threadIdx.x; i < c; i += RS_THREADS) {
    const uint64_t k = skey[i];
    out[gofs[pass_digit<HI>(k, sh, mask)] + i] = k;
  }
}

// One CTA sorts [0, n) of global arrays in place through tkeys/tvals (any n):
// each pass histograms everything, then ranks tile after tile in order with a
// running digit base.  Used for small sorts and for per-segment fix-ups.
static __device__ void cta_radix_sort_global(uint64_t *keys, uint32_t *vals, uint64_t *tkeys, uint32_t *tvals, int64_t n,
                                      int bit_lo, int nbits) {
  __shared__ uint32_t wcnt[RS_WARPS][RS_BINS];
  __shared__ uint32_t cnt[RS_BINS];
  __shared__ int64_t base[RS_BINS];
  __shared__ int64_t sh[33];
  uint64_t *src = keys, *dst = tkeys;
  uint32_t *vs = vals, *vd = tvals;
  const int passes = (nbits + 7) / 8;
  for (int p = 0; p < passes; ++p) {
    const int shift = bit_lo + 8 * p;
    const uint32_t mask = digit_mask(nbits, p);
    for (int b = threadIdx.x; b < RS_BINS; b += RS_THREADS) cnt[b] = 0;
    __syncthreads();
    // Eight loads in flight per thread before their counts (one dependent
    // L2 round trip per key otherwise bounds small sorts).
    for (int64_t i0 = 0; i0 < n; i0 += 8 * RS_THREADS) {
      uint64_t k[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int64_t i = i0 + u * RS_THREADS + threadIdx.x;
        k[u] = i < n ? src[i] : 0ull;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (i0 + u * RS_THREADS + threadIdx.x < n) atomicAdd(&cnt[digit_of(k[u], shift, mask)], 1u);
    }
    __syncthreads();
    {
      int64_t v = threadIdx.x < RS_BINS ? (int64_t)cnt[threadIdx.x] : 0;
      int64_t e = block_excl_scan<int64_t>(v, sh, (int64_t *)nullptr);
      if (threadIdx.x < RS_BINS) base[threadIdx.x] = e;
      __syncthreads();
    }
    for (int64_t t0 = 0; t0 < n; t0 += RS_TILE) {
      int64_t c = n - t0 < RS_TILE ? n - t0 : RS_TILE;
      uint64_t key[RS_ITEMS];
      uint32_t rank[RS_ITEMS];
      tile_rank(src, t0, c, shift, mask, key, rank, wcnt, cnt);
      const int w = threadIdx.x >> 5, l = lane_id();
      uint32_t val[RS_ITEMS];
#pragma unroll
      for (int q = 0; q < RS_ITEMS; ++q) {
        const int64_t idx = (int64_t)w * (32 * RS_ITEMS) + q * 32 + l;
        val[q] = vs && idx < c ? vs[t0 + idx] : 0u;
      }
#pragma unroll
      for (int q = 0; q < RS_ITEMS; ++q) {
        int64_t idx = (int64_t)w * (32 * RS_ITEMS) + q * 32 + l;
        if (idx < c) {
          int64_t pos = base[digit_of(key[q], shift, mask)] + rank[q];
          dst[pos] = key[q];
          if (vs) vd[pos] = val[q];
        }
      }
      __syncthreads();
      for (int b = threadIdx.x; b < RS_BINS; b += RS_THREADS) base[b] += cnt[b];
      __syncthreads();
    }
    uint64_t *tk = src; src = dst; dst = tk;
    uint32_t *tv = vs; vs = vd; vd = tv;
    __syncthreads();
  }
  if (passes & 1) {  // result sits in the temporaries: copy back, eight loads in flight per thread
    for (int64_t i0 = 0; i0 < n; i0 += 8 * RS_THREADS) {
      uint64_t k[8];
      uint32_t v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int64_t i = i0 + u * RS_THREADS + threadIdx.x;
        k[u] = i < n ? tkeys[i] : 0ull;
        v[u] = vals && i < n ? tvals[i] : 0u;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int64_t i = i0 + u * RS_THREADS + threadIdx.x;
        if (i < n) {
          keys[i] = k[u];
          if (vals) vals[i] = v[u];
        }
      }
    }
    __syncthreads();
  }
}

static __global__ void __launch_bounds__(RS_THREADS) k_rs_single(uint64_t *keys, uint32_t *vals, uint64_t *tkeys,
                                                          uint32_t *tvals, int64_t n, int bit_lo, int nbits) {
  pdl_entry();
  cta_radix_sort_global(keys, vals, tkeys, tvals, n, bit_lo, nbits);
}

// All-digit histogram of the keys a kernel writes, counted per CTA in shared
// memory and added to the sort's global histogram at the
// end, so that radix_sort(..., RS_PREP_HIST) needs no histogram pass.  g null:
// off (a kernel parameter, so uniform over the block).
struct KeyHist {
  uint32_t *g;
  int bit_lo, nbits;
};
using KeyHistSmem = uint32_t[RS_MAX_PASSES][RS_BINS];

__device__ __forceinline__ void khist_init(KeyHistSmem &h, const KeyHist &kh) {
  if (!kh.g) return;
  for (int b = threadIdx.x; b < RS_MAX_PASSES * RS_BINS; b += blockDim.x) (&h[0][0])[b] = 0;
  __syncthreads();
}

// Any subset of the block's threads may call it.
__device__ __forceinline__ void khist_add(KeyHistSmem &h, const KeyHist &kh, uint64_t key, bool valid) {
  if (!kh.g) return;
  if (!valid) return;
  const int passes = (kh.nbits + 7) / 8;
  for (int p = 0; p < passes; ++p) atomicAdd(&h[p][digit_of(key, kh.bit_lo + 8 * p, digit_mask(kh.nbits, p))], 1u);
}

// Called by every thread of the block after its last khist_add.
__device__ __forceinline__ void khist_flush(KeyHistSmem &h, const KeyHist &kh) {
  if (!kh.g) return;
  __syncthreads();
  const int n = ((kh.nbits + 7) / 8) * RS_BINS;
  for (int b = threadIdx.x; b < n; b += blockDim.x) {
    const uint32_t v = (&h[0][0])[b];
    if (v) atomicAdd(&kh.g[b], v);
  }
}

// Decoupled look-back over tiles taken in ticket order: returns the sum of
// the totals of every earlier tile.  status: one zeroed word per tile (flag
// in the top two bits: 1 = the tile's own total, 2 = the inclusive total;
// value below).  Every earlier tile's CTA is already running (ticket order),
// so the wait ends; it is bounded anyway (F_TIMEOUT in *err).
constexpr uint64_t LB_AGG = 1ull << 62, LB_INC = 2ull << 62, LB_VAL = (1ull << 62) - 1;
// Called by a whole warp (the same tile and total in every lane): lane l
// reads the status of tile k - l, so each step covers 32 earlier tiles; the
// nearest tile that has published its inclusive count ends the walk.  A
// step waits (bounded) only while a tile before that one has published
// nothing.  Returns the exclusive prefix in every lane.
__device__ __forceinline__ int64_t tile_lookback(uint64_t *status, int64_t tile, int64_t total, int32_t *err) {
  const int l = lane_id();
  if (tile == 0) {
    if (l == 0) *(volatile uint64_t *)&status[0] = LB_INC | (uint64_t)total;
    return 0;
  }
  if (l == 0) *(volatile uint64_t *)&status[tile] = LB_AGG | (uint64_t)total;
  int64_t excl = 0, k = tile - 1;
  long spins = 0;
  for (;;) {
    const int64_t idx = k - l;
    const uint64_t w = idx >= 0 ? *(volatile const uint64_t *)&status[idx] : LB_INC;  // before tile 0: inclusive 0
    const uint32_t inc = __ballot_sync(0xffffffffu, (w & LB_INC) != 0);
    const uint32_t unset = __ballot_sync(0xffffffffu, (w & (LB_AGG | LB_INC)) == 0);
    // Lanes up to the nearest inclusive one (all lanes if none).
    const uint32_t upto = inc ? (2u << (__ffs(inc) - 1)) - 1u : 0xffffffffu;
    if (unset & upto) {
      if (++spins > RS_WAIT_LIMIT) {
        if (l == 0) atomicOr(err, F_TIMEOUT);
        break;
      }
      __nanosleep(32);
      continue;
    }
    int64_t v = ((upto >> l) & 1u) ? (int64_t)(w & LB_VAL) : 0;
#pragma unroll
    for (int d = 16; d; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
    excl += v;
    if (inc) break;
    k -= 32;
  }
  if (l == 0) *(volatile uint64_t *)&status[tile] = LB_INC | (uint64_t)(excl + total);
  return excl;
}

// Scratch for radix_sort: a temporary of n keys and rs_meta_bytes(n) bytes
// (all-digit histogram, tile tickets, per-tile status words).  The sorted
// result ends in `keys`.  `err`: device flags word for a timed-out wait.
struct RadixScratch {
  uint64_t *tkeys;
  uint8_t *meta;
  int32_t *err;
};
inline int64_t rs_tiles(int64_t n) {  // tiles of a digit pass over n keys
  return n <= OS_SMALL_N ? (n + OS_SMALL_TILE - 1) / OS_SMALL_TILE : (n + OS_TILE - 1) / OS_TILE;
}
// Head of the scratch: the all-digit histogram, then 256 bytes holding the
// passes' tile tickets (word p) and the timed-out-pass mask (word
// RS_TMASK_WORD); the per-(tile, digit) status words follow.
constexpr int64_t RS_META_HEAD = RS_MAX_PASSES * RS_BINS * 4 + 256;
constexpr int RS_TMASK_WORD = 32;
static_assert(RS_MAX_PASSES <= RS_TMASK_WORD && (RS_TMASK_WORD + 1) * 4 <= 256, "sort scratch head layout");
// Room for the status words of a sort of any m <= n keys, whichever tile size
// m takes (callers size the scratch from an upper bound on the key count).
inline int64_t rs_meta_bytes(int64_t n) {
  const int64_t small = ((n < OS_SMALL_N ? n : OS_SMALL_N) + OS_SMALL_TILE - 1) / OS_SMALL_TILE;
  return RS_META_HEAD + (small + (n + OS_TILE - 1) / OS_TILE) * RS_BINS * 8;
}

// Clear the sort's scratch (unless `zeroed`: the caller cleared at least
// rs_meta_bytes(n) bytes of it) and return the histogram for a key generator
// to fill (KeyHist with g null when the sort will not use it: one-CTA sizes).
inline vr_status radix_prepare(int64_t n, int bit_lo, int nbits, const RadixScratch &sc, cudaStream_t s,
                               KeyHist *kh, bool zeroed = false) {
  *kh = KeyHist{nullptr, bit_lo, nbits};
  if (n <= 2 * RS_TILE || nbits <= 0) return VR_OK;
  if (!zeroed) VR_CUDA(cudaMemsetAsync(sc.meta, 0, (size_t)rs_meta_bytes(n), s));
  kh->g = (uint32_t *)sc.meta;
  return VR_OK;
}

// What the caller did to the scratch before radix_sort: nothing; cleared
// rs_meta_bytes(n) bytes of it; or radix_prepare plus a generator that filled
// the histogram.
enum RsPrep { RS_PREP_NONE, RS_PREP_ZEROED, RS_PREP_HIST };

// `prof`/`tag`: optional per-kernel timing ("<tag>.hist", ".pass").
// `sorted`: if given, receives the buffer holding the result (keys or
// sc.tkeys) and an odd pass count costs no copy back into keys.
inline vr_status radix_sort(uint64_t *keys, int64_t n, int bit_lo, int nbits, const RadixScratch &sc,
                            cudaStream_t s, Prof *prof = nullptr, const char *const *tag = nullptr,
                            RsPrep prep = RS_PREP_NONE, uint64_t **sorted = nullptr) {
  if (sorted) *sorted = keys;
  if (n <= 1 || nbits <= 0) return VR_OK;
  if (n <= 2 * RS_TILE) {
    launch_dep(k_rs_single, 1, RS_THREADS, 0, s, keys, nullptr, sc.tkeys, nullptr, n, bit_lo, nbits);
    count_launch(1);
    VR_CUDA(cudaGetLastError());
    return VR_OK;
  }
  const int64_t nt = rs_tiles(n);
  const int passes = (nbits + 7) / 8;
  uint32_t *hist = (uint32_t *)sc.meta;
  uint32_t *ticket = (uint32_t *)(sc.meta + RS_MAX_PASSES * RS_BINS * 4);
  uint32_t *tmask = ticket + RS_TMASK_WORD;  // passes that timed out (bit per pass)
  uint64_t *status = (uint64_t *)(sc.meta + RS_META_HEAD);
  int tk_ = -1;
  if (prep != RS_PREP_HIST) {
    tk_ = prof ? prof->begin(tag[0]) : -1;
    if (prep == RS_PREP_NONE) VR_CUDA(cudaMemsetAsync(sc.meta, 0, (size_t)rs_meta_bytes(n), s));
    const int64_t hcap = (int64_t)num_sms() * 8;
    const unsigned hg = (unsigned)(nt < hcap ? nt : hcap);
    launch_dep(k_rs_hist_all, hg, RS_THREADS, 0, s, keys, n, bit_lo, nbits, hist);
    count_launch(1);
    if (prof) prof->end(tk_);
  }
  uint64_t *src = keys, *dst = sc.tkeys;
  for (int p = 0; p < passes; ++p) {
    tk_ = prof ? prof->begin(tag[1]) : -1;
    const int sh = bit_lo + 8 * p;
    const uint32_t dm = digit_mask(nbits, p);
    RsStall stall{-1, RS_WAIT_LIMIT};
    const bool inj = take_rs_stall(nt, &stall);
    const int shp = sh >= 32 ? sh - 32 : sh;
#define VR_ONESWEEP(HI, IT, MB)                                                                                   \
  (inj ? launch_dep(k_rs_onesweep<HI, IT, MB, true>, (unsigned)nt, RS_THREADS, 0, s, src, dst, n, shp, dm, p,       \
                    hist + p * RS_BINS, status, ticket + p, sc.err, stall, tmask)                                   \
       : launch_dep(k_rs_onesweep<HI, IT, MB, false>, (unsigned)nt, RS_THREADS, 0, s, src, dst, n, shp, dm, p,      \
                    hist + p * RS_BINS, status, ticket + p, sc.err, stall, tmask))
    if (n <= OS_SMALL_N) {
      if (sh >= 32) VR_ONESWEEP(true, OS_SMALL_ITEMS, 8);
      else VR_ONESWEEP(false, OS_SMALL_ITEMS, 8);
    } else {
      if (sh >= 32) VR_ONESWEEP(true, OS_ITEMS, 4);
      else VR_ONESWEEP(false, OS_ITEMS, 4);
    }
#undef VR_ONESWEEP
    count_launch(1);
    if (prof) prof->end(tk_);
    VR_CUDA(cudaGetLastError());
    uint64_t *tk = src; src = dst; dst = tk;
  }
  if (sorted) *sorted = src;
  else if (passes & 1) VR_CUDA(cudaMemcpyAsync(keys, src, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, s));
  return VR_OK;
}

// ------------------------------------------------------- bitonic (smem)
// Sort cap (a power of two) pairs (key, val) ascending in shared memory; keys
// unique, slots past the live count already hold ~0 keys.
static __device__ void cta_bitonic(uint64_t *key, uint32_t *val, int cap) {
  for (int k = 2; k <= cap; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < cap; i += blockDim.x) {
        int x = i ^ j;
        if (x > i) {
          bool up = (i & k) == 0;
          uint64_t a = key[i], b = key[x];
          if ((a > b) == up) {
            key[i] = b; key[x] = a;
            uint32_t t = val[i]; val[i] = val[x]; val[x] = t;
          }
        }
      }
      __syncthreads();
    }
  }
}

}  // namespace vr
