// kernels.cuh -- device steps of the Vietoris-Rips build (arXiv 1809.04424,
// Sec. 2.1 construction; Sec. 3 / Sec. 4.4 ranking; Sec. 2.2 boundary).
//
// Layout in HBM for one cloud of n points (W = ceil(n/32) words per row):
//   X       n*d int32 (integer inputs) or float (float inputs), row-major
//   adj     n*W u32   kept-edge adjacency bitmap, symmetric, no diagonal
//   adjpre  n*W i32   exclusive prefix popcount of each row's words, so the
//                     rank of neighbour j in row i is adjpre + popc(word & below)
//   nbr_ptr n+1 i32   row starts of the neighbour CSR (neighbours ascending)
//   nbr_ord 2E  i32   order index of the edge behind each neighbour entry
//   keys    E   u64   (d2 key << 26) | i << 13 | j, i < j
// Every step is one kernel; the host only learns sizes at two sync points.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "prims.cuh"

namespace vr {

constexpr int ID_BITS = 13;
constexpr uint64_t ID_MASK = (1ull << ID_BITS) - 1;
constexpr int KEY_SHIFT = 2 * ID_BITS;  // d2 part of an edge key starts at bit 26
constexpr uint64_t INT_KEY_LIMIT = 1ull << 38;

// Parameters of the cap shared by the distance kernels.
struct Cap {
  int keep_all;     // maxrad = +inf
  uint64_t r2i;     // integer inputs: floor(fl(maxrad^2)) clamped to u64
  double r2;        // float inputs: fl(maxrad^2)
  double crel;      // float inputs: relative bound of the fp32 first pass
  float a_keep;     // float inputs: fp32 value at or below which a pair is certainly kept
  float a_drop;     // float inputs: fp32 value at or above which a pair is certainly dropped
  float r2f_dn;     // float inputs: largest float <= r2
  float r2f_up;     // float inputs: smallest float >= r2
};

// Absolute slack of the fp32 bound: covers underflow of tiny squares.
constexpr double F32_ABS_SLACK = 7.888609052210118e-31;  // 2^-100

// --------------------------------------------------------------- distances

// Exact integer squared distance, saturating at 2^64-1.  |x_i - x_j| < 2^32
// for int32 inputs, so every square fits in u64.
__device__ __forceinline__ uint64_t d2_int(const int32_t *xi, const int32_t *xj, int d) {
  uint64_t acc = 0;
  for (int k = 0; k < d; ++k) {
    int64_t t = (int64_t)xi[k] - (int64_t)xj[k];
    uint64_t m = (uint64_t)(t < 0 ? -t : t);
    uint64_t s = acc + m * m;
    acc = s < acc ? ~0ull : s;
  }
  return acc;
}

// fp32 first pass: acc = fma(t, t, acc) over coordinates in order, t = fl32
// difference.  The same sequence everywhere, so every kernel that evaluates a
// pair gets the same bits (the value is symmetric in i, j: t only flips sign).
__device__ __forceinline__ float d2_f32(const float *xi, const float *xj, int d) {
  float acc = 0.f;
  for (int k = 0; k < d; ++k) {
    float t = __fsub_rn(xi[k], xj[k]);
    acc = __fmaf_rn(t, t, acc);
  }
  return acc;
}

// Canonical FP64 squared distance: acc = 0; t = fl(x_ik - x_jk);
// acc = fl(acc + fl(t*t)) in coordinate order, each operation rounded to
// nearest, nothing fused.  This is the value float inputs are ranked by.
__device__ __forceinline__ double d2_f64(const float *xi, const float *xj, int d) {
  double acc = 0.0;
  for (int k = 0; k < d; ++k) {
    double t = __dsub_rn((double)xi[k], (double)xj[k]);
    acc = __dadd_rn(acc, __dmul_rn(t, t));
  }
  return acc;
}

// The same canonical value without FP64 instructions (B300 runs FP64 at a
// small fraction of its integer rate).  A positive double is held as (M, E)
// with M in [2^52, 2^53) and value M * 2^E; zero as M = 0.  Per coordinate:
//   t = x - y is exact as an integer D * 2^emin when the fp32 exponents are
//       within 29 of each other (|D| < 2^53), the case handled here;
//   s = RN(t*t): D^2 is exact in 128 bits, rounded to 53 bits, ties to even;
//   acc = RN(acc + s): both positive, aligned in 64 bits with 10 guard bits
//       and a sticky bit, at most one carry, rounded to 53 bits, ties to even.
// IEEE 754 round-to-nearest-even makes each step's result unique, so this
// equals the hardware sequence bit for bit.  Returns false (caller falls back
// to d2_f64) when some coordinate pair is outside the exact case.
__device__ __forceinline__ void f32_decode(float v, int64_t &mant, int &ex) {
  const uint32_t b = __float_as_uint(v);
  const int be = (int)((b >> 23) & 0xff);
  const int64_t m = (int64_t)(b & 0x7fffff);
  if (be == 0) { mant = m; ex = -149; }                 // zero or subnormal
  else { mant = m | 0x800000; ex = be - 150; }
  if (b >> 31) mant = -mant;
}

__device__ __forceinline__ void soft_round_u128(unsigned __int128 p, int e0, uint64_t &M, int &E) {
  // p * 2^e0 rounded to a 53-bit significand (p > 0).
  const uint64_t hi = (uint64_t)(p >> 64), lo = (uint64_t)p;
  const int L = hi ? 128 - __clzll(hi) : 64 - __clzll(lo);
  if (L <= 53) {
    M = lo << (53 - L);
    E = e0 - (53 - L);
    return;
  }
  const int sh = L - 53;
  uint64_t m = (uint64_t)(p >> sh);
  const unsigned __int128 rem = p & ((((unsigned __int128)1) << sh) - 1);
  const unsigned __int128 half = ((unsigned __int128)1) << (sh - 1);
  if (rem > half || (rem == half && (m & 1))) ++m;
  int e = e0 + sh;
  if (m == (1ull << 53)) { m >>= 1; ++e; }
  M = m;
  E = e;
}

__device__ __forceinline__ void soft_add(uint64_t &Ma, int &Ea, uint64_t Ms, int Es) {
  if (Ms == 0) return;
  if (Ma == 0) { Ma = Ms; Ea = Es; return; }
  uint64_t big = Ma, sm = Ms;
  int Eb = Ea, diff = Ea - Es;
  if (diff < 0) { big = Ms; sm = Ma; Eb = Es; diff = -diff; }
  const uint64_t b10 = big << 10;
  uint64_t s10 = sm << 10;
  if (diff >= 64) s10 = 1;                                // all of it is sticky
  else if (diff > 0) s10 = (s10 >> diff) | ((s10 & ((1ull << diff) - 1)) != 0);
  uint64_t sum = b10 + s10;
  if (sum >> 63) { sum = (sum >> 1) | (sum & 1); ++Eb; }
  uint64_t m = sum >> 10;
  const uint64_t rem = sum & 0x3ff;
  if (rem > 0x200 || (rem == 0x200 && (m & 1))) ++m;
  if (m == (1ull << 53)) { m >>= 1; ++Eb; }
  Ma = m;
  Ea = Eb;
}

__device__ __forceinline__ bool d2_f64_soft(const float *xi, const float *xj, int d, double &out) {
  uint64_t M = 0;
  int E = 0;
  for (int k = 0; k < d; ++k) {
    int64_t a, b;
    int ea, eb;
    f32_decode(xi[k], a, ea);
    f32_decode(xj[k], b, eb);
    int64_t D;
    int emin;
    if (a == 0 || b == 0) {                                // t = x or -y exactly
      D = a ? a : -b;
      emin = a ? ea : eb;
    } else {
      emin = min(ea, eb);
      const int da = ea - emin, db = eb - emin;
      if (da > 29 || db > 29) return false;               // t might round: not the exact case
      D = (a << da) - (b << db);                          // |D| < 2^54
    }
    const uint64_t ad = (uint64_t)(D < 0 ? -D : D);
    if (ad >> 53) return false;
    if (ad == 0) continue;
    uint64_t Ms;
    int Es;
    soft_round_u128((unsigned __int128)ad * ad, 2 * emin, Ms, Es);
    soft_add(M, E, Ms, Es);
  }
  if (M == 0) { out = 0.0; return true; }
  const uint64_t bits = ((uint64_t)(E + 52 + 1023) << 52) | (M & ((1ull << 52) - 1));
  out = __longlong_as_double((long long)bits);
  return true;
}

__device__ __forceinline__ double d2_canonical(const float *xi, const float *xj, int d) {
  double v;
  if (d2_f64_soft(xi, xj, d, v)) return v;
  return d2_f64(xi, xj, d);
}

// Bounds of the canonical value from the fp32 first pass A:
//   |A - D| <= ((d+2) u32 + O(u^2)) D + underflow, |F - D| <= (d+2) u64 D
// (D exact, F canonical FP64), so |A - F| <= crel * A + 2^-100 with
// crel = (d + 5) * 2^-24 (slack for the second-order terms).
__device__ __forceinline__ double f32_lo(float a, double crel) { return (double)a * (1.0 - crel) - F32_ABS_SLACK; }
__device__ __forceinline__ double f32_hi(float a, double crel) { return (double)a * (1.0 + crel) + F32_ABS_SLACK; }

// ------------------------------------------------------------------ stage

template <typename TIn, bool F>
__global__ void k_stage(const TIn *in, int64_t count, typename std::conditional<F, float, int32_t>::type *X,
                        DevStatus *st) {
  pdl_entry();
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < count; t += (int64_t)gridDim.x * blockDim.x) {
    if constexpr (F) {
      float v = (float)in[t];
      if (!isfinite(v)) raise_flag(st, F_NONFINITE);
      else if (fabsf(v) > (float)VR_MAX_F32_ABS) raise_flag(st, F_F32_RANGE);
      X[t] = v;
    } else {
      X[t] = (int32_t)in[t];
    }
  }
}

// ------------------------------------------------------- distance + bitmap
// One warp per 32x32 block (bi <= bj) of the pair matrix.  Lane l owns column
// j = 32*bj + l and walks the 32 rows i of the block; __ballot_sync of the
// keep test gives row i's bitmap word directly (the ballot/popc idea of the
// paper's init_supp kernel, Sec. 4.3), and each lane accumulates its own
// column word for the mirrored block, so both halves are written without
// atomics.  grid = (B, ceil(B/8)), 8 warps per CTA.

// STAGE8 (int8 input, d <= 4): Xv is the raw int8 input, converted as it is
// loaded, and the warps of the diagonal blocks also write the staged int32
// copy Xout (each row once) that the edge-key kernel reads: no staging launch.
template <bool F, int DR, bool STAGE8 = false>
__global__ void __launch_bounds__(256) k_dist_bitmap(const void *Xv, int n, int d, int W, Cap cap, uint32_t *adj,
                                                     DevStatus *st, int32_t *Xout = nullptr) {
  pdl_entry();
  using T = typename std::conditional<F, float, int32_t>::type;
  static_assert(!STAGE8 || (!F && DR > 0 && DR <= 4), "fused staging: int8 input, d <= 4");
  const T *X = (const T *)Xv;
  auto ld = [&](int64_t idx) -> T {
    if constexpr (STAGE8) return (T)((const int8_t *)Xv)[idx];
    else return X[idx];
  };
  const int bj = blockIdx.x;
  const int bi = blockIdx.y * 8 + (threadIdx.x >> 5);
  const int l = lane_id();
  if (bi > bj) return;
  const int j = bj * 32 + l;
  const bool jv = j < n;
  T xj[DR > 0 ? DR : 1];
  if constexpr (DR > 0) {
#pragma unroll
    for (int k = 0; k < DR; ++k) xj[k] = (jv && k < d) ? ld((int64_t)j * d + k) : T(0);
  }
  const T *pj = X + (int64_t)(jv ? j : 0) * d;
  uint32_t myrow = 0, mycol = 0;
  bool key_overflow = false;
  const int rows = min(32, n - bi * 32);
  // d <= 4: lane r holds row point bi*32 + r, broadcast by shuffles (all the
  // block's loads issued up front instead of one row at a time).
  constexpr bool SHFL = DR > 0 && DR <= 4;
  T xr[DR > 0 ? DR : 1];
  if constexpr (SHFL) {
    const int ir = bi * 32 + l;
#pragma unroll
    for (int k = 0; k < DR; ++k) xr[k] = (ir < n && k < d) ? ld((int64_t)ir * d + k) : T(0);
    if constexpr (STAGE8) {
      if (bi == bj && ir < n) {
#pragma unroll
        for (int k = 0; k < DR; ++k)
          if (k < d) Xout[(int64_t)ir * d + k] = (int32_t)xr[k];
      }
    }
  }
  for (int r = 0; r < rows; ++r) {
    const int i = bi * 32 + r;
    const T *pi = X + (int64_t)i * d;
    T xi[DR > 0 ? DR : 1];
    if constexpr (SHFL) {
#pragma unroll
      for (int k = 0; k < DR; ++k) xi[k] = __shfl_sync(0xffffffffu, xr[k], r);
    }
    bool kept = false;
    if (jv && j != i) {
      if constexpr (F) {
        float a;
        if constexpr (DR > 0) {
          a = 0.f;
#pragma unroll
          for (int k = 0; k < DR; ++k)
            if (k < d) {
              float t = __fsub_rn(SHFL ? xi[k] : pi[k], xj[k]);
              a = __fmaf_rn(t, t, a);
            }
        } else {
          a = d2_f32(pi, pj, d);
        }
        if (cap.keep_all || a <= cap.a_keep) kept = true;
        else if (a >= cap.a_drop) kept = false;
        else kept = d2_canonical(pi, pj, d) <= cap.r2;  // near the cap: decide exactly
      } else {
        uint64_t v;
        if constexpr (DR > 0) {
          v = 0;
#pragma unroll
          for (int k = 0; k < DR; ++k)
            if (k < d) {
              int64_t t = (int64_t)(SHFL ? xi[k] : pi[k]) - (int64_t)xj[k];
              uint64_t m = (uint64_t)(t < 0 ? -t : t);
              uint64_t s = v + m * m;
              v = s < v ? ~0ull : s;
            }
        } else {
          v = d2_int(pi, pj, d);
        }
        kept = cap.keep_all || v <= cap.r2i;
        if (kept && v >= INT_KEY_LIMIT) key_overflow = true;
      }
    }
    uint32_t word = __ballot_sync(0xffffffffu, kept);
    if (l == r) myrow = word;
    mycol |= (uint32_t)kept << r;
  }
  if (key_overflow) raise_flag(st, F_INT_KEY);
  const int i = bi * 32 + l;
  if (i < n) adj[(int64_t)i * W + bj] = myrow;
  if (bi < bj && jv) adj[(int64_t)j * W + bi] = mycol;
}

// ------------------------------------------------------------- row counts
// One warp per row: degree, number of neighbours above the row id, and the
// exclusive prefix popcount of the row's words.
// Row counts and both scans in one launch: every CTA does its rows; the last CTA
// to finish (ticket after a fence; no CTA waits for another) scans deg and up
// (n <= 8192) into nbr_ptr and lex_ptr and stores the edge count in st->E.
// adjx (optional): each row word beside its prefix count, {word, prefix},
// so that one 8-byte load gives a neighbour's rank (the max-edge final write).
static __global__ void __launch_bounds__(256) k_rows_scan(const uint32_t *adj, int n, int W, int32_t *adjpre,
                                                          int32_t *deg, int32_t *up, int32_t *nbr_ptr,
                                                          int64_t *lex_ptr, DevStatus *st, int2 *adjx) {
  pdl_entry();
  if (build_failed(st)) return;
  __shared__ int64_t sh[33];
  __shared__ unsigned int ticket;
  const int i = blockIdx.x * 8 + (threadIdx.x >> 5);
  const int l = lane_id();
  if (i < n) {
    // The row's words are all loaded first (W <= 256: at most 8 per lane).
    constexpr int RW = VR_MAX_POINTS / 32 / 32;
    uint32_t words[RW];
#pragma unroll
    for (int r = 0; r < RW; ++r) {
      const int w = r * 32 + l;
      words[r] = w < W ? adj[(int64_t)i * W + w] : 0u;
    }
    int carry = 0, upc = 0;
#pragma unroll
    for (int r = 0; r < RW; ++r) {
      const int w0 = r * 32;
      if (w0 >= W) break;
      const int w = w0 + l;
      const uint32_t word = words[r];
      const int c = __popc(word);
      const int inc = warp_incl_scan(c);
      if (w < W) {
        adjpre[(int64_t)i * W + w] = carry + inc - c;
        if (adjx) adjx[(int64_t)i * W + w] = make_int2((int)word, carry + inc - c);
      }
      carry += __shfl_sync(0xffffffffu, inc, 31);
      uint32_t m;
      const int lo = w * 32;
      if (lo > i) m = 0xffffffffu;
      else if (lo + 31 <= i) m = 0u;
      else m = ~((2u << (i & 31)) - 1u);
      upc += __popc(word & m);
    }
    upc = warp_sum(upc);
    if (l == 0) {
      deg[i] = carry;
      up[i] = upc;
      __threadfence();  // the last CTA reads deg and up
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) ticket = atomicAdd(&st->rows_done, 1u);
  __syncthreads();
  if (ticket != gridDim.x - 1) return;
  __threadfence();
  // Last CTA: chunks of 2048 entries staged in shared memory (coalesced,
  // bypassing L1 for the other CTAs' writes), 8 consecutive per thread.
  constexpr int PER = 8, CH = 256 * PER;
  __shared__ int32_t cd[CH], cu[CH];
  int64_t base_d = 0, base_u = 0, wedges = 0;
  for (int c0 = 0; c0 < n; c0 += CH) {
    for (int q = threadIdx.x; q < CH; q += 256) {
      const int j = c0 + q;
      cd[q] = j < n ? __ldcg(deg + j) : 0;
      cu[q] = j < n ? __ldcg(up + j) : 0;
    }
    __syncthreads();
    int64_t sd = 0, su = 0, sw = 0;
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int64_t dq = cd[threadIdx.x * PER + q];
      sd += dq;
      su += cu[threadIdx.x * PER + q];
      sw += dq * (dq - 1) / 2;
    }
    int64_t td, tu, tw;
    const int64_t ed = block_excl_scan<int64_t>(sd, sh, &td);
    const int64_t eu = block_excl_scan<int64_t>(su, sh, &tu);
    block_excl_scan<int64_t>(sw, sh, &tw);
    wedges += tw;
    int64_t rd = base_d + ed, ru = base_u + eu;
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int j = c0 + threadIdx.x * PER + q;
      if (j < n) {
        nbr_ptr[j] = (int32_t)rd;
        lex_ptr[j] = ru;
      }
      rd += cd[threadIdx.x * PER + q];
      ru += cu[threadIdx.x * PER + q];
    }
    base_d += td;
    base_u += tu;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    nbr_ptr[n] = (int32_t)base_d;
    lex_ptr[n] = base_u;
    st->E = base_u;
    st->wedges = wedges;
    st->rows_done = 0;  // ready for another launch on the same status word
  }
}

// Bits of the words of row b strictly above column b.
__device__ __forceinline__ uint32_t above_mask(int b, int w) {
  const int lo = w * 32;
  if (lo > b) return 0xffffffffu;
  if (lo + 31 <= b) return 0u;
  return ~((2u << (b & 31)) - 1u);
}

// Balanced walk over the set bits of one round of per-lane masks m (lane l
// owns word w0 + l): the round's candidates are taken 32 at a time, lane q
// taking the q-th, located by a 5-step search over the lanes' prefix counts
// and __fns inside the owner lane's mask.  Every lane does the same number of
// iterations whatever the bits' distribution.  Returns, per chunk, through
// the callback: ok (lane has a candidate), owner lane, bit.
struct BitChunk {
  int tot;     // candidates in the round
  int excl;    // this lane's exclusive prefix
};
__device__ __forceinline__ BitChunk bit_round(uint32_t m) {
  const int c = __popc(m);
  const int inc = warp_incl_scan(c);
  return BitChunk{__shfl_sync(0xffffffffu, inc, 31), inc - c};
}
__device__ __forceinline__ int bit_owner(const BitChunk &r, int q) {
  int owner = 0;
#pragma unroll
  for (int step = 16; step > 0; step >>= 1) {
    const int cand = owner + step;
    const int v = __shfl_sync(0xffffffffu, r.excl, cand & 31);
    if (cand < 32 && v <= q) owner = cand;
  }
  return owner;
}

// Compaction of one round of per-lane masks m (lane l owns word w): the
// columns w * 32 + bit of all set bits, in ascending order, land in the
// warp's buffer cb (room for 32 x 32), each lane appending its own bits at its
// exclusive prefix; returns the round's count.  The caller reads cb after a
// __syncwarp and issues another before the buffer is reused.  Cheaper than
// locating every candidate by search (bit_owner + __fns): a lane's loop runs
// over its own set bits only.
__device__ __forceinline__ int bit_compact(uint32_t m, int w, uint16_t *cb) {
  const int c = __popc(m);
  const int inc = warp_incl_scan(c);
  for (int p = inc - c; m; m &= m - 1) cb[p++] = (uint16_t)(w * 32 + __ffs(m) - 1);
  return __shfl_sync(0xffffffffu, inc, 31);
}
constexpr int CB_SLOTS = 1024;  // bit_compact buffer per warp

__device__ __forceinline__ int32_t bit_rank(const uint32_t *adj_row, const int32_t *pre_row, int c) {
  const int w = c >> 5, b = c & 31;
  return pre_row[w] + __popc(adj_row[w] & ((1u << b) - 1u));
}

// --------------------------------------------------------------- edge keys
// One warp per row i: every kept j > i, in ascending j, at its lexicographic
// position lex_ptr[i] + (rank of j in row i) - (neighbours <= i).
template <bool F>
__global__ void __launch_bounds__(256) k_edge_keys(const void *Xv, int n, int d, int W, const uint32_t *adj,
                                                   const int64_t *lex_ptr, uint64_t *keys, uint32_t *lexe,
                                                   int32_t *elp, KeyHist kh,
    const DevStatus *st) {
  pdl_entry();
  if (build_failed(st)) return;
  using T = typename std::conditional<F, float, int32_t>::type;
  __shared__ KeyHistSmem hs;
  __shared__ uint16_t cbuf[8][CB_SLOTS];
  khist_init(hs, kh);
  const T *X = (const T *)Xv;
  const int i = blockIdx.x * 8 + (threadIdx.x >> 5);
  const int l = lane_id();
  uint16_t *cb = cbuf[threadIdx.x >> 5];
  const uint32_t *row = adj + (int64_t)i * W;
  int64_t t = i < n ? lex_ptr[i] : 0;
  for (int w0 = (i + 1) >> 5; i < n && w0 < W; w0 += 32) {
    const int w = w0 + l;
    const uint32_t word = w < W ? row[w] & above_mask(i, w) : 0u;
    const int tot = bit_compact(word, w, cb);
    __syncwarp();
    for (int q0 = 0; q0 < tot; q0 += 32) {
      const int q = q0 + l;
      uint64_t key = 0;
      if (q < tot) {
        const int j = cb[q];
        uint64_t dk;
        if constexpr (F) dk = (uint64_t)__float_as_uint(d2_f32(X + (int64_t)i * d, X + (int64_t)j * d, d));
        else dk = d2_int(X + (int64_t)i * d, X + (int64_t)j * d, d);
        key = (dk << KEY_SHIFT) | ((uint64_t)i << ID_BITS) | (uint64_t)j;
        keys[t + q] = key;
        lexe[t + q] = ((uint32_t)i << ID_BITS) | (uint32_t)j;
        if (elp) elp[(int64_t)i * n + j] = (int32_t)(t + q);  // lexicographic position (tetrahedra)
      }
      khist_add(hs, kh, key, q < tot);
    }
    __syncwarp();
    t += tot;
  }
  khist_flush(hs, kh);
}

// ------------------------------------------------- distance-matrix input
// A square symmetric n x n matrix of edge values (int32, or float32 whose
// keys are the bits of the value: order-preserving for non-negative floats,
// -0 folded onto +0).  The strict upper triangle gives the edges.

template <bool F>
__device__ __forceinline__ uint32_t dmat_key(const void *Dv, int64_t idx) {
  if constexpr (F) return __float_as_uint(((const float *)Dv)[idx]) & 0x7fffffffu;
  else return (uint32_t)((const int32_t *)Dv)[idx];
}

// Value checks on 32 x 32 tiles: finite, non-negative, D[i][j] == D[j][i].
template <bool F>
static __global__ void __launch_bounds__(256) k_dmat_check(const void *Dv, int n, DevStatus *st) {
  pdl_entry();
  __shared__ float tf[32][33];
  __shared__ int32_t ti[32][33];
  const int nb = (n + 31) / 32;
  const int bi = blockIdx.x / nb, bj = blockIdx.x % nb;
  if (bi > bj) return;  // the tile pair (bi, bj) and its transpose, once
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  // Load the transposed tile D[bj*32 + r][bi*32 + c].
  for (int r = ty; r < 32; r += 8) {
    const int gi = bj * 32 + r, gj = bi * 32 + tx;
    if (gi < n && gj < n) {
      if constexpr (F) tf[r][tx] = ((const float *)Dv)[(int64_t)gi * n + gj];
      else ti[r][tx] = ((const int32_t *)Dv)[(int64_t)gi * n + gj];
    }
  }
  __syncthreads();
  bool bad = false, nonfinite = false;
  for (int r = ty; r < 32; r += 8) {
    const int gi = bi * 32 + r, gj = bj * 32 + tx;
    if (gi < n && gj < n) {
      if constexpr (F) {
        const float v = ((const float *)Dv)[(int64_t)gi * n + gj];
        if (!isfinite(v)) nonfinite = true;
        else if (v < 0.0f || v != tf[tx][r]) bad = true;
      } else {
        const int32_t v = ((const int32_t *)Dv)[(int64_t)gi * n + gj];
        if (v < 0 || v != ti[tx][r]) bad = true;
      }
    }
  }
  if (__any_sync(0xffffffffu, nonfinite) && tx == 0) raise_flag(st, F_NONFINITE);
  if (__any_sync(0xffffffffu, bad) && tx == 0) raise_flag(st, F_DMAT);
}

// Kept-edge bitmap: warp per row, one ballot per 32 columns (the matrix is
// symmetric, so rows give both halves).  keep iff key <= capkey (or all).
template <bool F>
static __global__ void __launch_bounds__(256) k_dmat_bitmap(const void *Dv, int n, int W, int keep_all,
                                                            uint32_t capkey, uint32_t *adj) {
  pdl_entry();
  const int i = blockIdx.x * 8 + (threadIdx.x >> 5), l = lane_id();
  if (i >= n) return;
  for (int w = 0; w < W; ++w) {
    const int j = w * 32 + l;
    bool keep = false;
    if (j < n && j != i) keep = keep_all || dmat_key<F>(Dv, (int64_t)i * n + j) <= capkey;
    const uint32_t b = __ballot_sync(0xffffffffu, keep);
    if (l == 0) adj[(int64_t)i * W + w] = b;
  }
}

// Edge keys in lexicographic order, warp per row (the walk of k_edge_keys
// with the matrix entry as the value).
template <bool F>
static __global__ void __launch_bounds__(256) k_dmat_keys(const void *Dv, int n, int W, const uint32_t *adj,
                                                          const int64_t *lex_ptr, uint64_t *keys, uint32_t *lexe,
                                                          int32_t *elp, KeyHist kh,
    const DevStatus *st) {
  pdl_entry();
  if (build_failed(st)) return;
  __shared__ KeyHistSmem hs;
  __shared__ uint16_t cbuf[8][CB_SLOTS];
  khist_init(hs, kh);
  const int i = blockIdx.x * 8 + (threadIdx.x >> 5);
  const int l = lane_id();
  uint16_t *cb = cbuf[threadIdx.x >> 5];
  const uint32_t *row = adj + (int64_t)i * W;
  int64_t t = i < n ? lex_ptr[i] : 0;
  for (int w0 = (i + 1) >> 5; i < n && w0 < W; w0 += 32) {
    const int w = w0 + l;
    const uint32_t word = w < W ? row[w] & above_mask(i, w) : 0u;
    const int tot = bit_compact(word, w, cb);
    __syncwarp();
    for (int q0 = 0; q0 < tot; q0 += 32) {
      const int q = q0 + l;
      uint64_t key = 0;
      if (q < tot) {
        const int j = cb[q];
        const uint64_t dk = dmat_key<F>(Dv, (int64_t)i * n + j);
        key = (dk << KEY_SHIFT) | ((uint64_t)i << ID_BITS) | (uint64_t)j;
        keys[t + q] = key;
        lexe[t + q] = ((uint32_t)i << ID_BITS) | (uint32_t)j;
        if (elp) elp[(int64_t)i * n + j] = (int32_t)(t + q);  // lexicographic position (tetrahedra)
      }
      khist_add(hs, kh, key, q < tot);
    }
    __syncwarp();
    t += tot;
  }
  khist_flush(hs, kh);
}

struct SoftAcc {
  uint64_t M;
  int E;
  bool ok;
};
__device__ __forceinline__ void soft_step(SoftAcc &s, float x, float y) {
  int64_t a, b;
  int ea, eb;
  f32_decode(x, a, ea);
  f32_decode(y, b, eb);
  int64_t D;
  int emin;
  if (a == 0 || b == 0) {
    D = a ? a : -b;
    emin = a ? ea : eb;
  } else {
    emin = min(ea, eb);
    const int da = ea - emin, db = eb - emin;
    if (da > 29 || db > 29) { s.ok = false; return; }
    D = (a << da) - (b << db);
  }
  const uint64_t ad = (uint64_t)(D < 0 ? -D : D);
  if (ad >> 53) { s.ok = false; return; }
  if (ad == 0) return;
  uint64_t Ms;
  int Es;
  soft_round_u128((unsigned __int128)ad * ad, 2 * emin, Ms, Es);
  soft_add(s.M, s.E, Ms, Es);
}
__device__ __forceinline__ double soft_value(const SoftAcc &s) {
  if (s.M == 0) return 0.0;
  return __longlong_as_double((long long)(((uint64_t)(s.E + 52 + 1023) << 52) | (s.M & ((1ull << 52) - 1))));
}

// Kept edges (i, j), i < j, in lexicographic order: warp per row i, every
// kept j > i in ascending j at lex_ptr[i] + k (and its position in the dense
// table elp, when given).
static __global__ void __launch_bounds__(256) k_lex_edges(int n, int W, const uint32_t *adj, const int64_t *lex_ptr,
                                                          uint32_t *lexe, int32_t *elp,
    const DevStatus *st) {
  pdl_entry();
  if (build_failed(st)) return;
  __shared__ uint16_t cbuf[8][CB_SLOTS];
  const int i = blockIdx.x * 8 + (threadIdx.x >> 5);
  const int l = lane_id();
  if (i >= n) return;  // whole warps
  uint16_t *cb = cbuf[threadIdx.x >> 5];
  const uint32_t *row = adj + (int64_t)i * W;
  int64_t t = lex_ptr[i];
  for (int w0 = (i + 1) >> 5; w0 < W; w0 += 32) {
    const int w = w0 + l;
    const uint32_t word = w < W ? row[w] & above_mask(i, w) : 0u;
    const int tot = bit_compact(word, w, cb);
    __syncwarp();
    for (int q = l; q < tot; q += 32) {
      const int j = cb[q];
      lexe[t + q] = ((uint32_t)i << ID_BITS) | (uint32_t)j;
      if (elp) elp[(int64_t)i * n + j] = (int32_t)(t + q);
    }
    __syncwarp();
    t += tot;
  }
}

// Float edge keys over the lexicographic edge list: warp per 32 consecutive
// kept edges (lane l takes position 32c + l), so every warp has the same work
// whatever the rows' degrees (warp per row left the densest rows' warps
// running long after the rest).  Both endpoints' coordinates are staged
// through shared memory 32 at a time with coalesced loads, all of a stage's
// loads in flight; each lane then walks its pair in coordinate order,
// evaluating the canonical FP64 sum (integer emulation, hardware FP64 only on
// the rare inexact case) and the fp32 first pass for the error statistic.
// Key = RN32(FP64 value) bits, i, j.  E comes from the status word (the
// launch may precede the host's read of it).
constexpr int EKF_WARPS = 4;
// EKF_HW_NUM chunks in EKF_HW_MOD are evaluated with the hardware FP64 pipe
// (the same canonical sequence: IEEE 754 makes every step's result unique),
// the others by the integer emulation: whole warps take one or the other, so
// the two pipes work at once.
constexpr int EKF_HW_MOD = 2, EKF_HW_NUM = 1;
static __global__ void __launch_bounds__(EKF_WARPS * 32) k_edge_keys_f32(const float *X, int d, const uint32_t *lexe,
                                                                         uint64_t *keys, double *d64_lex,
                                                                         DevStatus *st) {
  pdl_entry();
  if (build_failed(st)) return;
  __shared__ float ti[EKF_WARPS][32][33], tj[EKF_WARPS][32][33];
  const int wid = threadIdx.x >> 5, l = lane_id();
  const int64_t E = st->E, nch = (E + 31) / 32;
  float worst = 0.f;
  for (int64_t c = (int64_t)blockIdx.x * EKF_WARPS + wid; c < nch; c += (int64_t)gridDim.x * EKF_WARPS) {
    const int64_t t = c * 32 + l;
    const bool has = t < E;
    const uint32_t ab = lexe[has ? t : c * 32];  // idle lanes repeat the chunk's first pair
    const int i = (int)(ab >> ID_BITS), j = (int)(ab & ID_MASK);
    SoftAcc acc{0, 0, true};
    const bool hw = (c % EKF_HW_MOD) < EKF_HW_NUM;  // warp-uniform
    double acc64 = 0.0;
    float a = 0.f;
    for (int k0 = 0; k0 < d; k0 += 32) {
      const int kn = min(32, d - k0);
      float v[32];
#pragma unroll
      for (int rr = 0; rr < 32; ++rr) {
        const int jr = __shfl_sync(0xffffffffu, j, rr);
        v[rr] = l < kn ? __ldg(X + (int64_t)jr * d + k0 + l) : 0.f;
      }
#pragma unroll
      for (int rr = 0; rr < 32; ++rr) tj[wid][rr][l] = v[rr];
#pragma unroll
      for (int rr = 0; rr < 32; ++rr) {
        const int ir = __shfl_sync(0xffffffffu, i, rr);
        v[rr] = l < kn ? __ldg(X + (int64_t)ir * d + k0 + l) : 0.f;
      }
#pragma unroll
      for (int rr = 0; rr < 32; ++rr) ti[wid][rr][l] = v[rr];
      __syncwarp();
      if (hw) {
        for (int k = 0; k < kn; ++k) {
          const float xv = ti[wid][l][k], yv = tj[wid][l][k];
          const float tt = __fsub_rn(xv, yv);
          a = __fmaf_rn(tt, tt, a);
          const double t64 = __dsub_rn((double)xv, (double)yv);
          acc64 = __dadd_rn(acc64, __dmul_rn(t64, t64));
        }
      } else {
        for (int k = 0; k < kn; ++k) {
          const float xv = ti[wid][l][k], yv = tj[wid][l][k];
          const float tt = __fsub_rn(xv, yv);
          a = __fmaf_rn(tt, tt, a);
          if (acc.ok) soft_step(acc, xv, yv);
        }
      }
      __syncwarp();
    }
    if (has) {
      const double f = hw ? acc64 : acc.ok ? soft_value(acc) : d2_f64(X + (int64_t)i * d, X + (int64_t)j * d, d);
      d64_lex[t] = f;
      keys[t] = ((uint64_t)__float_as_uint(__double2float_rn(f)) << KEY_SHIFT) | ((uint64_t)i << ID_BITS) |
                (uint64_t)j;
      if (f > 0.0) {
        const float ff = (float)f, sf = sqrtf(ff);
        worst = fmaxf(worst, fabsf((float)((double)a - f)) / (sf * (sqrtf(a) + sf)));
      }
    }
  }
  worst = fmaxf(worst, __shfl_xor_sync(0xffffffffu, worst, 16));
  worst = fmaxf(worst, __shfl_xor_sync(0xffffffffu, worst, 8));
  worst = fmaxf(worst, __shfl_xor_sync(0xffffffffu, worst, 4));
  worst = fmaxf(worst, __shfl_xor_sync(0xffffffffu, worst, 2));
  worst = fmaxf(worst, __shfl_xor_sync(0xffffffffu, worst, 1));
  if (l == 0 && worst > 0.f)
    atomicMax((unsigned long long *)&st->max_rel_err_bits, (unsigned long long)__double_as_longlong((double)worst));
}

__device__ __forceinline__ int key_i(uint64_t k) { return (int)((k >> ID_BITS) & ID_MASK); }
__device__ __forceinline__ int key_j(uint64_t k) { return (int)(k & ID_MASK); }

// ---------------------------------------------------------- float repair
// After the sort by the fp32 first pass, every edge gets its canonical FP64
// value.  Neighbours whose first-pass intervals [lo, hi] overlap may be out
// of order; they form a repair group (a maximal run where each step's
// intervals overlap), re-sorted by (FP64 value, i, j).  Across a group
// boundary the FP64 values are strictly ordered already.
// After the sort: each edge's canonical value (computed in lexicographic
// order by k_edge_keys_f32) is fetched through its lex position.  Keys are
// RN32 of the canonical value, which is monotone, so different keys are
// already in FP64 order; only runs of equal keys need re-sorting by
// (FP64, i, j).
__device__ __forceinline__ double f64_of(uint64_t key, const double *d64_lex, const uint32_t *adj,
                                         const int32_t *adjpre, int W, const int32_t *deg, const int32_t *up,
                                         const int64_t *lex_ptr) {
  const int i = key_i(key), j = key_j(key);
  return d64_lex[lex_ptr[i] + bit_rank(adj + (int64_t)i * W, adjpre + (int64_t)i * W, j) - (deg[i] - up[i])];
}

__device__ __forceinline__ bool f64_less(double da, uint64_t ka, double db, uint64_t kb) {
  return da < db || (da == db && (ka & ((1ull << KEY_SHIFT) - 1)) < (kb & ((1ull << KEY_SHIFT) - 1)));
}

constexpr int REPAIR_SMALL = 32;
constexpr int REPAIR_MID = 2048;

struct F64Src {
  const double *d64_lex;
  const uint32_t *adj;
  const int32_t *adjpre;
  int W;
  const int32_t *deg, *up;
  const int64_t *lex_ptr;
  __device__ __forceinline__ double of(uint64_t key) const { return f64_of(key, d64_lex, adj, adjpre, W, deg, up, lex_ptr); }
};

// Thread per sorted position k.  A position whose fp32 key differs from both
// neighbours stands alone and fetches its FP64 value.  The first position of
// a run of equal keys finds the run's end by a galloping search; a run of up
// to REPAIR_SMALL edges is fetched and insertion-sorted by that thread, a
// longer one is queued as a (begin, size) pair for the CTA kernels, which
// fetch its values themselves.  Other positions inside runs do nothing.
static __global__ void k_f64_repair_small(uint64_t *keys, int64_t E, F64Src src, double *d64, int32_t *midq,
                                          int32_t *bigq, DevStatus *st) {
  pdl_entry();
  if (build_failed(st)) return;
  int64_t nt = 0;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < E; k += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t key = keys[k];
    const uint64_t top = key >> KEY_SHIFT;
    if (k > 0 && (keys[k - 1] >> KEY_SHIFT) == top) continue;
    if (k + 1 == E || (keys[k + 1] >> KEY_SHIFT) != top) {
      d64[k] = src.of(key);
      continue;
    }
    // keys[lo] is in the run; hi is past it (or E).
    int64_t lo = k + 1, step = 1;
    while (lo + step < E && (keys[lo + step] >> KEY_SHIFT) == top) {
      lo += step;
      step <<= 1;
    }
    int64_t hi = lo + step < E ? lo + step : E;
    while (hi - lo > 1) {
      const int64_t mid = lo + ((hi - lo) >> 1);
      if ((keys[mid] >> KEY_SHIFT) == top) lo = mid;
      else hi = mid;
    }
    const int64_t sz = hi - k;
    nt += sz;
    if (sz > REPAIR_MID) {
      const int q = (int)atomicAdd((unsigned long long *)&st->big_grp_count, 1ull);
      bigq[2 * q] = (int32_t)k;
      bigq[2 * q + 1] = (int32_t)sz;
      atomicMax((unsigned long long *)&st->big_grp_max, (unsigned long long)sz);
      continue;
    }
    if (sz > REPAIR_SMALL) {
      const int q = atomicAdd(&st->mid_grp_count, 1);
      midq[2 * q] = (int32_t)k;
      midq[2 * q + 1] = (int32_t)sz;
      continue;
    }
    d64[k] = src.of(key);
    for (int64_t x = k + 1; x < hi; ++x) {
      const uint64_t kx = keys[x];
      const double dx = src.of(kx);
      int64_t y = x - 1;
      while (y >= k && f64_less(dx, kx, d64[y], keys[y])) {
        keys[y + 1] = keys[y];
        d64[y + 1] = d64[y];
        --y;
      }
      keys[y + 1] = kx;
      d64[y + 1] = dx;
    }
  }
  if (nt) atomicAdd((unsigned long long *)&st->near_tie, (unsigned long long)nt);
}

// CTA per queued mid-size group: bitonic sort in shared memory on the pair
// (FP64 bits, i<<13|j) packed as two words; val = position in the group.
static __global__ void __launch_bounds__(256) k_repair_mid(const int32_t *midq, F64Src src, const DevStatus *st,
                                                    uint64_t *keys, double *d64) {
  pdl_entry();
  if (build_failed(st)) return;
  __shared__ uint64_t hi[REPAIR_MID];
  __shared__ uint32_t lo[REPAIR_MID];
  __shared__ uint32_t val[REPAIR_MID];
  const int nq = st->mid_grp_count;
  for (int q = blockIdx.x; q < nq; q += gridDim.x) {
    const int64_t b = midq[2 * q];
    const int s = midq[2 * q + 1];
    int cap = 1;
    while (cap < s) cap <<= 1;
    for (int t = threadIdx.x; t < cap; t += blockDim.x) {
      if (t < s) {
        const uint64_t kt = keys[b + t];
        const double dt = src.of(kt);
        d64[b + t] = dt;
        hi[t] = (uint64_t)__double_as_longlong(dt);
        lo[t] = (uint32_t)(kt & ((1ull << KEY_SHIFT) - 1));
      } else {
        hi[t] = ~0ull;
        lo[t] = ~0u;
      }
      val[t] = t;
    }
    __syncthreads();
    for (int k = 2; k <= cap; k <<= 1)
      for (int j = k >> 1; j > 0; j >>= 1) {
        for (int i = threadIdx.x; i < cap; i += blockDim.x) {
          int x = i ^ j;
          if (x > i) {
            bool up = (i & k) == 0;
            bool gt = hi[i] > hi[x] || (hi[i] == hi[x] && lo[i] > lo[x]);
            if (gt == up) {
              uint64_t th = hi[i]; hi[i] = hi[x]; hi[x] = th;
              uint32_t tl = lo[i]; lo[i] = lo[x]; lo[x] = tl;
              uint32_t tv = val[i]; val[i] = val[x]; val[x] = tv;
            }
          }
        }
        __syncthreads();
      }
    // Permute: keys' top bits and d64 follow val.  Read all first, then write.
    uint64_t kk[REPAIR_MID / 256];
    double dd[REPAIR_MID / 256];
    int c = 0;
    for (int t = threadIdx.x; t < s; t += blockDim.x, ++c) {
      kk[c] = keys[b + val[t]];
      dd[c] = d64[b + val[t]];
    }
    __syncthreads();
    c = 0;
    for (int t = threadIdx.x; t < s; t += blockDim.x, ++c) {
      keys[b + t] = kk[c];
      d64[b + t] = dd[c];
    }
    __syncthreads();
  }
}

// One CTA for the queued large groups (rare: massive near-ties): stable LSD
// sort by (i<<13|j), then by the FP64 bits, through global temporaries.
static __global__ void __launch_bounds__(RS_THREADS) k_repair_big(const int32_t *bigq, F64Src src,
                                                           const DevStatus *st, uint64_t *keys, double *d64,
                                                           uint64_t *k1, uint32_t *v1, uint64_t *k2, uint32_t *v2,
                                                           uint64_t *gk, double *gd) {
  pdl_entry();
  if (build_failed(st)) return;
  const int nq = (int)st->big_grp_count;
  for (int q = 0; q < nq; ++q) {
    const int64_t b = bigq[2 * q];
    const int64_t s = bigq[2 * q + 1];
    for (int64_t t = threadIdx.x; t < s; t += blockDim.x) {
      const uint64_t kt = keys[b + t];
      d64[b + t] = src.of(kt);
      k1[t] = kt & ((1ull << KEY_SHIFT) - 1);
      v1[t] = (uint32_t)t;
    }
    __syncthreads();
    cta_radix_sort_global(k1, v1, k2, v2, s, 0, KEY_SHIFT);
    for (int64_t t = threadIdx.x; t < s; t += blockDim.x) k1[t] = (uint64_t)__double_as_longlong(d64[b + v1[t]]);
    __syncthreads();
    cta_radix_sort_global(k1, v1, k2, v2, s, 0, 64);
    for (int64_t t = threadIdx.x; t < s; t += blockDim.x) {
      gk[t] = keys[b + v1[t]];
      gd[t] = d64[b + v1[t]];
    }
    __syncthreads();
    for (int64_t t = threadIdx.x; t < s; t += blockDim.x) {
      keys[b + t] = gk[t];
      d64[b + t] = gd[t];
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------ edge grades
// flag[k] = 1 where the squared distance differs from the previous edge's
// (or from 0 for k = 0): the dense rank is the running sum of flags.
// Grades and edge outputs in one launch: tiles of EG_TILE sorted keys (four
// per thread, 32 apart; 1024-key tiles measured 2 us faster than one key per
// thread on 75k edges: a shorter look-back chain) in ticket order; a key
// starts a new grade when its distance differs from the
// previous key's (the first distance > 0 also does: grade 0 is d = 0); the
// block scan of those flags plus the earlier tiles' counts (look-back) is the
// dense rank; then the outputs: verts, grade, colptr/rowidx ({i, j}), grade
// values and group starts, the neighbour CSR scatter and the dense tables.  lb: the
// tiles' zeroed status words followed by the ticket counter.  Every load of
// the outputs' inputs (keys, FP64 values, the endpoints' CSR offsets and
// {row word, prefix count} pairs) is issued before the look-back, so its
// latency overlaps warp 0's wait.
constexpr int EG_TILE = 1024;
template <bool F>
__global__ void __launch_bounds__(256) k_edge_grades(const uint64_t *__restrict__ keys,
                                                     const double *__restrict__ d64, int64_t E,
                                                     const int2 *__restrict__ adjx, int W,
                                                     const int32_t *__restrict__ nbr_ptr, int32_t *verts,
                                                     int32_t *grade, int64_t *colptr, int32_t *rowidx, double *gval,
                                                     int32_t *gstart, int32_t *nbr_ord, int32_t *eidx, int32_t *egd,
                                                     int n, int key_f32, uint64_t *lb, int64_t ntiles,
                                                     DevStatus *st) {
  pdl_entry();
  if (build_failed(st)) return;
  // Warp w of the tile takes the keys k0 + w * 32 * PER + 32 q + l (q < PER):
  // a new grade starts at a key whose value differs from its predecessor's;
  // each key's grade is the tile's prefix plus the flags up to it (ballots),
  // and consecutive lanes write consecutive entries of every output.
  constexpr int PER = EG_TILE / 256;
  __shared__ int64_t wpre[8];
  __shared__ int64_t tile_sh;
  if (threadIdx.x == 0) tile_sh = atomicAdd((unsigned long long *)&lb[ntiles], 1ull);
  __syncthreads();
  const int w = threadIdx.x >> 5, l = lane_id();
  const int64_t tile = tile_sh, kw = tile * EG_TILE + (int64_t)w * 32 * PER;
  uint64_t kq[PER];
  double dq[PER];
  uint32_t fm[PER];
  int wcnt = 0;
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int64_t k = kw + 32 * q + l;
    kq[q] = k < E ? keys[k] : 0ull;
    dq[q] = F && k < E ? d64[k] : 0.0;
  }
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int64_t k = kw + 32 * q + l;
    bool f = false;
    if (k < E) {
      if constexpr (F) f = k == 0 ? (dq[q] != 0.0) : (dq[q] != d64[k - 1]);
      else f = k == 0 ? ((kq[q] >> KEY_SHIFT) != 0) : ((kq[q] >> KEY_SHIFT) != (keys[k - 1] >> KEY_SHIFT));
    }
    fm[q] = __ballot_sync(0xffffffffu, f);
    wcnt += __popc(fm[q]);
  }
  // The scatter's inputs: each endpoint's CSR offset and the {row word,
  // prefix count} pair of the word holding the other endpoint.
  int32_t npi[PER], npj[PER];
  int2 ai[PER], aj[PER];
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int64_t k = kw + 32 * q + l;
    const int i = key_i(kq[q]), j = key_j(kq[q]);
    if (k < E) {
      npi[q] = nbr_ptr[i];
      npj[q] = nbr_ptr[j];
      ai[q] = adjx[(int64_t)i * W + (j >> 5)];
      aj[q] = adjx[(int64_t)j * W + (i >> 5)];
    } else {
      npi[q] = npj[q] = 0;
      ai[q] = aj[q] = make_int2(0, 0);
    }
  }
  if (l == 0) wpre[w] = wcnt;
  __syncthreads();
  if (w == 0) {
    const int64_t v = l < 8 ? wpre[l] : 0;
    const int64_t iv = warp_incl_scan(v);
    const int64_t tot = __shfl_sync(0xffffffffu, iv, 31);
    const int64_t pre = tile_lookback(lb, tile, tot, &st->flags);
    if (l < 8) wpre[l] = pre + iv - v;
  }
  __syncthreads();
  int64_t gbase = wpre[w];  // grades started before this warp's q-th group
  const uint32_t le = lanemask_lt() | (1u << l);
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int64_t k = kw + 32 * q + l;
    const int64_t g = gbase + __popc(fm[q] & le);
    gbase += __popc(fm[q]);
    if (k >= E) continue;
    const bool f = (fm[q] >> l) & 1u;
    const uint64_t key = kq[q];
    const int i = key_i(key), j = key_j(key);
    ((int2 *)verts)[k] = make_int2(i, j);
    ((int2 *)rowidx)[k] = make_int2(i, j);
    colptr[k] = 2 * k;
    grade[k] = (int32_t)g;
    if (f) {
      gval[g] = F ? dq[q]
                  : key_f32 ? (double)__uint_as_float((uint32_t)(key >> KEY_SHIFT)) : (double)(key >> KEY_SHIFT);
      gstart[g] = (int32_t)k;
    }
    nbr_ord[npi[q] + ai[q].y + __popc((uint32_t)ai[q].x & ((1u << (j & 31)) - 1u))] = (int32_t)k;
    nbr_ord[npj[q] + aj[q].y + __popc((uint32_t)aj[q].x & ((1u << (i & 31)) - 1u))] = (int32_t)k;
    if (eidx) {
      eidx[(int64_t)i * n + j] = (int32_t)k;
      egd[(int64_t)i * n + j] = (int32_t)g;
    }
    if (k == E - 1) {
      colptr[E] = 2 * E;
      gstart[g + 1] = (int32_t)E;
      st->ngrades = g + 1;
    }
    if (k == 0) {
      gval[0] = 0.0;
      gstart[0] = 0;
    }
  }
}

// Also clears `zero_words` words at `zero` (the triangle sort's scratch), so
// that no memset sits between the build's dependent launches.
static __global__ void k_vertices(int n, int32_t *verts, int32_t *grade, int64_t *tcol, int64_t T, uint64_t *zero,
                                  int64_t zero_words) {
  pdl_entry();
  if (tcol && blockIdx.x == 0 && threadIdx.x == 0) tcol[T] = 3 * T;  // closing colptr entry of dimension 2
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += stride) {
    verts[v] = (int32_t)v;
    grade[v] = 0;
  }
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < zero_words; i += stride) zero[i] = 0;
}

// -------------------------------------------------------------- triangles
// Edge e = (a, b) in filtration order.  The candidates c are the set bits of
// adj[a] & adj[b]; a triangle {a, b, c} is counted at e iff e is its largest
// edge in the total (grade, lex) order, i.e. ord(a,c) < e and ord(b,c) < e,
// so each triangle appears exactly once and its grade is grade(e).  One warp
// per edge; lane l takes word 32*r + l in round r, so the warp's output is in
// ascending c, which is already lexicographic for the sorted triple.

// Two enumeration orders (both exact):
//  * max-edge order (above): a triangle is produced by its largest edge, so
//    the output is already in (grade, lex) order when no grade group spans
//    several edges with triangles -- the case for float data;
//  * lex order: a triangle is produced by its first edge (a, b), a < b < c,
//    as the key grade << 39 | (a, b, c); a stable sort on the grade bits then
//    gives (grade, lex) with no merge -- the case for tie-heavy integer data.
// The mode is chosen on the device from the grade count (same rule on host).
constexpr int LEX_SHIFT = 3 * ID_BITS;
__device__ __forceinline__ uint64_t lex3(int a, int b, int c) {
  return ((uint64_t)a << (2 * ID_BITS)) | ((uint64_t)b << ID_BITS) | (uint64_t)c;
}

// Triangles in lexicographic order + a sort on the grade bits: chosen when
// more than 5% of edges share a grade (tie-heavy integer data: the max-edge
// output would need most grade groups merged), and always when the caller
// forces it (tetrahedra, which are generated from the lexicographic triangle
// list; clouds with sparse rows, where the time-sliced rows of the max-edge
// enumeration cost more than walking the few neighbours).
__host__ __device__ __forceinline__ bool lex_mode(int64_t E, int64_t ngrades, int force = 0) {
  return force || (E - (ngrades - 1)) * 20 > E;
}

__device__ __forceinline__ int64_t lex_pos(int a, int b, const uint32_t *adj, const int32_t *adjpre, int W,
                                           const int32_t *deg, const int32_t *up, const int64_t *lex_ptr) {
  return lex_ptr[a] + bit_rank(adj + (int64_t)a * W, adjpre + (int64_t)a * W, b) - (deg[a] - up[a]);
}

// Order index of kept edge (a, b), a < b: from the dense table when there is
// one (n <= DENSE_MAX_N), else through the neighbour CSR.
constexpr int DENSE_MAX_N = 8192;  // every cloud (n <= 8192): two n x n int32 tables, at most 512 MB
struct EdgeIndex {
  const int2 *adjx;  // {row word, prefix count} pairs, or null
  const uint32_t *adj;
  const int32_t *adjpre;
  const int32_t *nbr_ptr;
  const int32_t *nbr_ord;
  const int32_t *eidx;
  const int32_t *egd;     // dense (a, b) -> grade table (with eidx)
  const int32_t *egrade;  // grade by order index
  int W, n;
  template <bool DENSE>
  __device__ __forceinline__ int32_t ord(int a, int b) const {
    if constexpr (DENSE) return eidx[(int64_t)a * n + b];
    else return nbr_ord[nbr_ptr[a] + bit_rank(adj + (int64_t)a * W, adjpre + (int64_t)a * W, b)];
  }
  template <bool DENSE>
  __device__ __forceinline__ int32_t grade(int a, int b) const {
    if constexpr (DENSE) return egd[(int64_t)a * n + b];
    else return egrade[ord<false>(a, b)];
  }
};

// ---- max-edge enumeration through time-sliced adjacency
// In max-edge order a triangle {x, y, z} is produced by its largest edge
// e = (x, y) (order index e) and its third vertices are
//   S_e = { z : ord(x, z) < e and ord(y, z) < e } = B_x(e) & B_y(e),
// B_v(e) being the bitmap of v's neighbours through edges earlier than e.
// The edge orders are cut into S time slices of B consecutive edges; for
// each slice b >= 1 a snapshot holds every vertex's bitmap B_v(b * B) (edges
// of earlier slices), and every vertex's neighbour list is bucketed by slice.
// Then B_v(e) = snapshot_{e / B}[v] | { z in bucket (v, e / B) : ord < e }:
// one row read plus a short filtered bucket, no per-candidate lookup; S_e
// comes out as a bitmap, in ascending z (lexicographic within the edge).
constexpr int SNAP_MAX_S = 32;
struct SnapIdx {
  const uint32_t *snap;  // (S - 1) x n x Wp words: snapshot b (1 .. S - 1) at (b - 1) * n * Wp
  const uint64_t *bl;    // 2E entries (order << 32) | neighbour, vertex v's from nbr_ptr[v], by slice
  const int32_t *boff;   // n x (S + 1): slice starts within v's entries (relative to nbr_ptr[v])
  int S;
  int64_t B;
  int Wp;                // snapshot row stride: W rounded up to 16-byte words (4 words), padding zero
};
__host__ __device__ __forceinline__ int snap_stride(int W) { return (W + 3) & ~3; }

// One CTA per vertex v, one warp per 32-word round of v's row (blockDim =
// 32 * ceil(Wp / 32) <= 256): the CTA buckets v's neighbour entries by slice
// (a shared histogram, one prefix, shared cursors; the order inside a bucket
// is immaterial: buckets are filtered, not walked in order) and each warp
// writes its round's words of v's snapshot rows.  The histogram pass keeps
// the first SNAP_ORDC neighbour orders in shared memory, where the per-bit
// pass finds them (no dependent L2 load per set bit).  Dynamic shared
// memory: snap_build_smem(warps, S).  Runs in max-edge mode only (decided
// on the device, like the count kernel).
constexpr int SNAP_ORDC = 1024;
__host__ __device__ __forceinline__ size_t snap_build_smem(int warps, int S) {
  return (size_t)warps * (S - 1) * 32 * 4 + SNAP_ORDC * 4;
}
static __global__ void __launch_bounds__(256) k_snap_build(const uint32_t *adj, const int32_t *adjpre, int W, int n,
                                                           const int32_t *nbr_ptr, const int32_t *nbr_ord,
                                                           const DevStatus *st, int force_lex, int S, int64_t B,
                                                           uint32_t *snap, uint64_t *bl, int32_t *boff) {
  pdl_entry();
  if (build_failed(st)) return;
  if (lex_mode(st->E, st->ngrades, force_lex)) return;
  __shared__ int32_t cur[SNAP_MAX_S + 1];
  extern __shared__ uint32_t snap_sm[];
  const int nw = blockDim.x >> 5;
  int32_t *ordc = (int32_t *)(snap_sm + (size_t)nw * (S - 1) * 32);
  const int l = lane_id(), wid = threadIdx.x >> 5;
  uint32_t *sw = snap_sm + (size_t)wid * (S - 1) * 32;  // this warp: lane l's word in snapshot b at sw[(b - 1) * 32 + l]
  const int Wp = snap_stride(W);
  const int64_t nWp = (int64_t)n * Wp;
  const uint32_t Bu = (uint32_t)B;  // B <= E < 2^31: 32-bit divisions
  for (int64_t v = blockIdx.x; v < n; v += gridDim.x) {
    const int32_t ptr = nbr_ptr[v], deg = nbr_ptr[v + 1] - ptr;
    for (int b = threadIdx.x; b <= S; b += blockDim.x) cur[b] = 0;
    __syncthreads();
    for (int k = threadIdx.x; k < deg; k += blockDim.x) {
      const int32_t o = nbr_ord[ptr + k];
      if (k < SNAP_ORDC) ordc[k] = o;
      atomicAdd(&cur[(uint32_t)o / Bu], 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int32_t run = 0;
      for (int b = 0; b <= S; ++b) {
        boff[v * (S + 1) + b] = run;
        const int32_t c = cur[b];
        cur[b] = run;
        run += c;
      }
    }
    __syncthreads();
    const uint32_t *row = adj + v * W;
    const int32_t *pre = adjpre + v * W;
    const int w = wid * 32 + l;  // this lane's word
    if (wid * 32 < Wp) {
      uint32_t m = w < W ? row[w] : 0u;
      int32_t k = w < W ? pre[w] : 0;  // entry index of the word's lowest set bit
      for (int b = 0; b < S - 1; ++b) sw[b * 32 + l] = 0u;
      for (; m; m &= m - 1, ++k) {
        const int bit = __ffs(m) - 1;
        const int32_t o = k < SNAP_ORDC ? ordc[k] : nbr_ord[ptr + k];
        const int bb = (int)((uint32_t)o / Bu);
        const int32_t slot = atomicAdd(&cur[bb], 1);
        bl[ptr + slot] = ((uint64_t)(uint32_t)o << 32) | (uint32_t)(w * 32 + bit);
        for (int b = bb + 1; b < S; ++b) sw[(b - 1) * 32 + l] |= 1u << bit;
      }
      if (w < Wp)
        for (int b = 1; b < S; ++b) snap[(b - 1) * nWp + v * Wp + w] = sw[(b - 1) * 32 + l];
    }
    __syncthreads();
  }
}

template <bool DENSE>
static __global__ void __launch_bounds__(256, 6) k_tri_count(const int32_t *everts, const uint32_t *lexe, int64_t E,
                                                          const uint32_t *adj, const int32_t *adjpre, int W,
                                                          const int32_t *nbr_ptr, const int32_t *nbr_ord,
                                                          const DevStatus *st, int32_t *tcnt, int force_lex,
                                                          EdgeIndex ex, const int64_t *lex_ptr, int sparse,
                                                          SnapIdx sx, int me_claimed) {
  pdl_entry();
  if (build_failed(st)) return;
  const int l = lane_id();
  const int64_t nwarps = (int64_t)gridDim.x * 8;
  if (lex_mode(E, st->ngrades, force_lex) && sparse) {
    // Lex mode on sparse rows (fewer neighbours than bitmap words): the
    // candidates of edge e = (a, b) are a's neighbours above b, which are the
    // lexicographic edges after e in row a; each is one bit test in row b.
    // Four edges per warp at a time, their first rounds' loads together.
    constexpr int U = 4;
    for (int64_t e0 = (blockIdx.x * 8 + (threadIdx.x >> 5)) * (int64_t)U; e0 < E; e0 += nwarps * U) {
      int b[U], c[U], cnt[U];
      int64_t end[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const uint32_t ab = e0 + u < E ? lexe[e0 + u] : 0u;
        b[u] = (int)(ab & ID_MASK);
        end[u] = e0 + u < E ? lex_ptr[(ab >> ID_BITS) + 1] : 0;
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t q = e0 + u + 1 + l;
        c[u] = q < end[u] ? (int)(lexe[q] & ID_MASK) : -1;
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const bool ok = c[u] >= 0 && ((adj[(int64_t)b[u] * W + (c[u] >> 5)] >> (c[u] & 31)) & 1u);
        cnt[u] = __popc(__ballot_sync(0xffffffffu, ok));
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const uint32_t *rb = adj + (int64_t)b[u] * W;
        for (int64_t q0 = e0 + u + 1 + 32; q0 < end[u]; q0 += 32) {
          const int64_t q = q0 + l;
          bool ok = false;
          if (q < end[u]) {
            const int cv = (int)(lexe[q] & ID_MASK);
            ok = (rb[cv >> 5] >> (cv & 31)) & 1u;
          }
          cnt[u] += __popc(__ballot_sync(0xffffffffu, ok));
        }
      }
      if (l < U && e0 + l < E) tcnt[e0 + l] = l == 0 ? cnt[0] : l == 1 ? cnt[1] : l == 2 ? cnt[2] : cnt[3];
    }
    return;
  }
  if (lex_mode(E, st->ngrades, force_lex)) {
    // Lex mode: edges in lexicographic order, the count of edge e (its
    // triangles (a, b, c), c > b) at e: a popcount of the two rows above b.
    // Four edges per warp at a time with all their first-round loads in
    // flight together (one short dependent chain per edge otherwise leaves
    // the kernel latency-bound).
    constexpr int U = 4;
    for (int64_t e0 = (blockIdx.x * 8 + (threadIdx.x >> 5)) * (int64_t)U; e0 < E; e0 += nwarps * U) {
      int a[U], b[U], cnt[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const uint32_t ab = e0 + u < E ? lexe[e0 + u] : 0u;
        a[u] = (int)(ab >> ID_BITS);
        b[u] = (int)(ab & ID_MASK);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int w = (b[u] >> 5) + l;
        cnt[u] = e0 + u < E && w < W
                     ? __popc(adj[(int64_t)a[u] * W + w] & adj[(int64_t)b[u] * W + w] & above_mask(b[u], w))
                     : 0;
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const uint32_t *ra = adj + (int64_t)a[u] * W, *rb = adj + (int64_t)b[u] * W;
        for (int w = (b[u] >> 5) + l + 32; e0 + u < E && w < W; w += 32) cnt[u] += __popc(ra[w] & rb[w]);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) cnt[u] = warp_sum(cnt[u]);
      if (l < U && e0 + l < E) tcnt[e0 + l] = l == 0 ? cnt[0] : l == 1 ? cnt[1] : l == 2 ? cnt[2] : cnt[3];
    }
    return;
  }
  // Max-edge mode: edges in filtration order.  With Sx, Sy the slice
  // snapshot rows of x and y and Dx, Dy their bucket entries earlier than e
  // (disjoint from the snapshots; k_snap_build), the count of e = (x, y) is
  //   |Sx & Sy| + |Dy & Sx| + |Dx & B_y(e)|,
  // the last term by one adjacency bit and one order lookup per entry.  An
  // edge per 8 lanes (4 per warp): every load of an edge is independent of
  // the others, so each lane keeps many in flight (no shared memory, no
  // dependent chain beyond the edge's endpoints and bucket bounds).
  if (me_claimed) return;  // the claiming generator has written the counts
  const int sub = l >> 3, sl = l & 7;
  for (int64_t e = (blockIdx.x * 8 + (threadIdx.x >> 5)) * 4 + sub; e - sub < E; e += nwarps * 4) {
    int cnt = 0;
    if (e < E) {
      const int2 xy = ((const int2 *)everts)[e];
      const int x = xy.x, y = xy.y;
      const int b = (int)((uint32_t)e / (uint32_t)sx.B);  // e < E < 2^31
      const uint32_t *rx = b > 0 ? sx.snap + ((int64_t)(b - 1) * ex.n + x) * sx.Wp : nullptr;
      const uint32_t *ry = b > 0 ? sx.snap + ((int64_t)(b - 1) * ex.n + y) * sx.Wp : nullptr;
      if (b > 0) {
        const uint4 *vx = (const uint4 *)rx, *vy = (const uint4 *)ry;
#pragma unroll 4
        for (int q = sl; q < (sx.Wp >> 2); q += 8) {
          const uint4 a = vx[q], c = vy[q];
          cnt += __popc(a.x & c.x) + __popc(a.y & c.y) + __popc(a.z & c.z) + __popc(a.w & c.w);
        }
      }
      const int32_t *ox = sx.boff + (int64_t)x * (sx.S + 1) + b, *oy = sx.boff + (int64_t)y * (sx.S + 1) + b;
      const int32_t ox0 = ox[0], ox1 = ox[1], oy0 = oy[0], oy1 = oy[1];
      const uint64_t *lx = sx.bl + nbr_ptr[x], *ly = sx.bl + nbr_ptr[y];
      const uint32_t *ay = adj + (int64_t)y * W;
      for (int32_t k = ox0 + sl; k < ox1; k += 8) {
        const uint64_t t = lx[k];
        const int z = (int)(t & 0xffffu);
        const bool adjy = (ay[z >> 5] >> (z & 31)) & 1u;
        int32_t oyz;
        if constexpr (DENSE) oyz = ex.ord<true>(min(y, z), max(y, z));  // in the table; used only when adjacent
        else oyz = adjy ? ex.ord<false>(min(y, z), max(y, z)) : INT32_MAX;
        cnt += (int64_t)(t >> 32) < e && adjy && oyz < (int32_t)e;
      }
      if (b > 0)
        for (int32_t k = oy0 + sl; k < oy1; k += 8) {
          const uint64_t t = ly[k];
          const int z = (int)(t & 0xffffu);
          cnt += (int64_t)(t >> 32) < e && ((rx[z >> 5] >> (z & 31)) & 1u);
        }
    }
    cnt += __shfl_xor_sync(0xffffffffu, cnt, 1);
    cnt += __shfl_xor_sync(0xffffffffu, cnt, 2);
    cnt += __shfl_xor_sync(0xffffffffu, cnt, 4);
    if (sl == 0 && e < E) tcnt[e] = cnt;
  }
}

// Max-edge generation: an edge e = (x, y) per half-warp (16 lanes), edges in
// filtration order; its third vertices S_e = (Sx | Dx) & (Sy | Dy) in
// ascending z go out as keys (e << 32) | z at toff[e] on.  Lane s of the
// half owns the contiguous words [s K, s K + K) of both snapshot rows (K =
// Wp / 16, 16-byte loads); the bucket entries earlier than e are or-ed into
// two shared rows of the half; one scan of the lanes' bit counts places
// every lane's run of keys, which the lane writes in order.  The keys are
// in final (max-edge) order: no sort follows.
constexpr int MEG_KMAX = VR_MAX_POINTS / 32 / 16;  // words per lane and row at most

// Claimed key space (the generator run before any triangle count): a warp
// takes room for its edges' third vertices from one of CLAIM_CTRS counters
// (one 128-byte line each, chosen by the warp, so the atomics spread over
// L2), each owning a sub-buffer of sub_cap 16-bit slots.  It claims `chunk`
// slots at a time (or what its two current edges need, if more) and fills
// them over its iterations, so most iterations make no global atomic.  Edge
// e's third vertices, ascending, go to tz[kpos[e]] on and its count to
// tcnt[e]; a claim past its sub-buffer raises F_CLAIM and writes no vertex
// (the counts stay exact; the host then generates keys the counted way).
constexpr int CLAIM_CTRS = 32;
struct ClaimBuf {
  uint16_t *tz;
  int32_t *kpos;
  int32_t *tcnt;
  uint32_t *ctr;    // CLAIM_CTRS counters at a stride of 32 words, zero at the start
  int64_t sub_cap;  // 16-bit slots per counter
  int32_t chunk;    // slots a warp claims at a time (more when its two edges need more)
};

// KT: the key word (see k_tri_final_me); T: the key buffer's capacity in keys.
// K4: 16-byte chunks per lane and row, (Wp / 16 rounded up to whole chunks)
// / 4, from 1 to 4 (Wp <= 256).  CL: claimed key space (ClaimBuf; toff,
// tkeys, T and zbits unused), else keys at toff[e] from the triangle count.
template <typename KT, int K4, bool CL>
static __global__ void __launch_bounds__(256) k_tri_gen_me(const int32_t *everts, int64_t E, int W, int n,
                                                           const int32_t *nbr_ptr, const int64_t *toff, int64_t T,
                                                           KT *tkeys, int zbits, SnapIdx sx, DevStatus *st,
                                                           int force_lex, ClaimBuf cb) {
  pdl_entry();
  if (build_failed(st)) return;
  if (lex_mode(E, st->ngrades, force_lex)) return;  // (a launch ahead of the host's decision)
  constexpr int WMAX = VR_MAX_POINTS / 32;
  __shared__ uint4 drow[8][2][2 * WMAX / 4];  // per warp, per half: Dx then Dy (16-byte words)
  const int l = lane_id(), wid = threadIdx.x >> 5, half = l >> 4, s16 = l & 15;
  // Words per lane: K = 4 K4; a lane's chunks past Wp are neither loaded nor
  // used.
  static_assert(K4 >= 1 && 4 * K4 <= MEG_KMAX, "chunks per lane");
  constexpr int K = 4 * K4;
  const int Wp = sx.Wp;
  uint32_t *dx = (uint32_t *)drow[wid][half], *dy = dx + WMAX;
  const int64_t nwarps = (int64_t)gridDim.x * 8;
  const int hw = (int)((blockIdx.x * 8 + wid) % CLAIM_CTRS);
  int64_t cnext = 0, cend = 0;  // the warp's claimed slots [cnext, cend) in counter hw's space
  // Endpoints are loaded one iteration ahead.
  int64_t e = (blockIdx.x * 8 + wid) * 2 + half;
  int2 nxy = e < E ? ((const int2 *)everts)[e] : make_int2(0, 0);
  for (; e - half < E; e += nwarps * 2) {
    const bool live = e < E;
    const int x = nxy.x, y = nxy.y;
    const int b = live ? (int)((uint32_t)e / (uint32_t)sx.B) : 0;  // e < E < 2^31
    if (e + nwarps * 2 < E) nxy = ((const int2 *)everts)[e + nwarps * 2];
    // This lane's words [w0, w0 + K) of both rows (zero before the first
    // snapshot and past Wp), and its delta words cleared.
    const int w0 = s16 * K;
    uint32_t wx[K], wy[K];
    {
      const uint4 *vx = (const uint4 *)(sx.snap + ((int64_t)(b > 0 ? b - 1 : 0) * n + x) * Wp + w0);
      const uint4 *vy = (const uint4 *)(sx.snap + ((int64_t)(b > 0 ? b - 1 : 0) * n + y) * Wp + w0);
      const bool in = live && b > 0;
#pragma unroll
      for (int q = 0; q < K4; ++q) {
        uint4 a = make_uint4(0u, 0u, 0u, 0u), c = a;
        if (in && w0 + 4 * q < Wp) {
          a = vx[q];
          c = vy[q];
        }
        wx[4 * q] = a.x; wx[4 * q + 1] = a.y; wx[4 * q + 2] = a.z; wx[4 * q + 3] = a.w;
        wy[4 * q] = c.x; wy[4 * q + 1] = c.y; wy[4 * q + 2] = c.z; wy[4 * q + 3] = c.w;
        ((uint4 *)(dx + w0))[q] = make_uint4(0u, 0u, 0u, 0u);
        ((uint4 *)(dy + w0))[q] = make_uint4(0u, 0u, 0u, 0u);
      }
    }
    __syncwarp();
    if (live) {
      const int32_t *ox = sx.boff + (int64_t)x * (sx.S + 1) + b, *oy = sx.boff + (int64_t)y * (sx.S + 1) + b;
      const uint64_t *lx = sx.bl + nbr_ptr[x], *ly = sx.bl + nbr_ptr[y];
      const int32_t ox1 = ox[1], oy1 = oy[1];
      for (int32_t k = ox[0] + s16; k < ox1; k += 16) {
        const uint64_t t = lx[k];
        if ((int64_t)(t >> 32) < e) atomicOr(&dx[(t & 0xffffu) >> 5], 1u << (t & 31));
      }
      for (int32_t k = oy[0] + s16; k < oy1; k += 16) {
        const uint64_t t = ly[k];
        if ((int64_t)(t >> 32) < e) atomicOr(&dy[(t & 0xffffu) >> 5], 1u << (t & 31));
      }
    }
    __syncwarp();
    int c = 0;
#pragma unroll
    for (int q = 0; q < K4; ++q) {
      {
        const uint4 ddx = ((const uint4 *)(dx + w0))[q], ddy = ((const uint4 *)(dy + w0))[q];
        wx[4 * q] = (wx[4 * q] | ddx.x) & (wy[4 * q] | ddy.x);
        wx[4 * q + 1] = (wx[4 * q + 1] | ddx.y) & (wy[4 * q + 1] | ddy.y);
        wx[4 * q + 2] = (wx[4 * q + 2] | ddx.z) & (wy[4 * q + 2] | ddy.z);
        wx[4 * q + 3] = (wx[4 * q + 3] | ddx.w) & (wy[4 * q + 3] | ddy.w);
        c += __popc(wx[4 * q]) + __popc(wx[4 * q + 1]) + __popc(wx[4 * q + 2]) + __popc(wx[4 * q + 3]);
      }
    }
    int inc = c;  // inclusive scan over the half's 16 lanes
#pragma unroll
    for (int d = 1; d < 16; d <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, inc, d, 16);
      if (s16 >= d) inc += v;
    }
    if constexpr (CL) {
      // The half-warps' totals; a new claim when the warp's slots run short.
      const int t0 = __shfl_sync(0xffffffffu, inc, 15), t1 = __shfl_sync(0xffffffffu, inc, 31);
      const int need = t0 + t1;
      if (cnext + need > cend) {
        const int len = max(need, cb.chunk);
        uint32_t base = 0;
        if (l == 0) base = atomicAdd(cb.ctr + hw * 32, (uint32_t)len);
        cnext = __shfl_sync(0xffffffffu, base, 0);
        cend = cnext + len;
      }
      const bool fits = cend <= cb.sub_cap;
      const int64_t hb = (int64_t)hw * cb.sub_cap + cnext + (half ? t0 : 0);
      cnext += need;
      if (live && s16 == 0) {
        cb.tcnt[e] = half ? t1 : t0;
        cb.kpos[e] = (int32_t)hb;
      }
      if (!fits) {
        if (l == 0) raise_flag(st, F_CLAIM);
      } else if (live && c) {
        unsigned short *out = (unsigned short *)cb.tz + hb + inc - c;
#pragma unroll
        for (int k = 0; k < K; ++k) {
          const uint32_t zb = (uint32_t)(w0 + k) * 32u - 1u;
          for (uint32_t mm = wx[k]; mm; mm &= mm - 1) __stcs(out++, (unsigned short)(zb + __ffs(mm)));
        }
      }
    } else if (live && c) {
      const int64_t p = toff[e] + inc - c;
      if (p + c <= T) {
        if constexpr (sizeof(KT) == 8) {
          // Key (e << 32) | z stored as its two 32-bit halves.
          uint2 *out = (uint2 *)(tkeys + p);
          const uint32_t eh = (uint32_t)e;
#pragma unroll
          for (int k = 0; k < K; ++k) {
            const uint32_t zb = (uint32_t)(w0 + k) * 32u - 1u;
            for (uint32_t mm = wx[k]; mm; mm &= mm - 1) __stcs(out++, make_uint2(zb + __ffs(mm), eh));
          }
        } else {
          // Key (e << zbits) | z (z < 2^zbits).
          unsigned int *out = (unsigned int *)(tkeys + p);
          const uint32_t ek = ((uint32_t)e << zbits) - 1u;
#pragma unroll
          for (int k = 0; k < K; ++k) {
            const uint32_t zb = ek + (uint32_t)(w0 + k) * 32u;
            for (uint32_t mm = wx[k]; mm; mm &= mm - 1) __stcs(out++, zb + __ffs(mm));
          }
        }
      } else {
        raise_flag(st, F_INTERNAL);  // never write past the key array
      }
    }
    __syncwarp();
  }
}

// Lex-order generation: warp per edge (a, b), taken in lexicographic order
// (lexe); its triangles (a, b, c), c > b ascending, land at toff[e]; the key
// carries the triangle's grade (largest of its three edge grades).
// Coalesced chunked stores.  T: the key buffer's capacity
// (at least the triangle count).
template <bool DENSE>
static __global__ void __launch_bounds__(256) k_lex_tri_gen(const uint32_t *lexe, const int32_t *egrade, int64_t E,
                                                            const uint32_t *adj, const int32_t *adjpre, int W,
                                                            const int32_t *nbr_ptr, const int32_t *nbr_ord,
                                                            const int64_t *toff, int64_t T, uint64_t *tkeys,
                                                            EdgeIndex ex, DevStatus *st, int force_lex,
                                                            const int64_t *lex_ptr, int sparse) {
  pdl_entry();
  if (build_failed(st)) return;
  if (!lex_mode(E, st->ngrades, force_lex)) return;  // max-edge order (a launch ahead of the host's decision)
  if (sparse) {
    // Sparse rows (as in k_tri_count): the candidates c of edge (a, b) are
    // the lexicographic edges after it in row a, ascending; lane q tests the
    // q-th in row b, and the kept ones of a round take consecutive slots.
    const int l = lane_id();
    const uint32_t lt = lanemask_lt();
    const int64_t nwarps = (int64_t)gridDim.x * 8;
    for (int64_t e = blockIdx.x * 8 + (threadIdx.x >> 5); e < E; e += nwarps) {
      const uint32_t ab = lexe[e];
      const int a = (int)(ab >> ID_BITS), b = (int)(ab & ID_MASK);
      const int64_t end = lex_ptr[a + 1];
      const uint32_t *rb = adj + (int64_t)b * W;
      int64_t t = toff[e];
      const uint64_t kab = lex3(a, b, 0);
      const int32_t gab = ex.grade<DENSE>(a, b);
      for (int64_t q0 = e + 1; q0 < end; q0 += 32) {
        const int64_t q = q0 + l;
        bool ok = false;
        int cv = 0;
        if (q < end) {
          cv = (int)(lexe[q] & ID_MASK);
          ok = (rb[cv >> 5] >> (cv & 31)) & 1u;
        }
        const uint32_t bal = __ballot_sync(0xffffffffu, ok);
        if (ok) {
          const int64_t p = t + __popc(bal & lt);
          const int32_t g = max(gab, max(ex.grade<DENSE>(a, cv), ex.grade<DENSE>(b, cv)));
          if (p < T) tkeys[p] = ((uint64_t)g << LEX_SHIFT) | kab | (uint64_t)cv;
          else raise_flag(st, F_INTERNAL);  // never write past the key array
        }
        t += __popc(bal);
      }
    }
    return;
  }
  // Per warp: the third vertices of one 32-word chunk's candidates
  // (bit_compact); lane q takes candidates q, q + 32, ...
  __shared__ uint16_t cbuf[8][CB_SLOTS];
  const int l = lane_id(), wid = threadIdx.x >> 5;
  uint16_t *cb = cbuf[wid];
  const int64_t nwarps = (int64_t)gridDim.x * 8;
  for (int64_t e = blockIdx.x * 8 + wid; e < E; e += nwarps) {
    const uint32_t ab = lexe[e];
    const int a = (int)(ab >> ID_BITS), b = (int)(ab & ID_MASK);
    const int64_t t0 = toff[e];
    uint64_t *out = tkeys + t0;
    int64_t room = T - t0;  // keys that fit from out on
    const uint64_t kab = lex3(a, b, 0);
    const uint32_t *ra = adj + (int64_t)a * W, *rb = adj + (int64_t)b * W;
    const int32_t *pa = adjpre + (int64_t)a * W, *pb = adjpre + (int64_t)b * W;
    const int32_t *oa = nbr_ord + nbr_ptr[a], *ob = nbr_ord + nbr_ptr[b];
    const int32_t *ga = DENSE ? ex.egd + (int64_t)a * ex.n : nullptr;
    const int32_t *gb = DENSE ? ex.egd + (int64_t)b * ex.n : nullptr;
    const int32_t gab = ex.grade<DENSE>(a, b);
    for (int w0 = (b >> 5); w0 < W; w0 += 32) {
      const int w = w0 + l;
      const uint32_t vm = w < W ? (ra[w] & rb[w] & above_mask(b, w)) : 0u;
      const int tot = bit_compact(vm, w, cb);
      if (tot == 0) continue;
      __syncwarp();
      for (int q = l; q < tot; q += 32) {
        const int cv = cb[q];
        int32_t gac, gbc;
        if constexpr (DENSE) {
          gac = ga[cv];
          gbc = gb[cv];
        } else {
          const int ww = cv >> 5;
          const uint32_t below = (1u << (cv & 31)) - 1u;
          gac = egrade[oa[pa[ww] + __popc(ra[ww] & below)]];
          gbc = egrade[ob[pb[ww] + __popc(rb[ww] & below)]];
        }
        const int32_t g = max(gab, max(gac, gbc));
        if (q < room) out[q] = ((uint64_t)g << LEX_SHIFT) | kab | (uint64_t)cv;
        else raise_flag(st, F_INTERNAL);  // never write past the key array
      }
      __syncwarp();
      out += tot;
      room -= tot;
    }
  }
}

// Final write of lex-mode triangles, sorted by (grade, a, b, c): verts,
// grade, colptr and the boundary column (order indices of the three faces,
// ascending).  The output arrays start 16-byte aligned; a scalar tail.
__device__ __forceinline__ void tri_final_one(uint64_t k, const EdgeIndex &ex, int32_t *v, int32_t *r, int32_t &g,
                                              bool dense) {
  const int a = (int)((k >> (2 * ID_BITS)) & ID_MASK), b = (int)((k >> ID_BITS) & ID_MASK), c = (int)(k & ID_MASK);
  const int32_t o0 = dense ? ex.ord<true>(a, b) : ex.ord<false>(a, b);
  const int32_t o1 = dense ? ex.ord<true>(a, c) : ex.ord<false>(a, c);
  const int32_t o2 = dense ? ex.ord<true>(b, c) : ex.ord<false>(b, c);
  const int32_t lo = min(o0, min(o1, o2)), hi = max(o0, max(o1, o2));
  v[0] = a; v[1] = b; v[2] = c;
  r[0] = lo; r[1] = o0 + o1 + o2 - lo - hi; r[2] = hi;
  g = (int32_t)(k >> LEX_SHIFT);
}

// A warp takes 128 consecutive sorted triangles: lane l the pairs at 2l and
// 64 + 2l (16-byte key loads, consecutive lanes on consecutive addresses).
// Grades and colptr go out directly (8- and 16-byte stores, coalesced); the
// vertices and boundary rows (12 bytes per triangle) are staged in shared
// memory and written as 16-byte words by consecutive lanes, so every store
// instruction covers whole sectors (the kernel is bound by L1 sector
// throughput: the three order lookups per triangle are scattered).
template <bool DENSE>
static __global__ void __launch_bounds__(256) k_tri_final(const uint64_t *tkeys, int64_t T, EdgeIndex ex,
                                                          int32_t *tverts, int32_t *tgrade, int64_t *tcolptr,
                                                          int32_t *trow,
    const DevStatus *st) {
  pdl_entry();
  if (build_failed(st)) return;
  __shared__ int4 sv[8][96], sr[8][96];  // per warp: 128 triangles x 3 ints
  const int wid = threadIdx.x >> 5, l = lane_id();
  int32_t *svi = (int32_t *)sv[wid], *sri = (int32_t *)sr[wid];
  // Lane l takes triangles l, l + 32, l + 64, l + 96 of a chunk of 128
  // (coalesced 8-byte key loads; staging at stride 3 words, no bank
  // conflicts).
  const int64_t nch = T / 128;
  for (int64_t ch = blockIdx.x * 8 + wid; ch < nch; ch += (int64_t)gridDim.x * 8) {
    const int64_t base = ch * 128;
    uint64_t kk[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) kk[u] = tkeys[base + 32 * u + l];
    int32_t v[12], r[12], g[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) tri_final_one(kk[u], ex, v + 3 * u, r + 3 * u, g[u], DENSE);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int t = 32 * u + l;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        svi[3 * t + k] = v[3 * u + k];
        sri[3 * t + k] = r[3 * u + k];
      }
      tgrade[base + t] = g[u];
      tcolptr[base + t] = 3 * (base + t);
    }
    __syncwarp();
    int4 *gv = (int4 *)(tverts + 3 * base), *gr = (int4 *)(trow + 3 * base);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      gv[32 * k + l] = sv[wid][32 * k + l];
      gr[32 * k + l] = sr[wid][32 * k + l];
    }
    __syncwarp();
  }
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t p = nch * 128 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < T; p += stride) {
    int32_t v[3], r[3], g;
    tri_final_one(tkeys[p], ex, v, r, g, DENSE);
    tverts[3 * p] = v[0]; tverts[3 * p + 1] = v[1]; tverts[3 * p + 2] = v[2];
    trow[3 * p] = r[0]; trow[3 * p + 1] = r[1]; trow[3 * p + 2] = r[2];
    tgrade[p] = g;
    tcolptr[p] = 3 * p;
  }
}

// Final write of max-edge keys (e << 32) | z, already in (grade, lex) order
// up to tie groups: the edge's endpoints from the edge list, the two other
// faces' order indices from the neighbour CSR rows of x and of y (never the
// dense table).  Consecutive triangles mostly share their edge (x, y) and
// their z ascend, so a warp's 32 lookups fall in x's and y's compact rows (a
// few hundred bytes each: adjacency word, its prefix, the order entry) and
// the L1 sends a few line requests to L2 where the dense table's row would
// cost a 32-byte sector per lookup.  Same store pattern as k_tri_final (128
// triangles per warp, vertices and rows staged in shared memory for 16-byte
// stores).
// Triangle {x, y, z} with largest edge e = (x, y): sorted vertices and the
// ascending order indices of its faces.
__device__ __forceinline__ void tri_final_xyz(int32_t e, int x, int y, int z, const EdgeIndex &ex, int32_t *v,
                                              int32_t *r) {
  const int2 px = ex.adjx[(int64_t)x * ex.W + (z >> 5)], py = ex.adjx[(int64_t)y * ex.W + (z >> 5)];
  const uint32_t below = (1u << (z & 31)) - 1u;
  const int32_t oxz = ex.nbr_ord[ex.nbr_ptr[x] + px.y + __popc((uint32_t)px.x & below)];
  const int32_t oyz = ex.nbr_ord[ex.nbr_ptr[y] + py.y + __popc((uint32_t)py.x & below)];
  if (z < x) { v[0] = z; v[1] = x; v[2] = y; }
  else if (z < y) { v[0] = x; v[1] = z; v[2] = y; }
  else { v[0] = x; v[1] = y; v[2] = z; }
  r[0] = min(oxz, oyz); r[1] = max(oxz, oyz); r[2] = e;
}

__device__ __forceinline__ void tri_final_ez(int32_t e, int z, const int32_t *everts, const int32_t *egrade,
                                             const EdgeIndex &ex, int32_t *v, int32_t *r, int32_t &g) {
  const int2 xy = ((const int2 *)everts)[e];
  tri_final_xyz(e, xy.x, xy.y, z, ex, v, r);
  g = egrade[e];
}

__device__ __forceinline__ void tri_final_me_one(uint64_t k, int zbits, const int32_t *everts,
                                                 const int32_t *egrade, const EdgeIndex &ex, int32_t *v, int32_t *r,
                                                 int32_t &g) {
  tri_final_ez((int32_t)(k >> zbits), (int)(k & ((1ull << min(zbits, 16)) - 1ull)), everts, egrade, ex, v, r, g);
}

// KT: the key word, uint64_t ((e << 32) | z, zbits = 32) or uint32_t
// ((e << zbits) | z, when the edge count fits the bits that n leaves).
template <typename KT>
static __global__ void __launch_bounds__(256, 4) k_tri_final_me(const KT *tkeys, int zbits, int64_t T,
                                                                const int32_t *everts, const int32_t *egrade,
                                                                EdgeIndex ex, int32_t *tverts, int32_t *tgrade,
                                                                int64_t *tcolptr, int32_t *trow, const DevStatus *st) {
  pdl_entry();
  if (build_failed(st)) return;
  __shared__ int4 sv[8][96], sr[8][96];  // per warp: 128 triangles x 3 ints
  const int wid = threadIdx.x >> 5, l = lane_id();
  int32_t *svi = (int32_t *)sv[wid], *sri = (int32_t *)sr[wid];
  const int64_t nch = T / 128, cstride = (int64_t)gridDim.x * 8;
  // Keys are read once and the outputs written once: streaming hints keep
  // them from evicting the order table the lookups need from L2.  The next
  // chunk's keys are loaded while this one is processed.
  // Lane l takes triangles l, l + 32, l + 64, l + 96 of a chunk of 128:
  // coalesced key loads, and staging at stride 3 words (no bank conflicts).
  int64_t ch = blockIdx.x * 8 + wid;
  KT nk[4] = {0, 0, 0, 0};
  if (ch < nch) {
#pragma unroll
    for (int u = 0; u < 4; ++u) nk[u] = __ldcs(tkeys + ch * 128 + 32 * u + l);
  }
  for (; ch < nch; ch += cstride) {
    const int64_t base = ch * 128;
    KT kk[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) kk[u] = nk[u];
    if (ch + cstride < nch) {
#pragma unroll
      for (int u = 0; u < 4; ++u) nk[u] = __ldcs(tkeys + (ch + cstride) * 128 + 32 * u + l);
    }
    int32_t v[12], r[12], g[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) tri_final_me_one(kk[u], zbits, everts, egrade, ex, v + 3 * u, r + 3 * u, g[u]);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int t = 32 * u + l;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        svi[3 * t + k] = v[3 * u + k];
        sri[3 * t + k] = r[3 * u + k];
      }
      __stcs(tgrade + base + t, g[u]);
      __stcs((long long *)tcolptr + base + t, (long long)(3 * (base + t)));
    }
    __syncwarp();
    int4 *gv = (int4 *)(tverts + 3 * base), *gr = (int4 *)(trow + 3 * base);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      __stcs(gv + 32 * k + l, sv[wid][32 * k + l]);
      __stcs(gr + 32 * k + l, sr[wid][32 * k + l]);
    }
    __syncwarp();
  }
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t p = nch * 128 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < T; p += stride) {
    int32_t v[3], r[3], g;
    tri_final_me_one(tkeys[p], zbits, everts, egrade, ex, v, r, g);
    tverts[3 * p] = v[0]; tverts[3 * p + 1] = v[1]; tverts[3 * p + 2] = v[2];
    trow[3 * p] = r[0]; trow[3 * p + 1] = r[1]; trow[3 * p + 2] = r[2];
    tgrade[p] = g;
    tcolptr[p] = 3 * p;
  }
}

// Final write over claimed key space.  Edge e's third vertices are the
// 16-bit values at tz[kpos[e]] on (tcnt[e] of them, ascending) and its
// triangles take output positions toff[e] on.  A warp takes 32 consecutive
// edges: lane l holds edge e0 + l's endpoints, grade, count and key position
// in registers, and the group's triangles fill the contiguous output range
// toff[e0] .. toff[e0] + S.  The warp walks that range by the 128-position
// chunks of the whole output; lane l takes positions l, l + 32, l + 64,
// l + 96 of a chunk and finds each one's edge by a five-step search over the
// lanes' inclusive counts (shuffles only), so the only load before the face
// lookups is the third vertex.  The faces come from the CSR rows of x and y
// as in k_tri_final_me; chunks inside the range are staged in shared memory
// for 16-byte stores, the (at most two) chunks the range shares with its
// neighbours' are stored position by position.  ticket: a zeroed word.
static __global__ void __launch_bounds__(256, 4) k_tri_final_grp(const uint16_t *__restrict__ tz,
                                                                 const int32_t *__restrict__ kpos,
                                                                 const int32_t *__restrict__ tcnt,
                                                                 const int64_t *__restrict__ toff, int64_t E,
                                                                 const int32_t *everts, const int32_t *egrade,
                                                                 EdgeIndex ex, int32_t *tverts, int32_t *tgrade,
                                                                 int64_t *tcolptr, int32_t *trow,
                                                                 uint32_t *ticket, const DevStatus *st) {
  pdl_entry();
  if (build_failed(st)) return;
  __shared__ int4 sv[8][96], sr[8][96];  // per warp: 128 triangles x 3 ints
  const int wid = threadIdx.x >> 5, l = lane_id();
  int32_t *svi = (int32_t *)sv[wid], *sri = (int32_t *)sr[wid];
  // Groups are taken from a ticket (zero at the start), last group first:
  // the late edges of the filtration carry most triangles, so the heavy
  // groups go out first and the light ones even out the end.
  const int64_t ngroups = (E + 31) / 32;
  for (;;) {
    uint32_t tk = 0;
    if (l == 0) tk = atomicAdd(ticket, 1u);
    tk = __shfl_sync(0xffffffffu, tk, 0);
    if ((int64_t)tk >= ngroups) break;
    const int64_t e0 = (ngroups - 1 - (int64_t)tk) * 32;
    const int64_t e = e0 + l;
    const bool ev = e < E;
    const int32_t c = ev ? tcnt[e] : 0;
    const int32_t kp = ev ? kpos[e] : 0;
    const int2 xy = ev ? ((const int2 *)everts)[e] : make_int2(0, 0);
    const int32_t ge = ev ? egrade[e] : 0;
    const int64_t o0 = toff[e0];
    int32_t incl = c;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int32_t t = __shfl_up_sync(0xffffffffu, incl, d);
      if (l >= d) incl += t;
    }
    const int32_t excl = incl - c;
    const int32_t npx = ev ? ex.nbr_ptr[xy.x] : 0, npy = ev ? ex.nbr_ptr[xy.y] : 0;
    const int64_t oend = o0 + __shfl_sync(0xffffffffu, incl, 31);
    // Position p's edge j (lanes' inclusive counts at or below f = p - o0;
    // f < S keeps j <= 31) and third vertex, packed (j << 16) | z; the next
    // chunk's are fetched before this chunk's faces are looked up.
    auto fetch = [&](int64_t base, uint32_t *jz) {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int64_t p = base + 32 * u + l;
        const bool ok = p >= o0 && p < oend;
        const int32_t f = ok ? (int32_t)(p - o0) : 0;
        int j = 0;
#pragma unroll
        for (int step = 16; step; step >>= 1)
          if (__shfl_sync(0xffffffffu, incl, j + step - 1) <= f) j += step;
        const int32_t ej = __shfl_sync(0xffffffffu, excl, j), kj = __shfl_sync(0xffffffffu, kp, j);
        jz[u] = ((uint32_t)j << 16) | (ok ? (uint32_t)__ldcs(tz + kj + (f - ej)) : 0u);
      }
    };
    uint32_t jzc[4];
    fetch(o0 & ~int64_t(127), jzc);
    for (int64_t base = o0 & ~int64_t(127); base < oend; base += 128) {
      uint32_t jzn[4] = {0u, 0u, 0u, 0u};
      if (base + 128 < oend) fetch(base + 128, jzn);
      // The four positions' row words {adjacency word, prefix count} of x
      // and y are all loaded before any order entry (eight loads in flight
      // per lane at each level).  A position outside the range uses z = x:
      // x is one of y's neighbours and has y above it, so both lookups stay
      // inside the rows of x and y (the result is not stored).
      int32_t v[12], r[12], g[4];
      int2 pxa[4], pya[4];
      int32_t nxa[4], nya[4], za[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int64_t p = base + 32 * u + l;
        const bool ok = p >= o0 && p < oend;
        const int j = (int)(jzc[u] >> 16);
        const int xj = __shfl_sync(0xffffffffu, xy.x, j), yj = __shfl_sync(0xffffffffu, xy.y, j);
        nxa[u] = __shfl_sync(0xffffffffu, npx, j);
        nya[u] = __shfl_sync(0xffffffffu, npy, j);
        g[u] = __shfl_sync(0xffffffffu, ge, j);
        const int z = ok ? (int)(jzc[u] & 0xffffu) : xj;
        za[u] = z;
        pxa[u] = ex.adjx[(int64_t)xj * ex.W + (z >> 5)];
        pya[u] = ex.adjx[(int64_t)yj * ex.W + (z >> 5)];
        if (z < xj) { v[3 * u] = z; v[3 * u + 1] = xj; v[3 * u + 2] = yj; }
        else if (z < yj) { v[3 * u] = xj; v[3 * u + 1] = z; v[3 * u + 2] = yj; }
        else { v[3 * u] = xj; v[3 * u + 1] = yj; v[3 * u + 2] = z; }
        r[3 * u + 2] = (int32_t)(e0 + j);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const uint32_t below = (1u << (za[u] & 31)) - 1u;
        const int32_t oxz = ex.nbr_ord[nxa[u] + pxa[u].y + __popc((uint32_t)pxa[u].x & below)];
        const int32_t oyz = ex.nbr_ord[nya[u] + pya[u].y + __popc((uint32_t)pya[u].x & below)];
        r[3 * u] = min(oxz, oyz);
        r[3 * u + 1] = max(oxz, oyz);
      }
      if (base >= o0 && base + 128 <= oend) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int t = 32 * u + l;
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            svi[3 * t + k] = v[3 * u + k];
            sri[3 * t + k] = r[3 * u + k];
          }
          __stcs(tgrade + base + t, g[u]);
          __stcs((long long *)tcolptr + base + t, (long long)(3 * (base + t)));
        }
        __syncwarp();
        int4 *gv = (int4 *)(tverts + 3 * base), *gr = (int4 *)(trow + 3 * base);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          __stcs(gv + 32 * k + l, sv[wid][32 * k + l]);
          __stcs(gr + 32 * k + l, sr[wid][32 * k + l]);
        }
        __syncwarp();
      } else {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int64_t p = base + 32 * u + l;
          if (p >= o0 && p < oend) {
            tverts[3 * p] = v[3 * u]; tverts[3 * p + 1] = v[3 * u + 1]; tverts[3 * p + 2] = v[3 * u + 2];
            trow[3 * p] = r[3 * u]; trow[3 * p + 1] = r[3 * u + 1]; trow[3 * p + 2] = r[3 * u + 2];
            tgrade[p] = g[u];
            tcolptr[p] = 3 * p;
          }
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) jzc[u] = jzn[u];
    }
  }
}

// Per grade group: the triangles of a group that spans several edges with
// triangles must be merged into lexicographic order.  Queue such groups by
// size class: small (CTA sort in 24 KB of shared memory), mid (192 KB), big
// (one CTA per group, global temporaries).
constexpr int TRI_SMALL = 1024;
constexpr int TRI_MID = 8192;

static __global__ void k_tri_groups(const int32_t *gstart, const int32_t *tcnt, const int64_t *toff, int32_t *smallq,
                                    int32_t *midq, int32_t *bigq, DevStatus *st, int force_lex) {
  pdl_entry();
  if (build_failed(st)) return;
  if (blockIdx.x == 0 && threadIdx.x == 0) st->T = toff[st->E];  // triangle count
  const int64_t ngrades = st->ngrades;
  if (lex_mode(st->E, ngrades, force_lex)) return;  // lex mode needs no merge
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < ngrades; g += (int64_t)gridDim.x * blockDim.x) {
    const int32_t b = gstart[g], e = gstart[g + 1];
    if (e - b < 2) continue;
    int runs = 0;
    for (int32_t x = b; x < e && runs < 2; ++x) runs += tcnt[x] > 0;
    if (runs < 2) continue;
    const int64_t s = toff[e] - toff[b];
    if (s <= TRI_SMALL) {
      smallq[atomicAdd(&st->small_seg_count, 1)] = (int32_t)g;
    } else if (s <= TRI_MID) {
      midq[atomicAdd(&st->mid_seg_count, 1)] = (int32_t)g;
    } else {
      int q = (int)atomicAdd((unsigned long long *)&st->big_seg_count, 1ull);
      bigq[q] = (int32_t)g;
      atomicMax((unsigned long long *)&st->big_seg_max, (unsigned long long)s);
      atomicAdd((unsigned long long *)&st->big_seg_total, (unsigned long long)s);
    }
  }
}

// CTA per queued group: sort the segment by lexicographic key in shared
// memory and rewrite verts and rowidx (grade and colptr do not change).
// Dynamic shared memory: CAP * (8 + 4 + 12) bytes.
template <int CAP>
static __global__ void k_tri_fix_smem(const int32_t *gstart, const int64_t *toff, const int32_t *queue,
                                      const int32_t *count, int32_t *tverts, int32_t *trow,
    const DevStatus *st) {
  pdl_entry();
  if (build_failed(st)) return;
  extern __shared__ unsigned char smem[];
  uint64_t *key = (uint64_t *)smem;              // CAP
  uint32_t *val = (uint32_t *)(key + CAP);       // CAP
  int32_t *rows = (int32_t *)(val + CAP);        // 3 * CAP
  const int nq = *count;
  for (int q = blockIdx.x; q < nq; q += gridDim.x) {
    const int g = queue[q];
    const int64_t s0 = toff[gstart[g]];
    const int s = (int)(toff[gstart[g + 1]] - s0);
    int cap = 1;
    while (cap < s) cap <<= 1;
    for (int t = threadIdx.x; t < cap; t += blockDim.x) {
      if (t < s) {
        key[t] = lex3(tverts[3 * (s0 + t)], tverts[3 * (s0 + t) + 1], tverts[3 * (s0 + t) + 2]);
      } else {
        key[t] = ~0ull;
      }
      val[t] = t;
    }
    for (int t = threadIdx.x; t < 3 * s; t += blockDim.x) rows[t] = trow[3 * s0 + t];
    __syncthreads();
    cta_bitonic(key, val, cap);
    for (int t = threadIdx.x; t < s; t += blockDim.x) {
      const uint64_t k = key[t];
      const int64_t p = s0 + t;
      tverts[3 * p] = (int32_t)(k >> (2 * ID_BITS));
      tverts[3 * p + 1] = (int32_t)((k >> ID_BITS) & ID_MASK);
      tverts[3 * p + 2] = (int32_t)(k & ID_MASK);
      const uint32_t v = val[t];
      trow[3 * p] = rows[3 * v];
      trow[3 * p + 1] = rows[3 * v + 1];
      trow[3 * p + 2] = rows[3 * v + 2];
    }
    __syncthreads();
  }
}

// CTA per queued large group (in parallel): stable LSD sort of the 39-bit
// lexicographic keys through global temporaries indexed by absolute triangle
// position (each group owns the slice of its own segment).
static __global__ void __launch_bounds__(RS_THREADS) k_tri_fix_big(const int32_t *gstart, const int64_t *toff,
                                                                   const int32_t *bigq, const DevStatus *st,
                                                                   int32_t *tverts, int32_t *trow, uint64_t *k1,
                                                                   uint32_t *v1, uint64_t *k2, uint32_t *v2,
                                                                   int32_t *rtmp) {
  pdl_entry();
  if (build_failed(st)) return;
  const int nq = (int)st->big_seg_count;
  for (int q = blockIdx.x; q < nq; q += gridDim.x) {
    const int g = bigq[q];
    const int64_t s0 = toff[gstart[g]];
    const int64_t s = toff[gstart[g + 1]] - s0;
    uint64_t *K1 = k1 + s0, *K2 = k2 + s0;
    uint32_t *V1 = v1 + s0, *V2 = v2 + s0;
    int32_t *R = rtmp + 3 * s0;
    for (int64_t t = threadIdx.x; t < s; t += blockDim.x) {
      const int64_t p = s0 + t;
      K1[t] = lex3(tverts[3 * p], tverts[3 * p + 1], tverts[3 * p + 2]);
      V1[t] = (uint32_t)t;
      R[3 * t] = trow[3 * p];
      R[3 * t + 1] = trow[3 * p + 1];
      R[3 * t + 2] = trow[3 * p + 2];
    }
    __syncthreads();
    cta_radix_sort_global(K1, V1, K2, V2, s, 0, 3 * ID_BITS);
    for (int64_t t = threadIdx.x; t < s; t += blockDim.x) {
      const uint64_t k = K1[t];
      const int64_t p = s0 + t;
      tverts[3 * p] = (int32_t)(k >> (2 * ID_BITS));
      tverts[3 * p + 1] = (int32_t)((k >> ID_BITS) & ID_MASK);
      tverts[3 * p + 2] = (int32_t)(k & ID_MASK);
      const uint32_t v = V1[t];
      trow[3 * p] = R[3 * v];
      trow[3 * p + 1] = R[3 * v + 1];
      trow[3 * p + 2] = R[3 * v + 2];
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------- tetrahedra
// Tetrahedron (a,b,c,d), a<b<c<d: present iff its six edges are kept; grade =
// the largest edge grade.  Generated from the triangles in lexicographic
// order: triangle (a,b,c) at lexicographic position t takes the apexes d > c
// of N(a) & N(b) & N(c), so the tetrahedra come out in lexicographic order;
// a stable sort on the grade gives (grade, lex).  Faces are found through the
// triangles' apex lists: the triangles whose first edge is (x,y) occupy
// positions toff[lex_pos(x,y)] .. toff[lex_pos(x,y)+1] of the lexicographic
// list, apexes ascending.

constexpr uint64_t LEX3_MASK = (1ull << LEX_SHIFT) - 1;

__device__ __forceinline__ void lex3_unpack(uint64_t k, int &a, int &b, int &c) {
  a = (int)((k >> (2 * ID_BITS)) & ID_MASK);
  b = (int)((k >> ID_BITS) & ID_MASK);
  c = (int)(k & ID_MASK);
}

// Per lexicographic edge e = (x, y): word by word, the number of common
// neighbours above y in the words below (16-bit: n <= 8192).  A triangle
// (x, y, z)'s rank among edge e's triangles (z ascending) is then one read
// of this table plus a popcount, instead of a bisection in the triangle keys.
static __global__ void __launch_bounds__(256) k_lex_pre(const uint32_t *lexe, int64_t E, const uint32_t *adj, int W,
                                                        uint16_t *pre,
    const DevStatus *st) {
  pdl_entry();
  if (build_failed(st)) return;
  const int l = lane_id();
  const int64_t nwarps = (int64_t)gridDim.x * 8;
  for (int64_t e = blockIdx.x * 8 + (threadIdx.x >> 5); e < E; e += nwarps) {
    const uint32_t ab = lexe[e];
    const int x = (int)(ab >> ID_BITS), y = (int)(ab & ID_MASK);
    const uint32_t *rx = adj + (int64_t)x * W, *ry = adj + (int64_t)y * W;
    int carry = 0;
    for (int w0 = 0; w0 < W; w0 += 32) {
      const int w = w0 + l;
      const int c = w < W ? __popc(rx[w] & ry[w] & above_mask(y, w)) : 0;
      const int inc = warp_incl_scan(c);
      if (w < W) pre[e * W + w] = (uint16_t)(carry + inc - c);
      carry += __shfl_sync(0xffffffffu, inc, 31);
    }
  }
}

// Lexicographic position of triangle (x,y,z), x<y<z, all edges kept: the
// first edge's triangle offset plus z's rank among that edge's triangles
// (from the prefix table when given, else a bisection in the keys).
__device__ __forceinline__ int64_t tri_lexpos(int x, int y, int z, const uint64_t *tk_lex, const int64_t *toff,
                                              const uint32_t *adj, const int32_t *adjpre, int W, const int32_t *deg,
                                              const int32_t *up, const int64_t *lex_ptr, const int32_t *elp, int n,
                                              const uint16_t *pre) {
  const int64_t lp = elp ? (int64_t)elp[(int64_t)x * n + y] : lex_pos(x, y, adj, adjpre, W, deg, up, lex_ptr);
  if (pre) {
    const int w = z >> 5;
    const uint32_t m = adj[(int64_t)x * W + w] & adj[(int64_t)y * W + w] & above_mask(y, w) & ((1u << (z & 31)) - 1u);
    return toff[lp] + pre[lp * W + w] + __popc(m);
  }
  int64_t lo = toff[lp], hi = toff[lp + 1];
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if ((int)(tk_lex[mid] & ID_MASK) < z) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// Order index of each triangle by lexicographic position: the sorted
// triangle p has key (grade, lex3); its lexicographic position comes from the
// per-edge prefix table when there is one, else by bisection in the
// lexicographic key list.
static __global__ void k_tri_ordidx(const uint64_t *tk, int64_t T, const uint64_t *tk_lex, int32_t *ordidx,
                                    const int64_t *toff, const uint32_t *adj, const int32_t *adjpre, int W,
                                    const int32_t *deg, const int32_t *up, const int64_t *lex_ptr, const int32_t *elp,
                                    int n, const uint16_t *pre,
    const DevStatus *st) {
  pdl_entry();
  if (build_failed(st)) return;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < T; p += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t x = tk[p] & LEX3_MASK;
    int64_t lo;
    if (pre) {
      int a, b, c;
      lex3_unpack(x, a, b, c);
      lo = tri_lexpos(a, b, c, tk_lex, toff, adj, adjpre, W, deg, up, lex_ptr, elp, n, pre);
    } else {
      int64_t hi = T;
      lo = 0;
      while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if ((tk_lex[mid] & LEX3_MASK) < x) lo = mid + 1;
        else hi = mid;
      }
    }
    ordidx[lo] = (int32_t)p;
  }
}

// Tetrahedra per lexicographic triangle (warp per triangle).
static __global__ void __launch_bounds__(256) k_tet_count(const uint64_t *tk_lex, int64_t T, const uint32_t *adj,
                                                          int W, int32_t *cnt4,
    const DevStatus *st) {
  pdl_entry();
  if (build_failed(st)) return;
  const int l = lane_id();
  const int64_t nwarps = (int64_t)gridDim.x * 8;
  // Four triangles per warp at a time, their first-round loads in flight
  // together (as in k_tri_count's lex path).
  constexpr int U = 4;
  for (int64_t t0 = (blockIdx.x * 8 + (threadIdx.x >> 5)) * (int64_t)U; t0 < T; t0 += nwarps * U) {
    int a[U], b[U], c[U], n4[U];
#pragma unroll
    for (int u = 0; u < U; ++u) lex3_unpack(t0 + u < T ? tk_lex[t0 + u] : 0ull, a[u], b[u], c[u]);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int w = (c[u] >> 5) + l;
      n4[u] = t0 + u < T && w < W
                  ? __popc(adj[(int64_t)a[u] * W + w] & adj[(int64_t)b[u] * W + w] & adj[(int64_t)c[u] * W + w] &
                           above_mask(c[u], w))
                  : 0;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const uint32_t *ra = adj + (int64_t)a[u] * W, *rb = adj + (int64_t)b[u] * W, *rc = adj + (int64_t)c[u] * W;
      for (int w = (c[u] >> 5) + l + 32; t0 + u < T && w < W; w += 32) n4[u] += __popc(ra[w] & rb[w] & rc[w]);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) n4[u] = warp_sum(n4[u]);
    if (l < U && t0 + l < T) cnt4[t0 + l] = l == 0 ? n4[0] : l == 1 ? n4[1] : l == 2 ? n4[2] : n4[3];
  }
}

// Keys in lexicographic order.  packed (grades below 2^12): grade << 52 |
// a,b,c,d (13 bits each), so the sorted keys carry the vertices; otherwise
// grade << 32 | lexicographic position q, with the packed vertices at lex4[q].
constexpr int TET_PACK_SHIFT = 4 * ID_BITS;
template <bool DENSE>
static __global__ void __launch_bounds__(256) k_tet_gen(const uint64_t *tk_lex, int64_t T, const uint32_t *adj,
                                                        int W, const int32_t *tgrade, const int32_t *ordidx,
                                                        const int32_t *egrade, EdgeIndex ex, const int64_t *off4,
                                                        int64_t T4, uint64_t *keys4, uint64_t *lex4, int packed,
                                                        DevStatus *st) {
  pdl_entry();
  if (build_failed(st)) return;
  __shared__ uint16_t cbuf[8][CB_SLOTS];  // per warp: one chunk's fourth vertices (bit_compact)
  const int l = lane_id(), wid = threadIdx.x >> 5;
  uint16_t *cb = cbuf[wid];
  const int64_t nwarps = (int64_t)gridDim.x * 8;
  for (int64_t t = blockIdx.x * 8 + wid; t < T; t += nwarps) {
    const uint64_t k3 = tk_lex[t] & LEX3_MASK;
    int a, b, c;
    lex3_unpack(k3, a, b, c);
    const int32_t g3 = tgrade[ordidx[t]];
    const uint32_t *ra = adj + (int64_t)a * W, *rb = adj + (int64_t)b * W, *rc = adj + (int64_t)c * W;
    int64_t q0 = off4[t];
    for (int w0 = c >> 5; w0 < W; w0 += 32) {
      const int w = w0 + l;
      const uint32_t vm = w < W ? (ra[w] & rb[w] & rc[w] & above_mask(c, w)) : 0u;
      const int tot = bit_compact(vm, w, cb);
      if (tot == 0) continue;
      __syncwarp();
      for (int qq = l; qq < tot; qq += 32) {
        const int d = cb[qq];
        int32_t g = g3;
        g = max(g, ex.grade<DENSE>(a, d));
        g = max(g, ex.grade<DENSE>(b, d));
        g = max(g, ex.grade<DENSE>(c, d));
        const int64_t q = q0 + qq;
        if (q < T4) {
          const uint64_t v4 = (k3 << ID_BITS) | (uint64_t)d;
          if (packed) {
            keys4[q] = ((uint64_t)(uint32_t)g << TET_PACK_SHIFT) | v4;
          } else {
            keys4[q] = ((uint64_t)(uint32_t)g << 32) | (uint64_t)q;
            lex4[q] = v4;
          }
        } else {
          raise_flag(st, F_INTERNAL);  // never write past the key arrays
        }
      }
      __syncwarp();
      q0 += tot;
    }
  }
}

// Final write of the tetrahedra in (grade, lex) order: vertices, grade,
// colptr and the boundary column (order indices of the four triangles,
// ascending); thread p also closes colptr at T4.
static __global__ void k_tet_final(const uint64_t *keys4, int64_t T4, const uint64_t *lex4, const uint64_t *tk_lex,
                                   const int64_t *toff, const uint32_t *adj, const int32_t *adjpre, int W,
                                   const int32_t *deg, const int32_t *up, const int64_t *lex_ptr,
                                   const int32_t *ordidx, const int32_t *elp, int n, int packed,
                                   const uint16_t *pre, int32_t *verts, int32_t *grade, int64_t *colptr,
                                   int32_t *rowidx,
    const DevStatus *st) {
  pdl_entry();
  if (build_failed(st)) return;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < T4; p += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t key = keys4[p];
    const uint64_t v = packed ? key & ((1ull << TET_PACK_SHIFT) - 1) : lex4[key & 0xffffffffull];
    const int d = (int)(v & ID_MASK);
    int a, b, c;
    lex3_unpack(v >> ID_BITS, a, b, c);
    int32_t r[4];
    r[0] = ordidx[tri_lexpos(b, c, d, tk_lex, toff, adj, adjpre, W, deg, up, lex_ptr, elp, n, pre)];
    r[1] = ordidx[tri_lexpos(a, c, d, tk_lex, toff, adj, adjpre, W, deg, up, lex_ptr, elp, n, pre)];
    if (pre && elp) {
      // Faces (a, b, d) and (a, b, c) share their first edge: its position,
      // triangle offset and the two rows' words above b, read once.
      const int64_t lp = elp[(int64_t)a * n + b];
      const int64_t base = toff[lp];
      const uint32_t *ra = adj + (int64_t)a * W, *rb = adj + (int64_t)b * W;
      const int wc = c >> 5, wd = d >> 5;
      const uint32_t mc = ra[wc] & rb[wc] & above_mask(b, wc);
      const uint32_t md = wd == wc ? mc : ra[wd] & rb[wd] & above_mask(b, wd);
      const int64_t pc = base + pre[lp * W + wc] + __popc(mc & ((1u << (c & 31)) - 1u));
      const int64_t pd = base + (wd == wc ? pre[lp * W + wc] : pre[lp * W + wd]) + __popc(md & ((1u << (d & 31)) - 1u));
      r[2] = ordidx[pd];
      r[3] = ordidx[pc];
    } else {
      r[2] = ordidx[tri_lexpos(a, b, d, tk_lex, toff, adj, adjpre, W, deg, up, lex_ptr, elp, n, pre)];
      r[3] = ordidx[tri_lexpos(a, b, c, tk_lex, toff, adj, adjpre, W, deg, up, lex_ptr, elp, n, pre)];
    }
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int y = 0; y < 3 - x; ++y)
        if (r[y] > r[y + 1]) {
          const int32_t sw = r[y];
          r[y] = r[y + 1];
          r[y + 1] = sw;
        }
    // One 16-byte store each (the arrays start 16-byte aligned): consecutive
    // lanes then cover whole sectors.
    ((int4 *)verts)[p] = make_int4(a, b, c, d);
    grade[p] = (int32_t)(packed ? key >> TET_PACK_SHIFT : key >> 32);
    colptr[p] = 4 * p;
    ((int4 *)rowidx)[p] = make_int4(r[0], r[1], r[2], r[3]);
    if (p == T4 - 1) colptr[T4] = 4 * T4;
  }
}

}  // namespace vr
