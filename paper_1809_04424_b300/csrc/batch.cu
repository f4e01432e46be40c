// batch.cu -- many point clouds in two launches.
//
// vr_build_batch takes clouds concatenated row-wise with host offsets.  One
// CTA owns one cloud at a time, taking clouds from a work list ordered by
// descending size (longest first), and runs the whole build of that cloud
// with its bitmap, prefix counts and per-row arrays in shared memory and its
// longer arrays (keys, sort temporaries, neighbour CSR) in a per-CTA slice of
// global scratch that stays in L2:
//   k_batch_size  -- values check, kept-edge bitmap, E, and T as
//                    (sum over edges of |N(a) & N(b)|) / 3;
//   [one host sync: exact output arenas, per-cloud slices]
//   k_batch_build -- bitmap again, lexicographic edge keys, CTA radix sort on
//                    the distance bits, dense-rank grades, edge outputs and
//                    neighbour CSR, lexicographic triangle keys carrying the
//                    grade, CTA radix sort on the grade bits, final write.
// Triangles always take the lexicographic enumeration (exact with ties).
// A cloud beyond the fused limits (its bitmap, prefix counts and points above
// 200 KB of shared memory, or a float run of equal fp32 keys longer than 64)
// is rebuilt by the single-cloud path.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <numeric>
#include <type_traits>
#include <vector>

#include "complex.h"
#include "jobs.h"
#include "kernels.cuh"
#include "prof.h"

namespace vr {

constexpr int BT = RS_THREADS;  // 256: the CTA sort's tile ranking assumes it
constexpr int BWARPS = BT / 32;
constexpr size_t FUSED_SMEM = 200 * 1024;  // shared-memory budget of one fused cloud
constexpr int RUN_MAX = 64;     // longest float run of equal fp32 keys handled in-CTA

// Per-cloud descriptor (device and host copies).
struct CloudDesc {
  int64_t pt;                 // first row of the cloud in the concatenated points
  int32_t n, maxdim;
  int32_t keep_all, kbits;    // cap: keep everything; distance bits to sort
  double maxrad;              // as given
  uint64_t r2i;               // integer cap
  double r2;                  // float cap
  float a_keep, a_drop;       // float thresholds of the cap test
  int64_t E, T;               // sizes (sizing pass)
  int64_t eo, to, go, vo, co, ko;  // output offsets: edges, triangles, grade values, vertices, colptr
  int32_t flags;              // value / internal flags of this cloud
  int32_t fallback;           // 1: rebuild with the single-cloud path
  int64_t ngrades;
  double max_rel_err;
};

struct BatchOut {
  int32_t *everts, *egrade, *erow;
  int64_t *ecol;
  int32_t *tverts, *tgrade, *trow;
  int64_t *tcol;
  int32_t *vverts, *vgrade;
  double *gval;
};

// Per-CTA scratch slice layout (bytes from the slice base), sized from the
// batch's largest E and T.
struct ScratchLayout {
  int64_t keys, tkeys, d64lex, d64, flag, gex, nbr_ord, nbr_gr, gstart, tcnt, toff, tk, tk2, bytes;
};

static ScratchLayout scratch_layout(int64_t Emax, int64_t Tmax, bool F) {
  ScratchLayout L{};
  int64_t o = 0;
  auto take = [&](int64_t bytes) {
    int64_t at = o;
    o += (bytes + 255) / 256 * 256;
    return at;
  };
  const int64_t E1 = Emax + 2, T1 = std::max<int64_t>(Tmax, 1);
  L.keys = take(8 * E1);
  L.tkeys = take(8 * E1);
  L.d64lex = F ? take(8 * E1) : 0;
  L.d64 = F ? take(8 * E1) : 0;
  L.flag = take(4 * E1);
  L.gex = take(4 * E1);
  L.nbr_ord = take(8 * E1);
  L.nbr_gr = take(8 * E1);
  L.gstart = take(4 * E1);
  L.tcnt = take(4 * E1);
  L.toff = take(8 * E1);
  L.tk = take(8 * T1);
  L.tk2 = take(8 * T1);
  L.bytes = o;
  return L;
}

// ----------------------------------------------------------- CTA helpers

// Shared-memory layout of one fused cloud of up to nmax points (every region
// 16-byte aligned): bitmap u32, prefix counts u16, deg, up, row pointers
// (i32, n+2), lex pointers (i64, n+1), points (4 B each).
struct SmemLayout {
  size_t adj, pre, deg, up, nptr, lptr, X, bytes;
};
__host__ __device__ __forceinline__ size_t al16(size_t v) { return (v + 15) & ~(size_t)15; }
__host__ __device__ __forceinline__ SmemLayout smem_layout(int nmax, int d) {
  const size_t nw = (size_t)nmax * ((nmax + 31) / 32);
  SmemLayout L;
  L.adj = 0;
  L.pre = L.adj + al16(nw * 4);
  L.deg = L.pre + al16(nw * 2);
  L.up = L.deg + al16((size_t)nmax * 4);
  L.nptr = L.up + al16((size_t)nmax * 4);
  L.lptr = L.nptr + al16((size_t)(nmax + 2) * 4);
  L.X = L.lptr + al16((size_t)(nmax + 1) * 8);
  L.bytes = L.X + al16((size_t)nmax * d * 4);
  return L;
}

// Exclusive scan of in[0..L) into out[0..L], out[L] = total, by one CTA.
template <typename TI, typename TO>
__device__ void cta_scan(const TI *in, TO *out, int64_t L) {
  __shared__ int64_t sh[33];
  int64_t carry = 0;
  for (int64_t b0 = 0; b0 < L; b0 += BT) {
    const int64_t i = b0 + threadIdx.x;
    const int64_t v = i < L ? (int64_t)in[i] : 0;
    int64_t tot;
    const int64_t e = block_excl_scan<int64_t>(v, sh, &tot);
    if (i < L) out[i] = (TO)(carry + e);
    carry += tot;
  }
  if (threadIdx.x == 0) out[L] = (TO)carry;
  __syncthreads();
}

__device__ __forceinline__ int64_t cta_sum(int64_t v) {
  __shared__ int64_t sh[33];
  int64_t tot;
  block_excl_scan<int64_t>(v, sh, &tot);
  return tot;
}

__device__ __forceinline__ int32_t rank16(const uint32_t *row, const uint16_t *pre, int c) {
  const int w = c >> 5, b = c & 31;
  return (int32_t)pre[w] + __popc(row[w] & ((1u << b) - 1u));
}

// Stage points, bitmap (warp per 32x32 block of the upper triangle, ballot
// rows, lane-accumulated mirrored columns), all in shared memory.  I8 (int8
// source, d <= 4): the lane's column point sits in registers, the block's
// row points are broadcast by shuffles and the distance is 32-bit integer
// arithmetic (d^2 <= 4 * 255^2, far below the key limit).
template <bool F, bool I8 = false>
__device__ void cta_bitmap(const void *pts, const CloudDesc &c, int d, void *Xs, uint32_t *adj, int32_t *flags) {
  using T = typename std::conditional<F, float, int32_t>::type;
  const int n = c.n, W = (n + 31) / 32;
  T *X = (T *)Xs;
  for (int t = threadIdx.x; t < n * d; t += BT) {
    if constexpr (F) {
      const float v = ((const float *)pts)[c.pt * d + t];
      if (!isfinite(v)) atomicOr(flags, F_NONFINITE);
      else if (fabsf(v) > (float)VR_MAX_F32_ABS) atomicOr(flags, F_F32_RANGE);
      X[t] = v;
    }
  }
  __syncthreads();
  const int wid = threadIdx.x >> 5, l = lane_id();
  const int nblk = W * W;
  for (int blk = wid; blk < nblk; blk += BWARPS) {
    const int bi = blk / W, bj = blk % W;
    if (bi > bj) continue;
    const int j = bj * 32 + l;
    const bool jv = j < n;
    uint32_t myrow = 0, mycol = 0;
    bool over = false;
    const int rows = min(32, n - bi * 32);
    constexpr int DR = I8 ? 4 : 1;
    T xj[DR], xr[DR];
    if constexpr (I8) {
      const int ir = bi * 32 + l;
#pragma unroll
      for (int k = 0; k < DR; ++k) {
        xj[k] = (jv && k < d) ? X[j * d + k] : T(0);
        xr[k] = (ir < n && k < d) ? X[ir * d + k] : T(0);
      }
    }
    for (int r = 0; r < rows; ++r) {
      const int i = bi * 32 + r;
      bool kept = false;
      if constexpr (I8 && !F) {
        // All lanes shuffle (the row point of lane r), then decide.
        int32_t v = 0;
#pragma unroll
        for (int k = 0; k < DR; ++k) {
          const int32_t t = __shfl_sync(0xffffffffu, (int32_t)xr[k], r) - (int32_t)xj[k];
          v += t * t;
        }
        if (jv && j != i) kept = c.keep_all || (uint64_t)v <= c.r2i;
      } else if (jv && j != i) {
        if constexpr (F) {
          const float a = d2_f32(X + i * d, X + j * d, d);
          if (c.keep_all || a <= c.a_keep) kept = true;
          else if (a >= c.a_drop) kept = false;
          else kept = d2_canonical(X + i * d, X + j * d, d) <= c.r2;
        } else {
          const uint64_t v = d2_int(X + i * d, X + j * d, d);
          kept = c.keep_all || v <= c.r2i;
          if (kept && v >= INT_KEY_LIMIT) over = true;
        }
      }
      const uint32_t word = __ballot_sync(0xffffffffu, kept);
      if (l == r) myrow = word;
      mycol |= (uint32_t)kept << r;
    }
    if (over) atomicOr(flags, F_INT_KEY);
    const int i = bi * 32 + l;
    if (i < n) adj[i * W + bj] = myrow;
    if (bi < bj && jv) adj[j * W + bi] = mycol;
  }
  __syncthreads();
}

// Integer clouds are staged by a typed loop (int8 or int32 source).
template <typename TIn>
__device__ void cta_stage_int(const TIn *pts, const CloudDesc &c, int d, int32_t *X) {
  for (int t = threadIdx.x; t < c.n * d; t += BT) X[t] = (int32_t)pts[c.pt * d + t];
}

// Work list: clouds in descending size, fetched one per CTA iteration.
__device__ __forceinline__ int next_cloud(int *cursor, const int32_t *order, int n_clouds) {
  __shared__ int idx;
  if (threadIdx.x == 0) idx = atomicAdd(cursor, 1);
  __syncthreads();
  const int k = idx;
  __syncthreads();
  return k < n_clouds ? order[k] : -1;
}

// ------------------------------------------------------------------ sizing

template <bool F, typename TIn>
__device__ void batch_size_loop(const TIn *pts, int d, CloudDesc *desc, const int32_t *order, int n_clouds,
                                int *cursor, int nmax, unsigned char *smem) {
  const int Wmax = (nmax + 31) / 32;
  uint32_t *adj = (uint32_t *)smem;
  void *Xs = (void *)(smem + al16((size_t)nmax * Wmax * 4));
  __shared__ int32_t flags;
  for (int ci; (ci = next_cloud(cursor, order, n_clouds)) >= 0;) {
    CloudDesc &c = desc[ci];
    if (c.fallback) continue;
    if (threadIdx.x == 0) flags = 0;
    __syncthreads();
    if constexpr (!F) cta_stage_int<TIn>(pts, c, d, (int32_t *)Xs);
    if constexpr (std::is_same<TIn, int8_t>::value) {
      if (d <= 4) cta_bitmap<F, true>(pts, c, d, Xs, adj, &flags);
      else cta_bitmap<F>(pts, c, d, Xs, adj, &flags);
    } else {
      cta_bitmap<F>(pts, c, d, Xs, adj, &flags);
    }
    const int n = c.n, W = (n + 31) / 32;
    const int wid = threadIdx.x >> 5, l = lane_id();
    // E: upper-triangle bits; 3T: sum over edges (a < b) of |N(a) & N(b)|.
    int64_t e_loc = 0, t3_loc = 0;
    for (int a = wid; a < n; a += BWARPS) {
      const uint32_t *ra = adj + a * W;
      for (int w0 = (a + 1) >> 5; w0 < W; w0 += 32) {
        const int w = w0 + l;
        const uint32_t word = w < W ? ra[w] & above_mask(a, w) : 0u;
        e_loc += __popc(word);
        const BitChunk r = bit_round(word);
        for (int q0 = 0; q0 < r.tot; q0 += 32) {
          const int q = q0 + l;
          const int ow = bit_owner(r, q);
          const uint32_t om = __shfl_sync(0xffffffffu, word, ow);
          const int oex = __shfl_sync(0xffffffffu, r.excl, ow);
          if (q < r.tot) {
            const int b = (w0 + ow) * 32 + __fns(om, 0, q - oex + 1);
            const uint32_t *rb = adj + b * W;
            for (int x = 0; x < W; ++x) t3_loc += __popc(ra[x] & rb[x]);
          }
        }
      }
    }
    const int64_t E = cta_sum(e_loc), T3 = cta_sum(t3_loc);
    if (threadIdx.x == 0) {
      c.E = E;
      c.T = c.maxdim >= 2 ? T3 / 3 : 0;
      c.flags |= flags;
    }
    __syncthreads();
  }
}

template <bool F, typename TIn>
__global__ void __launch_bounds__(BT) k_batch_size(const TIn *pts, int d, CloudDesc *desc, const int32_t *order,
                                                   int n_clouds, int *cursor, int nmax) {
  extern __shared__ __align__(16) unsigned char smem[];
  batch_size_loop<F, TIn>(pts, d, desc, order, n_clouds, cursor, nmax, smem);
}

// ------------------------------------------------------------------- build

template <bool F, typename TIn>
__device__ void batch_build_loop(const TIn *pts, int d, CloudDesc *desc, const int32_t *order, int n_clouds,
                                 int *cursor, int nmax, unsigned char *scratch, const ScratchLayout &SL,
                                 const BatchOut &out, unsigned char *smem) {
  const SmemLayout SM = smem_layout(nmax, d);
  uint32_t *adj = (uint32_t *)(smem + SM.adj);
  uint16_t *pre = (uint16_t *)(smem + SM.pre);
  int32_t *deg = (int32_t *)(smem + SM.deg);
  int32_t *up = (int32_t *)(smem + SM.up);
  int32_t *nptr = (int32_t *)(smem + SM.nptr);
  int64_t *lptr = (int64_t *)(smem + SM.lptr);
  void *Xs = (void *)(smem + SM.X);
  __shared__ int32_t flags;
  __shared__ int64_t ngr;

  unsigned char *base = scratch + (size_t)blockIdx.x * SL.bytes;
  uint64_t *keys = (uint64_t *)(base + SL.keys), *tkeys = (uint64_t *)(base + SL.tkeys);
  double *d64lex = (double *)(base + SL.d64lex), *d64 = (double *)(base + SL.d64);
  int32_t *flag = (int32_t *)(base + SL.flag), *gex = (int32_t *)(base + SL.gex);
  int32_t *nbr_ord = (int32_t *)(base + SL.nbr_ord), *gstart = (int32_t *)(base + SL.gstart);
  int32_t *nbr_gr = (int32_t *)(base + SL.nbr_gr);  // the CSR's edge grades, beside nbr_ord
  int32_t *tcnt = (int32_t *)(base + SL.tcnt);
  int64_t *toff = (int64_t *)(base + SL.toff);
  uint64_t *tk = (uint64_t *)(base + SL.tk), *tk2 = (uint64_t *)(base + SL.tk2);
  const int wid = threadIdx.x >> 5, l = lane_id();
  const uint32_t lt = lanemask_lt();

  for (int ci; (ci = next_cloud(cursor, order, n_clouds)) >= 0;) {
    CloudDesc &c = desc[ci];
    if (c.fallback || c.flags) continue;
    if (threadIdx.x == 0) {
      flags = 0;
      ngr = 1;
    }
    __syncthreads();
    const int n = c.n, W = (n + 31) / 32;
    if constexpr (!F) cta_stage_int<TIn>(pts, c, d, (int32_t *)Xs);
    if constexpr (std::is_same<TIn, int8_t>::value) {
      if (d <= 4) cta_bitmap<F, true>(pts, c, d, Xs, adj, &flags);
      else cta_bitmap<F>(pts, c, d, Xs, adj, &flags);
    } else {
      cta_bitmap<F>(pts, c, d, Xs, adj, &flags);
    }
    using TX = typename std::conditional<F, float, int32_t>::type;
    const TX *X = (const TX *)Xs;

    // Row counts and prefix popcounts (u16: n <= 1024).
    for (int i = wid; i < n; i += BWARPS) {
      int carry = 0, upc = 0;
      for (int w0 = 0; w0 < W; w0 += 32) {
        const int w = w0 + l;
        const uint32_t word = w < W ? adj[i * W + w] : 0u;
        const int cc = __popc(word), inc = warp_incl_scan(cc);
        if (w < W) pre[i * W + w] = (uint16_t)(carry + inc - cc);
        carry += __shfl_sync(0xffffffffu, inc, 31);
        upc += __popc(word & above_mask(i, w));
      }
      upc = warp_sum(upc);
      if (l == 0) {
        deg[i] = carry;
        up[i] = upc;
      }
    }
    __syncthreads();
    cta_scan<int32_t, int32_t>(deg, nptr, n);
    cta_scan<int32_t, int64_t>(up, lptr, n);
    const int64_t E = lptr[n];
    if (E != c.E) {
      if (threadIdx.x == 0) c.flags |= F_INTERNAL;
      continue;
    }

    // Lexicographic edge keys (float: canonical FP64 value alongside).
    for (int i = wid; i < n; i += BWARPS) {
      int64_t t = lptr[i];
      for (int w0 = (i + 1) >> 5; w0 < W; w0 += 32) {
        const int w = w0 + l;
        const uint32_t word = w < W ? adj[i * W + w] & above_mask(i, w) : 0u;
        const BitChunk r = bit_round(word);
        for (int q0 = 0; q0 < r.tot; q0 += 32) {
          const int q = q0 + l;
          const int ow = bit_owner(r, q);
          const uint32_t om = __shfl_sync(0xffffffffu, word, ow);
          const int oex = __shfl_sync(0xffffffffu, r.excl, ow);
          if (q < r.tot) {
            const int j = (w0 + ow) * 32 + __fns(om, 0, q - oex + 1);
            uint64_t dk;
            if constexpr (F) {
              const double f = d2_canonical(X + i * d, X + j * d, d);
              d64lex[t + q] = f;
              dk = (uint64_t)__float_as_uint(__double2float_rn(f));
            } else {
              dk = d2_int(X + i * d, X + j * d, d);
            }
            keys[t + q] = (dk << KEY_SHIFT) | ((uint64_t)i << ID_BITS) | (uint64_t)j;
          }
        }
        t += r.tot;
      }
    }
    __syncthreads();
    cta_radix_sort_global(keys, nullptr, tkeys, nullptr, E, KEY_SHIFT, c.kbits);

    if constexpr (F) {
      // Canonical values in sorted order; re-sort runs of equal fp32 keys by
      // (FP64 value, i, j).  A run longer than RUN_MAX sends the cloud to the
      // single-cloud path.
      for (int64_t k = threadIdx.x; k < E; k += BT) {
        const uint64_t key = keys[k];
        const int i = (int)((key >> ID_BITS) & ID_MASK), j = (int)(key & ID_MASK);
        d64[k] = d64lex[lptr[i] + rank16(adj + i * W, pre + i * W, j) - (deg[i] - up[i])];
      }
      __syncthreads();
      for (int64_t k = threadIdx.x; k < E; k += BT) {
        const uint64_t dk = keys[k] >> KEY_SHIFT;
        if (k > 0 && (keys[k - 1] >> KEY_SHIFT) == dk) continue;  // not a run start
        int64_t e = k + 1;
        while (e < E && (keys[e] >> KEY_SHIFT) == dk && e - k <= RUN_MAX) ++e;
        if (e - k > RUN_MAX) {
          atomicOr(&flags, F_OVERFLOW);
          continue;
        }
        for (int64_t x = k + 1; x < e; ++x) {
          const uint64_t kx = keys[x];
          const double dx = d64[x];
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
      __syncthreads();
      if (flags & F_OVERFLOW) {
        if (threadIdx.x == 0) c.fallback = 1;
        continue;
      }
    }

    // Dense-rank grades, edge outputs, grade values, neighbour CSR.
    for (int64_t k = threadIdx.x; k < E; k += BT) {
      int f;
      if constexpr (F) f = k == 0 ? (d64[0] != 0.0) : (d64[k] != d64[k - 1]);
      else f = k == 0 ? ((keys[0] >> KEY_SHIFT) != 0) : ((keys[k] >> KEY_SHIFT) != (keys[k - 1] >> KEY_SHIFT));
      flag[k] = f;
    }
    __syncthreads();
    cta_scan<int32_t, int32_t>(flag, gex, E);
    for (int64_t k = threadIdx.x; k < E; k += BT) {
      const uint64_t key = keys[k];
      const int i = (int)((key >> ID_BITS) & ID_MASK), j = (int)(key & ID_MASK);
      const int g = gex[k + 1];
      const int64_t p = c.eo + k;
      out.everts[2 * p] = i;
      out.everts[2 * p + 1] = j;
      out.erow[2 * p] = i;
      out.erow[2 * p + 1] = j;
      out.ecol[c.co + k] = 2 * k;
      out.egrade[p] = g;
      if (flag[k]) {
        double v;
        if constexpr (F) v = d64[k];
        else v = (double)(key >> KEY_SHIFT);
        out.gval[c.go + g] = v;
        gstart[g] = (int32_t)k;
      }
      const int32_t si = nptr[i] + rank16(adj + i * W, pre + i * W, j);
      const int32_t sj = nptr[j] + rank16(adj + j * W, pre + j * W, i);
      nbr_ord[si] = (int32_t)k;
      nbr_ord[sj] = (int32_t)k;
      nbr_gr[si] = g;
      nbr_gr[sj] = g;
      if (k == E - 1) ngr = g + 1;
    }
    if (threadIdx.x == 0) {
      out.gval[c.go] = 0.0;
      out.ecol[c.co + E] = 2 * E;
    }
    for (int v = threadIdx.x; v < n; v += BT) {
      out.vverts[c.vo + v] = v;
      out.vgrade[c.vo + v] = 0;
    }
    __syncthreads();
    const int64_t ngrades = ngr;

    const int64_t T = c.T;
    if (c.maxdim >= 2) {
      if (threadIdx.x == 0) out.tcol[c.ko + T] = 3 * T;
      // Lex counts: triangle (a, b, c'), a < b < c', counted at its first
      // edge.  Warp per row a, lane per kept b > a (lexicographic position
      // lptr[a] + rank), all from the shared-memory bitmap.
      for (int a = wid; a < n; a += BWARPS) {
        int64_t e = lptr[a];
        for (int w0 = (a + 1) >> 5; w0 < W; w0 += 32) {
          const int w = w0 + l;
          const uint32_t word = w < W ? adj[a * W + w] & above_mask(a, w) : 0u;
          const BitChunk r = bit_round(word);
          for (int q0 = 0; q0 < r.tot; q0 += 32) {
            const int q = q0 + l;
            const int ow = bit_owner(r, q);
            const uint32_t om = __shfl_sync(0xffffffffu, word, ow);
            const int oex = __shfl_sync(0xffffffffu, r.excl, ow);
            if (q < r.tot) {
              const int b = (w0 + ow) * 32 + __fns(om, 0, q - oex + 1);
              int cnt = 0;
              for (int x = b >> 5; x < W; ++x) cnt += __popc(adj[a * W + x] & adj[b * W + x] & above_mask(b, x));
              tcnt[e + q] = cnt;
            }
          }
          e += r.tot;
        }
      }
      __syncthreads();
      cta_scan<int32_t, int64_t>(tcnt, toff, E);
      if (toff[E] != T) {
        if (threadIdx.x == 0) c.flags |= F_INTERNAL;
        continue;
      }
      // Keys grade << 39 | (a, b, c'): warp per row a, lane per kept b > a
      // (lexicographic position lptr[a] + rank); each lane walks its edge's
      // triangles (c' ascending) itself, the two other grades read from the
      // CSR's grade copy, so the lanes' loads overlap instead of one edge's
      // few triangles holding the whole warp.
      for (int a = wid; a < n; a += BWARPS) {
        const int32_t *ga = nbr_gr + nptr[a];
        int64_t e = lptr[a];
        for (int w0 = (a + 1) >> 5; w0 < W; w0 += 32) {
          const int w = w0 + l;
          const uint32_t word = w < W ? adj[a * W + w] & above_mask(a, w) : 0u;
          const BitChunk r = bit_round(word);
          for (int q0 = 0; q0 < r.tot; q0 += 32) {
            const int q = q0 + l;
            const int ow = bit_owner(r, q);
            const uint32_t om = __shfl_sync(0xffffffffu, word, ow);
            const int oex = __shfl_sync(0xffffffffu, r.excl, ow);
            if (q < r.tot) {
              const int b = (w0 + ow) * 32 + __fns(om, 0, q - oex + 1);
              const int32_t gab = ga[rank16(adj + a * W, pre + a * W, b)];
              const int32_t *gb = nbr_gr + nptr[b];
              int64_t t = toff[e + q];
              for (int x = b >> 5; x < W; ++x) {
                uint32_t m = adj[a * W + x] & adj[b * W + x] & above_mask(b, x);
                while (m) {
                  const int cv = x * 32 + __ffs(m) - 1;
                  m &= m - 1;
                  const int32_t gac = ga[rank16(adj + a * W, pre + a * W, cv)];
                  const int32_t gbc = gb[rank16(adj + b * W, pre + b * W, cv)];
                  if (t < T) tk[t] = ((uint64_t)max(gab, max(gac, gbc)) << LEX_SHIFT) | lex3(a, b, cv);
                  ++t;
                }
              }
            }
          }
          e += r.tot;
        }
      }
      __syncthreads();
      int gbits = 1;
      while ((1ll << gbits) < ngrades) ++gbits;
      cta_radix_sort_global(tk, nullptr, tk2, nullptr, T, LEX_SHIFT, gbits);
      for (int64_t p = threadIdx.x; p < T; p += BT) {
        const uint64_t k = tk[p];
        const int a = (int)((k >> (2 * ID_BITS)) & ID_MASK), b = (int)((k >> ID_BITS) & ID_MASK),
                  cc = (int)(k & ID_MASK);
        const int32_t o0 = nbr_ord[nptr[a] + rank16(adj + a * W, pre + a * W, b)];
        const int32_t o1 = nbr_ord[nptr[a] + rank16(adj + a * W, pre + a * W, cc)];
        const int32_t o2 = nbr_ord[nptr[b] + rank16(adj + b * W, pre + b * W, cc)];
        const int32_t lo = min(o0, min(o1, o2)), hi = max(o0, max(o1, o2));
        const int64_t q = c.to + p;
        out.tverts[3 * q] = a;
        out.tverts[3 * q + 1] = b;
        out.tverts[3 * q + 2] = cc;
        out.tgrade[q] = (int32_t)(k >> LEX_SHIFT);
        out.tcol[c.ko + p] = 3 * p;
        out.trow[3 * q] = lo;
        out.trow[3 * q + 1] = o0 + o1 + o2 - lo - hi;
        out.trow[3 * q + 2] = hi;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      c.ngrades = ngrades;
      c.flags |= flags;
    }
    __syncthreads();
  }
  (void)lt;
}

template <bool F, typename TIn>
__global__ void __launch_bounds__(BT) k_batch_build(const TIn *pts, int d, CloudDesc *desc, const int32_t *order,
                                                    int n_clouds, int *cursor, int nmax, unsigned char *scratch,
                                                    ScratchLayout SL, BatchOut out) {
  extern __shared__ __align__(16) unsigned char smem[];
  batch_build_loop<F, TIn>(pts, d, desc, order, n_clouds, cursor, nmax, scratch, SL, out, smem);
}

// ------------------------------------------------------- one-launch batch
// The whole batch in one persistent launch of co-resident CTAs (cooperative):
//   phase 1: every cloud of the work list sized (bitmap, E, T);
//   grid barrier; CTA 0 lays the clouds' output slices out in cloud order
//   (exclusive scans of their sizes) and checks them against the arenas'
//   and the per-CTA scratch's capacities; grid barrier;
//   phase 2: every cloud built into its slice (skipped, with the overflow
//   word set, when a capacity is short: the host then grows the arenas and
//   relaunches phase 2 alone).
// Inputs, outputs and capacities are read from a parameter block in device
// memory, so that one captured graph serves every batch of the same shape.
struct BatchParams {
  const void *pts;
  int32_t n_clouds;
  BatchOut out;
  unsigned char *scratch;
  ScratchLayout SL;
  int64_t cap[6];     // arena capacities: edges, triangles, vertices, grade values, edge colptr, triangle colptr
  int64_t emax_cap;   // per-CTA scratch: largest E and T of one cloud
  int64_t tmax_cap;
};
// Control words of a launch: [0] sizing cursor, [1] build cursor, [2..3]
// grid barrier, [4] flags (F_TIMEOUT), [5] overflow, then (64-bit, from
// word 6) the totals of the six arenas and the largest E and T.
constexpr int BC_WORDS = 6 + 2 * 8;
static_assert(sizeof(int64_t) * 8 == sizeof(unsigned int) * (BC_WORDS - 6), "control words: eight 64-bit totals");
constexpr uint64_t BATCH_BARRIER_NS = 30ull * 1000 * 1000 * 1000;  // 30 s

__device__ bool batch_grid_barrier(unsigned int *bar, int32_t *err) {
  __threadfence();
  __syncthreads();
  __shared__ int s_ok;
  if (threadIdx.x == 0) {
    volatile unsigned int *gen = bar + 1;
    const unsigned int g = *gen;
    __threadfence();
    if (atomicAdd(bar, 1u) == gridDim.x - 1) {
      bar[0] = 0;
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      // Bounded by time, not by polls: a CTA may legitimately wait here for
      // as long as the slowest CTA's last cloud takes.
      uint64_t t0, t;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
      while (*gen == g) {
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        if (t - t0 > BATCH_BARRIER_NS) {  // every CTA then leaves the launch
          atomicOr(err, F_TIMEOUT);
          break;
        }
        __nanosleep(256);
      }
    }
    __threadfence();
    s_ok = *(volatile int32_t *)err == 0;
  }
  __syncthreads();
  return s_ok != 0;
}

// CTA 0: output slices of the clouds in cloud order, totals and maxima.
__device__ void batch_layout(CloudDesc *desc, int n_clouds, const BatchParams &p, unsigned int *ctr) {
  __shared__ int64_t sh[33];
  int64_t base[6] = {0, 0, 0, 0, 0, 0};
  int64_t emax = 0, tmax = 0;
  for (int b0 = 0; b0 < n_clouds; b0 += BT) {
    const int i = b0 + threadIdx.x;
    int64_t v[6] = {0, 0, 0, 0, 0, 0};
    bool act = false;
    if (i < n_clouds) {
      const CloudDesc &c = desc[i];
      act = !(c.fallback || c.flags);
      if (act) {
        v[0] = c.E;
        v[1] = c.T;
        v[2] = c.n;
        v[3] = c.E + 1;
        v[4] = c.E + 1;
        v[5] = c.maxdim >= 2 ? c.T + 1 : 0;
        emax = max(emax, c.E);
        tmax = max(tmax, c.T);
      }
    }
    int64_t ex[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      int64_t tot;
      ex[k] = block_excl_scan<int64_t>(v[k], sh, &tot) + base[k];
      base[k] += tot;
    }
    if (act) {
      CloudDesc &c = desc[i];
      c.eo = ex[0];
      c.to = ex[1];
      c.vo = ex[2];
      c.go = ex[3];
      c.co = ex[4];
      c.ko = ex[5];
    }
  }
  // Maxima over the CTA (shared atomics).
  __shared__ unsigned long long smax[2];
  if (threadIdx.x == 0) smax[0] = smax[1] = 0;
  __syncthreads();
  atomicMax(&smax[0], (unsigned long long)emax);
  atomicMax(&smax[1], (unsigned long long)tmax);
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t *tot = (int64_t *)(ctr + 6);
    bool over = smax[0] > (unsigned long long)p.emax_cap || smax[1] > (unsigned long long)p.tmax_cap;
    for (int k = 0; k < 6; ++k) {
      tot[k] = base[k];
      over |= base[k] > p.cap[k];
    }
    tot[6] = (int64_t)smax[0];
    tot[7] = (int64_t)smax[1];
    ctr[5] = over ? 1u : 0u;
  }
}

// phases: bit 0 sizing + layout, bit 1 build.
template <bool F, typename TIn>
__global__ void __launch_bounds__(BT) k_batch_all(const BatchParams *P, int d, CloudDesc *desc, const int32_t *order,
                                                  int nmax, unsigned int *ctr, int phases) {
  extern __shared__ __align__(16) unsigned char smem[];
  const BatchParams p = *P;
  const int n_clouds = p.n_clouds;
  int32_t *err = (int32_t *)(ctr + 4);
  if (phases & 1) {
    batch_size_loop<F, TIn>((const TIn *)p.pts, d, desc, order, n_clouds, (int *)ctr, nmax, smem);
    if (!batch_grid_barrier(ctr + 2, err)) return;
    if (blockIdx.x == 0) batch_layout(desc, n_clouds, p, ctr);
    if (!batch_grid_barrier(ctr + 2, err)) return;
  }
  if (phases & 2) {
    if (*(volatile unsigned int *)(ctr + 5)) return;  // a capacity is short: the host relaunches
    batch_build_loop<F, TIn>((const TIn *)p.pts, d, desc, order, n_clouds, (int *)(ctr + 1), nmax, p.scratch, p.SL,
                             p.out, smem);
  }
}

}  // namespace vr

// ================================================================== host

#include <memory>
#include <mutex>

namespace vr {

template <typename T>
static vr_status dalloc(std::vector<void *> &v, T **p, int64_t count, cudaStream_t s) {
  size_t bytes = sizeof(T) * (size_t)std::max<int64_t>(count, 1);
  cudaError_t e = dev_malloc((void **)p, bytes, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error("device allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? VR_ERR_OOM : VR_ERR_CUDA;
  }
  v.push_back(*p);
  return VR_OK;
}

static void free_all(std::vector<void *> &v, cudaStream_t s) {
  for (void *p : v) cudaFreeAsync(p, s);
  v.clear();
}

static void thresholds_host(double r2, double crel, float *a_keep, float *a_drop) {
  auto hi = [&](float a) { return (double)a * (1.0 + crel) + F32_ABS_SLACK; };
  auto lo = [&](float a) { return (double)a * (1.0 - crel) - F32_ABS_SLACK; };
  float k = (float)((r2 - F32_ABS_SLACK) / (1.0 + crel));
  if (k < 0.f) k = 0.f;
  while (k > 0.f && hi(k) > r2) k = std::nextafter(k, -INFINITY);
  while (hi(std::nextafter(k, INFINITY)) <= r2) k = std::nextafter(k, INFINITY);
  if (hi(k) > r2) k = -1.f;
  float dr = (float)((r2 + F32_ABS_SLACK) / (1.0 - crel));
  while (lo(dr) <= r2) dr = std::nextafter(dr, INFINITY);
  while (dr > 0.f && lo(std::nextafter(dr, -INFINITY)) > r2) dr = std::nextafter(dr, -INFINITY);
  *a_keep = k;
  *a_drop = dr;
}

static int bitlen64(uint64_t v) { return v ? 64 - __builtin_clzll(v) : 0; }

// Shared memory of one fused cloud.
size_t fused_smem(int n, int d) { return smem_layout(n, d).bytes; }
bool fused_fits(int n, int d) { return fused_smem(n, d) <= FUSED_SMEM; }

// Fill a cloud descriptor from its request; false (with the error set) on a
// bad argument.
vr_status make_desc(CloudDesc &c, int64_t pt, int64_t n, int d, vr_dtype dtype, int maxdim, double maxrad) {
  memset(&c, 0, sizeof(c));
  if (n < 1 || n > VR_MAX_POINTS) { set_error("cloud with %lld points", (long long)n); return VR_ERR_RANGE; }
  if (maxdim < 0) { set_error("maxdim < 0"); return VR_ERR_ARG; }
  if (maxdim > VR_MAX_DIM_BATCH) { set_error("maxdim above 2 is not offered for batches"); return VR_ERR_UNSUPPORTED; }
  if (std::isnan(maxrad) || maxrad < 0) { set_error("maxrad must be >= 0 and not NaN"); return VR_ERR_ARG; }
  c.pt = pt;
  c.n = (int32_t)n;
  c.maxdim = maxdim;
  c.maxrad = maxrad;
  const double r2 = maxrad * maxrad;
  c.keep_all = std::isinf(r2) ? 1 : 0;
  c.r2 = r2;
  if (dtype == VR_F32) {
    if (!c.keep_all && r2 >= 1e38) c.keep_all = 1;
    if (!c.keep_all) thresholds_host(r2, (d + 5) * std::ldexp(1.0, -24), &c.a_keep, &c.a_drop);
    c.kbits = 31;
  } else {
    uint64_t bound = dtype == VR_I8 ? (uint64_t)d * 255ull * 255ull : INT_KEY_LIMIT - 1;
    if (!c.keep_all) {
      const double f = std::floor(r2);
      c.r2i = f >= 18446744073709551615.0 ? ~0ull : (uint64_t)f;
      bound = std::min(bound, c.r2i);
    }
    c.kbits = std::max(1, bitlen64(bound));
  }
  c.fallback = fused_fits(c.n, d) ? 0 : 1;
  return VR_OK;
}

// Output arenas of one batch, shared by the per-cloud results through
// reference counting; released (stream-ordered on `stream`) with the last.
struct Arenas {
  std::vector<void *> ptrs;
  cudaStream_t stream = nullptr;
  ~Arenas() {
    for (void *p : ptrs) cudaFreeAsync(p, stream);
    cudaGetLastError();
  }
};

// Test hook (vr_inject_admission_refusals): the next k admission decisions
// of the request server refuse every cloud of their batch.
static std::atomic<int64_t> g_inj_refuse{0};
void inject_admission_refusals(int64_t k) { g_inj_refuse.store(k, std::memory_order_relaxed); }
static bool take_refusal() {
  int64_t k = g_inj_refuse.load(std::memory_order_relaxed);
  while (k > 0)
    if (g_inj_refuse.compare_exchange_weak(k, k - 1, std::memory_order_relaxed)) return true;
  return false;
}

// Bytes of output a fused cloud writes.
int64_t cloud_out_bytes(const CloudDesc &c) {
  return c.E * (8 + 4 + 8 + 8 + 8) + c.T * (12 + 4 + 12 + 8) + c.n * 8 + 16;
}

// One batch in three asynchronous steps, each ending with an event:
// size -> build (with memory admission) -> finish.
struct BatchJob {
  cudaStream_t s = nullptr;
  int d = 0;
  vr_dtype dtype = VR_I8;
  const void *dpts = nullptr;
  std::vector<CloudDesc> hd;
  CloudDesc *hpin = nullptr;   // optional pinned mirror of hd (async copies)
  int32_t *hord = nullptr;     // optional pinned work-list order
  std::vector<void *> ws;
  CloudDesc *dd = nullptr;
  int32_t *dorder = nullptr;
  int *cursor = nullptr;
  std::shared_ptr<Arenas> ar;
  BatchOut o{};
  int64_t out_bytes = 0;       // admitted output bytes
  cudaEvent_t ev = nullptr;
  int dev = 0;

  ~BatchJob() {
    free_all(ws, s);
    if (ev) cudaEventDestroy(ev);
  }
  CloudDesc *host_descs() { return hpin ? hpin : hd.data(); }

  template <bool F, typename TIn>
  vr_status launch_size() {
    const int nc = (int)hd.size();
    int nmax = 1;
    for (auto &c : hd)
      if (!c.fallback) nmax = std::max(nmax, c.n);
    const int Wmax = (nmax + 31) / 32;
    std::vector<int32_t> order(nc);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return hd[x].n > hd[y].n; });
    int32_t *ord = order.data();
    if (hord) {
      memcpy(hord, order.data(), sizeof(int32_t) * nc);
      ord = hord;
    }
    VR_TRY(dalloc(ws, &dd, nc, s));
    VR_TRY(dalloc(ws, &dorder, nc, s));
    VR_TRY(dalloc(ws, &cursor, 2, s));
    if (hpin) memcpy(hpin, hd.data(), sizeof(CloudDesc) * nc);
    VR_CUDA(cudaMemcpyAsync(dd, host_descs(), sizeof(CloudDesc) * nc, cudaMemcpyHostToDevice, s));
    VR_CUDA(cudaMemcpyAsync(dorder, ord, sizeof(int32_t) * nc, cudaMemcpyHostToDevice, s));
    VR_CUDA(cudaMemsetAsync(cursor, 0, 2 * sizeof(int), s));
    int nsm = 0;
    VR_CUDA(cudaGetDevice(&dev));
    VR_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const size_t smem = al16((size_t)nmax * Wmax * 4) + al16((size_t)nmax * d * 4);
    VR_CUDA(cudaFuncSetAttribute(k_batch_size<F, TIn>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per = 0;
    VR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch_size<F, TIn>, BT, smem));
    const int grid = std::max(1, std::min(nc, nsm * std::max(per, 1)));
    k_batch_size<F, TIn><<<grid, BT, smem, s>>>((const TIn *)dpts, d, dd, dorder, nc, cursor, nmax);
    count_launch();
    VR_CUDA(cudaGetLastError());
    VR_CUDA(cudaMemcpyAsync(host_descs(), dd, sizeof(CloudDesc) * nc, cudaMemcpyDeviceToHost, s));
    if (!ev) VR_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    VR_CUDA(cudaEventRecord(ev, s));
    return VR_OK;
  }

  // After the sizing event.  Admits clouds in order while their output fits
  // `budget` bytes (the first cloud always fits); the others are marked
  // deferred (fallback = 2) and returned in `deferred`.
  template <bool F, typename TIn>
  vr_status launch_build(int64_t budget, std::vector<int> *deferred) {
    const int nc = (int)hd.size();
    if (hpin) memcpy(hd.data(), hpin, sizeof(CloudDesc) * nc);
    int64_t Etot = 0, Ttot = 0, Vtot = 0, Gtot = 0, Ctot = 0, Ktot = 0, Emax = 0, Tmax = 0;
    int nmax = 1;
    bool any = false;
    const bool refuse_all = deferred && take_refusal();
    for (int ci = 0; ci < nc; ++ci) {
      CloudDesc &c = hd[ci];
      if (c.fallback || c.flags) continue;
      const int64_t ob = cloud_out_bytes(c);
      if (deferred && (refuse_all || (any && out_bytes + ob > budget))) {
        c.fallback = 2;
        deferred->push_back(ci);
        continue;
      }
      any = true;
      out_bytes += ob;
      c.eo = Etot;
      c.to = Ttot;
      c.vo = Vtot;
      c.go = Gtot;
      c.co = Ctot;
      c.ko = Ktot;
      Etot += c.E;
      Ttot += c.T;
      Vtot += c.n;
      Gtot += c.E + 1;
      Ctot += c.E + 1;
      Ktot += c.maxdim >= 2 ? c.T + 1 : 0;
      Emax = std::max(Emax, c.E);
      Tmax = std::max(Tmax, c.T);
      nmax = std::max(nmax, c.n);
    }
    ar = std::make_shared<Arenas>();
    ar->stream = s;
    VR_TRY(dalloc(ar->ptrs, &o.everts, 2 * Etot, s));
    VR_TRY(dalloc(ar->ptrs, &o.egrade, Etot, s));
    VR_TRY(dalloc(ar->ptrs, &o.erow, 2 * Etot, s));
    VR_TRY(dalloc(ar->ptrs, &o.ecol, Ctot, s));
    VR_TRY(dalloc(ar->ptrs, &o.tverts, 3 * Ttot, s));
    VR_TRY(dalloc(ar->ptrs, &o.tgrade, Ttot, s));
    VR_TRY(dalloc(ar->ptrs, &o.trow, 3 * Ttot, s));
    VR_TRY(dalloc(ar->ptrs, &o.tcol, Ktot, s));
    VR_TRY(dalloc(ar->ptrs, &o.vverts, Vtot, s));
    VR_TRY(dalloc(ar->ptrs, &o.vgrade, Vtot, s));
    VR_TRY(dalloc(ar->ptrs, &o.gval, Gtot, s));
    if (!any) {
      // Nothing admitted: finish() reads the descriptors back from the pinned
      // mirror, so it must carry the deferral marks set above.
      if (hpin) memcpy(hpin, hd.data(), sizeof(CloudDesc) * nc);
      VR_CUDA(cudaEventRecord(ev, s));
      return VR_OK;
    }
    const ScratchLayout SL = scratch_layout(Emax, Tmax, F);
    const size_t smem = fused_smem(nmax, d);
    VR_CUDA(cudaFuncSetAttribute(k_batch_build<F, TIn>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per = 0, nsm = 0;
    VR_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    VR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch_build<F, TIn>, BT, smem));
    const int grid = std::max(1, std::min(nc, nsm * std::max(per, 1)));
    unsigned char *scratch;
    VR_TRY(dalloc(ws, &scratch, (int64_t)grid * SL.bytes, s));
    if (hpin) memcpy(hpin, hd.data(), sizeof(CloudDesc) * nc);
    VR_CUDA(cudaMemcpyAsync(dd, host_descs(), sizeof(CloudDesc) * nc, cudaMemcpyHostToDevice, s));
    k_batch_build<F, TIn><<<grid, BT, smem, s>>>((const TIn *)dpts, d, dd, dorder, nc, cursor + 1, nmax, scratch,
                                                 SL, o);
    count_launch();
    VR_CUDA(cudaGetLastError());
    VR_CUDA(cudaMemcpyAsync(host_descs(), dd, sizeof(CloudDesc) * nc, cudaMemcpyDeviceToHost, s));
    VR_CUDA(cudaEventRecord(ev, s));
    return VR_OK;
  }

  vr_status size_async() {
    if (dtype == VR_F32) return launch_size<true, float>();
    if (dtype == VR_I8) return launch_size<false, int8_t>();
    return launch_size<false, int32_t>();
  }
  vr_status build_async(int64_t budget, std::vector<int> *deferred) {
    if (dtype == VR_F32) return launch_build<true, float>(budget, deferred);
    if (dtype == VR_I8) return launch_build<false, int8_t>(budget, deferred);
    return launch_build<false, int32_t>(budget, deferred);
  }

  // After the build event: one result per cloud (views sharing the arenas;
  // clouds the fused path declined are built by the single-cloud path here,
  // synchronously on the job's stream).  Deferred clouds get no result.
  void finish(std::vector<vr_complex *> &views, std::vector<vr_status> &status) {
    const int nc = (int)hd.size();
    if (hpin) memcpy(hd.data(), hpin, sizeof(CloudDesc) * nc);
    views.assign(nc, nullptr);
    status.assign(nc, VR_OK);
    for (int ci = 0; ci < nc; ++ci) {
      CloudDesc &c = hd[ci];
      if (c.fallback == 2) continue;
      vr_complex *v = nullptr;
      vr_status st = VR_OK;
      if (c.flags && !(c.flags & F_OVERFLOW)) {
        st = flags_to_status(c.flags);
      } else if (c.fallback) {
        v = new vr_complex();
        v->device = dev;
        const size_t es = dtype == VR_I8 ? 1 : 4;
        st = build_cloud((const unsigned char *)dpts + (size_t)c.pt * d * es, c.n, d, dtype, c.maxdim, c.maxrad, s, v);
        if (st != VR_OK) {
          for (void *p : v->allocs) cudaFreeAsync(p, s);
          delete v;
          v = nullptr;
        }
      } else {
        v = new vr_complex();
        v->owned = false;
        v->arena = ar;
        v->device = dev;
        v->n = c.n;
        v->d = d;
        v->maxdim = c.maxdim;
        v->stream = s;
        v->count[0] = c.n;
        v->count[1] = c.maxdim >= 1 ? c.E : 0;
        v->count[2] = c.maxdim >= 2 ? c.T : 0;
        v->verts[0] = o.vverts + c.vo;
        v->grade[0] = o.vgrade + c.vo;
        v->verts[1] = o.everts + 2 * c.eo;
        v->grade[1] = o.egrade + c.eo;
        v->colptr[1] = o.ecol + c.co;
        v->rowidx[1] = o.erow + 2 * c.eo;
        if (c.maxdim >= 2) {
          v->verts[2] = o.tverts + 3 * c.to;
          v->grade[2] = o.tgrade + c.to;
          v->colptr[2] = o.tcol + c.ko;
          v->rowidx[2] = o.trow + 3 * c.to;
        }
        v->grade_value = o.gval + c.go;
        v->ngrades = c.ngrades;
        v->stats.kept_edges = c.E;
        v->stats.triangles = c.T;
        v->stats.ngrades = c.ngrades;
      }
      views[ci] = v;
      status[ci] = st;
    }
    free_all(ws, s);
  }
};

std::unique_ptr<BatchJob> new_batch_job() { return std::unique_ptr<BatchJob>(new BatchJob()); }

// ------------------------------------------------------- one-launch engine
// A batch shape: CTAs per SM of the persistent launch and the work-list
// order (0: largest cloud first, 1: input order).

// Device buffers, pinned mirrors and the captured graph of one shape:
// (device, dtype, d, largest fused cloud class, cloud-count class, shape).
// The graph copies the parameter block, descriptors and work list in,
// clears the control words, launches k_batch_all (both phases) and copies
// the descriptors and control words out; it only ever reads its inputs from
// the pinned mirrors, so it replays for any batch of its class.
struct BatchEngine {
  int dev = -1;
  vr_dtype dtype = VR_I8;
  int d = 0, nmax = 0, nc_cap = 0, grid = 0;
  vr_batch_shape shape{0, 0};
  size_t smem = 0;
  CloudDesc *d_desc = nullptr;
  int32_t *d_order = nullptr;
  unsigned int *d_ctr = nullptr;
  BatchParams *d_par = nullptr;
  unsigned char *h_mem = nullptr;  // pinned: params, control words, descriptors, work list
  BatchParams *h_par = nullptr;
  unsigned int *h_ctr = nullptr;
  CloudDesc *h_desc = nullptr;
  int32_t *h_order = nullptr;
  unsigned char *scratch = nullptr;
  int64_t scratch_bytes = 0;
  int64_t hint[6] = {0, 0, 0, 0, 0, 0};  // arena capacities that held the last batches
  int64_t emax_hint = 0, tmax_hint = 0;
  bool hinted = false, busy = false;
  cudaGraphExec_t exec = nullptr;
  bool graph_failed = false;
  ~BatchEngine() {
    if (exec) cudaGraphExecDestroy(exec);
    cudaDeviceSynchronize();
    for (void *p : {(void *)d_desc, (void *)d_order, (void *)d_ctr, (void *)d_par, (void *)scratch})
      if (p) cudaFree(p);
    if (h_mem) cudaFreeHost(h_mem);
    cudaGetLastError();
  }
};

static std::mutex g_eng_mu;
static std::vector<std::unique_ptr<BatchEngine>> g_engines;
static thread_local vr_batch_shape g_pinned_shape{0, 0};
struct TuneRec {
  int dev;
  vr_dtype dtype;
  int d, nmax;
  vr_batch_shape best;
  std::vector<std::pair<vr_batch_shape, double>> cand;
};
static std::vector<TuneRec> g_tuned;
static thread_local vr_batch_shape g_last_shape{0, 0};
static thread_local TuneRec g_last_tune{};  // the tuner's record of the last batch's class (cand empty: none)

template <bool F, typename TIn>
static void *batch_all_fn() { return (void *)k_batch_all<F, TIn>; }
static void *batch_kernel(vr_dtype dt) {
  if (dt == VR_F32) return batch_all_fn<true, float>();
  if (dt == VR_I8) return batch_all_fn<false, int8_t>();
  return batch_all_fn<false, int32_t>();
}

// Largest CTAs per SM the persistent launch can keep co-resident.
static int batch_max_per_sm(vr_dtype dt, size_t smem) {
  void *fn = batch_kernel(dt);
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  int per = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, BT, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return per;
}

static vr_status launch_all(BatchEngine &g, int phases, cudaStream_t s) {
  void *fn = batch_kernel(g.dtype);
  int d = g.d, nmax = g.nmax;
  void *args[] = {&g.d_par, &d, &g.d_desc, &g.d_order, &nmax, &g.d_ctr, &phases};
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(g.grid);
  cfg.blockDim = dim3(BT);
  cfg.dynamicSmemBytes = g.smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  VR_CUDA(cudaLaunchKernelExC(&cfg, fn, args));
  count_launch();
  return VR_OK;
}

static vr_status make_engine(BatchEngine &g, cudaStream_t s) {
  VR_CUDA(cudaFuncSetAttribute(batch_kernel(g.dtype), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g.smem));
  VR_CUDA(cudaMalloc((void **)&g.d_desc, sizeof(CloudDesc) * g.nc_cap));
  VR_CUDA(cudaMalloc((void **)&g.d_order, sizeof(int32_t) * g.nc_cap));
  VR_CUDA(cudaMalloc((void **)&g.d_ctr, sizeof(unsigned int) * BC_WORDS));
  VR_CUDA(cudaMalloc((void **)&g.d_par, sizeof(BatchParams)));
  // Pinned layout: parameter block, control words, descriptors, work list
  // (each 256-byte aligned).
  auto up256 = [](size_t v) { return (v + 255) & ~(size_t)255; };
  const size_t o_ctr = up256(sizeof(BatchParams));
  const size_t o_desc = o_ctr + up256(sizeof(unsigned int) * BC_WORDS);
  const size_t o_order = o_desc + up256(sizeof(CloudDesc) * g.nc_cap);
  const size_t hb = o_order + up256(sizeof(int32_t) * g.nc_cap);
  VR_CUDA(cudaMallocHost((void **)&g.h_mem, hb));
  memset(g.h_mem, 0, hb);
  g.h_par = (BatchParams *)g.h_mem;
  g.h_ctr = (unsigned int *)(g.h_mem + o_ctr);
  g.h_desc = (CloudDesc *)(g.h_mem + o_desc);
  g.h_order = (int32_t *)(g.h_mem + o_order);
  // The graph of both phases (falls back to plain launches if it cannot be
  // captured).
  cudaStream_t cs = nullptr;
  cudaGraph_t graph = nullptr;
  bool ok = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) == cudaSuccess &&
            cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
  if (ok) {
    cudaMemcpyAsync(g.d_par, g.h_par, sizeof(BatchParams), cudaMemcpyHostToDevice, cs);
    cudaMemcpyAsync(g.d_desc, g.h_desc, sizeof(CloudDesc) * g.nc_cap, cudaMemcpyHostToDevice, cs);
    cudaMemcpyAsync(g.d_order, g.h_order, sizeof(int32_t) * g.nc_cap, cudaMemcpyHostToDevice, cs);
    cudaMemsetAsync(g.d_ctr, 0, sizeof(unsigned int) * BC_WORDS, cs);
    const vr_status ls = launch_all(g, 3, cs);
    cudaMemcpyAsync(g.h_desc, g.d_desc, sizeof(CloudDesc) * g.nc_cap, cudaMemcpyDeviceToHost, cs);
    cudaMemcpyAsync(g.h_ctr, g.d_ctr, sizeof(unsigned int) * BC_WORDS, cudaMemcpyDeviceToHost, cs);
    ok = cudaStreamEndCapture(cs, &graph) == cudaSuccess && ls == VR_OK && graph &&
         cudaGraphInstantiate(&g.exec, graph, 0) == cudaSuccess;
  }
  if (graph) cudaGraphDestroy(graph);
  if (cs) cudaStreamDestroy(cs);
  if (!ok) {
    g.exec = nullptr;
    g.graph_failed = true;
  }
  cudaGetLastError();
  (void)s;
  return VR_OK;
}

// Check out the engine of a shape (made on first use; a second user of a
// busy engine gets a private one, released after the call).
static BatchEngine *get_engine(int dev, vr_dtype dt, int d, int nmax, int nc, vr_batch_shape sh, cudaStream_t s,
                               std::unique_ptr<BatchEngine> &priv, vr_status *err) {
  int nc_cap = 64;
  while (nc_cap < nc) nc_cap *= 2;
  const size_t smem = smem_layout(nmax, d).bytes;
  const int per = batch_max_per_sm(dt, smem);
  if (per < 1) {
    set_error("the batch kernel does not fit one SM with %zu bytes of shared memory", smem);
    *err = VR_ERR_INTERNAL;
    return nullptr;
  }
  const int cps = std::min(per, std::max(1, sh.ctas_per_sm));
  {
    std::lock_guard<std::mutex> lk(g_eng_mu);
    for (auto &e : g_engines)
      if (e->dev == dev && e->dtype == dt && e->d == d && e->nmax == nmax && e->nc_cap == nc_cap &&
          e->shape.ctas_per_sm == cps && e->shape.order == sh.order && !e->busy) {
        e->busy = true;
        *err = VR_OK;
        return e.get();
      }
  }
  std::unique_ptr<BatchEngine> g(new BatchEngine());
  g->dev = dev;
  g->dtype = dt;
  g->d = d;
  g->nmax = nmax;
  g->nc_cap = nc_cap;
  g->shape = vr_batch_shape{cps, sh.order};
  g->smem = smem;
  g->grid = num_sms() * cps;
  *err = make_engine(*g, s);
  if (*err != VR_OK) return nullptr;
  g->busy = true;
  std::lock_guard<std::mutex> lk(g_eng_mu);
  if (g_engines.size() < 32) {
    g_engines.push_back(std::move(g));
    return g_engines.back().get();
  }
  priv = std::move(g);
  return priv.get();
}

static void release_engine(BatchEngine *g) {
  std::lock_guard<std::mutex> lk(g_eng_mu);
  g->busy = false;
}

// Scratch for the per-CTA slices (largest E and T of one cloud).
static vr_status engine_scratch(BatchEngine &g, int64_t emax, int64_t tmax, bool F) {
  const ScratchLayout SL = scratch_layout(emax, tmax, F);
  const int64_t need = (int64_t)g.grid * SL.bytes;
  if (need > g.scratch_bytes) {
    if (g.scratch) {
      VR_CUDA(cudaStreamSynchronize(nullptr));
      cudaFree(g.scratch);
      g.scratch = nullptr;
      g.scratch_bytes = 0;
    }
    VR_CUDA(cudaMalloc((void **)&g.scratch, (size_t)need));
    g.scratch_bytes = need;
  }
  g.emax_hint = emax;
  g.tmax_hint = tmax;
  g.h_par->scratch = g.scratch;
  g.h_par->SL = SL;
  g.h_par->emax_cap = emax;
  g.h_par->tmax_cap = tmax;
  return VR_OK;
}

// Output arenas of capacities cap[6] (edges, triangles, vertices, grade
// values, edge colptr, triangle colptr), shared by the batch's results.
static vr_status alloc_arenas(std::shared_ptr<Arenas> &ar, BatchOut &o, const int64_t cap[6], cudaStream_t s) {
  ar = std::make_shared<Arenas>();
  ar->stream = s;
  VR_TRY(dalloc(ar->ptrs, &o.everts, 2 * cap[0], s));
  VR_TRY(dalloc(ar->ptrs, &o.egrade, cap[0], s));
  VR_TRY(dalloc(ar->ptrs, &o.erow, 2 * cap[0], s));
  VR_TRY(dalloc(ar->ptrs, &o.ecol, cap[4], s));
  VR_TRY(dalloc(ar->ptrs, &o.tverts, 3 * cap[1], s));
  VR_TRY(dalloc(ar->ptrs, &o.tgrade, cap[1], s));
  VR_TRY(dalloc(ar->ptrs, &o.trow, 3 * cap[1], s));
  VR_TRY(dalloc(ar->ptrs, &o.tcol, cap[5], s));
  VR_TRY(dalloc(ar->ptrs, &o.vverts, cap[2], s));
  VR_TRY(dalloc(ar->ptrs, &o.vgrade, cap[2], s));
  VR_TRY(dalloc(ar->ptrs, &o.gval, cap[3], s));
  return VR_OK;
}

// One batch on one engine: returns the device time of the launch(es) in *ms
// (events around the graph or the launches) when ms is given.
static vr_status run_engine(BatchEngine &g, BatchJob &job, cudaStream_t s, float *ms) {
  const int nc = (int)job.hd.size();
  const bool F = g.dtype == VR_F32;
  memcpy(g.h_desc, job.hd.data(), sizeof(CloudDesc) * nc);
  std::vector<int32_t> order(nc);
  std::iota(order.begin(), order.end(), 0);
  if (g.shape.order == 0)
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return job.hd[x].n > job.hd[y].n; });
  memcpy(g.h_order, order.data(), sizeof(int32_t) * nc);
  BatchParams &P = *g.h_par;
  P.pts = job.dpts;
  P.n_clouds = nc;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (ms) {
    VR_CUDA(cudaEventCreate(&e0));
    VR_CUDA(cudaEventCreate(&e1));
  }
  auto finish_events = [&]() {
    if (ms && e0) {
      cudaEventSynchronize(e1);
      cudaEventElapsedTime(ms, e0, e1);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  };
  if (!g.hinted) {
    // First batch of this engine: size it alone for exact capacities.
    VR_TRY(engine_scratch(g, 1, 1, F));
    for (int k = 0; k < 6; ++k) P.cap[k] = INT64_MAX;
    VR_CUDA(cudaMemcpyAsync(g.d_par, g.h_par, sizeof(BatchParams), cudaMemcpyHostToDevice, s));
    VR_CUDA(cudaMemcpyAsync(g.d_desc, g.h_desc, sizeof(CloudDesc) * nc, cudaMemcpyHostToDevice, s));
    VR_CUDA(cudaMemcpyAsync(g.d_order, g.h_order, sizeof(int32_t) * nc, cudaMemcpyHostToDevice, s));
    VR_CUDA(cudaMemsetAsync(g.d_ctr, 0, sizeof(unsigned int) * BC_WORDS, s));
    VR_TRY(launch_all(g, 1, s));
    VR_CUDA(cudaMemcpyAsync(g.h_ctr, g.d_ctr, sizeof(unsigned int) * BC_WORDS, cudaMemcpyDeviceToHost, s));
    VR_CUDA(cudaStreamSynchronize(s));
    if (g.h_ctr[4]) {
      finish_events();
      return flags_to_status((int32_t)g.h_ctr[4]);
    }
    const int64_t *tot = (const int64_t *)(g.h_ctr + 6);
    for (int k = 0; k < 6; ++k) g.hint[k] = tot[k];
    g.emax_hint = tot[6];
    g.tmax_hint = tot[7];
    g.hinted = true;
  }
  VR_TRY(engine_scratch(g, std::max<int64_t>(g.emax_hint, 1), std::max<int64_t>(g.tmax_hint, 1), F));
  int64_t cap[6];
  for (int k = 0; k < 6; ++k) cap[k] = std::max<int64_t>(g.hint[k], 1);
  VR_TRY(alloc_arenas(job.ar, job.o, cap, s));
  P.out = job.o;
  for (int k = 0; k < 6; ++k) P.cap[k] = cap[k];
  if (ms) VR_CUDA(cudaEventRecord(e0, s));
  if (g.exec) {
    VR_CUDA(cudaGraphLaunch(g.exec, s));
    count_launch();
  } else {
    VR_CUDA(cudaMemcpyAsync(g.d_par, g.h_par, sizeof(BatchParams), cudaMemcpyHostToDevice, s));
    VR_CUDA(cudaMemcpyAsync(g.d_desc, g.h_desc, sizeof(CloudDesc) * g.nc_cap, cudaMemcpyHostToDevice, s));
    VR_CUDA(cudaMemcpyAsync(g.d_order, g.h_order, sizeof(int32_t) * g.nc_cap, cudaMemcpyHostToDevice, s));
    VR_CUDA(cudaMemsetAsync(g.d_ctr, 0, sizeof(unsigned int) * BC_WORDS, s));
    VR_TRY(launch_all(g, 3, s));
    VR_CUDA(cudaMemcpyAsync(g.h_desc, g.d_desc, sizeof(CloudDesc) * g.nc_cap, cudaMemcpyDeviceToHost, s));
    VR_CUDA(cudaMemcpyAsync(g.h_ctr, g.d_ctr, sizeof(unsigned int) * BC_WORDS, cudaMemcpyDeviceToHost, s));
  }
  if (ms) VR_CUDA(cudaEventRecord(e1, s));
  VR_CUDA(cudaStreamSynchronize(s));
  if (g.h_ctr[4]) {
    finish_events();
    return flags_to_status((int32_t)g.h_ctr[4]);
  }
  const int64_t *tot = (const int64_t *)(g.h_ctr + 6);
  if (g.h_ctr[5]) {
    // A capacity was short: exact arenas (and scratch), phase 2 again.
    for (int k = 0; k < 6; ++k) cap[k] = std::max<int64_t>(tot[k], 1);
    job.ar.reset();
    VR_TRY(alloc_arenas(job.ar, job.o, cap, s));
    VR_TRY(engine_scratch(g, std::max<int64_t>(tot[6], 1), std::max<int64_t>(tot[7], 1), F));
    P.out = job.o;
    for (int k = 0; k < 6; ++k) P.cap[k] = cap[k];
    g.h_ctr[1] = 0;
    g.h_ctr[5] = 0;
    VR_CUDA(cudaMemcpyAsync(g.d_par, g.h_par, sizeof(BatchParams), cudaMemcpyHostToDevice, s));
    VR_CUDA(cudaMemcpyAsync(g.d_ctr, g.h_ctr, sizeof(unsigned int) * BC_WORDS, cudaMemcpyHostToDevice, s));
    VR_TRY(launch_all(g, 2, s));
    VR_CUDA(cudaMemcpyAsync(g.h_desc, g.d_desc, sizeof(CloudDesc) * nc, cudaMemcpyDeviceToHost, s));
    VR_CUDA(cudaMemcpyAsync(g.h_ctr, g.d_ctr, sizeof(unsigned int) * BC_WORDS, cudaMemcpyDeviceToHost, s));
    if (ms) VR_CUDA(cudaEventRecord(e1, s));
    VR_CUDA(cudaStreamSynchronize(s));
    if (g.h_ctr[4]) {
      finish_events();
      return flags_to_status((int32_t)g.h_ctr[4]);
    }
  }
  // Capacities for the next batches: what this one needed, plus slack.
  for (int k = 0; k < 6; ++k) g.hint[k] = std::max(g.hint[k], tot[k] + tot[k] / 16);
  g.emax_hint = std::max(g.emax_hint, tot[6]);
  g.tmax_hint = std::max(g.tmax_hint, tot[7]);
  memcpy(job.hd.data(), g.h_desc, sizeof(CloudDesc) * nc);
  finish_events();
  return VR_OK;
}

// The shapes the tuner tries for a class: every CTAs-per-SM count the
// launch allows, in both work-list orders.
static std::vector<vr_batch_shape> tune_candidates(int per) {
  std::vector<vr_batch_shape> v;
  for (int k = 1; k <= per; ++k)
    for (int o = 0; o < 2; ++o) v.push_back(vr_batch_shape{k, o});
  return v;
}

// The batch through the one-launch engine.  Shape: the pinned one, else the
// tuned one of the batch's class (device, dtype, d, largest fused cloud
// rounded up to 64 points); a class seen for the first time is tuned now:
// each candidate shape builds the whole batch twice and the second run's
// device time counts (the first carries the engine's one-off sizing and
// graph instantiation).
static vr_status batch_onelaunch(BatchJob &job, cudaStream_t s) {
  int nmax = 0;
  for (auto &c : job.hd)
    if (!c.fallback) nmax = std::max(nmax, c.n);
  if (nmax == 0) {  // nothing for the fused kernels: the single-cloud path builds every cloud
    const int64_t cap[6] = {1, 1, 1, 1, 1, 1};
    return alloc_arenas(job.ar, job.o, cap, s);
  }
  int ncls = (nmax + 63) / 64 * 64;
  if (!fused_fits(ncls, job.d)) ncls = nmax;
  vr_batch_shape sh = g_pinned_shape;
  g_last_tune = TuneRec{};
  if (sh.ctas_per_sm <= 0) {
    bool found = false;
    {
      std::lock_guard<std::mutex> lk(g_eng_mu);
      for (auto &t : g_tuned)
        if (t.dev == job.dev && t.dtype == job.dtype && t.d == job.d && t.nmax == ncls) {
          sh = t.best;
          g_last_tune = t;
          found = true;
        }
    }
    if (!found) {
      TuneRec rec{job.dev, job.dtype, job.d, ncls, vr_batch_shape{0, 0}, {}};
      const int per = batch_max_per_sm(job.dtype, smem_layout(ncls, job.d).bytes);
      double best = 1e300;
      for (const vr_batch_shape &cand : tune_candidates(std::max(per, 1))) {
        std::unique_ptr<BatchEngine> priv;
        vr_status es;
        BatchEngine *g = get_engine(job.dev, job.dtype, job.d, ncls, (int)job.hd.size(), cand, s, priv, &es);
        if (!g) return es;
        float ms = 0.f;
        vr_status rs = VR_OK;
        for (int rep = 0; rep < 2 && rs == VR_OK; ++rep) {
          BatchJob tj;
          tj.s = s;
          tj.d = job.d;
          tj.dtype = job.dtype;
          tj.dpts = job.dpts;
          tj.dev = job.dev;
          tj.hd = job.hd;
          rs = run_engine(*g, tj, s, &ms);
        }
        release_engine(g);
        if (rs != VR_OK) return rs;
        rec.cand.push_back({g->shape, (double)ms});
        if (ms < best) {
          best = ms;
          rec.best = g->shape;
        }
      }
      sh = rec.best;
      std::lock_guard<std::mutex> lk(g_eng_mu);
      g_tuned.push_back(rec);
      g_last_tune = rec;
      // Keep the winner's engine only: the others hold per-CTA scratch.
      for (size_t k = 0; k < g_engines.size();) {
        BatchEngine &e = *g_engines[k];
        if (!e.busy && e.dev == job.dev && e.dtype == job.dtype && e.d == job.d && e.nmax == ncls &&
            !(e.shape.ctas_per_sm == sh.ctas_per_sm && e.shape.order == sh.order))
          g_engines.erase(g_engines.begin() + k);
        else
          ++k;
      }
    }
  }
  std::unique_ptr<BatchEngine> priv;
  vr_status es;
  BatchEngine *g = get_engine(job.dev, job.dtype, job.d, ncls, (int)job.hd.size(), sh, s, priv, &es);
  if (!g) return es;
  const vr_status rs = run_engine(*g, job, s, nullptr);
  g_last_shape = g->shape;
  release_engine(g);
  return rs;
}

// ---- asynchronous job interface (jobs.h)
struct Job {
  BatchJob b;
};

vr_status check_cloud_args(int64_t n, int d, vr_dtype dtype, int maxdim, double maxrad) {
  if (dtype != VR_I8 && dtype != VR_I32 && dtype != VR_F32) { set_error("unknown dtype"); return VR_ERR_ARG; }
  if (d < 1) { set_error("d = %d must be >= 1", d); return VR_ERR_ARG; }
  CloudDesc c;
  return make_desc(c, 0, n, d, dtype, maxdim, maxrad);
}

size_t job_pinned_bytes(size_t n_clouds) { return n_clouds * (sizeof(CloudDesc) + sizeof(int32_t)) + 64; }

Job *job_create(cudaStream_t s, const void *dpts, int d, vr_dtype dtype, const std::vector<JobCloud> &clouds,
                void *pinned, vr_status *err) {
  Job *j = new Job();
  if (pinned) {
    j->b.hpin = (CloudDesc *)pinned;
    j->b.hord = (int32_t *)((char *)pinned + clouds.size() * sizeof(CloudDesc));
  }
  j->b.s = s;
  j->b.d = d;
  j->b.dtype = dtype;
  j->b.dpts = dpts;
  j->b.hd.resize(clouds.size());
  for (size_t i = 0; i < clouds.size(); ++i) {
    const JobCloud &c = clouds[i];
    const vr_status st = make_desc(j->b.hd[i], c.pt, c.n, d, dtype, c.maxdim, c.maxrad);
    if (st != VR_OK) {
      *err = st;
      delete j;
      return nullptr;
    }
  }
  *err = VR_OK;
  return j;
}
vr_status job_size_async(Job *j) { return j->b.size_async(); }
vr_status job_build_async(Job *j, int64_t budget, std::vector<int> *deferred) {
  return j->b.build_async(budget, deferred);
}
bool job_ready(Job *j) {
  const cudaError_t e = cudaEventQuery(j->b.ev);
  if (e == cudaErrorNotReady) {
    cudaGetLastError();
    return false;
  }
  return true;
}
int64_t job_out_bytes(Job *j) { return j->b.out_bytes; }
void job_finish(Job *j, std::vector<vr_complex *> &results, std::vector<vr_status> &status, bool detach) {
  j->b.finish(results, status);
  if (detach) {
    if (j->b.ar) j->b.ar->stream = nullptr;
    for (vr_complex *v : results)
      if (v) v->stream = nullptr;
  }
}
void job_destroy(Job *j) { delete j; }

}  // namespace vr

struct vr_batch {
  int32_t n_clouds = 0;
  cudaStream_t stream = nullptr;
  std::vector<void *> allocs;              // the input copy, if any
  std::vector<vr_complex *> views;         // one per cloud
  std::vector<vr_status> status;           // per cloud
  int64_t total_simplices = 0;
};

// ================================================================ C ABI

using namespace vr;

extern "C" {

vr_status vr_build_batch(const void *points, const int64_t *offsets, int32_t n_clouds, int32_t d, vr_dtype dtype,
                         const int32_t *maxdim, const double *maxrad, vr_stream_t stream, vr_batch **out) {
  if (!out) { set_error("out is NULL"); return VR_ERR_ARG; }
  *out = nullptr;
  if (!points || !offsets) { set_error("points or offsets is NULL"); return VR_ERR_ARG; }
  if (n_clouds < 1) { set_error("n_clouds = %d must be >= 1", n_clouds); return VR_ERR_ARG; }
  if (d < 1) { set_error("d = %d must be >= 1", d); return VR_ERR_ARG; }
  if (dtype != VR_I8 && dtype != VR_I32 && dtype != VR_F32) { set_error("unknown dtype"); return VR_ERR_ARG; }
  if (offsets[0] != 0) { set_error("offsets[0] must be 0"); return VR_ERR_ARG; }
  int dev = 0;
  VR_CUDA(cudaGetDevice(&dev));
  auto job = new_batch_job();
  job->dev = dev;
  job->hd.resize(n_clouds);
  for (int i = 0; i < n_clouds; ++i)
    VR_TRY(make_desc(job->hd[i], offsets[i], offsets[i + 1] - offsets[i], d, dtype, maxdim ? maxdim[i] : 2,
                     maxrad ? maxrad[i] : INFINITY));
  keep_pool_warm();
  cudaStream_t s = (cudaStream_t)stream;
  vr_batch *b = new (std::nothrow) vr_batch();
  if (!b) { set_error("host allocation failed"); return VR_ERR_OOM; }
  b->n_clouds = n_clouds;
  b->stream = s;
  const size_t es = dtype == VR_I8 ? 1 : 4;
  const size_t bytes = (size_t)offsets[n_clouds] * d * es;
  const void *dpts = points;
  cudaPointerAttributes pa;
  const bool on_dev = cudaPointerGetAttributes(&pa, points) == cudaSuccess &&
                      (pa.type == cudaMemoryTypeDevice || pa.type == cudaMemoryTypeManaged);
  cudaGetLastError();
  if (!on_dev) {
    void *p = nullptr;
    if (dev_malloc(&p, bytes, s) != cudaSuccess) {
      cudaGetLastError();
      delete b;
      set_error("device allocation for the input copy failed");
      return VR_ERR_OOM;
    }
    b->allocs.push_back(p);
    cudaMemcpyAsync(p, points, bytes, cudaMemcpyHostToDevice, s);
    dpts = p;
  }
  job->s = s;
  job->d = d;
  job->dtype = dtype;
  job->dpts = dpts;
  vr_status st = batch_onelaunch(*job, s);
  if (st != VR_OK) {
    vr_batch_free(b);
    return st;
  }
  job->finish(b->views, b->status);
  for (vr_complex *v : b->views)
    if (v) {
      v->in_batch = true;
      b->total_simplices += v->count[0] + v->count[1] + v->count[2];
    }
  *out = b;
  return VR_OK;
}

vr_status vr_batch_set_shape(const vr_batch_shape *shape) {
  if (shape && shape->ctas_per_sm > 0 && (shape->order < 0 || shape->order > 1)) {
    set_error("order %d outside {0, 1}", shape->order);
    return VR_ERR_ARG;
  }
  g_pinned_shape = shape ? *shape : vr_batch_shape{0, 0};
  if (g_pinned_shape.ctas_per_sm < 0) g_pinned_shape.ctas_per_sm = 0;
  return VR_OK;
}

vr_status vr_batch_get_shape(vr_batch_shape *used, int32_t *n_cand, vr_batch_shape *cand, double *cand_ms,
                             int32_t max_cand) {
  if (used) *used = g_last_shape;
  const int nc = (int)g_last_tune.cand.size();
  if (n_cand) *n_cand = nc;
  for (int k = 0; k < nc && k < max_cand; ++k) {
    if (cand) cand[k] = g_last_tune.cand[k].first;
    if (cand_ms) cand_ms[k] = g_last_tune.cand[k].second;
  }
  return VR_OK;
}

vr_status vr_batch_tune_reset(void) {
  std::lock_guard<std::mutex> lk(g_eng_mu);
  g_tuned.clear();
  return VR_OK;
}

vr_status vr_batch_get(const vr_batch *b, int32_t cloud, const vr_complex **view, vr_status *cloud_status) {
  if (!b || !view) { set_error("NULL argument"); return VR_ERR_ARG; }
  if (cloud < 0 || cloud >= b->n_clouds) { set_error("cloud %d outside [0, %d)", cloud, b->n_clouds); return VR_ERR_ARG; }
  *view = b->views[cloud];
  if (cloud_status) *cloud_status = b->status[cloud];
  return VR_OK;
}

vr_status vr_batch_info(const vr_batch *b, int32_t *n_clouds, int64_t *total_simplices, int32_t *n_failed) {
  if (!b) { set_error("NULL batch"); return VR_ERR_ARG; }
  if (n_clouds) *n_clouds = b->n_clouds;
  if (total_simplices) *total_simplices = b->total_simplices;
  if (n_failed) {
    int32_t f = 0;
    for (auto s : b->status) f += s != VR_OK;
    *n_failed = f;
  }
  return VR_OK;
}

void vr_batch_free(vr_batch *b) {
  if (!b) return;
  for (vr_complex *v : b->views) {
    if (!v) continue;
    if (v->owned)
      for (void *p : v->allocs) cudaFreeAsync(p, b->stream);
    delete v;
  }
  free_all(b->allocs, b->stream);
  cudaGetLastError();
  delete b;
}

}  // extern "C"
