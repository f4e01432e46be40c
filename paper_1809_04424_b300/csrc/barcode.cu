// barcode.cu -- persistence barcodes of a built complex on the GPU.
//
// The reduction of the filtered boundary matrix over F2 (Algorithm 1; the
// pivot/bar rule of Fig. 4's caption) pairs simplices (s, j): s of
// dimension k is the low of the reduced column j of dimension k+1, and
// [grade(s), grade(j)) is a bar.  The pairing does not depend on which
// left-to-right column additions reach the reduced form, so it is computed
// here by two parallel routes that reach the same pairs:
//
//  * dimension 0 (vertices x edges): the reduced column of edge j is
//    {root(A), root(B)} when j joins components A and B (roots = the
//    smallest vertex id, the oldest vertex), so j kills max(root(A),
//    root(B)); edges inside one component reduce to zero.  The killing edges
//    are the minimum spanning forest under the edge order (Boruvka rounds,
//    order index as the unique weight); one CTA then replays the forest
//    edges in order with a union-find to name the killed vertices.
//  * dimension 1 (edges x triangles): the coboundary matrix (the boundary
//    matrix transposed with both orders reversed; the cohomology variant of
//    the same reduction) is reduced instead.  Columns are the edges outside
//    the forest (forest edges reduce to zero there: clearing), youngest
//    first; a column lists the triangles containing the edge, its pivot is
//    the oldest.  Columns are taken in processing order in batches: each
//    column of a batch adds final columns owning its pivot (every addition
//    uses a final column, as in the sequential algorithm), then one CTA
//    finalises the longest prefix of the batch whose pivots differ; the
//    first column whose pivot repeats a younger one adds that (now final)
//    column on the next pass.  Column sums go to a growing pool.
//
// Bars are listed in the order of the killing simplex, then the essential
// (never killed) positive simplices in their own order; zero-length bars are
// dropped.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <vector>

#include "complex.h"
#include "prims.cuh"
#include "prof.h"

namespace vr {

constexpr int BC_THREADS = 256;

static unsigned bc_grid(int64_t work) {
  const int64_t g = (work + BC_THREADS - 1) / BC_THREADS;
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(g, (int64_t)num_sms() * 16));
}

// ------------------------------------------------------------ dimension 0

static __global__ void k_bv_init(int n, int32_t *comp, int32_t *best) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    comp[v] = v;
    best[v] = INT_MAX;
  }
}

// Each component's lightest (oldest) edge to another component.
static __global__ void k_bv_choose(const int32_t *everts, int64_t E, const int32_t *comp, int32_t *best) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < E; j += (int64_t)gridDim.x * blockDim.x) {
    const int ca = comp[everts[2 * j]], cb = comp[everts[2 * j + 1]];
    if (ca != cb) {
      atomicMin(&best[ca], (int32_t)j);
      atomicMin(&best[cb], (int32_t)j);
    }
  }
}

// Root c hooks onto the component across its chosen edge (a mutual choice
// keeps the smaller root); the edge joins the forest.  Reads comp, writes next.
static __global__ void k_bv_hook(const int32_t *everts, int n, const int32_t *comp, const int32_t *best,
                                 int32_t *next, uint8_t *msf, int32_t *changed) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
    int32_t to = comp[c];
    if (to == c && best[c] != INT_MAX) {
      const int32_t j = best[c];
      msf[j] = 1;
      const int ca = comp[everts[2 * j]], cb = comp[everts[2 * j + 1]];
      const int other = ca == c ? cb : ca;
      if (!(best[other] == j && c < other)) to = other;
      *changed = 1;
    }
    next[c] = to;
  }
}

// comp[v] = the root reached through next (a forest: hooks never close a cycle).
static __global__ void k_bv_jump(int n, const int32_t *next, int32_t *comp, int32_t *best) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    int r = next[v];
    for (int guard = 0; next[r] != r && guard < 8192; ++guard) r = next[r];
    comp[v] = r;
    best[v] = INT_MAX;
  }
}

// Replay the forest edges in filtration order (one thread; n <= 8192 vertices
// in shared memory): edge j joining roots ra, rb kills max(ra, rb).
static __global__ void __launch_bounds__(32) k_elder(const int32_t *everts, const int32_t *fedges, const int64_t *nf,
                                                     int n, int32_t *killed_by_edge) {
  __shared__ int32_t parent[VR_MAX_POINTS];
  for (int v = threadIdx.x; v < n; v += 32) parent[v] = v;
  __syncwarp();
  if (threadIdx.x != 0) return;
  const int m = (int)*nf;
  for (int q = 0; q < m; ++q) {
    const int32_t j = fedges[q];
    int a = everts[2 * j], b = everts[2 * j + 1];
    while (parent[a] != a) { parent[a] = parent[parent[a]]; a = parent[a]; }
    while (parent[b] != b) { parent[b] = parent[parent[b]]; b = parent[b]; }
    const int s = max(a, b), r = min(a, b);
    parent[s] = r;
    killed_by_edge[j] = s;
  }
}

static __global__ void k_u8_to_i32(const uint8_t *f, int64_t L, int32_t *o) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < L; q += (int64_t)gridDim.x * blockDim.x)
    o[q] = f[q];
}

// Indices q with flag[q] set, in order (pos = exclusive scan of flag).
static __global__ void k_compact_idx(const int32_t *flag, const int64_t *pos, int64_t L, int32_t *out) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < L; q += (int64_t)gridDim.x * blockDim.x)
    if (flag[q]) out[pos[q]] = (int32_t)q;
}

// ------------------------------------------------------------ dimension 1

// Coboundary entries (face, coface) in coface order; `faces` faces per
// coface in its boundary column.
static __global__ void k_cob_keys(const int32_t *rows, int64_t T, int faces, uint64_t *keys, int32_t *cnt) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < faces * T;
       p += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t e = (uint32_t)rows[p];
    keys[p] = ((uint64_t)e << 32) | (uint64_t)(p / faces);
    atomicAdd(&cnt[e], 1);
  }
}

static __global__ void k_cob_cols(const uint64_t *keys, int64_t L, int32_t *pool) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < L; p += (int64_t)gridDim.x * blockDim.x)
    pool[p] = (int32_t)(uint32_t)keys[p];
}

// Columns of the reduction: the positive simplices (not killing one of the
// dimension below: neg8 != 0 / neg32 >= 0 mark the negative ones) with their
// coface list.
static __global__ void k_col_init(int64_t E, const uint8_t *neg8, const int32_t *neg32, const int32_t *cptr,
                                  int64_t *coff, int32_t *clen) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x) {
    const bool neg = (neg8 && neg8[e]) || (neg32 && neg32[e] >= 0);
    coff[e] = cptr[e];
    clen[e] = neg ? 0 : cptr[e + 1] - cptr[e];
  }
}

// Active columns (outside the forest, with cofaces), ascending edge order.
static __global__ void k_active_flags(int64_t E, const int32_t *clen, int32_t *flag) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x)
    flag[e] = clen[e] > 0;
}

constexpr int BC_BATCH = 1024;
// Working columns of at least g_dense_min entries continue as bitsets
// (negative: never); the slots take at most DENSE_BITS_MAX bytes.
static int64_t g_dense_min = 4096;
constexpr int64_t DENSE_BITS_MAX = int64_t(1) << 30;

// Symmetric difference of two ascending lists A (la) and B (lb) into out by
// one CTA of BC_THREADS threads, in merge-path tiles of BC_TILE merged
// entries: both slices of a tile are staged in shared memory (coalesced),
// each thread merges BC_PER consecutive entries (A first on ties, so an
// entry present in both lists is an A entry directly followed by the equal B
// entry), drops the entries that cancel, and a block scan places the rest.
// Returns the output length (to every thread).
// A column's chain of additions is serial, so one column gets a whole
// 1024-thread CTA (the longest chains decide the reduction's time).
constexpr int BR_THREADS = 1024;
constexpr int BC_PER = 16;
constexpr int BC_TILE = BR_THREADS * BC_PER;

struct SymdiffSmem {
  int32_t a[BC_TILE], b[BC_TILE];
  int64_t sh[33];
  int64_t split[BR_THREADS + 1];  // A entries before each tile boundary of a group of tiles
};
constexpr size_t BR_SMEM = sizeof(SymdiffSmem) + 64;

// Entries of A before merged position d (A first on ties).
__device__ __forceinline__ int64_t merge_split(const int32_t *A, int64_t la, const int32_t *B, int64_t lb, int64_t d) {
  int64_t lo = d - lb > 0 ? d - lb : 0, hi = d < la ? d : la;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (__ldcg(A + mid) <= __ldcg(B + (d - mid - 1))) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

__device__ int64_t cta_symdiff(const int32_t *A, int64_t la, const int32_t *B, int64_t lb, int32_t *out,
                               SymdiffSmem &S) {
  int64_t written = 0;
  const int64_t L = la + lb;
  for (int64_t g0 = 0; g0 < L; g0 += (int64_t)BC_TILE * BR_THREADS) {
    // The boundaries of up to BR_THREADS tiles, one binary search per thread.
    {
      const int64_t d = g0 + (int64_t)threadIdx.x * BC_TILE;
      S.split[threadIdx.x] = merge_split(A, la, B, lb, d < L ? d : L);
      if (threadIdx.x == 0) {
        const int64_t dl = g0 + (int64_t)BR_THREADS * BC_TILE;
        S.split[BR_THREADS] = merge_split(A, la, B, lb, dl < L ? dl : L);
      }
    }
    __syncthreads();
    for (int t = 0; t < BR_THREADS; ++t) {
      const int64_t d0 = g0 + (int64_t)t * BC_TILE;
      if (d0 >= L) break;
      const int64_t d1 = d0 + BC_TILE < L ? d0 + BC_TILE : L;
      const int64_t a0 = S.split[t], a1 = S.split[t + 1];  // split[t + 1] was taken at d1
      const int64_t b0 = d0 - a0, b1 = d1 - a1;
      const int na = (int)(a1 - a0), nb = (int)(b1 - b0);
      for (int q = threadIdx.x; q < na; q += BR_THREADS) S.a[q] = __ldcg(A + a0 + q);
      for (int q = threadIdx.x; q < nb; q += BR_THREADS) S.b[q] = __ldcg(B + b0 + q);
      const int32_t prevA = a0 > 0 ? __ldcg(A + a0 - 1) : -1;    // last A entry before the tile
      const int32_t nextB = b1 < lb ? __ldcg(B + b1) : INT_MAX;  // first B entry after the tile
      __syncthreads();
      // This thread's merged positions [p0, p1) of the tile: one pass counts
      // the entries that survive, a block scan places them, a second pass
      // writes them (no per-thread buffer).
      const int p0 = threadIdx.x * BC_PER, p1 = min(p0 + BC_PER, na + nb);
      int ia0 = 0, ib0 = 0;
      if (p0 < p1) {
        int lo = p0 - nb > 0 ? p0 - nb : 0, hi = p0 < na ? p0 : na;
        while (lo < hi) {
          const int mid = (lo + hi) >> 1;
          if (S.a[mid] <= S.b[p0 - mid - 1]) lo = mid + 1;
          else hi = mid;
        }
        ia0 = lo;
        ib0 = p0 - lo;
      }
      int nk = 0;
      {
        int ia = ia0, ib = ib0;
        for (int p = p0; p < p1; ++p) {
          const bool takeA = ib >= nb || (ia < na && S.a[ia] <= S.b[ib]);
          if (takeA) {
            const int32_t x = S.a[ia];
            nk += (ib < nb ? S.b[ib] : nextB) != x;
            ++ia;
          } else {
            const int32_t y = S.b[ib];
            nk += (ia > 0 ? S.a[ia - 1] : prevA) != y;
            ++ib;
          }
        }
      }
      int64_t tot;
      const int64_t off = block_excl_scan<int64_t>((int64_t)nk, S.sh, &tot);
      {
        int ia = ia0, ib = ib0;
        int32_t *o = out + written + off;
        for (int p = p0; p < p1; ++p) {
          const bool takeA = ib >= nb || (ia < na && S.a[ia] <= S.b[ib]);
          if (takeA) {
            const int32_t x = S.a[ia];
            if ((ib < nb ? S.b[ib] : nextB) != x) *o++ = x;
            ++ia;
          } else {
            const int32_t y = S.b[ib];
            if ((ia > 0 ? S.a[ia - 1] : prevA) != y) *o++ = y;
            ++ib;
          }
        }
      }
      written += tot;
      __syncthreads();
    }
  }
  return written;
}

// Smallest set bit at index >= from in the bitset bs (WT words), or
// INT_MAX; one CTA, 1024 words per round (the bits are updated by atomics,
// so they are read from L2).
__device__ int32_t bits_first_from(const uint32_t *bs, int64_t WT, int32_t from, int *s_piv) {
  const int64_t ws = from >> 5;
  for (int64_t w0 = ws; w0 < WT; w0 += BR_THREADS) {
    const int64_t w = w0 + threadIdx.x;
    uint32_t v = w < WT ? __ldcg(bs + w) : 0u;
    if (w == ws) v &= ~((1u << (from & 31)) - 1u);
    if (threadIdx.x == 0) *s_piv = INT_MAX;
    __syncthreads();
    if (v) atomicMin(s_piv, (int)(w * 32 + __ffs(v) - 1));
    __syncthreads();
    const int r = *s_piv;
    __syncthreads();
    if (r != INT_MAX) return r;
  }
  return INT_MAX;
}

// Reduce the non-final columns of batch positions [p0, p1) (position p is
// edge act[P-1-p]: youngest first) against final columns, one CTA per
// column: while the pivot has a final owner, add that column (into fresh
// pool space).  No pool space: *overflow, the column keeps its last value.
// A column of at least dense_min entries (dense_min >= 0) that has an
// addition to make continues as a bitset over the nrows rows in one of
// nslots slots of `bits` (slot taken from *slot_ctr): each addition then
// flips the added column's entries (its length, not the sum of both) and the
// pivot moves to the next set bit; the bitset goes back to a sorted list in
// fresh pool space at the end.  (Long-lived working columns meet many short
// final columns: on the n = 1000 torus the merges moved 950M entries for
// 1.25M entries added.)
__device__ void batch_reduce_phase(const int32_t *act, int64_t P, int64_t p0, int64_t p1, int64_t *coff,
                                   int32_t *clen, int32_t *pool, int64_t cap, unsigned long long *top,
                                   const int32_t *final_owner, const uint8_t *fin, int32_t *overflow, int64_t nrows,
                                   uint32_t *bits, int nslots, int *slot_ctr, int64_t dense_min, SymdiffSmem &S) {
  __shared__ int64_t s_o, s_at, s_p;
  __shared__ int s_slot, s_piv;
  // The grid's CTAs take the batch's columns by ticket (slot_ctr[1]).
  for (;;) {
    if (threadIdx.x == 0) s_p = p0 + (int64_t)atomicAdd(slot_ctr + 1, 1);
    __syncthreads();
    const int64_t p = s_p;
    __syncthreads();
    if (p >= p1) return;
    const int64_t e = act[P - 1 - p];
    if (__ldcg(fin + e)) continue;
    int64_t la = __ldcg(clen + e), oa = __ldcg(coff + e);
    bool moved = false;
    while (la > 0) {
      if (threadIdx.x == 0) {
        const int32_t o = __ldcg(final_owner + __ldcg(pool + oa));
        s_o = o;
        s_at = -1;
        s_slot = -1;
        if (o >= 0) {
          bool dense = false;
          if (bits && dense_min >= 0 && la >= dense_min) {
            const int sl = atomicAdd(slot_ctr, 1);
            if (sl < nslots) {
              s_slot = sl;
              dense = true;
            }
          }
          if (!dense) {
            const int64_t need = la + __ldcg(clen + o);
            const int64_t at = (int64_t)atomicAdd(top, (unsigned long long)need);
            if (at + need > cap) *overflow = 1;
            else s_at = at;
          }
        }
      }
      __syncthreads();
      const int64_t o = s_o, at = s_at;
      const int slot = s_slot;
      __syncthreads();
      if (o < 0) break;
      if (slot >= 0) {
        // Dense continuation of this column's chain.
        const int64_t WT = (nrows + 31) / 32;
        uint32_t *bs = bits + (size_t)slot * WT;
        for (int64_t w = threadIdx.x; w < WT; w += BR_THREADS) bs[w] = 0u;
        __syncthreads();
        for (int64_t i = threadIdx.x; i < la; i += BR_THREADS) {
          const int32_t x = __ldcg(pool + oa + i);
          atomicOr(bs + (x >> 5), 1u << (x & 31));
        }
        __syncthreads();
        int32_t piv = __ldcg(pool + oa);
        int64_t oo = o;
        for (;;) {
          const int64_t ob = __ldcg(coff + oo), lb = __ldcg(clen + oo);
          for (int64_t i = threadIdx.x; i < lb; i += BR_THREADS) {
            const int32_t x = __ldcg(pool + ob + i);
            atomicXor(bs + (x >> 5), 1u << (x & 31));
          }
          __syncthreads();
          piv = bits_first_from(bs, WT, piv, &s_piv);
          if (piv == INT_MAX) break;
          if (threadIdx.x == 0) s_o = __ldcg(final_owner + piv);
          __syncthreads();
          oo = s_o;
          __syncthreads();
          if (oo < 0) break;
        }
        // Back to a sorted list: per-thread runs of words, counted, placed.
        const int64_t per = (WT + BR_THREADS - 1) / BR_THREADS;
        const int64_t w0 = (int64_t)threadIdx.x * per, w1 = w0 + per < WT ? w0 + per : WT;
        int64_t cnt = 0;
        for (int64_t w = w0; w < w1; ++w) cnt += __popc(__ldcg(bs + w));
        int64_t tot;
        const int64_t off = block_excl_scan<int64_t>(cnt, S.sh, &tot);
        if (threadIdx.x == 0) {
          s_at = -1;
          if (tot > 0) {
            const int64_t a2 = (int64_t)atomicAdd(top, (unsigned long long)tot);
            if (a2 + tot > cap) *overflow = 1;
            else s_at = a2;
          }
        }
        __syncthreads();
        const int64_t a2 = s_at;
        if (tot == 0) {
          la = 0;
          moved = true;
        } else if (a2 >= 0) {
          int32_t *out = pool + a2 + off;
          for (int64_t w = w0; w < w1; ++w) {
            uint32_t v = __ldcg(bs + w);
            while (v) {
              *out++ = (int32_t)(w * 32 + __ffs(v) - 1);
              v &= v - 1;
            }
          }
          oa = a2;
          la = tot;
          moved = true;
        }
        break;  // (no pool space: the column keeps its last list and comes back next pass)
      }
      if (at < 0) break;
      const int64_t k = cta_symdiff(pool + oa, la, pool + __ldcg(coff + o), __ldcg(clen + o), pool + at, S);
      oa = at;
      la = k;
      moved = true;
    }
    if (moved && threadIdx.x == 0) {
      coff[e] = oa;
      clen[e] = (int32_t)la;
    }
  }
}

// One CTA: finalise the longest prefix of the batch's non-final columns whose
// pivots differ from every younger non-final column's (empty columns are
// final at once).  *remaining = the batch's non-final columns afterwards.
__device__ void batch_finalize_phase(const int32_t *act, int64_t P, int64_t p0, int64_t p1, const int64_t *coff,
                                     const int32_t *clen, const int32_t *pool, int32_t *final_owner, uint8_t *fin,
                                     const int32_t *overflow, int32_t *remaining) {
  static_assert(BR_THREADS == BC_BATCH, "one thread per column of a batch");
  __shared__ int32_t piv[BC_BATCH];
  __shared__ int32_t first_conflict;
  __shared__ int32_t left;
  const int i = threadIdx.x;
  const int64_t p = p0 + i;
  const bool mine = p < p1;
  const int64_t e = mine ? act[P - 1 - p] : -1;
  const bool open = mine && !__ldcg(fin + e);
  piv[i] = open && __ldcg(clen + e) > 0 ? __ldcg(pool + __ldcg(coff + e)) : -1;
  if (i == 0) {
    first_conflict = BC_BATCH;
    left = 0;
  }
  __syncthreads();
  if (__ldcg(overflow)) {  // a column could not finish its additions: no finalising this pass
    if (open) atomicAdd(&left, 1);
    __syncthreads();
    if (i == 0) *remaining = left;
    return;
  }
  bool conflict = false;
  if (piv[i] >= 0)
    for (int j = 0; j < i; ++j)
      if (piv[j] == piv[i]) {
        conflict = true;
        break;
      }
  if (conflict) atomicMin(&first_conflict, i);
  __syncthreads();
  if (open) {
    if (i < first_conflict) {
      if (piv[i] >= 0) final_owner[piv[i]] = (int32_t)e;
      fin[e] = 1;
    } else {
      atomicAdd(&left, 1);
    }
  }
  __syncthreads();
  if (i == 0) *remaining = left;
}

// Grid-wide barrier of a co-resident grid (cooperative launch): arrival
// count and generation in global memory; the wait is bounded (F_TIMEOUT in
// *err, then every CTA leaves the reduction).  Every thread fences its writes
// first; data other CTAs write during the launch is read through L2 (__ldcg).
constexpr long BAR_WAIT_LIMIT = 1l << 26;
__device__ bool grid_barrier(unsigned int *bar, int32_t *err) {
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
      long spins = 0;
      while (*gen == g) {
        if (++spins > BAR_WAIT_LIMIT) {
          atomicOr(err, F_TIMEOUT);
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    s_ok = *(volatile int32_t *)err == 0;
  }
  __syncthreads();
  return s_ok != 0;
}

// The whole column reduction from batch position *cursor on, in one launch
// of co-resident CTAs: per batch, passes of (every CTA reduces columns by
// ticket; CTA 0 finalises the longest conflict-free prefix) until the batch
// has no open column.  It returns to the host, with *cursor at the batch to
// redo or take next, when the pool is over half full or an addition found no
// room (the host compacts the pool and relaunches), or when a batch does not
// settle (*cursor = -1).  ctr: [0] bitset slots, [1] column tickets,
// [2..3] barrier, [4] stop.
static __global__ void __launch_bounds__(BR_THREADS) k_reduce_all(const int32_t *act, int64_t P, int64_t *cursor,
                                                                  int64_t *coff, int32_t *clen, int32_t *pool,
                                                                  int64_t cap, unsigned long long *top,
                                                                  int32_t *final_owner, uint8_t *fin,
                                                                  int32_t *overflow, int32_t *remaining,
                                                                  int64_t nrows, uint32_t *bits, int nslots,
                                                                  unsigned int *ctr, int64_t dense_min, int32_t *err) {
  extern __shared__ __align__(16) unsigned char br_smem[];
  SymdiffSmem &S = *reinterpret_cast<SymdiffSmem *>(br_smem);
  int *slot_ctr = (int *)ctr;
  unsigned int *bar = ctr + 2;
  for (int64_t p0 = *(volatile int64_t *)cursor; p0 < P; p0 += BC_BATCH) {
    const int64_t p1 = p0 + BC_BATCH < P ? p0 + BC_BATCH : P;
    for (int64_t pass = 0;; ++pass) {
      batch_reduce_phase(act, P, p0, p1, coff, clen, pool, cap, top, final_owner, fin, overflow, nrows, bits, nslots,
                         slot_ctr, dense_min, S);
      if (!grid_barrier(bar, err)) return;
      if (blockIdx.x == 0) {
        batch_finalize_phase(act, P, p0, p1, coff, clen, pool, final_owner, fin, overflow, remaining);
        __syncthreads();
        if (threadIdx.x == 0) {
          slot_ctr[0] = 0;
          slot_ctr[1] = 0;
          const bool full = *(volatile int32_t *)overflow != 0 ||
                            *(volatile unsigned long long *)top > (unsigned long long)cap / 2;
          const bool settled = *(volatile int32_t *)remaining == 0;
          // leave for the host: compaction (redo this batch if unsettled, else
          // start at the next), or a batch that does not settle
          if (full) *cursor = settled ? p1 : p0;
          else if (!settled && pass > BC_BATCH + 8) *cursor = -1;
          else *cursor = settled ? p1 : p0;
          ctr[4] = (full || (!settled && pass > BC_BATCH + 8)) ? 1u : 0u;
        }
      }
      if (!grid_barrier(bar, err)) return;
      const int64_t cur = *(volatile int64_t *)cursor;
      if (*(volatile unsigned int *)(ctr + 4) != 0) return;
      if (cur != p0) break;  // settled: next batch
    }
  }
}

// Move the live columns to the front of a new pool.
static __global__ void k_compact(int64_t E, const int64_t *coff, const int32_t *clen, const int64_t *noff,
                                 const int32_t *pool, int32_t *npool, int64_t *coff_out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x) {
    const int32_t l = clen[e];
    const int64_t src = coff[e], dst = noff[e];
    for (int32_t q = 0; q < l; ++q) npool[dst + q] = pool[src + q];
    coff_out[e] = dst;
  }
}

static __global__ void k_pairs1(int64_t E, const int64_t *coff, const int32_t *clen, const int32_t *pool,
                                int32_t *pair_tri, int32_t *pair_edge) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x) {
    if (clen[e] > 0) {
      const int32_t t = pool[coff[e]];
      pair_tri[t] = (int32_t)e;
      pair_edge[e] = t;
    }
  }
}

// ------------------------------------------------------------------ bars

// Bar candidates of one dimension in output order: finite bars indexed by
// the killing simplex (m1 candidates), then essential ones (m0 candidates).
struct BarSrc {
  int dim, maxdim;
  int64_t m0, m1;                 // simplices of dimension dim / dim+1
  const int32_t *g0, *g1;         // their grades
  const int32_t *killer_of;       // per (dim+1)-simplex: the dim-simplex it kills (-1: none)
  const uint8_t *neg8;            // negative dim-simplices (they kill one of dimension dim-1) ...
  const int32_t *neg32;           // ... as a flag array or as a partner array (>= 0)
  const int32_t *kill;            // per dim-simplex: the (dim+1)-simplex killing it (-1: none)
};

__device__ __forceinline__ bool bar_at(const BarSrc &b, int64_t q, int32_t &birth, int32_t &death) {
  if (q < b.m1) {  // finite bar killed by simplex q of dimension dim+1
    const int32_t s = b.killer_of[q];
    if (s < 0) return false;
    birth = b.g0[s];
    death = b.g1[q];
    return birth != death;
  }
  const int64_t s = q - b.m1;  // essential: positive and never killed
  if (b.neg8 && b.neg8[s]) return false;
  if (b.neg32 && b.neg32[s] >= 0) return false;
  if (b.kill && b.kill[s] >= 0) return false;
  birth = b.g0[s];
  death = -1;
  return true;
}

static __global__ void k_bar_flags(BarSrc b, int32_t *flag) {
  const int64_t L = b.m1 + b.m0;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < L; q += (int64_t)gridDim.x * blockDim.x) {
    int32_t x, y;
    flag[q] = bar_at(b, q, x, y) ? 1 : 0;
  }
}

static __global__ void k_bar_write(BarSrc b, const int64_t *pos, int32_t *birth, int32_t *death) {
  const int64_t L = b.m1 + b.m0;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < L; q += (int64_t)gridDim.x * blockDim.x) {
    int32_t x, y;
    if (bar_at(b, q, x, y)) {
      birth[pos[q]] = x;
      death[pos[q]] = y;
    }
  }
}

// dim 0 helper: per vertex, whether some forest edge killed it (-1 = never).
static __global__ void k_killed_vertices(int64_t E, const int32_t *killed_by_edge, int32_t *vkill) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < E; j += (int64_t)gridDim.x * blockDim.x)
    if (killed_by_edge[j] >= 0) vkill[killed_by_edge[j]] = (int32_t)j;
}

// ------------------------------------------------------------------ host

struct Dev {
  cudaStream_t s;
  std::vector<void *> tmp;
  explicit Dev(cudaStream_t st) : s(st) {}
  ~Dev() {
    for (void *p : tmp) cudaFreeAsync(p, s);
  }
  void release(void *p) {
    for (auto &q : tmp)
      if (q == p) {
        cudaFreeAsync(p, s);
        q = tmp.back();
        tmp.pop_back();
        return;
      }
  }
  template <typename T>
  vr_status get(T **p, int64_t count, bool keep = false, std::vector<void *> *owner = nullptr) {
    const size_t bytes = sizeof(T) * (size_t)std::max<int64_t>(count, 1);
    cudaError_t e = dev_malloc((void **)p, bytes, s);
    if (e != cudaSuccess) {
      cudaGetLastError();
      set_error("barcode: device allocation of %zu bytes failed", bytes);
      return e == cudaErrorMemoryAllocation ? VR_ERR_OOM : VR_ERR_CUDA;
    }
    if (keep) owner->push_back(*p);
    else tmp.push_back(*p);
    return VR_OK;
  }
};

static vr_status read_i32(const int32_t *d, int32_t *h, cudaStream_t s) {
  VR_CUDA(cudaMemcpyAsync(h, d, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  VR_CUDA(cudaStreamSynchronize(s));
  return VR_OK;
}

// Pairs of dimension k (k-simplices x (k+1)-simplices) by the batch-ordered
// coboundary reduction.  E = number of k-simplices (columns), T = number of
// (k+1)-simplices (rows); a column is cleared when its k-simplex is negative
// (neg8[s] != 0 or neg32[s] >= 0: it kills a (k-1)-simplex).  Outputs, kept
// on the complex: pair_tri[j] = the k-simplex the (k+1)-simplex j kills,
// pair_edge[s] = the (k+1)-simplex killing s (-1: none).
static vr_status reduce_cohomology(vr_complex *c, int k, cudaStream_t s, Dev &dv, Prof &prof, const uint8_t *neg8,
                                   const int32_t *neg32, int32_t *&pair_tri, int32_t *&pair_edge) {
  const int64_t E = c->count[k], T = c->count[k + 1];
  {
    prof.begin(k == 1 ? "bars.coboundary" : "bars.coboundary2");
    VR_TRY(dv.get(&pair_tri, T, true, &c->bar_allocs));
    VR_TRY(dv.get(&pair_edge, E, true, &c->bar_allocs));
    VR_CUDA(cudaMemsetAsync(pair_tri, 0xff, sizeof(int32_t) * T, s));
    VR_CUDA(cudaMemsetAsync(pair_edge, 0xff, sizeof(int32_t) * E, s));
    // Coboundary lists: (edge, triangle) entries sorted by edge, stable in t.
    const int64_t L = (int64_t)(k + 2) * T;
    uint64_t *keys;
    int32_t *cnt, *cptr;
    RadixScratch rs{};
    int32_t *sflags;
    VR_TRY(dv.get(&keys, L));
    VR_TRY(dv.get(&rs.tkeys, L));
    VR_TRY(dv.get(&rs.meta, rs_meta_bytes(L)));
    VR_TRY(dv.get(&sflags, 1));
    VR_CUDA(cudaMemsetAsync(sflags, 0, sizeof(int32_t), s));
    rs.err = sflags;
    VR_TRY(dv.get(&cnt, E));
    VR_TRY(dv.get(&cptr, E + 1));
    VR_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * E, s));
    k_cob_keys<<<bc_grid(L), BC_THREADS, 0, s>>>(c->rowidx[k + 1], T, k + 2, keys, cnt);
    count_launch();
    int ebits = 1;
    while ((1ll << ebits) < E) ++ebits;
    VR_TRY(radix_sort(keys, L, 32, ebits, rs, s));
    int64_t *bs;
    VR_TRY(dv.get(&bs, scan_tmp_slots(E)));
    VR_TRY((scan_exclusive<int32_t, int32_t>(cnt, cptr, E, bs, s)));
    // The pool: the initial columns, then room for column sums.
    int64_t cap = std::max<int64_t>(4 * L, 1 << 20);
    int32_t *pool;
    VR_TRY(dv.get(&pool, cap));
    k_cob_cols<<<bc_grid(L), BC_THREADS, 0, s>>>(keys, L, pool);
    count_launch();
    int64_t *coff;
    int32_t *clen;
    unsigned long long *top;
    int32_t *overflow;
    VR_TRY(dv.get(&coff, E));
    VR_TRY(dv.get(&clen, E));
    VR_TRY(dv.get(&top, 1));
    VR_TRY(dv.get(&overflow, 1));
    const unsigned long long top0 = (unsigned long long)L;
    VR_CUDA(cudaMemcpyAsync(top, &top0, sizeof(top0), cudaMemcpyHostToDevice, s));
    k_col_init<<<bc_grid(E), BC_THREADS, 0, s>>>(E, neg8, neg32, cptr, coff, clen);
    count_launch();
    VR_CUDA(cudaGetLastError());
    prof.end();

    prof.begin(k == 1 ? "bars.reduce" : "bars.reduce2");
    // Active columns in ascending edge order; processing takes them from the
    // youngest.
    int32_t *aflag, *act, *final_owner, *rem;
    int64_t *apos, *abs_;
    uint8_t *fin;
    VR_TRY(dv.get(&aflag, E));
    VR_TRY(dv.get(&apos, E + 1));
    VR_TRY(dv.get(&abs_, scan_tmp_slots(E)));
    VR_TRY(dv.get(&act, E));
    VR_TRY(dv.get(&final_owner, T));
    VR_TRY(dv.get(&fin, E));
    VR_TRY(dv.get(&rem, 1));
    VR_CUDA(cudaMemsetAsync(final_owner, 0xff, sizeof(int32_t) * T, s));
    VR_CUDA(cudaMemsetAsync(fin, 0, E, s));
    k_active_flags<<<bc_grid(E), BC_THREADS, 0, s>>>(E, clen, aflag);
    count_launch();
    VR_TRY((scan_exclusive<int32_t, int64_t>(aflag, apos, E, abs_, s)));
    k_compact_idx<<<bc_grid(E), BC_THREADS, 0, s>>>(aflag, apos, E, act);
    count_launch();
    int64_t P = 0;
    VR_CUDA(cudaMemcpyAsync(&P, apos + E, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    VR_CUDA(cudaStreamSynchronize(s));
    // Bitset slots for the long working columns (one per CTA of a launch, up
    // to BC_BATCH, at most DENSE_BITS_MAX bytes in all).
    const int64_t WT = (T + 31) / 32;
    const int64_t dense_min = g_dense_min;
    int nslots = 0;
    uint32_t *bits = nullptr;
    int *slot_ctr = nullptr;  // [0]: bitset slots taken, [1]: column tickets (per launch)
    VR_TRY(dv.get(&slot_ctr, 2));
    if (dense_min >= 0 && T > 0) {
      nslots = (int)std::min<int64_t>(BC_BATCH, std::max<int64_t>(1, DENSE_BITS_MAX / (WT * 4)));
      VR_TRY(dv.get(&bits, (int64_t)nslots * WT));
    }
    int nsm = 0, dev = 0;
    VR_CUDA(cudaGetDevice(&dev));
    VR_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    // One cooperative launch reduces batch after batch; it comes back only
    // to have the pool compacted (then it is launched again from *cursor).
    int64_t *cursor;
    unsigned int *ctr;
    int32_t *rerr;
    VR_TRY(dv.get(&cursor, 1));
    VR_TRY(dv.get(&ctr, 5));
    VR_TRY(dv.get(&rerr, 1));
    VR_CUDA(cudaMemsetAsync(cursor, 0, sizeof(int64_t), s));
    VR_CUDA(cudaMemsetAsync(rerr, 0, sizeof(int32_t), s));
    VR_CUDA(cudaFuncSetAttribute(k_reduce_all, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)BR_SMEM));
    int per = 0;
    VR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_reduce_all, BR_THREADS, BR_SMEM));
    const unsigned rgrid = (unsigned)std::max(1, nsm * std::max(per, 1));
    for (int launch = 0;; ++launch) {
      if (launch > 1 << 20) {
        set_error("barcode: the column reduction did not finish");
        return VR_ERR_INTERNAL;
      }
      VR_CUDA(cudaMemsetAsync(overflow, 0, sizeof(int32_t), s));
      VR_CUDA(cudaMemsetAsync(ctr, 0, 5 * sizeof(unsigned int), s));
      int64_t a_P = P, a_cap = cap, a_T = T, a_dmin = dense_min;
      int a_nslots = nslots;
      void *args[] = {&act, &a_P, &cursor, &coff, &clen, &pool, &a_cap, &top, &final_owner, &fin, &overflow, &rem,
                      &a_T, &bits, &a_nslots, &ctr, &a_dmin, &rerr};
      VR_CUDA(cudaLaunchCooperativeKernel((const void *)k_reduce_all, dim3(rgrid), dim3(BR_THREADS), args, BR_SMEM, s));
      count_launch();
      int64_t hcur = 0;
      int32_t herr = 0;
      VR_CUDA(cudaMemcpyAsync(&hcur, cursor, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
      VR_CUDA(cudaMemcpyAsync(&herr, rerr, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
      VR_CUDA(cudaStreamSynchronize(s));
      VR_TRY(flags_to_status(herr));
      if (hcur < 0) {
        set_error("barcode: a batch of the column reduction did not settle");
        return VR_ERR_INTERNAL;
      }
      if (hcur >= P) break;
      // The pool is over half full (or an addition found no room): compact
      // the live columns into a pool four times the live size (and at least
      // as large as before).
      int64_t *noff, *nbs;
      VR_TRY(dv.get(&noff, E + 1));
      VR_TRY(dv.get(&nbs, scan_tmp_slots(E)));
      VR_TRY((scan_exclusive<int32_t, int64_t>(clen, noff, E, nbs, s)));
      int64_t live = 0;
      VR_CUDA(cudaMemcpyAsync(&live, noff + E, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
      VR_CUDA(cudaStreamSynchronize(s));
      const int64_t ncap = std::max<int64_t>(cap, 4 * live + (1 << 20));
      int32_t *npool;
      int64_t *ncoff;
      VR_TRY(dv.get(&npool, ncap));
      VR_TRY(dv.get(&ncoff, E));
      k_compact<<<bc_grid(E), BC_THREADS, 0, s>>>(E, coff, clen, noff, pool, npool, ncoff);
      count_launch();
      VR_CUDA(cudaGetLastError());
      dv.release(pool);
      dv.release(coff);
      dv.release(noff);
      dv.release(nbs);
      pool = npool;
      coff = ncoff;
      cap = ncap;
      const unsigned long long t0 = (unsigned long long)live;
      VR_CUDA(cudaMemcpyAsync(top, &t0, sizeof(t0), cudaMemcpyHostToDevice, s));
    }
    k_pairs1<<<bc_grid(E), BC_THREADS, 0, s>>>(E, coff, clen, pool, pair_tri, pair_edge);
    count_launch();
    VR_CUDA(cudaGetLastError());
    int32_t hs = 0;
    VR_TRY(read_i32(sflags, &hs, s));
    VR_TRY(flags_to_status(hs));
    prof.end();
  }
  return VR_OK;
}

// Pairs of dimension 0 (killed vertex per edge) and, for maxdim 2, of
// dimension 1 (edge per triangle and triangle per edge).  Kept on the complex.
static vr_status compute_pairs(vr_complex *c, cudaStream_t s) {
  Dev dv(s);
  Prof prof(s);
  const int n = c->n;
  const int64_t E = c->maxdim >= 1 ? c->count[1] : 0;
  const int64_t T = c->maxdim >= 2 ? c->count[2] : 0;
  int32_t *killed_by_edge = nullptr, *vkill = nullptr;
  uint8_t *msf = nullptr;
  int32_t *pair_tri = nullptr, *pair_edge = nullptr;
  VR_TRY(dv.get(&killed_by_edge, E, true, &c->bar_allocs));
  VR_TRY(dv.get(&vkill, n, true, &c->bar_allocs));
  VR_TRY(dv.get(&msf, E, true, &c->bar_allocs));
  VR_CUDA(cudaMemsetAsync(killed_by_edge, 0xff, sizeof(int32_t) * std::max<int64_t>(E, 1), s));
  VR_CUDA(cudaMemsetAsync(vkill, 0xff, sizeof(int32_t) * n, s));
  VR_CUDA(cudaMemsetAsync(msf, 0, std::max<int64_t>(E, 1), s));
  int32_t *hflag = nullptr;
  VR_CUDA(cudaMallocHost((void **)&hflag, sizeof(int32_t)));
  struct HostFree {
    int32_t *p;
    ~HostFree() { cudaFreeHost(p); }
  } hf{hflag};

  if (E > 0) {
    // Boruvka rounds for the spanning forest.
    prof.begin("bars.forest");
    int32_t *comp, *best, *next, *changed;
    VR_TRY(dv.get(&comp, n));
    VR_TRY(dv.get(&best, n));
    VR_TRY(dv.get(&next, n));
    VR_TRY(dv.get(&changed, 1));
    k_bv_init<<<bc_grid(n), BC_THREADS, 0, s>>>(n, comp, best);
    count_launch();
    for (int round = 0; round < 64; ++round) {
      VR_CUDA(cudaMemsetAsync(changed, 0, sizeof(int32_t), s));
      k_bv_choose<<<bc_grid(E), BC_THREADS, 0, s>>>(c->verts[1], E, comp, best);
      k_bv_hook<<<bc_grid(n), BC_THREADS, 0, s>>>(c->verts[1], n, comp, best, next, msf, changed);
      k_bv_jump<<<bc_grid(n), BC_THREADS, 0, s>>>(n, next, comp, best);
      count_launch(3);
      VR_CUDA(cudaGetLastError());
      VR_TRY(read_i32(changed, hflag, s));
      if (!*hflag) break;
    }
    prof.end();
    // Forest edges in order, then the elder rule.
    prof.begin("bars.elder");
    int32_t *flag, *fedges;
    int64_t *bs;
    VR_TRY(dv.get(&flag, E));
    VR_TRY(dv.get(&fedges, n));
    int64_t *fpos;
    VR_TRY(dv.get(&fpos, E + 1));
    VR_TRY(dv.get(&bs, scan_tmp_slots(E)));
    k_u8_to_i32<<<bc_grid(E), BC_THREADS, 0, s>>>(msf, E, flag);
    count_launch();
    VR_TRY((scan_exclusive<int32_t, int64_t>(flag, fpos, E, bs, s)));
    k_compact_idx<<<bc_grid(E), BC_THREADS, 0, s>>>(flag, fpos, E, fedges);
    count_launch();
    k_elder<<<1, 32, 0, s>>>(c->verts[1], fedges, fpos + E, n, killed_by_edge);
    k_killed_vertices<<<bc_grid(E), BC_THREADS, 0, s>>>(E, killed_by_edge, vkill);
    count_launch(2);
    VR_CUDA(cudaGetLastError());
    prof.end();
  }

  if (T > 0) VR_TRY(reduce_cohomology(c, 1, s, dv, prof, msf, nullptr, pair_tri, pair_edge));
  int32_t *pair_tet = nullptr, *pair_tri2 = nullptr;
  if (c->maxdim >= 3 && c->count[3] > 0 && T > 0)
    VR_TRY(reduce_cohomology(c, 2, s, dv, prof, nullptr, pair_tri, pair_tet, pair_tri2));
  c->pair_tet = pair_tet;
  c->pair_tri2 = pair_tri2;
  c->killed_by_edge = killed_by_edge;
  c->vkill = vkill;
  c->msf = msf;
  c->pair_tri = pair_tri;
  c->pair_edge = pair_edge;
  c->pairs_done = true;
  VR_CUDA(cudaStreamSynchronize(s));
  return VR_OK;
}

vr_status complex_barcode(vr_complex *c, int dim, cudaStream_t s, int64_t *nbars) {
  if (!c->pairs_done) VR_TRY(compute_pairs(c, s));
  if (c->nbars[dim] >= 0) {
    *nbars = c->nbars[dim];
    return VR_OK;
  }
  BarSrc b{};
  b.dim = dim;
  b.maxdim = c->maxdim;
  b.m0 = c->count[dim];
  b.g0 = c->grade[dim];
  if (dim < c->maxdim) {
    b.killer_of = dim == 0 ? c->killed_by_edge : dim == 1 ? c->pair_tri : c->pair_tet;
    if (b.killer_of) {
      b.m1 = c->count[dim + 1];
      b.g1 = c->grade[dim + 1];
    }
  }
  if (dim == 0) b.kill = c->maxdim >= 1 ? c->vkill : nullptr;
  if (dim == 1) {
    b.neg8 = c->msf;
    b.kill = c->maxdim >= 2 ? c->pair_edge : nullptr;
  }
  if (dim == 2) {
    b.neg32 = c->pair_tri;
    b.kill = c->maxdim >= 3 ? c->pair_tri2 : nullptr;
  }
  if (dim == 3) b.neg32 = c->pair_tet;
  Dev dv(s);
  const int64_t L = b.m0 + b.m1;
  int32_t *flag;
  int64_t *pos, *bs;
  VR_TRY(dv.get(&flag, L));
  VR_TRY(dv.get(&pos, L + 1));
  VR_TRY(dv.get(&bs, scan_tmp_slots(L)));
  k_bar_flags<<<bc_grid(L), BC_THREADS, 0, s>>>(b, flag);
  count_launch();
  VR_TRY((scan_exclusive<int32_t, int64_t>(flag, pos, L, bs, s)));
  int64_t nb = 0;
  VR_CUDA(cudaMemcpyAsync(&nb, pos + L, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  VR_CUDA(cudaStreamSynchronize(s));
  int32_t *birth, *death;
  VR_TRY(dv.get(&birth, nb, true, &c->bar_allocs));
  VR_TRY(dv.get(&death, nb, true, &c->bar_allocs));
  k_bar_write<<<bc_grid(L), BC_THREADS, 0, s>>>(b, pos, birth, death);
  count_launch();
  VR_CUDA(cudaGetLastError());
  VR_CUDA(cudaStreamSynchronize(s));
  c->bar_birth[dim] = birth;
  c->bar_death[dim] = death;
  c->nbars[dim] = nb;
  *nbars = nb;
  return VR_OK;
}

}  // namespace vr

extern "C" vr_status vr_set_barcode_dense_min(int64_t min_entries) {
  vr::g_dense_min = min_entries;
  return VR_OK;
}
