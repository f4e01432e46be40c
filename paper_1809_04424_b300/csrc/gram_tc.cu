// gram_tc.cu -- the kept-edge bitmap from Gram tiles on the tensor cores.
//
// d^2(i,j) = |y_i|^2 + |y_j|^2 - 2 <y_i, y_j>, y = x - c (c a common centre:
// distances do not change).  One CTA per 128x128 tile of the pair matrix
// (upper triangle of tiles): TMA brings the two 128-row operand tiles (bf16,
// 64 coordinates, 128-byte swizzle) into shared memory, one thread issues
// tcgen05.mma (kind::f16, bf16 x bf16 -> fp32 accumulator in TMEM), and eight
// warps read the accumulator back with tcgen05.ld (two per TMEM lane quarter,
// each taking half of the tile's columns), one pair row per thread.
//
// int8 inputs: coordinates are exact in bf16, their products exact in fp32
// and every partial sum stays below 2^24, so the squared distances are
// exact integers and the cap test is exact.
// float inputs: y is split as hi + lo (two bf16 values, ~16 significant
// bits) and the Gram is hi.hi + hi.lo + lo.hi (three MMAs into one
// accumulator).  The computed d^2 is within beta = 4e-4 (|y_i|^2 + |y_j|^2) of
// the canonical FP64 value (bound below).  The tile compares fp32 d^2 -/+ beta
// with the floats just below / above r^2 (their few roundings, < 1e-6
// (|y_i|^2 + |y_j|^2), sit inside beta's margin); pairs left in between go to
// a list that k_band_patch decides with the exact canonical value (integer
// emulation of the FP64 sequence), so the bitmap is exact.  A list overflow
// makes the host redo the bitmap on the CUDA cores.
//
// Bound, per pair, with S = |y_i| + |y_j|, eta = 1.01 * 2^-16 (split plus
// centring error per coordinate, relative): representation 2 eta S^2; dropped
// lo.lo term 2 * 2^-16 S^2/4; fp32 accumulation of 3K = 192 products, taken as
// 192 * 2^-22 per term (truncating adders allowed) * S^2/4 * 1.1 * 2; norms
// K * 2^-24 S^2; final subtraction 3 * 2^-23 S^2 -- in all below 7e-5 S^2 <=
// 1.4e-4 (|y_i|^2 + |y_j|^2), so beta has more than 2x margin; a test measures
// the observed error against beta on adversarial inputs.
// Three-way split (vr_set_gram_split(3)): y = hi + mid + lo holds y's 24
// significant bits exactly, the dropped mid.lo, lo.mid, lo.lo terms are below
// 2^-23 S^2 / 4, and the accumulation bound doubles (6K = 384 products):
// still below 7.5e-5 S^2, inside the same beta.  It shrinks the observed
// error (no truncated lo.lo), not the band: the bound is the accumulation's.
//
// Every wait (TMA and MMA completion) is bounded; on a timeout the kernel
// raises F_TIMEOUT, releases its TMEM and returns.
#include <atomic>

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "complex.h"
#include "kernels.cuh"
#include "prof.h"

namespace vr {

constexpr int TC_TILE = 128;        // rows (and columns) of a pair tile
constexpr int TC_K = 64;            // coordinates per operand row (padded)
constexpr int TC_ROW_BYTES = TC_K * 2;
constexpr int TC_OPERAND_BYTES = TC_TILE * TC_ROW_BYTES;  // 16 KB
constexpr uint32_t TC_TMEM_COLS = 128;
constexpr int TC_THREADS = 256;     // 8 warps: two per TMEM lane quarter, each half the columns
constexpr long TC_WAIT_LIMIT = 1l << 22;
constexpr float TC_BETA = 4e-4f;

// ------------------------------------------------------------- PTX helpers

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
// Bounded wait for the phase with the given parity; false on timeout.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, long limit = TC_WAIT_LIMIT) {
  for (long it = 0; it < limit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
          dst),
      "l"((uint64_t)map), "r"(bar), "r"(x), "r"(y)
      : "memory");
}

// Shared-memory matrix descriptor of a K-major bf16 tile written by TMA with
// 128-byte swizzle: start address, leading offset (unused with this swizzle,
// 16 B), stride offset 1024 B (8 rows of 128 B), descriptor version 1,
// layout type 2 (128-byte swizzle).
__device__ __forceinline__ uint64_t umma_desc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3fff);
  d |= (uint64_t)1 << 16;                 // leading byte offset 16 B (>> 4)
  d |= (uint64_t)(1024 >> 4) << 32;       // stride byte offset
  d |= (uint64_t)1 << 46;                 // version
  d |= (uint64_t)2 << 61;                 // 128-byte swizzle
  return d;
}

// Instruction descriptor: D fp32, A and B bf16, both K-major, N = 128, M = 128.
constexpr uint32_t TC_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TC_TILE >> 3) << 17) |
                              ((uint32_t)(TC_TILE >> 4) << 24);

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          tmem_d),
      "l"(adesc), "l"(bdesc), "r"(TC_IDESC), "r"(accumulate));
}
__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int k = 0; k < 32; ++k) v[k] = __uint_as_float(r[k]);
}

// ----------------------------------------------------------------- kernels

// Operand preparation: y = x - c, hi = bf16(y), lo = bf16(y - hi) (float), or
// hi = x exactly (int8); rows padded to 64 coordinates and to whole tiles.
// norm = |hi + lo|^2 in fp32 (fma in coordinate order).
// Three-way split (Xm non-null): y = hi + mid + lo, mid = bf16(y - hi),
// lo = bf16(y - hi - mid) (24 significant bits: y itself).
template <bool F>
// One warp per padded row: lane l owns coordinates 2l and 2l+1 (bf16x2
// stores, coalesced), |y_i|^2 by a warp sum of the split values.
__global__ void k_gram_prep(const void *Xv, int n, int d, int npad, const float *centre, __nv_bfloat16 *Xh,
                            __nv_bfloat16 *Xl, float *norm, __nv_bfloat16 *Xm) {
  pdl_entry();
  const int lane = threadIdx.x & 31;
  for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < npad; i += (gridDim.x * blockDim.x) >> 5) {
    float hi[2] = {0.f, 0.f}, mid[2] = {0.f, 0.f}, lo[2] = {0.f, 0.f};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int k = 2 * lane + h;
      if (i < n && k < d) {
        if constexpr (F) {
          const float y = __fsub_rn(((const float *)Xv)[(int64_t)i * d + k], centre[k]);
          hi[h] = __bfloat162float(__float2bfloat16_rn(y));
          if (Xm) {
            mid[h] = __bfloat162float(__float2bfloat16_rn(__fsub_rn(y, hi[h])));
            lo[h] = __bfloat162float(__float2bfloat16_rn(__fsub_rn(__fsub_rn(y, hi[h]), mid[h])));
          } else {
            lo[h] = __bfloat162float(__float2bfloat16_rn(__fsub_rn(y, hi[h])));
          }
        } else {
          hi[h] = (float)((const int32_t *)Xv)[(int64_t)i * d + k];
        }
      }
    }
    ((__nv_bfloat162 *)(Xh + (int64_t)i * TC_K))[lane] = __floats2bfloat162_rn(hi[0], hi[1]);
    if constexpr (F) ((__nv_bfloat162 *)(Xl + (int64_t)i * TC_K))[lane] = __floats2bfloat162_rn(lo[0], lo[1]);
    if (F && Xm) ((__nv_bfloat162 *)(Xm + (int64_t)i * TC_K))[lane] = __floats2bfloat162_rn(mid[0], mid[1]);
    const float x0 = __fadd_rn(__fadd_rn(hi[0], mid[0]), lo[0]), x1 = __fadd_rn(__fadd_rn(hi[1], mid[1]), lo[1]);
    const float acc = warp_sum(__fmaf_rn(x1, x1, x0 * x0));
    if (lane == 0) norm[i] = acc;
  }
}

// Exact decision of the pairs the Gram tiles left within beta of the cap:
// the canonical FP64 value (hardware FP64: the list is a small fraction of
// the pairs), bits ORed into both rows.
__global__ void k_band_patch(const float *X, int d, int W, double r2, const uint64_t *band, const DevStatus *st,
                             uint64_t band_cap, uint32_t *adj) {
  pdl_entry();
  if (build_failed(st)) return;  // a timed-out tile left its bitmap words unwritten
  const uint64_t cnt = min((unsigned long long)st->band_count, (unsigned long long)band_cap);
  // Pair t goes to CTA t mod grid: a short list still spreads over every SM
  // (its FP64 chains, not its loads, set the time).
  for (uint64_t t = threadIdx.x * (uint64_t)gridDim.x + blockIdx.x; t < cnt; t += (uint64_t)gridDim.x * blockDim.x) {
    const int i = (int)(band[t] >> 32), j = (int)(band[t] & 0xffffffffu);
    if (d2_f64(X + (int64_t)i * d, X + (int64_t)j * d, d) <= r2) {
      atomicOr(&adj[(int64_t)i * W + (j >> 5)], 1u << (j & 31));
      atomicOr(&adj[(int64_t)j * W + (i >> 5)], 1u << (i & 31));
    }
  }
}

// Centre c = mean of up to 256 evenly spaced points (one CTA).  Any c gives
// the same distances; one near the middle of the cloud keeps |y|, and with it
// the width of the near-cap band, small.  Also clears the near-cap count.
constexpr int TC_CENTRE_SAMPLE = 256;
__global__ void __launch_bounds__(1024) k_gram_centre(const float *X, int n, int d, float *centre, DevStatus *st) {
  pdl_entry();
  if (threadIdx.x == 0) st->band_count = 0;
  __shared__ float part[32][TC_K];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m = min(n, TC_CENTRE_SAMPLE);
  float a0 = 0.f, a1 = 0.f;
  for (int s = warp; s < m; s += 32) {
    const int64_t r = (int64_t)s * n / m;
    if (lane < d) a0 += X[r * d + lane];
    if (lane + 32 < d) a1 += X[r * d + lane + 32];
  }
  part[warp][lane] = a0;
  part[warp][lane + 32] = a1;
  __syncthreads();
  if (threadIdx.x < d) {
    float t = 0.f;
    for (int w = 0; w < 32; ++w) t += part[w][threadIdx.x];
    centre[threadIdx.x] = t / (float)m;
  }
}

struct TcSmem {
  uint32_t ah, bh, al, bl, am, bm, bar_tma, bar_mma, tslot;
};

// Accuracy counters of the validation variant.
struct GramAcc {
  unsigned int worst_norm;       // float bits: max |d2_tc - d2_fp64| / (|y_i|^2 + |y_j|^2), all pairs
  unsigned int worst_rel_d;      // float bits: max |d_tc - d_fp64| / d_fp64, kept pairs
  unsigned long long kept;       // pairs with d2_fp64 <= r2
  unsigned long long band;       // pairs the tiles leave to the exact decision
};

// One CTA (TC_THREADS) per upper-triangle tile pair (ti <= tj).  Float
// pairs within beta of the cap are appended to `band` (decided exactly by
// k_band_patch); VALIDATE instead computes the canonical value of every pair
// and records the worst observed |d2_tc - d2_fp64| / (|y_i|^2 + |y_j|^2).
// INJ (test hook, vr_inject_gram_stall): CTA `stall_tile` issues no MMA and
// no completion, so its waits run out after `wait_limit` polls.
// S3: three-way split (hi, mid, lo), six products hh, hm, mh, hl, lh, mm.
template <bool F, bool VALIDATE, bool INJ = false, bool S3 = false>
__global__ void __launch_bounds__(TC_THREADS) k_gram_bitmap_tc(const __grid_constant__ CUtensorMap tmh,
                                                        const __grid_constant__ CUtensorMap tml, const void *Xv,
                                                        int n, int d, int W, int nt, Cap cap, const float *norm,
                                                        uint32_t *adj, DevStatus *st, uint64_t *band,
                                                        uint64_t band_cap, GramAcc *acc_out,
                                                        int stall_tile = -1, long wait_limit = TC_WAIT_LIMIT,
                                                        const __grid_constant__ CUtensorMap tmm = CUtensorMap{}) {
  // Only the stalled CTA's completion wait takes the short limit: every other
  // wait guards a TMA load or an MMA that is really in flight.
  const bool stalled = INJ && (int)blockIdx.x == stall_tile;
  extern __shared__ unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // Tile pair from the linear block index.
  int ti = 0, rem = blockIdx.x;
  while (rem >= nt - ti) {
    rem -= nt - ti;
    ++ti;
  }
  const int tj = ti + rem;

  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023) & ~1023u;  // 128-byte swizzle wants 1024-byte alignment
  TcSmem S;
  S.ah = base;
  S.bh = base + TC_OPERAND_BYTES;
  S.al = base + 2 * TC_OPERAND_BYTES;
  S.bl = base + 3 * TC_OPERAND_BYTES;
  S.am = base + 4 * TC_OPERAND_BYTES;
  S.bm = base + 5 * TC_OPERAND_BYTES;
  S.bar_tma = base + (S3 ? 6 : 4) * TC_OPERAND_BYTES;
  S.bar_mma = S.bar_tma + 8;
  S.tslot = S.bar_tma + 16;
  uint32_t *tslot_ptr = (uint32_t *)(smem_raw + (S.tslot - raw));

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(S.tslot),
                 "r"(TC_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (threadIdx.x == 32) {
    mbar_init(S.bar_tma, 1);
    mbar_init(S.bar_mma, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *(volatile uint32_t *)tslot_ptr;
  // TMEM and barriers are set up while the operand preparation finishes.
  pdl_entry();

  if (threadIdx.x == 0) {
    const uint32_t bytes = (S3 ? 6 : F ? 4 : 2) * TC_OPERAND_BYTES;
    mbar_expect_tx(S.bar_tma, bytes);
    tma_load_2d(S.ah, &tmh, 0, ti * TC_TILE, S.bar_tma);
    tma_load_2d(S.bh, &tmh, 0, tj * TC_TILE, S.bar_tma);
    if (F) {
      tma_load_2d(S.al, &tml, 0, ti * TC_TILE, S.bar_tma);
      tma_load_2d(S.bl, &tml, 0, tj * TC_TILE, S.bar_tma);
    }
    if (S3) {
      tma_load_2d(S.am, &tmm, 0, ti * TC_TILE, S.bar_tma);
      tma_load_2d(S.bm, &tmm, 0, tj * TC_TILE, S.bar_tma);
    }
    if (stalled) {
      // Test hook: the operands arrived (waited for, so nothing is in flight
      // when TMEM is released), but no MMA and no completion are issued.
      if (!mbar_wait(S.bar_tma, 0)) raise_flag(st, F_TIMEOUT);
    } else if (mbar_wait(S.bar_tma, 0)) {
      tc_fence_after();
      uint32_t acc = 0;
      // Products: hi.hi, hi.lo, lo.hi (two-way split) or hi.hi, hi.mid,
      // mid.hi, hi.lo, lo.hi, mid.mid (three-way split).
      const uint32_t As[6] = {S.ah, S.ah, S.al, S.ah, S.am, S.am};
      const uint32_t Bs[6] = {S.bh, S.bl, S.bh, S.bm, S.bh, S.bm};
      const int nprod = S3 ? 6 : F ? 3 : 1;
      for (int p = 0; p < nprod; ++p)
        for (int k = 0; k < TC_K / 16; ++k) {
          umma_bf16(tmem, umma_desc_sw128(As[p] + 32 * k), umma_desc_sw128(Bs[p] + 32 * k), acc);
          acc = 1;
        }
      umma_commit(S.bar_mma);
    } else {
      raise_flag(st, F_TIMEOUT);
      mbar_arrive(S.bar_mma);  // release the other threads; nothing was issued
    }
  }
  const bool ok = mbar_wait(S.bar_mma, 0, stalled ? wait_limit : TC_WAIT_LIMIT);
  tc_fence_after();
  if (!ok && lane == 0) raise_flag(st, F_TIMEOUT);

  if (ok && !(*(volatile int32_t *)&st->flags & F_TIMEOUT)) {
    // Warp w reads TMEM lanes 32 (w % 4) .. +31 (the lane quarter its warp
    // index allows) and columns 64 (w / 4) .. +63.
    const int q = warp & 3, half = warp >> 2;
    const int i = ti * TC_TILE + q * 32 + lane;  // this thread's pair row
    const float ni = i < n ? norm[i] : 0.f;
    const bool diag = ti == tj;
    unsigned int worst = 0, worst_rel = 0;
    unsigned int kept_cnt = 0, band_cnt = 0;
    for (int c0 = half * (TC_TILE / 2); c0 < (half + 1) * (TC_TILE / 2); c0 += 32) {
      float g[32];
      tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c0, g);
      uint32_t rowword = 0, bandword = 0;
#pragma unroll
      for (int c = 0; c < 32; ++c) {
        const int j = tj * TC_TILE + c0 + c;
        bool kept = false, in_band = false;
        if (i < n && j < n && i != j) {
          const float nj = norm[j];
          const float d2 = __fsub_rn(__fadd_rn(ni, nj), 2.f * g[c]);
          if constexpr (F) {
            const float beta = TC_BETA * (ni + nj);
            if (cap.keep_all || __fadd_rn(d2, beta) <= cap.r2f_dn) kept = true;
            else if (__fsub_rn(d2, beta) > cap.r2f_up) kept = false;
            else in_band = i < j;  // a diagonal tile sees the pair twice: record it once
            if constexpr (VALIDATE) {
              const double f = d2_canonical((const float *)Xv + (int64_t)i * d, (const float *)Xv + (int64_t)j * d, d);
              const float r = (float)(fabs((double)d2 - f) / ((double)ni + (double)nj + 1e-30));
              worst = max(worst, __float_as_uint(r));
              if (i < j && (cap.keep_all || f <= cap.r2)) {
                ++kept_cnt;
                if (f > 0.0) {
                  const double dt = sqrt(fmax((double)d2, 0.0)), df = sqrt(f);
                  worst_rel = max(worst_rel, __float_as_uint((float)(fabs(dt - df) / df)));
                }
              }
              band_cnt += in_band;
            }
          } else {
            const uint64_t v = (uint64_t)(int64_t)d2;  // exact: every term is an integer below 2^24
            kept = cap.keep_all || v <= cap.r2i;
          }
        }
        rowword |= (uint32_t)kept << c;
        bandword |= (uint32_t)in_band << c;
      }
      // The chunk's near-cap pairs: one warp-aggregated append.
      if constexpr (F && !VALIDATE) {
        const int nb = __popc(bandword);
        const int incl = warp_incl_scan(nb);
        const int tot = __shfl_sync(0xffffffffu, incl, 31);
        if (tot) {
          uint64_t at = 0;
          if (lane == 31) at = atomicAdd((unsigned long long *)&st->band_count, (unsigned long long)tot);
          at = __shfl_sync(0xffffffffu, at, 31) + (uint64_t)(incl - nb);
          for (uint32_t m = bandword; m; m &= m - 1, ++at) {
            const int j = tj * TC_TILE + c0 + __ffs(m) - 1;
            if (at < band_cap) band[at] = ((uint64_t)i << 32) | (uint32_t)j;
            else raise_flag(st, F_OVERFLOW);
          }
        }
      }
      // Mirrored column words: the 32 x 32 bit transpose of the lanes' row
      // words (lane c gets bit r = row r's bit c), by five shuffle rounds.
      uint32_t mirror = rowword;
#pragma unroll
      for (int sh = 16; sh >= 1; sh >>= 1) {
        const uint32_t m = sh == 16 ? 0x0000ffffu : sh == 8 ? 0x00ff00ffu : sh == 4 ? 0x0f0f0f0fu
                         : sh == 2 ? 0x33333333u : 0x55555555u;
        const uint32_t y = __shfl_xor_sync(0xffffffffu, mirror, sh);
        mirror = (lane & sh) ? (mirror & ~m) | ((y & ~m) >> sh) : (mirror & m) | ((y & m) << sh);
      }
      // Padded columns of the last tile map past the row's W words: skip them.
      const int wr = (tj * TC_TILE + c0) / 32, wm = (ti * TC_TILE + q * 32) / 32;
      if (i < n && wr < W) adj[(int64_t)i * W + wr] = rowword;
      const int jrow = tj * TC_TILE + c0 + lane;
      if (!diag && jrow < n && wm < W) adj[(int64_t)jrow * W + wm] = mirror;
    }
    if constexpr (VALIDATE) {
      if (worst) atomicMax(&acc_out->worst_norm, worst);
      if (worst_rel) atomicMax(&acc_out->worst_rel_d, worst_rel);
      const unsigned int kc = warp_sum((int)kept_cnt), bc = warp_sum((int)band_cnt);
      if (lane == 0) {
        if (kc) atomicAdd(&acc_out->kept, (unsigned long long)kc);
        if (bc) atomicAdd(&acc_out->band, (unsigned long long)bc);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS) : "memory");
  }
}

// ----------------------------------------------------------------- host

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
    cudaGetLastError();
  }
  return fn;
}

static vr_status make_map(CUtensorMap *m, void *base, int npad) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) {
    set_error("cuTensorMapEncodeTiled is not available");
    return VR_ERR_CUDA;
  }
  const cuuint64_t dims[2] = {(cuuint64_t)TC_K, (cuuint64_t)npad};
  const cuuint64_t strides[1] = {(cuuint64_t)TC_ROW_BYTES};
  const cuuint32_t box[2] = {(cuuint32_t)TC_K, (cuuint32_t)TC_TILE};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, dims, strides, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed (%d)", (int)r);
    return VR_ERR_CUDA;
  }
  return VR_OK;
}

static int g_gram_mode = 0;  // 0 auto, 1 tensor cores where eligible, 2 CUDA cores

// Test hook: takes (and disarms) an armed Gram stall for a launch of `tiles`
// tiles (api.cu, vr_inject_gram_stall).
bool take_gram_stall(int tiles, int *tile, long *limit);

// Tensor-core tiles pay off once there are enough 128x128 tiles to fill the
// GPU (two per SM); mode 1 forces them wherever they apply.
bool gram_tc_eligible(vr_dtype dtype, int n, int d) {
  if (g_gram_mode == 2) return false;
  if (!(d <= TC_K && (dtype == VR_I8 || dtype == VR_F32))) return false;
  if (g_gram_mode == 1) return true;
  // Automatic choice: the tiles cost the same for any d up to TC_K (the
  // contraction is padded), the CUDA-core pair loop grows with d; measured on
  // float clouds of 3000-7322 points the CUDA cores are ahead up to d = 16
  // (by 1-5 %) and the tiles from d = 32 (by 5 %).  Enough tiles to fill the
  // SMs twice, too.
  if (d <= 16) return false;
  const int nt = (n + TC_TILE - 1) / TC_TILE;
  return nt * (nt + 1) / 2 >= 2 * num_sms();
}

// Float split: 2 = two-way (hi, lo; three products, the default), 3 =
// three-way (hi, mid, lo; six products).  Process-wide.
static int g_gram_split = 2;

template <bool F, bool VALIDATE, bool INJ, bool S3>
static cudaError_t launch_tiles(int ntiles, size_t smem, cudaStream_t s, const CUtensorMap &mh, const CUtensorMap &ml,
                                const CUtensorMap &mm, const void *X, int n, int d, int W, int nt, const Cap &cap,
                                const float *norm, uint32_t *adj, DevStatus *st, uint64_t *band, uint64_t band_cap,
                                GramAcc *acc, int stall_tile, long stall_limit) {
  // The shared-memory size is fixed per kernel: set once per device.
  static std::atomic<uint64_t> set_on{0};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 64 || !((set_on.load() >> dev) & 1u)) {
    e = cudaFuncSetAttribute(k_gram_bitmap_tc<F, VALIDATE, INJ, S3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
    if (dev < 64) set_on.fetch_or(1ull << dev);
  }
  e = launch_dep(k_gram_bitmap_tc<F, VALIDATE, INJ, S3>, ntiles, TC_THREADS, smem, s, mh, ml, X, n, d, W, nt, cap,
                 norm, adj, st, band, band_cap, acc, stall_tile, stall_limit, mm);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

// Bitmap of kept pairs on the tensor cores.  X is the staged point array
// (int32 for int8 input, float for float input).  `acc` non-null turns on
// validation (float only: every pair's canonical value, accuracy counters).
// split3: three-way float split (six products).
vr_status gram_bitmap_tc(const void *X, int n, int d, bool F, const Cap &cap, uint32_t *adj, DevStatus *st,
                         cudaStream_t s, GramAcc *acc, int split = 0) {
  const bool S3 = F && (split ? split == 3 : g_gram_split == 3);
  const int W = (n + 31) / 32;
  const int nt = (n + TC_TILE - 1) / TC_TILE;
  const int npad = nt * TC_TILE;
  const int ntiles = nt * (nt + 1) / 2;
  const uint64_t npairs = (uint64_t)n * (n - 1) / 2;
  const uint64_t band_cap = std::min<uint64_t>(npairs, std::max<uint64_t>(1u << 20, npairs / 16));
  const bool want_band = F && !acc;
  // One allocation: operands (hi, lo, mid), norms, centre, near-cap list.
  auto up256 = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const size_t opb = up256((size_t)npad * TC_ROW_BYTES);
  const size_t o_l = opb, o_m = 2 * opb, o_norm = (S3 ? 3 : 2) * opb, o_c = o_norm + up256((size_t)npad * 4),
               o_band = o_c + up256((size_t)TC_K * 4), total = o_band + (want_band ? band_cap * 8 : 0);
  char *blk = nullptr;
  auto release = [&]() {
    if (blk) cudaFreeAsync(blk, s);
  };
  auto fail = [&](cudaError_t e) {
    cudaGetLastError();
    release();
    return cuda_status(e, "gram_bitmap_tc", __FILE__, __LINE__);
  };
  cudaError_t e;
  if ((e = dev_malloc((void **)&blk, total, s)) != cudaSuccess) return fail(e);
  __nv_bfloat16 *Xh = (__nv_bfloat16 *)blk, *Xl = (__nv_bfloat16 *)(blk + o_l);
  __nv_bfloat16 *Xm = S3 ? (__nv_bfloat16 *)(blk + o_m) : nullptr;
  float *norm = (float *)(blk + o_norm), *centre = (float *)(blk + o_c);
  uint64_t *band = want_band ? (uint64_t *)(blk + o_band) : nullptr;
  CUtensorMap mh, ml, mm;
  vr_status vs = make_map(&mh, Xh, npad);
  if (vs == VR_OK) vs = make_map(&ml, Xl, npad);
  if (vs == VR_OK) vs = make_map(&mm, S3 ? Xm : Xh, npad);
  if (vs != VR_OK) {
    release();
    return vs;
  }
  if (F) {
    if ((e = launch_dep(k_gram_centre, 1, 1024, 0, s, (const float *)X, n, d, centre, st)) != cudaSuccess)
      return fail(e);
    if ((e = launch_dep(k_gram_prep<true>, (npad + 7) / 8, 256, 0, s, X, n, d, npad, (const float *)centre, Xh, Xl,
                        norm, Xm)) != cudaSuccess)
      return fail(e);
  } else {
    if ((e = launch_dep(k_gram_prep<false>, (npad + 7) / 8, 256, 0, s, X, n, d, npad, (const float *)centre, Xh, Xl,
                        norm, (__nv_bfloat16 *)nullptr)) != cudaSuccess)
      return fail(e);
  }
  count_launch(F ? 2 : 1);
  const size_t smem = (S3 ? 6 : 4) * TC_OPERAND_BYTES + 1024 + 64;
  int stall_tile = -1;
  long stall_limit = TC_WAIT_LIMIT;
  const bool inj = !acc && take_gram_stall(ntiles, &stall_tile, &stall_limit);
#define VR_TILES(FF, VV, II, SS) \
  launch_tiles<FF, VV, II, SS>(ntiles, smem, s, mh, ml, mm, X, n, d, W, nt, cap, norm, adj, st, band, band_cap, acc, \
                               stall_tile, stall_limit)
  if (F && acc) e = S3 ? VR_TILES(true, true, false, true) : VR_TILES(true, true, false, false);
  else if (F && inj) e = S3 ? VR_TILES(true, false, true, true) : VR_TILES(true, false, true, false);
  else if (F) e = S3 ? VR_TILES(true, false, false, true) : VR_TILES(true, false, false, false);
  else if (inj) e = VR_TILES(false, false, true, false);
  else e = VR_TILES(false, false, false, false);
#undef VR_TILES
  count_launch();
  if (e != cudaSuccess) return fail(e);
  if (want_band) {
    e = launch_dep(k_band_patch, num_sms() * 4, 256, 0, s, (const float *)X, d, W, cap.r2, (const uint64_t *)band,
                   (const DevStatus *)st, band_cap, adj);
    count_launch();
    if (e != cudaSuccess) return fail(e);
  }
  release();
  return VR_OK;
}

}  // namespace vr

extern "C" {

vr_status vr_set_gram_path(int32_t mode) {
  if (mode < 0 || mode > 2) {
    vr::set_error("gram path mode %d outside 0..2", mode);
    return VR_ERR_ARG;
  }
  vr::g_gram_mode = mode;
  return VR_OK;
}

vr_status vr_set_gram_split(int32_t split) {
  if (split != 2 && split != 3) {
    vr::set_error("gram split %d: 2 (hi, lo) or 3 (hi, mid, lo)", split);
    return VR_ERR_ARG;
  }
  vr::g_gram_split = split;
  return VR_OK;
}

}  // extern "C"

// Accuracy of the float Gram tiles against the canonical FP64 values.
extern "C" vr_status vr_gram_accuracy_check(const float *points, int32_t n, int32_t d, double maxrad, int32_t split,
                                            vr_stream_t stream, vr_gram_accuracy *out) {
  using namespace vr;
  if (!points || !out || n < 2 || n > VR_MAX_POINTS || d < 1 || d > TC_K || !(maxrad >= 0) ||
      (split != 0 && split != 2 && split != 3)) {
    set_error("bad argument (n in [2, 8192], 1 <= d <= 64, maxrad >= 0, split 0/2/3, device float points)");
    return VR_ERR_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const int W = (n + 31) / 32;
  uint32_t *adj = nullptr;
  DevStatus *st = nullptr;
  GramAcc *acc = nullptr;
  auto release = [&]() {
    for (void *p : {(void *)adj, (void *)st, (void *)acc})
      if (p) cudaFreeAsync(p, s);
  };
  cudaError_t e = dev_malloc((void **)&adj, (size_t)n * W * 4, s);
  if (e == cudaSuccess) e = dev_malloc((void **)&st, sizeof(DevStatus), s);
  if (e == cudaSuccess) e = dev_malloc((void **)&acc, sizeof(GramAcc), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(st, 0, sizeof(DevStatus), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(acc, 0, sizeof(GramAcc), s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    release();
    set_error("accuracy check workspace: %s", cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? VR_ERR_OOM : VR_ERR_CUDA;
  }
  // The build's cap parameters for these points.
  Cap cap{};
  const double r2 = maxrad * maxrad;
  cap.keep_all = std::isinf(r2) || r2 >= 1e38 ? 1 : 0;
  cap.r2 = r2;
  if (!cap.keep_all) {
    cap.r2f_dn = (float)r2;
    if ((double)cap.r2f_dn > r2) cap.r2f_dn = std::nextafter(cap.r2f_dn, -INFINITY);
    cap.r2f_up = (float)r2;
    if ((double)cap.r2f_up < r2) cap.r2f_up = std::nextafter(cap.r2f_up, INFINITY);
  }
  vr_status r = gram_bitmap_tc(points, n, d, true, cap, adj, st, s, acc, split);
  GramAcc h{};
  int32_t flags = 0;
  if (r == VR_OK) {
    e = cudaMemcpyAsync(&h, acc, sizeof(GramAcc), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&flags, &st->flags, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) r = cuda_status(e, "accuracy check", __FILE__, __LINE__);
  }
  release();
  if (r != VR_OK) return r;
  if (flags) return flags_to_status(flags);
  float wn, wr;
  memcpy(&wn, &h.worst_norm, 4);
  memcpy(&wr, &h.worst_rel_d, 4);
  out->max_norm_err = wn;
  out->max_rel_d_err = wr;
  out->beta = TC_BETA;
  out->kept_pairs = (int64_t)h.kept;
  out->band_pairs = (int64_t)h.band;
  return VR_OK;
}

extern "C" vr_status vr_gram_error_check(const float *points, int32_t n, int32_t d, vr_stream_t stream,
                                         double *worst_ratio, double *beta_ratio) {
  if (!worst_ratio) {
    vr::set_error("worst_ratio is NULL");
    return VR_ERR_ARG;
  }
  vr_gram_accuracy a{};
  VR_TRY(vr_gram_accuracy_check(points, n, d, INFINITY, 0, stream, &a));
  *worst_ratio = a.max_norm_err;
  if (beta_ratio) *beta_ratio = a.beta;
  return VR_OK;
}
