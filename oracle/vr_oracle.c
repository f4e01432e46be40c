/*
 * vr_oracle.c -- plain, slow, obviously correct CPU oracle of the
 * Vietoris-Rips filtered-complex build (arXiv 1809.04424).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * benchmark's CPU-baseline leg, never by the product path.  It shares no code
 * with the CUDA library.  Build with -ffp-contract=off (no fused multiply-add)
 * so that the float distance follows the canonical rounding sequence below.
 *
 * Steps, in the order the definitions give them:
 *   1. squared distance of every pair i<j        (Sec. 2.1; ranks use d^2)
 *   2. radius cap, inclusive                      (Sec. 2.1 threshold reading)
 *   3. grades = dense rank of d^2 in {0} U kept   (Sec. 3 "symmat", Sec. 4.4)
 *   4. edges sorted by (grade, i, j)
 *   5. triangles by brute force, grade = max edge grade, sorted (grade, a,b,c)
 *   6. vertices in id order, grade 0
 *   7. boundary matrix over F2 in CSC             (Sec. 2.2, Sec. 4.5 "mod 2")
 *   8. (self-checks only) Algorithm 1 and the pivot -> bar rule of Fig. 4.
 * Every parity function is pinned by tests against closed forms, invariants
 * and brute force; none is "parity unpinned".
 */
#include "vr_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;

enum { ERR_ARG = -1, ERR_UNSUPPORTED = -2, ERR_OOM = -4 };

/* ------------------------------------------------------------------ step 1 */

/* Integer squared distance, exact: sum over coordinates of (x_ik - x_jk)^2.
 * Differences of int32 values fit in int64, their squares in u64, and the sum
 * is accumulated in 128 bits, so nothing rounds. */
static u128 d2_int(const void *pts, int32_t d, int32_t dtype, int32_t i,
                   int32_t j) {
  u128 acc = 0;
  for (int32_t k = 0; k < d; ++k) {
    int64_t a, b;
    if (dtype == VRO_I8) {
      a = ((const int8_t *)pts)[(int64_t)i * d + k];
      b = ((const int8_t *)pts)[(int64_t)j * d + k];
    } else {
      a = ((const int32_t *)pts)[(int64_t)i * d + k];
      b = ((const int32_t *)pts)[(int64_t)j * d + k];
    }
    int64_t t = a - b;
    uint64_t m = (uint64_t)(t < 0 ? -t : t);
    acc += (u128)m * (u128)m;
  }
  return acc;
}

/* Float squared distance, the canonical FP64 sequence: acc = 0; for k in
 * order: t = fl(x_ik - x_jk); acc = fl(acc + fl(t*t)).  Each operation rounds
 * to nearest; nothing is fused. */
static double d2_f32(const float *pts, int32_t d, int32_t i, int32_t j) {
  double acc = 0.0;
  for (int32_t k = 0; k < d; ++k) {
    double t = (double)pts[(int64_t)i * d + k] - (double)pts[(int64_t)j * d + k];
    double sq = t * t;
    acc = acc + sq;
  }
  return acc;
}

double vro_pair_d2(const void *pts, int32_t d, int32_t dtype, int32_t i,
                   int32_t j) {
  if (dtype == VRO_F32) return d2_f32((const float *)pts, d, i, j);
  return (double)d2_int(pts, d, dtype, i, j);
}

/* ------------------------------------------------------------------ step 3 */

static int cmp_u128(const void *a, const void *b) {
  u128 x = *(const u128 *)a, y = *(const u128 *)b;
  return x < y ? -1 : (x > y ? 1 : 0);
}
static int cmp_f64(const void *a, const void *b) {
  double x = *(const double *)a, y = *(const double *)b;
  return x < y ? -1 : (x > y ? 1 : 0);
}

/* Sorted distinct set {0} U values, in place; returns its size. */
static int64_t distinct_u128(u128 *v, int64_t m) {
  v[m] = 0; /* caller leaves one spare slot for the 0 */
  qsort(v, (size_t)(m + 1), sizeof(u128), cmp_u128);
  int64_t w = 0;
  for (int64_t t = 0; t <= m; ++t)
    if (w == 0 || v[t] != v[w - 1]) v[w++] = v[t];
  return w;
}
static int64_t distinct_f64(double *v, int64_t m) {
  v[m] = 0.0;
  qsort(v, (size_t)(m + 1), sizeof(double), cmp_f64);
  int64_t w = 0;
  for (int64_t t = 0; t <= m; ++t)
    if (w == 0 || v[t] != v[w - 1]) v[w++] = v[t];
  return w;
}
/* Position of x in the sorted distinct array v[0..w) (x is a member). */
static int64_t find_u128(const u128 *v, int64_t w, u128 x) {
  int64_t lo = 0, hi = w - 1;
  while (lo < hi) {
    int64_t mid = (lo + hi) / 2;
    if (v[mid] < x) lo = mid + 1; else hi = mid;
  }
  return lo;
}
static int64_t find_f64(const double *v, int64_t w, double x) {
  int64_t lo = 0, hi = w - 1;
  while (lo < hi) {
    int64_t mid = (lo + hi) / 2;
    if (v[mid] < x) lo = mid + 1; else hi = mid;
  }
  return lo;
}

int vro_dense_rank(const double *values, int64_t m, int64_t *rank) {
  if (m < 0 || (m > 0 && (!values || !rank))) return ERR_ARG;
  for (int64_t t = 0; t < m; ++t)
    if (!(values[t] >= 0.0)) return ERR_ARG;
  double *v = (double *)malloc(sizeof(double) * (size_t)(m + 1));
  if (!v) return ERR_OOM;
  if (m) memcpy(v, values, sizeof(double) * (size_t)m);
  int64_t w = distinct_f64(v, m);
  for (int64_t t = 0; t < m; ++t) rank[t] = find_f64(v, w, values[t]);
  free(v);
  return 0;
}

/* ---------------------------------------------------------------- steps 4-5 */

typedef struct { int32_t g, a, b, c, d; } simp;

static int cmp_simp(const void *x, const void *y) {
  const simp *p = (const simp *)x, *q = (const simp *)y;
  if (p->g != q->g) return p->g < q->g ? -1 : 1;
  if (p->a != q->a) return p->a < q->a ? -1 : 1;
  if (p->b != q->b) return p->b < q->b ? -1 : 1;
  if (p->c != q->c) return p->c < q->c ? -1 : 1;
  if (p->d != q->d) return p->d < q->d ? -1 : 1;
  return 0;
}

static int cmp_i64pair(const void *x, const void *y) {
  const int64_t *p = (const int64_t *)x, *q = (const int64_t *)y;
  return p[0] < q[0] ? -1 : p[0] > q[0];
}

static void clear(vro_complex *c) { memset(c, 0, sizeof(*c)); }

void vro_free(vro_complex *c) {
  if (!c) return;
  for (int k = 0; k <= VRO_MAXDIM; ++k) {
    free(c->verts[k]);
    free(c->grade[k]);
    free(c->colptr[k]);
    free(c->rowidx[k]);
  }
  free(c->grade_value);
  clear(c);
}

void vro_free_buf(void *p) { free(p); }

/* Steps 3-7 from the kept pairs (ei[t] < ej[t], value di[t] (integer) or
 * df[t] (float), t < m, in (i, j) order).  Takes ownership of the four
 * arrays. */
static int finish_build(vro_complex *out, int32_t n, int32_t maxdim, int is_float, int32_t *ei, int32_t *ej,
                        u128 *di, double *df, int64_t m) {
  int32_t *eg = NULL;
  /* Step 3: grade of an edge = rank of its value (d^2 for points) in the
   * sorted distinct set {0} U {kept values}; grade_value[g] = the g-th
   * member. */
  eg = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m + 1));
  int64_t ng = 0;
  if (!eg) goto oom_pairs;
  if (is_float) {
    double *v = (double *)malloc(sizeof(double) * (size_t)(m + 1));
    if (!v) goto oom_pairs;
    if (m) memcpy(v, df, sizeof(double) * (size_t)m);
    ng = distinct_f64(v, m);
    for (int64_t t = 0; t < m; ++t) eg[t] = (int32_t)find_f64(v, ng, df[t]);
    out->grade_value = v;
  } else {
    u128 *v = (u128 *)malloc(sizeof(u128) * (size_t)(m + 1));
    if (!v) goto oom_pairs;
    if (m) memcpy(v, di, sizeof(u128) * (size_t)m);
    ng = distinct_u128(v, m);
    for (int64_t t = 0; t < m; ++t) eg[t] = (int32_t)find_u128(v, ng, di[t]);
    out->grade_value = (double *)malloc(sizeof(double) * (size_t)ng);
    if (!out->grade_value) { free(v); goto oom_pairs; }
    for (int64_t g = 0; g < ng; ++g) out->grade_value[g] = (double)v[g];
    free(v);
  }
  out->ngrades = ng;
  free(di); di = NULL;
  free(df); df = NULL;

  if (maxdim >= 1) {
    /* Step 4: edges in (grade, i, j) order. */
    simp *es = (simp *)malloc(sizeof(simp) * (size_t)(m + 1));
    if (!es) goto oom_pairs;
    for (int64_t t = 0; t < m; ++t) { es[t].g = eg[t]; es[t].a = ei[t]; es[t].b = ej[t]; es[t].c = 0; es[t].d = 0; }
    qsort(es, (size_t)m, sizeof(simp), cmp_simp);
    out->count[1] = m;
    out->verts[1] = (int32_t *)malloc(sizeof(int32_t) * (size_t)(2 * m + 1));
    out->grade[1] = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m + 1));
    out->colptr[1] = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m + 1));
    out->rowidx[1] = (int32_t *)malloc(sizeof(int32_t) * (size_t)(2 * m + 1));
    if (!out->verts[1] || !out->grade[1] || !out->colptr[1] || !out->rowidx[1]) { free(es); goto oom_pairs; }
    for (int64_t t = 0; t < m; ++t) {
      out->verts[1][2 * t] = es[t].a;
      out->verts[1][2 * t + 1] = es[t].b;
      out->grade[1][t] = es[t].g;
      /* Step 7, dimension 1: the boundary of edge (i,j) is {i, j}; vertices
       * are ordered by id, so the rows are i then j. */
      out->colptr[1][t] = 2 * t;
      out->rowidx[1][2 * t] = es[t].a;
      out->rowidx[1][2 * t + 1] = es[t].b;
    }
    out->colptr[1][m] = 2 * m;

    if (maxdim >= 2) {
      /* Order index of every kept edge, -1 where no edge. */
      int32_t *ord = (int32_t *)malloc(sizeof(int32_t) * (size_t)n * (size_t)n);
      if (!ord) { free(es); goto oom_pairs; }
      for (int64_t t = 0; t < (int64_t)n * n; ++t) ord[t] = -1;
      for (int64_t t = 0; t < m; ++t) {
        ord[(int64_t)es[t].a * n + es[t].b] = (int32_t)t;
        ord[(int64_t)es[t].b * n + es[t].a] = (int32_t)t;
      }
      /* Step 5: a triangle (i,j,k), i<j<k, is present iff all three edges
       * are kept (Sec. 2.1); its grade is the largest edge grade. */
      int64_t cap = 1024, T = 0;
      simp *ts = (simp *)malloc(sizeof(simp) * (size_t)cap);
      if (!ts) { free(ord); free(es); goto oom_pairs; }
      for (int64_t t = 0; t < m; ++t) {
        int32_t i = es[t].a, j = es[t].b;
        for (int32_t k = j + 1; k < n; ++k) {
          int32_t oik = ord[(int64_t)i * n + k], ojk = ord[(int64_t)j * n + k];
          if (oik < 0 || ojk < 0) continue;
          if (T == cap) {
            cap *= 2;
            simp *nt = (simp *)realloc(ts, sizeof(simp) * (size_t)cap);
            if (!nt) { free(ts); free(ord); free(es); goto oom_pairs; }
            ts = nt;
          }
          int32_t g = es[t].g;
          if (es[oik].g > g) g = es[oik].g;
          if (es[ojk].g > g) g = es[ojk].g;
          ts[T].g = g; ts[T].a = i; ts[T].b = j; ts[T].c = k; ts[T].d = 0;
          ++T;
        }
      }
      qsort(ts, (size_t)T, sizeof(simp), cmp_simp);
      out->count[2] = T;
      out->verts[2] = (int32_t *)malloc(sizeof(int32_t) * (size_t)(3 * T + 1));
      out->grade[2] = (int32_t *)malloc(sizeof(int32_t) * (size_t)(T + 1));
      out->colptr[2] = (int64_t *)malloc(sizeof(int64_t) * (size_t)(T + 1));
      out->rowidx[2] = (int32_t *)malloc(sizeof(int32_t) * (size_t)(3 * T + 1));
      if (!out->verts[2] || !out->grade[2] || !out->colptr[2] || !out->rowidx[2]) {
        free(ts); free(ord); free(es); goto oom_pairs;
      }
      for (int64_t t = 0; t < T; ++t) {
        int32_t a = ts[t].a, b = ts[t].b, c = ts[t].c;
        out->verts[2][3 * t] = a;
        out->verts[2][3 * t + 1] = b;
        out->verts[2][3 * t + 2] = c;
        out->grade[2][t] = ts[t].g;
        /* Step 7, dimension 2: the faces (b,c), (a,c), (a,b), as edge order
         * indices, listed ascending. */
        int32_t r[3] = {ord[(int64_t)b * n + c], ord[(int64_t)a * n + c],
                        ord[(int64_t)a * n + b]};
        for (int x = 0; x < 3; ++x)
          for (int y = x + 1; y < 3; ++y)
            if (r[y] < r[x]) { int32_t s = r[x]; r[x] = r[y]; r[y] = s; }
        out->colptr[2][t] = 3 * t;
        out->rowidx[2][3 * t] = r[0];
        out->rowidx[2][3 * t + 1] = r[1];
        out->rowidx[2][3 * t + 2] = r[2];
      }
      out->colptr[2][T] = 3 * T;

      if (maxdim >= 3) {
        /* Tetrahedra (a,b,c,d), a<b<c<d: present iff all six edges are kept;
         * grade = the largest edge grade (= the largest face grade). */
        int64_t *lexkey = (int64_t *)malloc(sizeof(int64_t) * (size_t)(T + 1));
        int64_t *lexord = (int64_t *)malloc(sizeof(int64_t) * (size_t)(T + 1));
        int64_t qcap = 1024, Q = 0;
        simp *qs = (simp *)malloc(sizeof(simp) * (size_t)qcap);
        if (!lexkey || !lexord || !qs) { free(lexkey); free(lexord); free(qs); free(ts); free(ord); free(es); goto oom_pairs; }
        /* Order index of a triangle from its vertices: triangles sorted by
         * their lexicographic key, searched by bisection. */
        for (int64_t t = 0; t < T; ++t) lexord[t] = t;
        const int64_t nn = n;
        for (int64_t t = 0; t < T; ++t) lexkey[t] = ((int64_t)ts[t].a * nn + ts[t].b) * nn + ts[t].c;
        /* insertion into lexicographic order via qsort on (key, index) pairs */
        int64_t *pairs = (int64_t *)malloc(sizeof(int64_t) * 2 * (size_t)(T + 1));
        if (!pairs) { free(lexkey); free(lexord); free(qs); free(ts); free(ord); free(es); goto oom_pairs; }
        for (int64_t t = 0; t < T; ++t) { pairs[2 * t] = lexkey[t]; pairs[2 * t + 1] = t; }
        qsort(pairs, (size_t)T, 2 * sizeof(int64_t), cmp_i64pair);
        for (int64_t t = 0; t < T; ++t) { lexkey[t] = pairs[2 * t]; lexord[t] = pairs[2 * t + 1]; }
        free(pairs);
        for (int64_t t = 0; t < T; ++t) {
          const int32_t a = ts[t].a, b = ts[t].b, c = ts[t].c;
          for (int32_t dv = c + 1; dv < n; ++dv) {
            const int32_t oad = ord[(int64_t)a * n + dv], obd = ord[(int64_t)b * n + dv], ocd = ord[(int64_t)c * n + dv];
            if (oad < 0 || obd < 0 || ocd < 0) continue;
            if (Q == qcap) {
              qcap *= 2;
              simp *nq = (simp *)realloc(qs, sizeof(simp) * (size_t)qcap);
              if (!nq) { free(lexkey); free(lexord); free(qs); free(ts); free(ord); free(es); goto oom_pairs; }
              qs = nq;
            }
            int32_t g = ts[t].g;
            if (es[oad].g > g) g = es[oad].g;
            if (es[obd].g > g) g = es[obd].g;
            if (es[ocd].g > g) g = es[ocd].g;
            qs[Q].g = g; qs[Q].a = a; qs[Q].b = b; qs[Q].c = c; qs[Q].d = dv;
            ++Q;
          }
        }
        qsort(qs, (size_t)Q, sizeof(simp), cmp_simp);
        out->count[3] = Q;
        out->verts[3] = (int32_t *)malloc(sizeof(int32_t) * (size_t)(4 * Q + 1));
        out->grade[3] = (int32_t *)malloc(sizeof(int32_t) * (size_t)(Q + 1));
        out->colptr[3] = (int64_t *)malloc(sizeof(int64_t) * (size_t)(Q + 1));
        out->rowidx[3] = (int32_t *)malloc(sizeof(int32_t) * (size_t)(4 * Q + 1));
        if (!out->verts[3] || !out->grade[3] || !out->colptr[3] || !out->rowidx[3]) {
          free(lexkey); free(lexord); free(qs); free(ts); free(ord); free(es); goto oom_pairs;
        }
        for (int64_t t = 0; t < Q; ++t) {
          const int32_t a = qs[t].a, b = qs[t].b, c = qs[t].c, dv = qs[t].d;
          out->verts[3][4 * t] = a;
          out->verts[3][4 * t + 1] = b;
          out->verts[3][4 * t + 2] = c;
          out->verts[3][4 * t + 3] = dv;
          out->grade[3][t] = qs[t].g;
          /* Step 7, dimension 3: the faces (b,c,d), (a,c,d), (a,b,d), (a,b,c)
           * as triangle order indices, listed ascending. */
          int64_t fk[4] = {((int64_t)b * nn + c) * nn + dv, ((int64_t)a * nn + c) * nn + dv,
                           ((int64_t)a * nn + b) * nn + dv, ((int64_t)a * nn + b) * nn + c};
          int32_t r[4];
          for (int x = 0; x < 4; ++x) {
            int64_t lo = 0, hi = T;
            while (lo < hi) { int64_t mid = (lo + hi) / 2; if (lexkey[mid] < fk[x]) lo = mid + 1; else hi = mid; }
            r[x] = (int32_t)lexord[lo];
          }
          for (int x = 0; x < 4; ++x)
            for (int y = x + 1; y < 4; ++y)
              if (r[y] < r[x]) { int32_t sw = r[x]; r[x] = r[y]; r[y] = sw; }
          out->colptr[3][t] = 4 * t;
          for (int x = 0; x < 4; ++x) out->rowidx[3][4 * t + x] = r[x];
        }
        out->colptr[3][Q] = 4 * Q;
        free(lexkey);
        free(lexord);
        free(qs);
      }
      free(ts);
      free(ord);
    }
    free(es);
  }
  free(eg);
  free(ei);
  free(ej);
  return 0;

oom_pairs:
  free(eg); free(ei); free(ej); free(di); free(df);
  vro_free(out);
  return ERR_OOM;
}

int vro_build(const void *pts, int32_t n, int32_t d, int32_t dtype,
              int32_t maxdim, double maxrad, vro_complex *out) {
  if (!out) return ERR_ARG;
  clear(out);
  if (!pts || n < 1 || d < 1) return ERR_ARG;
  if (dtype != VRO_I8 && dtype != VRO_I32 && dtype != VRO_F32) return ERR_ARG;
  if (maxdim < 0) return ERR_ARG;
  if (maxdim > VRO_MAXDIM) return ERR_UNSUPPORTED;
  if (isnan(maxrad) || maxrad < 0.0) return ERR_ARG;
  const int is_float = (dtype == VRO_F32);
  if (is_float)
    for (int64_t t = 0; t < (int64_t)n * d; ++t)
      if (!isfinite(((const float *)pts)[t])) return ERR_ARG;

  out->n = n;
  out->d = d;
  out->maxdim = maxdim;

  /* Step 6: vertices in id order, all at grade 0. */
  out->count[0] = n;
  out->verts[0] = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
  out->grade[0] = (int32_t *)calloc((size_t)n, sizeof(int32_t));
  if (!out->verts[0] || !out->grade[0]) { vro_free(out); return ERR_OOM; }
  for (int32_t v = 0; v < n; ++v) out->verts[0][v] = v;

  /* Steps 1-2: every pair i<j, its squared distance, kept iff d^2 <= r^2.
   * Float: r2 = fl(maxrad*maxrad).  Integer: r2i = floor(fl(maxrad*maxrad)),
   * which for an integer d^2 is the same test. */
  const double r2 = maxrad * maxrad;
  const int keep_all = isinf(r2);
  u128 r2i = 0;
  int keep_all_int = keep_all;
  if (!is_float && !keep_all) {
    double f = floor(r2);
    if (f >= 3.0e38) keep_all_int = 1; else r2i = (u128)f;
  }
  int64_t npairs = (int64_t)n * (n - 1) / 2;
  int32_t *ei = (int32_t *)malloc(sizeof(int32_t) * (size_t)(npairs + 1));
  int32_t *ej = (int32_t *)malloc(sizeof(int32_t) * (size_t)(npairs + 1));
  u128 *di = is_float ? NULL : (u128 *)malloc(sizeof(u128) * (size_t)(npairs + 1));
  double *df = is_float ? (double *)malloc(sizeof(double) * (size_t)(npairs + 1)) : NULL;
  if (!ei || !ej || (!di && !df)) goto oom_pairs;
  int64_t m = 0;
  for (int32_t i = 0; i < n; ++i)
    for (int32_t j = i + 1; j < n; ++j) {
      if (is_float) {
        double v = d2_f32((const float *)pts, d, i, j);
        if (keep_all || v <= r2) { ei[m] = i; ej[m] = j; df[m] = v; ++m; }
      } else {
        u128 v = d2_int(pts, d, dtype, i, j);
        if (keep_all_int || v <= r2i) { ei[m] = i; ej[m] = j; di[m] = v; ++m; }
      }
    }

  return finish_build(out, n, maxdim, is_float, ei, ej, di, df, m);

oom_pairs:
  free(ei); free(ej); free(di); free(df);
  vro_free(out);
  return ERR_OOM;
}

/* Distance-matrix input (the paper's Sec. 3: Eirene also takes a square
 * symmetric matrix, typically of pairwise distances).  Readings: the strict
 * upper triangle D[i][j], i < j, gives the edge values; the matrix must be
 * exactly symmetric with finite non-negative entries; the diagonal is
 * ignored (vertices at grade 0); an edge is kept iff D[i][j] <= maxrad; the
 * grades rank the values themselves (no squaring), grade_value[g] = the g-th
 * distinct value of {0} U {kept values}. */
int vro_build_dmat(const void *D, int32_t n, int32_t dtype, int32_t maxdim, double maxrad, vro_complex *out) {
  if (!out) return ERR_ARG;
  clear(out);
  if (!D || n < 1) return ERR_ARG;
  if (dtype != VRO_I32 && dtype != VRO_F32) return ERR_ARG;
  if (maxdim < 0) return ERR_ARG;
  if (maxdim > VRO_MAXDIM) return ERR_UNSUPPORTED;
  if (isnan(maxrad) || maxrad < 0.0) return ERR_ARG;
  const int is_float = (dtype == VRO_F32);
  for (int32_t i = 0; i < n; ++i)
    for (int32_t j = 0; j < n; ++j) {
      if (is_float) {
        const float v = ((const float *)D)[(int64_t)i * n + j], w = ((const float *)D)[(int64_t)j * n + i];
        if (!isfinite(v) || v < 0.0f || v != w) return ERR_ARG;
      } else {
        const int32_t v = ((const int32_t *)D)[(int64_t)i * n + j], w = ((const int32_t *)D)[(int64_t)j * n + i];
        if (v < 0 || v != w) return ERR_ARG;
      }
    }
  out->n = n;
  out->d = 0;
  out->maxdim = maxdim;
  out->count[0] = n;
  out->verts[0] = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
  out->grade[0] = (int32_t *)calloc((size_t)n, sizeof(int32_t));
  if (!out->verts[0] || !out->grade[0]) { vro_free(out); return ERR_OOM; }
  for (int32_t v = 0; v < n; ++v) out->verts[0][v] = v;
  const int64_t npairs = (int64_t)n * (n - 1) / 2;
  int32_t *ei = (int32_t *)malloc(sizeof(int32_t) * (size_t)(npairs + 1));
  int32_t *ej = (int32_t *)malloc(sizeof(int32_t) * (size_t)(npairs + 1));
  u128 *di = is_float ? NULL : (u128 *)malloc(sizeof(u128) * (size_t)(npairs + 1));
  double *df = is_float ? (double *)malloc(sizeof(double) * (size_t)(npairs + 1)) : NULL;
  if (!ei || !ej || (!di && !df)) {
    free(ei); free(ej); free(di); free(df);
    vro_free(out);
    return ERR_OOM;
  }
  int64_t m = 0;
  for (int32_t i = 0; i < n; ++i)
    for (int32_t j = i + 1; j < n; ++j) {
      const double v = is_float ? (double)((const float *)D)[(int64_t)i * n + j]
                                : (double)((const int32_t *)D)[(int64_t)i * n + j];
      if (v <= maxrad) {
        ei[m] = i;
        ej[m] = j;
        if (is_float) df[m] = v;
        else di[m] = (u128)((const int32_t *)D)[(int64_t)i * n + j];
        ++m;
      }
    }
  return finish_build(out, n, maxdim, is_float, ei, ej, di, df, m);
}

/* ------------------------------------------------------------------ step 8 */

/* A sparse F2 column: sorted row indices. */
typedef struct { int64_t len, cap; int64_t *r; } col_t;

static int col_push(col_t *c, int64_t x) {
  if (c->len == c->cap) {
    int64_t nc = c->cap ? 2 * c->cap : 4;
    int64_t *nr = (int64_t *)realloc(c->r, sizeof(int64_t) * (size_t)nc);
    if (!nr) return ERR_OOM;
    c->r = nr; c->cap = nc;
  }
  c->r[c->len++] = x;
  return 0;
}

/* c <- c + p over F2: symmetric difference of two sorted lists. */
static int col_add(col_t *c, const col_t *p) {
  col_t out = {0, 0, NULL};
  int64_t x = 0, y = 0;
  while (x < c->len || y < p->len) {
    int64_t v;
    if (y == p->len || (x < c->len && c->r[x] < p->r[y])) v = c->r[x++];
    else if (x == c->len || p->r[y] < c->r[x]) v = p->r[y++];
    else { ++x; ++y; continue; } /* equal rows cancel mod 2 */
    if (col_push(&out, v)) { free(out.r); return ERR_OOM; }
  }
  free(c->r);
  *c = out;
  return 0;
}

/* Algorithm 1 on the boundary matrix of dimension k (columns = k-simplices
 * in filtration order, rows = (k-1)-simplices in filtration order).  Over F2
 * the multiplier c is 1, so "R[:,i] - c R[:,j]" is an addition.  Outputs, per
 * column, its low (-1 for a zero column). */
static int reduce_dim(const vro_complex *cx, int32_t k, int64_t *low) {
  int64_t m = cx->count[k], rows = cx->count[k - 1];
  col_t *R = (col_t *)calloc((size_t)(m + 1), sizeof(col_t));
  int64_t *owner = (int64_t *)malloc(sizeof(int64_t) * (size_t)(rows + 1));
  if (!R || !owner) { free(R); free(owner); return ERR_OOM; }
  for (int64_t r = 0; r < rows; ++r) owner[r] = -1;
  int rc = 0;
  for (int64_t j = 0; j < m && !rc; ++j) {
    for (int64_t p = cx->colptr[k][j]; p < cx->colptr[k][j + 1]; ++p)
      if ((rc = col_push(&R[j], cx->rowidx[k][p]))) break;
    /* While another earlier column has the same low, add it. */
    while (!rc && R[j].len > 0 && owner[R[j].r[R[j].len - 1]] >= 0)
      rc = col_add(&R[j], &R[owner[R[j].r[R[j].len - 1]]]);
    if (rc) break;
    if (R[j].len > 0) { low[j] = R[j].r[R[j].len - 1]; owner[low[j]] = j; }
    else low[j] = -1;
  }
  for (int64_t j = 0; j < m; ++j) free(R[j].r);
  free(R);
  free(owner);
  return rc;
}

/* Bars of dimension `dim`: a pivot (low(j) = s, column j of dimension dim+1)
 * is the bar [grade(s), grade(j)) (Fig. 4's caption reads pivot (v3, e5) as
 * the bar (3, 5)); a positive dim-simplex (zero reduced column) that is no
 * pivot row lives forever.  Zero-length bars are dropped. */
int vro_barcode(const vro_complex *c, int32_t dim, int64_t *nbars,
                int64_t **birth, int64_t **death) {
  if (!c || !nbars || !birth || !death || dim < 0 || dim > c->maxdim) return ERR_ARG;
  int64_t m = c->count[dim];
  int64_t *lowk = NULL, *lowk1 = NULL;
  char *positive = (char *)malloc((size_t)m + 1);
  char *killed = (char *)calloc((size_t)m + 1, 1);
  int64_t *b = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m + 1));
  int64_t *e = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m + 1));
  if (!positive || !killed || !b || !e) goto oom;
  if (dim == 0) {
    memset(positive, 1, (size_t)m);
  } else {
    lowk = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m + 1));
    if (!lowk || reduce_dim(c, dim, lowk)) goto oom;
    for (int64_t j = 0; j < m; ++j) positive[j] = (lowk[j] < 0);
  }
  int64_t nb = 0;
  if (dim < c->maxdim) {
    int64_t m1 = c->count[dim + 1];
    lowk1 = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m1 + 1));
    if (!lowk1 || reduce_dim(c, dim + 1, lowk1)) goto oom;
    for (int64_t j = 0; j < m1; ++j) {
      if (lowk1[j] < 0) continue;
      killed[lowk1[j]] = 1;
      int64_t gb = c->grade[dim][lowk1[j]], gd = c->grade[dim + 1][j];
      if (gb != gd) { b[nb] = gb; e[nb] = gd; ++nb; }
    }
  }
  for (int64_t s = 0; s < m; ++s)
    if (positive[s] && !killed[s]) { b[nb] = c->grade[dim][s]; e[nb] = -1; ++nb; }
  free(lowk); free(lowk1); free(positive); free(killed);
  *nbars = nb;
  *birth = b;
  *death = e;
  return 0;
oom:
  free(lowk); free(lowk1); free(positive); free(killed); free(b); free(e);
  return ERR_OOM;
}
