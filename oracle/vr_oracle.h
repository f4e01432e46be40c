/*
 * vr_oracle.h -- plain CPU oracle for the Vietoris-Rips filtered-complex build.
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the independent checker that the
 * CUDA path is compared against.  Only the test suite, the package smoke check
 * and the CPU-baseline leg of the benchmark may load it; the product path never
 * does.  It shares no code, header, table or helper with the CUDA library.
 *
 * What it computes (arXiv 1809.04424):
 *   - Sec. 2.1 "Homological Persistence": an edge joins two points closer than
 *     the threshold, a triangle is present when its three edges are, and the
 *     threshold acts as time, so every simplex enters at the time of its
 *     longest edge.
 *   - Sec. 3 (the Eirene call): the output is an integer rank matrix of the
 *     distances ("symmat") plus per-dimension filtration grades.
 *   - Sec. 4.4 (sortperm): ranking the distances is a sort permutation.
 *   - Sec. 2.2: the filtered boundary matrix D, stored here in CSC over F2.
 *   - Algorithm 1 (column algorithm) and the pivot/bar rule of Fig. 4's caption:
 *     used only to turn the complex into barcodes for self-checks.
 *
 * Readings where the paper is silent (each restated in the .c file):
 *   cap inclusive (d <= maxrad); equal squared distances share a grade (dense
 *   rank over {0} U {kept d^2}); order within a dimension is (grade, vertex
 *   tuple lexicographic); a simplex's grade is its largest edge grade; maxdim
 *   is the top simplex dimension; a bar is [grade(low(j)), grade(j)).
 *
 * All functions return 0 on success and a negative code on a bad argument.
 */
#ifndef VR_ORACLE_H
#define VR_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Element types of the input point array (row-major n x d). */
#define VRO_I8 1
#define VRO_I32 2
#define VRO_F32 3

#define VRO_MAXDIM 3

typedef struct {
  int32_t n, d, maxdim;
  int64_t count[VRO_MAXDIM + 1];   /* number of k-simplices                  */
  int32_t *verts[VRO_MAXDIM + 1];  /* count[k] x (k+1), ascending per simplex */
  int32_t *grade[VRO_MAXDIM + 1];  /* count[k]                               */
  int64_t *colptr[VRO_MAXDIM + 1]; /* count[k]+1 for k >= 1; NULL for k = 0   */
  int32_t *rowidx[VRO_MAXDIM + 1]; /* (k+1)*count[k] for k >= 1               */
  int64_t ngrades;
  double *grade_value;             /* squared distance of each grade         */
} vro_complex;

/* Build the filtered complex (steps 1-7 of the oracle).  `pts` is a host
 * array of n*d elements of type `dtype`.  maxrad = +inf keeps every pair. */
int vro_build(const void *pts, int32_t n, int32_t d, int32_t dtype,
              int32_t maxdim, double maxrad, vro_complex *out);
void vro_free(vro_complex *c);

/* The same complex from a square symmetric n x n matrix of edge values
 * (host, row-major, VRO_I32 or VRO_F32): the strict upper triangle gives the
 * edges, kept iff value <= maxrad; grades rank the values (no squaring).
 * Asymmetric, negative or non-finite entries: a bad-argument code. */
int vro_build_dmat(const void *D, int32_t n, int32_t dtype, int32_t maxdim, double maxrad, vro_complex *out);

/* Squared distance of one pair, as step 1 defines it (integer: exact, as a
 * double that is exact below 2^53; float: canonical FP64 sequence). */
double vro_pair_d2(const void *pts, int32_t d, int32_t dtype, int32_t i,
                   int32_t j);

/* Dense rank of `m` non-negative values inside {0} U values (step 3):
 * rank[t] = number of distinct members of {0} U values below values[t]. */
int vro_dense_rank(const double *values, int64_t m, int64_t *rank);

/* Barcode of dimension `dim` (0 <= dim <= maxdim) by Algorithm 1 over F2.
 * Bars are [birth, death) in grades, death = -1 for an infinite bar;
 * zero-length bars are dropped.  Arrays are malloc'd; free with vro_free_buf. */
int vro_barcode(const vro_complex *c, int32_t dim, int64_t *nbars,
                int64_t **birth, int64_t **death);
void vro_free_buf(void *p);

#ifdef __cplusplus
}
#endif
#endif
