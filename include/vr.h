/*
 * vr.h -- C ABI of the B300 Vietoris-Rips filtered-complex builder.
 *
 * One call builds, on the GPU, the filtered Vietoris-Rips complex of a point
 * cloud up to simplex dimension 2 and its boundary matrix over F2:
 *
 *   - an edge {i,j} is present when |x_i - x_j| <= maxrad, a triangle when its
 *     three edges are (arXiv 1809.04424, Sec. 2.1 "Homological Persistence":
 *     the threshold acts as time, so a simplex enters with its longest edge);
 *   - the edge lengths are ranked into integer filtration grades, the rank
 *     matrix Eirene returns as "symmat" with per-dimension "filtration" grades
 *     (Sec. 3; ranking is the sort permutation of Sec. 4.4).  Equal squared
 *     distances share a grade; grade 0 is squared distance 0 and holds every
 *     vertex; grade g >= 1 is the g-th smallest distinct positive squared
 *     distance among the kept edges;
 *   - each dimension's simplices are listed in (grade, vertex tuple
 *     lexicographic) order, vertices ascending inside a simplex, a triangle's
 *     grade being its largest edge grade;
 *   - the boundary matrix D of Sec. 2.2 is stored per dimension k >= 1 in CSC
 *     over F2 (no values; Sec. 4.5 works mod 2 on CSC): column j lists the
 *     order indices of the k+1 faces of simplex j in the (k-1) order,
 *     ascending, and colptr[j] = (k+1) * j.
 *
 * Distances: integer inputs use exact integer squared distances; float32
 * inputs are ranked by the FP64 value acc = 0; for each coordinate k:
 * t = fl(x_ik - x_jk); acc = fl(acc + fl(t*t)) (round to nearest, nothing
 * fused), so equal ranks are bit-reproducible.  Every result is exactly that
 * of this definition: there is no approximation in any output.
 *
 * Errors: every entry point returns a vr_status; on failure vr_last_error()
 * gives a message for the calling thread and no output is produced.  Device
 * errors that a kernel detects (bad values, range) are returned by the call
 * that launched it, which synchronises on its stream before returning.
 * Thread safety: calls may come from several threads; results are separate
 * objects.  All device work is ordered on the stream passed in.
 */
#ifndef VR_H
#define VR_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define VR_API __attribute__((visibility("default")))
#else
#define VR_API
#endif

/* A cudaStream_t (same type); NULL is the legacy default stream. */
typedef struct CUstream_st *vr_stream_t;

typedef enum vr_status {
  VR_OK = 0,
  VR_ERR_ARG = 1,         /* bad argument or non-finite input value          */
  VR_ERR_RANGE = 2,       /* size or value beyond the documented limits      */
  VR_ERR_UNSUPPORTED = 3, /* valid request this build does not offer         */
  VR_ERR_OOM = 4,         /* device or host allocation failed                */
  VR_ERR_CUDA = 5,        /* CUDA runtime error                              */
  VR_ERR_TIMEOUT = 6,     /* result not ready within the time given          */
  VR_ERR_BUSY = 7,        /* queue full; try again later                     */
  VR_ERR_INTERNAL = 8     /* invariant violated inside the library           */
} vr_status;

typedef enum vr_dtype { VR_I8 = 1, VR_I32 = 2, VR_F32 = 3 } vr_dtype;

/* Limits.  Vertex ids travel in 13-bit fields of 64-bit sort keys. */
#define VR_MAX_POINTS 8192
#define VR_MAX_DIM_SIMPLEX 3
/* vr_build_batch and the server build up to triangles. */
#define VR_MAX_DIM_BATCH 2
/* Integer squared distances of kept edges must be below 2^38. */
#define VR_MAX_INT_D2_BITS 38
/* |float coordinate| must not exceed 2^50 (fp32 squares stay finite). */
#define VR_MAX_F32_ABS 1125899906842624.0

typedef struct vr_complex vr_complex;

/* View of one dimension of a result.  Pointers are DEVICE pointers owned by
 * the vr_complex; they stay valid until vr_complex_free. */
typedef struct vr_dim_view {
  int32_t k;              /* simplex dimension                                */
  int64_t count;          /* number of k-simplices                            */
  const int32_t *verts;   /* count x (k+1), row-major, ascending per simplex  */
  const int32_t *grade;   /* count                                            */
  const int64_t *colptr;  /* count+1 (k >= 1); NULL for k = 0                 */
  const int32_t *rowidx;  /* (k+1)*count face order indices (k >= 1); else NULL */
} vr_dim_view;

/* Build statistics of one result (host values). */
typedef struct vr_build_stats {
  int64_t kept_edges;       /* edges after the cap                            */
  int64_t triangles;        /* 2-simplices (0 when maxdim < 2)                */
  int64_t ngrades;          /* distinct grades, including grade 0             */
  int64_t near_tie_edges;   /* float input: edges re-sorted by their FP64 value */
  double max_rel_dist_err;  /* float input: max |d_approx - d_fp64| / d_fp64
                               over kept edges of the fp32 first-pass value  */
  int64_t tri_order;        /* how a single-cloud build ordered its triangles
                               (no counterpart in the paper): 0 none or not
                               reported, 1 lexicographic generation + stable
                               grade sort, 2 max-edge order with counted keys,
                               3 max-edge order in claimed key space          */
} vr_build_stats;

/* Build the filtered complex of one point cloud.
 *   points  n x d row-major elements of `dtype`, in device memory or in host
 *           memory (pageable or pinned; detected per call and copied in on
 *           `stream`).  Borrowed: it must stay valid until the call returns.
 *   n       1 .. VR_MAX_POINTS, else VR_ERR_RANGE.
 *   d       >= 1, else VR_ERR_ARG.
 *   maxdim  top simplex dimension, 0 .. 3 (3: tetrahedra, whose boundary
 *           columns list the order indices of their four triangles); above
 *           3 gives VR_ERR_UNSUPPORTED.
 *   maxrad  inclusive radius cap (keep |x_i - x_j| <= maxrad).  +INFINITY
 *           keeps every pair.  NaN or negative gives VR_ERR_ARG.  Integer
 *           inputs keep d^2 <= floor(fl(maxrad*maxrad)); float inputs keep
 *           d^2_fp64 <= fl(maxrad*maxrad).
 *   stream  all device work runs on it; the call waits for it to learn sizes.
 *   out     receives a new result, owned by the caller, released with
 *           vr_complex_free.
 * Value errors found on the device: a non-finite float coordinate gives
 * VR_ERR_ARG; |float coordinate| > VR_MAX_F32_ABS, an integer kept d^2 >=
 * 2^VR_MAX_INT_D2_BITS, or more than 2^31-1 simplices of one dimension give
 * VR_ERR_RANGE.  Device memory exhaustion gives VR_ERR_OOM. */
VR_API vr_status vr_build(const void *points, int32_t n, int32_t d, vr_dtype dtype,
                   int32_t maxdim, double maxrad, vr_stream_t stream,
                   vr_complex **out);

/* Build the filtered complex of a square symmetric matrix of edge values
 * (Sec. 3: Eirene takes a point cloud or a square symmetric matrix, typically
 * of pairwise distances, e.g. Hamming distances between sequences).
 *   D       n x n row-major, VR_I32 or VR_F32 (else VR_ERR_ARG), device or
 *           host memory (detected and copied in on `stream`).  Borrowed until
 *           the call returns.
 *   n       1 .. VR_MAX_POINTS, else VR_ERR_RANGE.
 *   maxdim  0 .. 3 as for vr_build.
 *   maxrad  inclusive cap on the VALUE (keep D[i][j] <= maxrad, no squaring);
 *           +INFINITY keeps every pair.
 * Edges come from the strict upper triangle (i < j); the diagonal is ignored
 * (vertices at grade 0).  Grades rank the values themselves: dense rank over
 * {0} U {kept values}; grade_values() returns the values.  Every entry must
 * be finite and non-negative and D[i][j] == D[j][i] exactly (-0 counts as
 * 0); otherwise VR_ERR_ARG, found on the device.  Other behaviour as vr_build
 * (ownership, sizes, errors); the build statistics' near-tie and distance
 * error fields are 0 (the keys are the exact values). */
VR_API vr_status vr_build_dmat(const void *D, int32_t n, vr_dtype dtype, int32_t maxdim,
                               double maxrad, vr_stream_t stream, vr_complex **out);

/* Persistence barcode of dimension `dim` (0 <= dim <= maxdim) of a built
 * complex, computed on the device (Algorithm 1 over F2 and the pivot/bar
 * rule of Fig. 4: a pivot (s, j) of the reduced boundary matrix is the bar
 * [grade(s), grade(j)); a positive simplex never killed is [grade, inf)).
 * The persistence pairs of every dimension are computed on the first call
 * and kept on the complex; the bars of each dimension on their first request.
 *   - Bars: first the finite ones in the order of the killing simplex, then
 *     the infinite ones in the order of the born simplex; zero-length bars
 *     are dropped; grades are the complex's integer filtration grades.
 *     `dim` = maxdim reports the top dimension's positive simplices (the
 *     complex is the maxdim skeleton, nothing kills them).
 *   - *nbars receives the count.  Synchronous on `stream` (NULL: the
 *     complex's stream).  Results of vr_build_batch views: VR_ERR_UNSUPPORTED.
 * vr_complex_bars gives device pointers (int32 birth and death grades, death
 * -1 for an infinite bar), valid until vr_complex_free; _to_host copies them
 * into caller buffers of nbars entries each.  Both need a prior
 * vr_complex_barcode of that dimension, else VR_ERR_ARG. */
VR_API vr_status vr_complex_barcode(vr_complex *c, int32_t dim, vr_stream_t stream, int64_t *nbars);
VR_API vr_status vr_complex_bars(const vr_complex *c, int32_t dim, const int32_t **birth,
                                 const int32_t **death, int64_t *nbars);
VR_API vr_status vr_complex_bars_to_host(const vr_complex *c, int32_t dim, int32_t *birth,
                                         int32_t *death);

/* Fill `view` for dimension k (0 <= k <= maxdim, else VR_ERR_ARG). */
VR_API vr_status vr_complex_dim(const vr_complex *c, int32_t k, vr_dim_view *view);

/* Device pointer to the squared distance of every grade (grade_value[0] = 0)
 * and the number of grades. */
VR_API vr_status vr_complex_grade_values(const vr_complex *c, const double **values,
                                  int64_t *ngrades);

/* Host-side sizes: counts[k] for k = 0..3 (0 above maxdim) and maxdim. */
VR_API vr_status vr_complex_counts(const vr_complex *c, int64_t counts[VR_MAX_DIM_SIMPLEX + 1],
                            int32_t *maxdim);

VR_API vr_status vr_complex_stats(const vr_complex *c, vr_build_stats *stats);

/* Waits for the build's stream and reports what the device found after the
 * build's last size read (vr_build returns before its last kernels finish):
 * VR_ERR_TIMEOUT if a bounded device wait gave up, VR_ERR_INTERNAL if an
 * internal check failed; then the arrays hold no valid result.  VR_OK
 * otherwise.  vr_complex_to_host reports the same on its own. */
VR_API vr_status vr_complex_status(const vr_complex *c);

/* Copy dimension k to host arrays sized as in vr_dim_view (any may be NULL;
 * colptr/rowidx are ignored for k = 0).  Synchronous on the build stream;
 * returns vr_complex_status's error if the device raised one late. */
VR_API vr_status vr_complex_to_host(const vr_complex *c, int32_t k, int32_t *verts,
                             int32_t *grade, int64_t *colptr, int32_t *rowidx);

/* Copy the grade values (ngrades doubles) to host memory. */
VR_API vr_status vr_complex_grade_values_to_host(const vr_complex *c, double *values);

/* Release a result (stream-ordered on the stream it was built on, which must
 * still exist).  NULL is ignored. */
VR_API void vr_complex_free(vr_complex *c);

/* ---- Batches: many clouds in one persistent launch.
 * vr_build_batch builds the complex of each of n_clouds clouds concatenated
 * row-wise in `points` (d coordinates each, one dtype; device or host
 * memory), cloud c being rows [offsets[c], offsets[c+1]) of a HOST array of
 * n_clouds+1 row offsets (offsets[0] = 0).  maxdim and maxrad are HOST arrays
 * of n_clouds values (NULL: 2 and +INFINITY for every cloud); their meaning is
 * that of vr_build.  Each cloud's result is exactly vr_build's.
 *   - One cooperative launch of co-resident CTAs takes the clouds from a work
 *     list: it sizes every cloud, lays their output slices out on the device
 *     (grid barrier, exclusive scans), and builds every cloud into its slice,
 *     one CTA per cloud with its working set in shared memory.  The launch
 *     and its copies are a CUDA graph captured once per batch class and
 *     replayed.  Output arenas are sized from earlier batches of the class;
 *     a batch that outgrows them is built again into exact arenas (the first
 *     batch of a class is sized first).  Clouds too large for one CTA take
 *     the single-cloud path.  The call synchronises on `stream` once (twice
 *     for a batch that outgrows the arenas).
 *   - Launch shape (CTAs per SM, work-list order): tuned on the first batch
 *     of each class (every candidate builds the batch; the fastest is kept
 *     for the process), or pinned by vr_batch_set_shape. */
typedef struct vr_batch_shape {
  int32_t ctas_per_sm; /* CTAs of the persistent launch per SM (<= 0: tuned) */
  int32_t order;       /* work list: 0 largest cloud first, 1 input order   */
} vr_batch_shape;
/* Pin the shape of later batches on this thread (NULL or ctas_per_sm <= 0:
 * the tuned shape; a count above what fits is clamped).  Bad order:
 * VR_ERR_ARG. */
VR_API vr_status vr_batch_set_shape(const vr_batch_shape *shape);
/* The shape the last batch on this thread used, and, when its class was
 * tuned, the candidates with their measured device times in ms (up to
 * max_cand of them; *n_cand gets the count, 0 if the class was pinned). */
VR_API vr_status vr_batch_get_shape(vr_batch_shape *used, int32_t *n_cand, vr_batch_shape *cand,
                                    double *cand_ms, int32_t max_cand);
/* Forget every tuned shape: the next batch of each class tunes again. */
VR_API vr_status vr_batch_tune_reset(void);
/* Argument errors fail the whole call; a value error (non-finite float, ...)
 * fails only its cloud, reported by vr_batch_get. */
typedef struct vr_batch vr_batch;
VR_API vr_status vr_build_batch(const void *points, const int64_t *offsets,
                                int32_t n_clouds, int32_t d, vr_dtype dtype,
                                const int32_t *maxdim, const double *maxrad,
                                vr_stream_t stream, vr_batch **out);
/* The result of one cloud: a view owned by the batch (do not pass it to
 * vr_complex_free; it lives until vr_batch_free), and the cloud's status
 * (view NULL when that status is not VR_OK). */
VR_API vr_status vr_batch_get(const vr_batch *b, int32_t cloud,
                              const vr_complex **view, vr_status *cloud_status);
VR_API vr_status vr_batch_info(const vr_batch *b, int32_t *n_clouds,
                               int64_t *total_simplices, int32_t *n_failed);
VR_API void vr_batch_free(vr_batch *b);

/* ---- Serving: continuous batching of requests.
 * A server owns worker threads and CUDA streams on one device.  Requests
 * (one cloud each) are queued by vr_serve_submit, which copies the points
 * (host or device memory) before returning.  Waiting requests of one
 * (dtype, d) class are formed into micro-batches while earlier ones run; a
 * batch's clouds are admitted by their exact output size against the memory
 * budget left by the batches in flight (the rest wait for the next batch),
 * and up to n_streams batches overlap on the device.  Clouds too large for
 * the batch kernels are built by n_large_workers threads, each on a stream
 * of its own.  Every
 * result equals vr_build's for the same request. */
typedef struct vr_server vr_server;
typedef struct vr_server_opts {
  int64_t mem_budget_bytes; /* output bytes in flight (<= 0: 8 GiB)          */
  int32_t max_queue;        /* waiting requests before VR_ERR_BUSY (<= 0: 65536) */
  int32_t n_streams;        /* batches in flight (<= 0: 3)                  */
  int32_t max_batch_clouds; /* clouds per micro-batch (<= 0: 512)           */
  int32_t device;           /* CUDA device (< 0: the current one)           */
  int32_t n_large_workers;  /* threads for clouds too large to batch (<= 0: 4) */
} vr_server_opts;
VR_API vr_status vr_server_create(const vr_server_opts *opts, vr_server **out);
/* Queue one request; *ticket identifies it.  VR_ERR_BUSY when the queue is
 * full; argument errors as in vr_build. */
VR_API vr_status vr_serve_submit(vr_server *srv, const void *points, int32_t n,
                                 int32_t d, vr_dtype dtype, int32_t maxdim,
                                 double maxrad, uint64_t *ticket);
/* Wait up to timeout_us for a ticket: VR_OK with *out (owned by the caller,
 * release with vr_complex_free), VR_ERR_TIMEOUT if not ready, or the
 * request's own error.  A ticket is delivered once. */
VR_API vr_status vr_serve_poll(vr_server *srv, uint64_t ticket,
                               int64_t timeout_us, vr_complex **out);
/* Counters of a server since its creation (a snapshot; for monitoring). */
typedef struct vr_server_stats {
  int64_t submitted;     /* requests accepted by vr_serve_submit             */
  int64_t completed;     /* results delivered with VR_OK                     */
  int64_t failed;        /* results delivered with an error                  */
  int64_t deferred;      /* clouds sent back to the queue by memory admission */
  int64_t batches;       /* micro-batches launched                           */
  int64_t large_builds;  /* requests built alone (too large for the batch kernels) */
  int64_t queued;        /* requests waiting now                             */
} vr_server_stats;
VR_API vr_status vr_server_get_stats(vr_server *srv, vr_server_stats *out);

/* Finish the work in flight and release the server (undelivered results are
 * freed). */
VR_API vr_status vr_server_destroy(vr_server *srv);

/* Barcode reduction: a working column reaching min_entries entries continues
 * as a bitset over its rows (each later addition then costs the added
 * column's length); negative: never, 0: always.  Default 4096.  Process-wide;
 * the bars are identical either way. */
VR_API vr_status vr_set_barcode_dense_min(int64_t min_entries);

/* Distance tiles: 0 = automatic (tensor-core Gram tiles for int8 or float
 * input with 16 < d <= 64 and enough 128-point tiles to fill the SMs twice,
 * CUDA cores otherwise), 1 = tensor-core tiles whenever d <= 64 (int8 or
 * float), 2 = CUDA cores always.  Process-wide; results are identical either
 * way. */
VR_API vr_status vr_set_gram_path(int32_t mode);

/* Max-edge triangle keys (the per-triangle word the generator writes in
 * output order and the final write reads; no counterpart in the paper):
 * 0 = automatic, (e << zbits) | z in 32 bits whenever the kept-edge count
 * fits the 32 - bitlen(n - 1) bits left beside the vertex, else
 * (e << 32) | z; 8 = always the 64-bit form.  Process-wide; results are
 * identical either way.  VR_ERR_ARG for any other value. */
VR_API vr_status vr_set_tri_key_width(int32_t bytes);

/* Max-edge triangle key space (no counterpart in the paper): 0 = automatic,
 * the generator runs before any triangle count and claims room for each
 * edge's third vertices (16 bits each) from striped counters in the
 * bound-sized key buffer, its exact per-edge counts then scanned into the
 * output offsets; 1 = counted, a triangle count and its scan first, then the
 * generator writes keys at the scanned offsets; 2 = claimed with tiny
 * sub-buffers (64 slots per counter), so that claims run out and the counted
 * generator takes over, for tests of that path.  Process-wide; results are
 * identical in every mode.  VR_ERR_ARG for any other value. */
VR_API vr_status vr_set_tri_claim(int32_t mode);

/* Float split of the tensor-core distance tiles (no counterpart in the
 * paper): 2 = two-way, y = hi + lo (bf16 each; products hi.hi, hi.lo,
 * lo.hi; the default), 3 = three-way, y = hi + mid + lo (six products).
 * Process-wide.  Either split decides the same pairs: pairs within the
 * tiles' error bound of the cap are decided by the canonical FP64 value. */
VR_API vr_status vr_set_gram_split(int32_t split);

/* Accuracy of the float tensor-core distance tiles (no counterpart in the
 * paper).  For device float points (n <= 8192, d <= 64) and a radius cap,
 * the tiles of the given split (0: the current one) are run with every
 * pair's canonical FP64 value beside them.  Synchronous; for tests and
 * measurement. */
typedef struct vr_gram_accuracy {
  double max_rel_d_err;  /* max |d_tc - d_fp64| / d_fp64 over the kept pairs */
  double max_norm_err;   /* max |d2_tc - d2_fp64| / (|y_i|^2 + |y_j|^2), all pairs */
  double beta;           /* the tiles' bound on the latter (their cap test uses it) */
  int64_t kept_pairs;    /* pairs with d_fp64 <= maxrad */
  int64_t band_pairs;    /* pairs within beta of the cap: decided by the FP64 value */
} vr_gram_accuracy;
VR_API vr_status vr_gram_accuracy_check(const float *points, int32_t n, int32_t d, double maxrad,
                                        int32_t split, vr_stream_t stream, vr_gram_accuracy *out);

/* Validation of the float Gram-tile error bound (no counterpart in the
 * paper): for device float points (n <= 8192, d <= 64) compute every pair's
 * tensor-core value and canonical FP64 value and return the worst
 * |d2_tc - d2_fp64| / (|y_i|^2 + |y_j|^2) observed, and the ratio beta the
 * build's cap test assumes (pairs within beta of the cap are decided with the
 * exact value).  Synchronous; for tests. */
VR_API vr_status vr_gram_error_check(const float *points, int32_t n, int32_t d,
                                     vr_stream_t stream, double *worst_ratio,
                                     double *beta_ratio);

/* Measurement support (no counterpart in the paper's API; its Sec. 4 profiles
 * with Julia's sampling profiler).  When enabled, every build records a CUDA
 * event pair around each phase on its own stream (events from a reused
 * pool); the elapsed times are added to a process-wide table of
 * (phase name, total ms, calls, kernel launches) when the table is next read
 * (vr_profile_phases / vr_profile_phase / vr_profile_reset wait for the
 * recorded events).  A profiled build adds event records, no
 * synchronisation.  vr_launch_count() is the number
 * of kernels this library has launched in the process (always counted). */
VR_API void vr_profile_enable(int32_t on);
/* Time only the phases named in `names` (comma-separated, e.g.
 * "tri_final,tri_sort.pass"); NULL or "" times every phase. */
VR_API void vr_profile_select(const char *names);
VR_API void vr_profile_reset(void);
VR_API int32_t vr_profile_phases(void);
VR_API vr_status vr_profile_phase(int32_t i, const char **name, double *total_ms,
                                  int64_t *calls, int64_t *launches);
VR_API int64_t vr_launch_count(void);

/* Sort without allocating.  The paper has no counterpart of this entry point.
 * It exists for callers that cannot allocate device memory when they need
 * the sort: a host framework whose caching allocator already owns the GPU's
 * memory, or a service that fixes its memory budget at start-up and cannot
 * afford the device-wide synchronisation cudaMalloc/cudaFree may cause.
 *
 * Stable LSD radix sort, in place, of n caller-owned 64-bit keys (DEVICE
 * memory) on bits [bit_lo, bit_lo + nbits), ascending; keys equal on those
 * bits keep their input order.  With edge keys (d2 << 26) | (i << 13) | j
 * written in (i, j) order and bits [26, 26 + bits of d2), the result is the
 * (distance, i, j) edge order vr_build produces.
 *   - n <= VR_NOALLOC_MAX_KEYS, else VR_ERR_RANGE; bit range inside [0, 64),
 *     else VR_ERR_ARG.  Asynchronous on `stream`.
 *   - Temporary storage is one fixed array in the library's device memory
 *     (VR_NOALLOC_MAX_KEYS keys, 1 MiB per GPU that loads the library, kept
 *     until the process exits).  The call allocates nothing and frees
 *     nothing.  The first call on a device looks up that array's device
 *     address (set-up once per device); make that first call before any
 *     stream capture.
 *   - Every call on a device shares the array and leaves its contents behind;
 *     nothing in it needs to start at zero.  Calls that overlap on the GPU
 *     (other streams, other threads) race on it: order them. */
#define VR_NOALLOC_MAX_KEYS 131072
VR_API vr_status vr_sort_keys_noalloc(uint64_t *keys, int64_t n, int32_t bit_lo,
                                      int32_t nbits, vr_stream_t stream);

/* The builder's multi-CTA sort, exposed as a primitive (the paper orders
 * simplices by (grade, lexicographic position); this is the stable sort that
 * realises it on packed keys).  Stable LSD radix sort, in place, of n
 * caller-owned 64-bit keys (DEVICE memory) on bits [bit_lo, bit_lo + nbits),
 * ascending; keys equal on those bits keep their input order; bits outside
 * the range never take part.
 *   - One histogram pass over all digits, then one launch per 8-bit digit;
 *     tiles of 4096 keys find their output offsets by looking back over
 *     earlier tiles' published counts (bounded waits).
 *   - Workspace (n keys + about 2 KB per tile) comes from the stream-ordered
 *     pool of the current device and is released before return.
 *   - Synchronous: returns once the sort on `stream` has finished.
 *   - n < 0, NULL keys with n > 0, or a bit range outside [0, 64): VR_ERR_ARG;
 *     n >= 2^31: VR_ERR_RANGE; no memory: VR_ERR_OOM; a bounded wait that gave
 *     up: VR_ERR_TIMEOUT (keys then unspecified). */
VR_API vr_status vr_sort_keys(uint64_t *keys, int64_t n, int32_t bit_lo, int32_t nbits,
                              vr_stream_t stream);

/* Message for the last failing call on this thread ("" if none). */
VR_API const char *vr_last_error(void);
VR_API const char *vr_status_string(vr_status s);

#ifdef __cplusplus
}
#endif
#endif /* VR_H */
