/*
 * rips.h -- C ABI of the GB300 Vietoris–Rips persistence library (librips.so).
 *
 * Problem (Bauer, "Ripser: efficient computation of Vietoris–Rips persistence
 * barcodes", arXiv 1908.02518): given a finite metric space as an n x n
 * distance matrix, compute the persistence barcodes H_0 .. H_dim_max, with
 * coefficients in the prime field Z/p, of the Vietoris–Rips filtration
 * Rips_t(X) = { nonempty S : diam S <= t }  (Section 2, "Simplicial complexes and
 * filtrations").  Bars are the intervals [f(sigma_i), f(sigma_j)) of the
 * persistence pairs of the lexicographically refined filtration with
 * f(sigma_i) < f(sigma_j), plus the essential intervals [f(sigma_i), inf)
 * (Section 2, Proposition on simplexwise refinements).  Zero-length intervals
 * are dropped.  f is the FP32 diameter, so every bar endpoint is a copy of an
 * input entry (or 0 for H_0 births).
 *
 * Simplices are named by their index in the combinatorial number system
 * (Section 2): the simplex on vertices a_0 < ... < a_d has index
 * sum_l C(a_l, l+1).
 *
 * Common conventions for every entry point:
 *  - dist: n x n row-major FP32; only the strict lower triangle dist[i*n + j]
 *    with i > j is read; the diagonal and the upper triangle are ignored.
 *    Entries must be finite and >= 0 (NaN, inf or negative -> RIPS_ERR_BAD_ARG).
 *  - threshold: simplices with diameter <= threshold are included (Section 2).
 *    +inf or NaN means "no threshold": the enclosing radius
 *    min_x max_{y != x} d(x, y) is used, beyond which the complex is a cone and
 *    the barcode cannot change (Section 4, "Input").  A negative threshold is
 *    RIPS_ERR_BAD_ARG.
 *  - p: prime, 2 <= p < 65536 (Section 4, "Coefficients"); otherwise
 *    RIPS_ERR_BAD_MODULUS.
 *  - dim_max >= 0 and n >= 1, else RIPS_ERR_BAD_ARG.  n is at most 46340 (the
 *    n x n rank matrix and the neighbour lists use 32-bit offsets); dim_max is at
 *    most 7.  C(n, dim_max + 2) must be below 2^63 and
 *    every filtration key (diameter rank bits + simplex index bits) must fit in
 *    64 bits, else RIPS_ERR_OVERFLOW (the paper uses 64-bit indices, Section 4).
 *  - Every function returns RIPS_OK (0) on success or a negative status and
 *    never throws.  Calls on the same device are serialised internally; work is
 *    issued on the given CUDA stream (NULL = legacy default stream).
 *  - All computation runs on the current CUDA device.  Result objects are owned
 *    by the library until rips_result_free.
 */
#ifndef RIPS_H
#define RIPS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RIPS_API __attribute__((visibility("default")))

enum rips_status {
  RIPS_OK = 0,
  RIPS_ERR_BAD_ARG = -1,        /* invalid size, pointer, distance or threshold */
  RIPS_ERR_BAD_MODULUS = -2,    /* p not a prime in [2, 65536) */
  RIPS_ERR_OVERFLOW = -3,       /* simplex index or filtration key exceeds 64 bits */
  RIPS_ERR_OOM = -4,            /* device or host allocation failed */
  RIPS_ERR_CUDA = -5,           /* a CUDA runtime call failed */
  RIPS_ERR_DEVICE_TIMEOUT = -6, /* a bounded device loop hit its iteration limit */
  RIPS_ERR_INTERNAL = -7        /* an internal consistency check failed */
};

/* One bar of the barcode.  death = +inf for an essential class. */
typedef struct rips_bar {
  int32_t dim;            /* homology dimension of the bar */
  float birth;            /* diameter of the birth simplex (0 in H_0) */
  float death;            /* diameter of the death simplex, +inf if essential */
  int32_t cloud;          /* cloud number in a batched call, 0 otherwise */
  uint64_t birth_simplex; /* index of the birth simplex (a dim-simplex) */
  uint64_t death_simplex; /* index of the death simplex (a (dim+1)-simplex), UINT64_MAX if essential */
} rips_bar_t;

/* Per-dimension counters, the categories of Table 2 of the paper. */
typedef struct rips_stats {
  int64_t simplices;        /* d-simplices with diameter <= threshold */
  int64_t apparent_cofacet; /* of which in a zero apparent pair (sigma, tau) as sigma */
  int64_t apparent_facet;   /* of which in a zero apparent pair (rho, sigma) as sigma */
  int64_t cleared;          /* of which pivots of the (d-1)-reduction found in its table */
  int64_t columns;          /* columns reduced: the rest */
  int64_t emergent;         /* columns whose first pivot was never contested */
  int64_t pairs;            /* persistence pairs (d, d+1) found by the reduction */
  int64_t zero_pairs;       /* of which zero persistence */
  int64_t essential;        /* essential classes in dimension d */
  int64_t reduction_steps;  /* column additions performed */
  int64_t rounds;           /* claim/reduce rounds of the reduction */
  int64_t longest_chain;    /* most additions made by one column in one round */
  int64_t compacted_entries;/* working-column entries merged by run compactions */
  int64_t added_entries;    /* entries of the columns added to working columns, summed */
} rips_stats_t;

typedef struct rips_result rips_result_t;

/*
 * rips_barcodes -- barcode of one distance matrix held in HOST memory.
 * Defined by: Section 2 (the Rips filtration of a finite metric space, its
 * lexicographic refinement, and the barcode of a filtration read off the
 * persistence pairs of a reduced boundary matrix), Section 4 "Input" (distance
 * matrix, threshold, enclosing radius) and "Coefficients" (Z/p).
 * dist: n x n FP32, HOST, read only, owned by the caller.  The matrix is copied
 * to the device on the legacy default stream; the bars are copied back and the
 * call returns when they are on the host.
 * out: receives a new result object owned by the caller until
 * rips_result_free (NULL on failure).
 */
RIPS_API int rips_barcodes(const float* dist, int64_t n, int32_t dim_max, float threshold,
                           uint32_t p, rips_result_t** out);

/* rips_barcodes_device -- the same problem (Section 2; Section 4 "Input",
 * "Coefficients") for a distance matrix already in DEVICE memory (read only,
 * owned by the caller), with the work issued on `cuda_stream` (a cudaStream_t,
 * or NULL); returns when the bars are on the host. */
RIPS_API int rips_barcodes_device(const float* d_dist, int64_t n, int32_t dim_max, float threshold,
                                  uint32_t p, void* cuda_stream, rips_result_t** out);

/*
 * rips_barcodes_packed -- the same problem for a distance matrix given as its
 * strict lower or upper triangle, packed row by row (the triangular input
 * formats of Section 4, "Input"): layout RIPS_LOWER_TRIANGLE holds d(1,0),
 * d(2,0), d(2,1), d(3,0), ...; RIPS_UPPER_TRIANGLE holds d(0,1), d(0,2), ...,
 * d(0,n-1), d(1,2), ....  d_packed: n(n-1)/2 FP32 entries in DEVICE memory
 * (read only, owned by the caller; may be NULL when n = 1); the matrix is
 * expanded into library-owned device memory on cuda_stream.  Entry rules,
 * threshold, p, statuses and the result as for rips_barcodes; an unknown
 * layout is RIPS_ERR_BAD_ARG.
 */
enum rips_layout { RIPS_LOWER_TRIANGLE = 0, RIPS_UPPER_TRIANGLE = 1 };
RIPS_API int rips_barcodes_packed(const float* d_packed, int64_t n, int32_t layout, int32_t dim_max,
                                  float threshold, uint32_t p, void* cuda_stream, rips_result_t** out);

/*
 * rips_barcodes_sparse -- the barcode of a sparse distance matrix (Section 4,
 * "Input": a sparse matrix, where a missing entry is an infinite distance),
 * without any n x n array: memory grows with the number of edges, not with n^2.
 * d_i, d_j, d_len: m entries in DEVICE memory (read only, owned by the caller),
 * entry e the edge {d_i[e], d_j[e]} of length d_len[e]; 0 <= i, j < n, i != j,
 * each unordered pair at most once, lengths finite and >= 0 (else
 * RIPS_ERR_BAD_ARG).  Entries longer than the threshold are left out; with no
 * threshold (+inf or NaN) every entry is kept (the enclosing radius does not
 * apply).  n at most 92681.  Rank lookups search the sorted neighbour lists
 * instead of reading a rank matrix.  Every filtration key must still fit in 64
 * bits (diameter rank bits + simplex index bits; RIPS_ERR_OVERFLOW otherwise),
 * which bounds n at a given density and dimension.  Statuses and the result as
 * for rips_barcodes_device.
 */
RIPS_API int rips_barcodes_sparse(const int32_t* d_i, const int32_t* d_j, const float* d_len, int64_t m, int64_t n,
                                  int32_t dim_max, float threshold, uint32_t p, void* cuda_stream,
                                  rips_result_t** out);

/*
 * rips_barcodes_sparse_points -- the same for a point cloud (n points of k FP32
 * coordinates, DEVICE, row-major) and a finite threshold: the pairs within the
 * threshold are found on the device tile by tile (distances by the rule of
 * rips_distance_matrix_device) and only they are kept.  An infinite or NaN
 * threshold is RIPS_ERR_BAD_ARG (the cloud would be dense).  The result feeds
 * rips_barcodes_backward with the same points.
 */
RIPS_API int rips_barcodes_sparse_points(const float* d_points, int64_t n, int32_t k, int32_t dim_max,
                                         float threshold, uint32_t p, void* cuda_stream, rips_result_t** out);

/*
 * rips_distance_matrix_device -- the finite metric space of a point cloud
 * (Section 4 "Input" accepts point clouds as well as distance matrices):
 * Euclidean distances of n points with k FP32
 * coordinates each (row-major, DEVICE memory) into d_dist (n x n, DEVICE,
 * written in full).  Each entry is computed in float64 from the FP32
 * coordinates (squared differences summed in coordinate order, each operation
 * separately rounded, then a correctly rounded square root) and rounded to FP32.
 */
RIPS_API int rips_distance_matrix_device(const float* d_points, int64_t n, int32_t k, float* d_dist,
                                         void* cuda_stream);

/*
 * rips_barcodes_batched -- barcodes (Section 2) of `batch` independent point
 * clouds (Section 4 "Input") in one pass.  d_points: all clouds' FP32 coordinates concatenated (DEVICE, row-major,
 * k per point); d_offsets: batch+1 point offsets (HOST).  The distances of every
 * cloud are computed on the device by the rule of rips_distance_matrix_device.
 * The bars of cloud c carry cloud = c.  Status as for rips_barcodes; every
 * cloud must satisfy its size rules, and with batch > 1 every cloud has at
 * most 12800 points.
 */
RIPS_API int rips_barcodes_batched(const float* d_points, const int64_t* offsets, int32_t batch,
                                   int32_t k, int32_t dim_max, float threshold, uint32_t p,
                                   void* cuda_stream, rips_result_t** out);

/*
 * rips_barcodes_batched_dists -- barcodes (Section 2) of `batch` independent
 * finite metric spaces given as distance matrices (Section 4 "Input"), in one
 * pass.  d_dists: HOST array of `batch` DEVICE pointers, matrix c being
 * ns[c] x ns[c] FP32 row-major with the conventions of rips_barcodes (strict
 * lower triangle read, not modified, owned by the caller); ns: HOST array of
 * the sizes.  Threshold, p and dim_max apply to every cloud.  The matrices are
 * gathered into library-owned device memory on cuda_stream, then processed
 * together as in rips_barcodes_batched; the bars of cloud c carry cloud = c.
 * Status as for rips_barcodes_batched.
 */
RIPS_API int rips_barcodes_batched_dists(const float* const* d_dists, const int64_t* ns, int32_t batch,
                                         int32_t dim_max, float threshold, uint32_t p, void* cuda_stream,
                                         rips_result_t** out);

/*
 * rips_barcodes_backward -- gradient of a loss L(bars) with respect to the
 * point coordinates of the clouds of a result computed by
 * rips_barcodes_batched (or by rips_barcodes_device on distances produced by
 * rips_distance_matrix_device, with batch = 1).  d_points and k are the
 * coordinates the distances were computed from (DEVICE, as for the forward).
 * grad_birth, grad_death: dL/dbirth and dL/ddeath per bar, in the order of
 * rips_result_bars over all clouds (DEVICE, FP32; essential deaths ignored).
 * Each finite bar endpoint is the length of one critical edge, the longest
 * edge of its simplex (ties: the edge with the smallest index).  The gradient
 * is scattered into d_grad_points (same layout as d_points, DEVICE, FP32,
 * accumulated: the caller zeroes it) through d|x_a - x_b| / dx_a.
 * If d_grad_dist is not NULL it receives dL/d dist[i][j] (i > j) for each cloud's
 * n x n block laid out back to back (DEVICE, FP32, accumulated).
 */
RIPS_API int rips_barcodes_backward(const rips_result_t* res, const float* d_points, int32_t k,
                                    const float* grad_birth, const float* grad_death,
                                    float* d_grad_points, float* d_grad_dist, void* cuda_stream);

/*
 * rips_barcodes_backward_dist -- gradient of a loss L(bars) with respect to
 * the distance matrices themselves, for callers that hold only the matrices.
 * Works for a result of any forward entry point.  The paper has no backward
 * pass; it rests on Section 2: a finite bar endpoint is the diameter of its
 * birth or death simplex, i.e. the entry of D at one critical edge -- the
 * longest edge of that simplex on the FP32 matrix the forward read, ties
 * broken towards the smallest edge index (the edge that enters the refined
 * filtration last).  d_dists: HOST array of one DEVICE pointer per cloud of the
 * result (the matrices the forward read, n_c x n_c FP32, not modified);
 * grad_birth, grad_death: DEVICE FP32, one entry per bar in the order of
 * rips_result_bars over all clouds (NULL: zero; essential deaths ignored);
 * d_grad_dists: HOST array of one DEVICE pointer per cloud, an n_c x n_c FP32
 * matrix into whose strict lower triangle dL/dD[a][b] (a > b) is accumulated
 * (the caller zeroes it).  Returns when the work on cuda_stream is done.
 */
RIPS_API int rips_barcodes_backward_dist(const rips_result_t* res, const float* const* d_dists,
                                         const float* grad_birth, const float* grad_death, float* const* d_grad_dists,
                                         void* cuda_stream);

/*
 * rips_h0_barcode_noalloc -- the dimension-0 barcode of one distance matrix
 * without allocating any memory.  The paper has no counterpart: it exists for
 * callers that cannot allocate device memory while they run (a serving process
 * whose memory pool already owns the whole device, a real-time loop that must
 * not wait on cudaMalloc / cudaFree, which may synchronise the device).  All
 * intermediate data lives in a fixed file-scope device array (about 3.3 MB,
 * held by every GPU that loads the library until the process exits), so n is
 * at most RIPS_NOALLOC_MAX_N; larger n returns RIPS_ERR_BAD_ARG.
 * d_dist: n x n FP32 (DEVICE, strict lower triangle read, as for
 * rips_barcodes; a NaN, infinite or negative entry returns RIPS_ERR_BAD_ARG);
 * threshold as for rips_barcodes.  d_bars: DEVICE room for n bars, receives
 * the H0 bars (forest edges in filtration order, then the essential classes);
 * d_nbars: DEVICE uint32, the bar count.  Work is issued on cuda_stream and the
 * call waits for that stream before it returns.  Every call reuses the same
 * array (which keeps the last call's contents) and resets what must start at
 * zero: calls that overlap on the GPU (other streams or threads) race and must
 * not be made.  The first call on a device looks the array's address up with
 * that device current and keeps it; make that first call before any stream
 * capture begins, and make no call after cudaDeviceReset.  Status: as for
 * rips_barcodes (RIPS_ERR_DEVICE_TIMEOUT for a bounded wait that ran out,
 * RIPS_ERR_OOM for a capacity limit, RIPS_ERR_INTERNAL otherwise).
 */
#define RIPS_NOALLOC_MAX_N 512
RIPS_API int rips_h0_barcode_noalloc(const float* d_dist, int64_t n, float threshold, rips_bar_t* d_bars,
                                     uint32_t* d_nbars, void* cuda_stream);

/* Result accessors: the barcode as a list of intervals (Section 2, the
 * Proposition on simplexwise refinements; zero-length intervals dropped).
 * Number of bars of cloud `cloud` in dimension `dim` (dim = -1: all dims);
 * cloud = -1: all clouds.  Negative status on a bad argument. */
RIPS_API int64_t rips_result_num_bars(const rips_result_t* res, int32_t cloud, int32_t dim);

/* Host pointer to those bars (owned by the result), ordered by cloud, then
 * dimension, then birth, death and birth simplex index; NULL if none. */
RIPS_API const rips_bar_t* rips_result_bars(const rips_result_t* res, int32_t cloud, int32_t dim);

/* Number of clouds, dim_max and the effective threshold of cloud `cloud`. */
RIPS_API int32_t rips_result_num_clouds(const rips_result_t* res);
RIPS_API int32_t rips_result_dim_max(const rips_result_t* res);
RIPS_API float rips_result_threshold(const rips_result_t* res, int32_t cloud);

/* Statistics of cloud `cloud` in dimension `dim`: the pair categories of
 * Table 2 (apparent, cleared, emergent, columns reduced) and reduction
 * counters. */
RIPS_API int rips_result_stats(const rips_result_t* res, int32_t cloud, int32_t dim,
                               rips_stats_t* out);

/* Device-side timing of the last call's phases in milliseconds (CUDA events on
 * the call's stream), for profiling: index 0 = prologue + H_0, then one entry
 * per dimension 1..dim_max.  Returns the number of entries written. */
RIPS_API int32_t rips_result_phase_ms(const rips_result_t* res, float* out, int32_t cap);

/* Kernel classes for rips_result_kernel_ms. */
enum rips_kernel_class {
  RIPS_K_PROLOGUE = 0,  /* validation, radius, edge keys, ranks, rank matrix, neighbours */
  RIPS_K_EDGE_SORT = 1, /* radix sort of the edges into filtration order */
  RIPS_K_H0 = 2,        /* spanning forest and elder rule */
  RIPS_K_ENUMERATE = 3, /* d-simplex enumeration */
  RIPS_K_APPARENT = 4,  /* zero-apparent-pair / clearing test and compaction */
  RIPS_K_COL_SORT = 5,  /* radix sort of the columns into processing order */
  RIPS_K_PIVOT_INIT = 6,/* first pivots (emergent shortcut) */
  RIPS_K_REDUCE = 7,    /* claim and reduce rounds */
  RIPS_K_READOUT = 8,   /* bars and statistics */
  RIPS_KERNEL_CLASSES = 9
};

/* Profiling aid (no counterpart in the paper): when enabled, every later call
 * records CUDA events on its stream around the launches of each kernel class.
 * Returns the previous setting. */
RIPS_API int rips_set_kernel_timing(int enable);

/* Total device time (ms) and number of timed regions of kernel class `cls` in
 * the call that produced `res` (zero when timing was off). */
RIPS_API int rips_result_kernel_ms(const rips_result_t* res, int32_t cls, float* ms, int64_t* regions);

RIPS_API void rips_result_free(rips_result_t* res);

/* Human-readable name of a status code (static string). */
RIPS_API const char* rips_status_string(int status);

/* Number of kernel launches issued by this library on the calling thread
 * since the last reset (a profiling aid). */
RIPS_API int64_t rips_kernel_launch_count(int reset);

/* Launch and scheduling parameters of one dimension's kernels.  The paper has
 * no counterpart: these are implementation choices, and no setting changes any
 * result (bars and statistics other than timings are identical).  They are
 * looked up per dimension d >= 1 and per the largest cloud size n of a call. */
typedef struct rips_tuning {
  int32_t warp_chain_limit;     /* additions one warp makes on a column before a block takes it over (>= 1) */
  int32_t warp_merge_max;       /* largest merge of working-column runs one warp makes (>= 1) */
  int32_t reduce_blocks_per_sm; /* blocks per SM of the reduction (0: as many as fit) */
  int32_t scan_blocks_per_sm;   /* blocks per SM of the enumeration and test kernels (1..64) */
} rips_tuning_t;

/* Use `t` for dimension `dim` (1..7) when the largest cloud of a call has
 * n_lo <= n <= n_hi points.  Entries added later take precedence.  The table
 * is process-wide and guarded by a lock.  RIPS_ERR_BAD_ARG on out-of-range
 * fields. */
RIPS_API int rips_set_tuning(int32_t dim, int64_t n_lo, int64_t n_hi, const rips_tuning_t* t);

/* The parameters a call with largest cloud size n would use in dimension dim
 * (the built-in defaults when no entry matches). */
RIPS_API int rips_get_tuning(int32_t dim, int64_t n, rips_tuning_t* out);

/* Forget every entry (back to the built-in defaults). */
RIPS_API void rips_clear_tuning(void);

/* Bounds of the library's waits and first buffer sizes.  The paper has no
 * counterpart.  Every device wait is bounded: a block waiting at the
 * reduction's grid barrier gives up (and the call returns
 * RIPS_ERR_DEVICE_TIMEOUT) when no block has made progress for barrier_wait_ns,
 * and one column's chain of additions gives up after chain_ns.  Setting them
 * small, or the arena and pivot table tiny, injects the failures the library
 * must report cleanly (a timeout status, an arena that is grown and the
 * dimension redone, RIPS_ERR_OOM for a full table) without faulting or hanging
 * the GPU; the defaults (all fields 0) never trigger them in normal use. */
typedef struct rips_limits {
  uint64_t barrier_wait_ns; /* 0: 30 s */
  uint64_t chain_ns;        /* 0: 600 s */
  uint64_t arena_entries;   /* first reduction-arena size in entries (0: from the column count) */
  uint64_t table_slots;     /* pivot-table capacity, a power of two (0: 2 x columns, rounded up) */
} rips_limits_t;

/* Process-wide; RIPS_ERR_BAD_ARG if table_slots is not 0 or a power of two. */
RIPS_API int rips_set_limits(const rips_limits_t* limits);
RIPS_API int rips_get_limits(rips_limits_t* out);

/* Ablation switches (the experiment of Table 3 of the paper): with
 * RIPS_OPT_NO_APPARENT the zero-persistence apparent pairs of Section 3.5 are
 * not skipped -- every simplex that is not cleared becomes a column and every
 * pivot is owned through the pivot table; with RIPS_OPT_NO_EMERGENT the first
 * pivot of a column is found by scanning its whole coboundary instead of
 * stopping at the first cofacet of the column's own diameter (the emergent-pair
 * shortcut of Section 3.5).  Neither switch changes any bar; the statistics of
 * Table 2 (rips_result_stats) show what each shortcut saved.  The library keeps
 * the coboundary implicit and the reduced columns R_j in every setting (it does
 * not store V, so R cannot be discarded).  Process-wide, later calls only;
 * batch plans ignore the switches.  RIPS_ERR_BAD_ARG on an unknown bit. */
enum rips_option { RIPS_OPT_NO_APPARENT = 1, RIPS_OPT_NO_EMERGENT = 2 };
RIPS_API int rips_set_options(uint32_t flags);
RIPS_API uint32_t rips_get_options(void);

/* Batch plans (the batched problem of rips_barcodes_batched for barcodes H0 and
 * H1, with every launch fixed in advance).  A plan is made once for a list of
 * cloud sizes (`offsets`, batch + 1 point offsets as in rips_barcodes_batched),
 * k coordinates, a threshold and p; it allocates every buffer for the worst
 * case (all C(n, 2) edges of every cloud), at most 12800 points per cloud.
 * rips_batch_plan_run enqueues the whole forward for new point coordinates
 * (same sizes) on the caller's stream without any host synchronisation or
 * allocation, so it may be captured into a CUDA graph and replayed;
 * rips_batch_plan_result waits for the stream and returns the last run's bars
 * and statistics as a result (for the accessors and rips_barcodes_backward).
 * The reduction's arena is fixed too: arena_entries entries of 12 bytes (0:
 * 384 per edge, within 40 % of the free device memory; the arena keeps every
 * intermediate run of a reduction, 150 to 250 entries per edge on the 256-cloud
 * mix of circles, tori and cubes); a run that needs more
 * reports RIPS_ERR_OOM from rips_batch_plan_result.  A plan is used by one
 * stream at a time. */
typedef struct rips_batch_plan rips_batch_plan_t;
RIPS_API int rips_batch_plan_create(const int64_t* offsets, int32_t batch, int32_t k, float threshold, uint32_t p,
                                    int64_t arena_entries, rips_batch_plan_t** out);
RIPS_API int rips_batch_plan_run(rips_batch_plan_t* plan, const float* d_points, void* cuda_stream);
RIPS_API int rips_batch_plan_result(rips_batch_plan_t* plan, void* cuda_stream, rips_result_t** out);
RIPS_API void rips_batch_plan_free(rips_batch_plan_t* plan);

#ifdef __cplusplus
}
#endif
#endif /* RIPS_H */
