/*
 * CPU oracle for Vietoris–Rips persistence barcodes (test infrastructure).
 *
 * This is the plain, slow, single-threaded reference against which the CUDA
 * library is checked.  Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg may load it; the product path never does.  It shares no code,
 * header, table or helper with the CUDA library.
 *
 * Two methods compute the same barcode:
 *   ORACLE_DEF  explicit filtration boundary matrix of the (dim_max+1)-skeleton
 *               reduced by the standard algorithm (Algorithm 1, Section 3.1) in
 *               homology; pairs and essential indices by the pivot proposition.
 *   ORACLE_COH  cohomology with clearing (Algorithm 2 applied to coboundary
 *               matrices in increasing dimension, Sections 3.2-3.4): columns are
 *               the uncleared d-simplices in reverse filtration order, their
 *               coboundaries are generated on the fly, V is stored for death
 *               columns only and R = D V is recomputed when a column is added.
 *               Dimension 0 uses Kruskal with union-find (Section 4, "Persistence
 *               pairs").  No apparent-pair or emergent-pair shortcut is taken.
 *
 * Input: n x n row-major FP32 distance matrix; only the strict lower triangle
 * (entry [i*n + j] with i > j) is read.  threshold = +inf or NaN means "none",
 * in which case the enclosing radius min_x max_y d(x, y) is used (Section 4,
 * "Input").  Simplices with diameter <= threshold are included (Section 2).
 */
#ifndef RIPS_ORACLE_H
#define RIPS_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORACLE_DEF = 0, ORACLE_COH = 1, ORACLE_KEEP_ZERO = 0x10 /* flag: list zero-persistence pairs too */ };

typedef struct {
  int32_t dim;
  float birth;
  float death;             /* +inf for an essential class */
  int64_t birth_simplex;   /* combinatorial index of the birth simplex (dim) */
  int64_t death_simplex;   /* index of the death simplex (dim+1), -1 if essential */
} oracle_bar;

typedef struct {
  int64_t simplices;       /* d-simplices with diam <= t */
  int64_t columns;         /* columns reduced (after clearing) */
  int64_t pairs;           /* persistence pairs with birth in dim d (zero ones included) */
  int64_t zero_pairs;      /* of which persistence is zero */
  int64_t essential;       /* essential classes in dim d */
  int64_t apparent_zero;   /* ORACLE_DEF only: zero-persistence apparent pairs (d, d+1) */
  int64_t additions;       /* column additions made by the reduction */
} oracle_dim_stats;

typedef struct oracle_result oracle_result;

/* Returns 0 on success, negative on bad arguments (-1), overflow (-2), or
 * allocation failure (-3). */
int oracle_barcodes(const float* dist, int64_t n, int32_t dim_max, float threshold,
                    uint32_t p, int32_t method, oracle_result** out);
int64_t oracle_result_num_bars(const oracle_result* r);
const oracle_bar* oracle_result_bars(const oracle_result* r);
float oracle_result_threshold(const oracle_result* r);
int oracle_result_stats(const oracle_result* r, int32_t dim, oracle_dim_stats* out);
void oracle_result_free(oracle_result* r);

/* Representative cocycles (ORACLE_COH only; Sections 3.1 and 3.4): for a bar of
 * dimension d >= 1, the column V_j of the coboundary reduction whose column j
 * is the bar's birth simplex, so that R_j = delta V_j.  An essential bar's
 * cocycle has a zero coboundary; a finite bar's coboundary vanishes on every
 * (d+1)-simplex older than its death simplex and not on the death simplex.
 * Entries are (d-simplex index, coefficient in Z/p), increasing index. */
typedef struct {
  int64_t idx;
  uint32_t c;
} oracle_cocycle_entry;
/* Copies up to cap entries of bar `bar`'s cocycle; returns its length (0 for
 * H0 bars and for the ORACLE_DEF method), -1 on bad arguments. */
int64_t oracle_result_cocycle(const oracle_result* r, int64_t bar, int64_t* idx_out, uint32_t* coef_out,
                              int64_t cap);

/* Combinatorial number system (Section 2): index of the simplex with vertices
 * verts[0..d] (any order, distinct). */
int64_t oracle_simplex_index(const int64_t* verts, int32_t d);
/* Vertices of the d-simplex with the given index, in decreasing order. */
int oracle_simplex_vertices(int64_t index, int32_t d, int64_t n, int64_t* verts_out);

/* Filtration of the maxdim-skeleton of Rips_t in the lexicographically refined
 * order (diameter, then dimension, then reverse colexicographic index).
 * Writes up to cap entries and returns the total count (negative on error). */
int64_t oracle_filtration(const float* dist, int64_t n, int32_t maxdim, float threshold,
                          int32_t* out_dim, int64_t* out_index, float* out_diam, int64_t cap);

/* Apparent pairs of that filtration (Definition in Section 3.5), as filtration
 * positions (sigma, tau).  Returns the count (negative on error). */
int64_t oracle_apparent_pairs(const float* dist, int64_t n, int32_t maxdim, float threshold,
                              int64_t* out_sigma, int64_t* out_tau, int64_t cap);

/* Filtration boundary matrix of that filtration with Z/p coefficients, as
 * (row position, column position, coefficient) triples in column order.
 * Returns the number of nonzero entries (negative on error). */
int64_t oracle_boundary_matrix(const float* dist, int64_t n, int32_t maxdim, float threshold,
                               uint32_t p, int64_t* out_row, int64_t* out_col,
                               uint32_t* out_coeff, int64_t cap);

/* Number of d-simplices of Rips_t (diam <= t). */
int64_t oracle_count_simplices(const float* dist, int64_t n, int32_t d, float threshold);

/* Enclosing radius min_x max_{y != x} d(x, y) (0 for n = 1). */
float oracle_enclosing_radius(const float* dist, int64_t n);

#ifdef __cplusplus
}
#endif
#endif
