// Internal declarations shared by the CUDA translation units of librips.
//
// Layout conventions used throughout:
//  * R (rank matrix): n x n uint32, full and symmetric.  R[i*n+j] is the rank of
//    the edge length d(i,j) among the distinct edge lengths <= threshold, in
//    increasing order, or RANK_INF if d(i,j) > threshold or i == j.  Every
//    simplex diameter is an edge length, so comparing ranks compares diameters
//    exactly (Section 2: the Rips filtration is the sublevel filtration of the
//    diameter), and all later kernels work on integers only.
//  * Binomial table: uint64, k-major: binom[k*(n+1) + i] = C(i, k) for
//    0 <= k <= kmax, 0 <= i <= n (saturating at UINT64_MAX).
//  * A d-simplex is identified by its index in the combinatorial number system
//    (Section 2) and carries the rank of its diameter.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/rips.h"

namespace rips {

constexpr uint32_t RANK_INF = 0xFFFFFFFFu;
constexpr uint64_t IDX_NONE = ~0ull;
constexpr int MAX_DIM = 8;  // largest simplex dimension handled (vertices per simplex <= 9)

// device error flag bits (written with atomicOr into Workspace::d_err)
enum : uint32_t {
  ERRF_TIMEOUT = 1u,       // a bounded loop hit its limit
  ERRF_TABLE_FULL = 2u,    // a hash table is full
  ERRF_INTERNAL = 4u,      // consistency check failed
  ERRF_ARENA = 8u,         // V arena exhausted (retry after growth)
  ERRF_BAD_INPUT = 16u,    // NaN / negative / infinite distance
  ERRF_OUT_OVERFLOW = 32u  // an output list exceeded its capacity (retry after growth)
};

// ------------------------------------------------------------------ kernel launch accounting
void note_launch();

// ------------------------------------------------------------------ device helpers
__device__ __forceinline__ uint64_t binom(const uint64_t* __restrict__ tab, int stride, int i, int k) {
  return tab[(size_t)k * stride + i];
}

// Largest v in [lo, hi] with C(v, k) <= N (the Lemma of Section 4,
// "Vertices and simplices"), by binary search.  Requires C(lo, k) <= N.
__device__ __forceinline__ int max_vertex(const uint64_t* __restrict__ tab, int stride, int lo, int hi,
                                          int k, uint64_t N) {
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (binom(tab, stride, mid, k) <= N) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Vertices of the d-simplex with index N, written in decreasing order
// v[0] > v[1] > ... > v[d].
__device__ __forceinline__ void decode_simplex(const uint64_t* __restrict__ tab, int stride, int n,
                                               uint64_t N, int d, int* v) {
  int hi = n - 1;
  for (int k = d + 1; k >= 1; --k) {
    int x = max_vertex(tab, stride, k - 1, hi, k, N);
    v[d + 1 - k] = x;
    N -= binom(tab, stride, x, k);
    hi = x - 1;
  }
}

// Z/p helpers (p < 2^16 so products fit in 32 bits)
__device__ __forceinline__ uint32_t mod_inv(uint32_t a, uint32_t p) {
  // extended Euclid on (a, p), p prime, a != 0
  int32_t t = 0, nt = 1;
  int32_t r = (int32_t)p, nr = (int32_t)(a % p);
  while (nr != 0) {
    int32_t q = r / nr;
    int32_t tmp = t - q * nt;
    t = nt;
    nt = tmp;
    tmp = r - q * nr;
    r = nr;
    nr = tmp;
  }
  if (t < 0) t += (int32_t)p;
  return (uint32_t)t;
}

__device__ __forceinline__ void set_error(uint32_t* err, uint32_t bit) { atomicOr(err, bit); }

__host__ __device__ __forceinline__ int bit_width64(uint64_t x) {
  int b = 0;
  while (x) {
    ++b;
    x >>= 1;
  }
  return b;
}

// ------------------------------------------------------------------ host-side launchers
// (defined in the .cu files; every launcher returns a cudaError_t of the launch)

// ------------------------------------------------------------------ clouds
// Every call works on a batch of independent clouds (one cloud for the
// single-matrix entry points).  Cloud c owns n_c vertices; its n_c x n_c
// distance and rank matrices start at element roff; its vertices are the global
// rows voff .. voff + n_c - 1 of the neighbour-list CSR; its edges are the
// positions eoff .. eoff + m_c - 1 of the sorted edge list.  A simplex is named
// by (cloud << shift) | local combinatorial index.
struct CloudInfo {
  int n;
  uint32_t voff;
  uint64_t roff;
  uint32_t eoff;
  uint32_t m;
  float t_eff;
  uint32_t pad;
};

// rips_prologue.cu (all kernels run over every cloud of the batch)
cudaError_t launch_binomial_table(uint64_t* tab, int n, int kmax, cudaStream_t s);
cudaError_t launch_cloud_vertices(const CloudInfo* clouds, int nclouds, uint32_t* vcloud, cudaStream_t s);
cudaError_t launch_validate_rowmax(const float* D, const CloudInfo* clouds, const uint32_t* tile_off, int nclouds,
                                   uint32_t tiles, uint32_t* rowmax_bits, uint32_t* err, cudaStream_t s);
cudaError_t launch_threshold(const uint32_t* rowmax_bits, CloudInfo* clouds, int nclouds, float threshold,
                             cudaStream_t s);
cudaError_t launch_edge_keys(const float* D, const CloudInfo* clouds, const uint32_t* vcloud, uint32_t nverts,
                             int edge_bits, uint64_t* keys, uint32_t* count, uint32_t* cloud_count, uint32_t cap,
                             cudaStream_t s);
cudaError_t launch_assign_ranks(const uint64_t* sorted_keys, uint32_t num_edges, int edge_bits, uint32_t* flags,
                                uint32_t* scan_tmp, uint32_t* edge_rank, float* rank_value, uint32_t* num_ranks,
                                cudaStream_t s);
cudaError_t launch_fill_rank_matrix(const uint64_t* sorted_keys, const uint32_t* edge_rank, uint32_t num_edges,
                                    int edge_bits, const CloudInfo* clouds, uint32_t* R, cudaStream_t s);
cudaError_t launch_neighbor_counts(const uint32_t* R, const CloudInfo* clouds, const uint32_t* vcloud,
                                   uint32_t nverts, uint32_t* deg, uint32_t* max_deg, cudaStream_t s);
cudaError_t launch_neighbor_fill(const uint32_t* R, const CloudInfo* clouds, const uint32_t* vcloud, uint32_t nverts,
                                 const uint32_t* off, uint32_t* nbr, cudaStream_t s);
cudaError_t launch_distance_matrix(const float* pts, int n, int k, float* D, cudaStream_t s);
// sparse inputs (one cloud): edge keys of a (i, j, length) list or of a point
// cloud's pairs within t, appended at *count (capacity cap; the count may
// exceed cap, nothing past it is written); neighbour lists with ranks
cudaError_t launch_coo_edge_keys(const int32_t* ei, const int32_t* ej, const float* len, uint64_t m, int n, float t,
                                 int eb, uint64_t* keys, uint32_t* count, uint32_t cap, uint32_t* err, cudaStream_t s);
cudaError_t launch_point_edges(const float* pts, int n, int k, float t, int eb, uint64_t* keys, uint32_t* count,
                               uint32_t cap, cudaStream_t s);
cudaError_t launch_sparse_degrees(const uint64_t* keys, uint32_t m, int eb, uint32_t* deg, cudaStream_t s);
cudaError_t launch_sparse_fill(const uint64_t* keys, const uint32_t* erank, uint32_t m, int eb, const uint32_t* off,
                               uint32_t* cursor, uint64_t* nkey, uint32_t* nval, cudaStream_t s);
cudaError_t launch_sparse_unpack(const uint64_t* nkey, const uint32_t* nval, uint32_t q, uint32_t* nbr,
                                 uint32_t* nrank, cudaStream_t s);
cudaError_t launch_max(const uint32_t* x, uint32_t n, uint32_t* out, cudaStream_t s);
// packed strict triangle (lower: row by row from row 1; upper: row by row to row n-2) -> strict lower triangle of D
cudaError_t launch_unpack_triangle(const float* packed, int n, int upper, float* D, cudaStream_t s);
cudaError_t launch_pad_past_count(uint64_t* keys, const uint32_t* count, uint64_t cap, cudaStream_t s);
cudaError_t launch_cloud_edge_offsets(CloudInfo* clouds, const uint32_t* ccounts, int nclouds, cudaStream_t s);
cudaError_t launch_distance_matrices(const float* pts, int k, const CloudInfo* clouds, const uint32_t* tile_off,
                                     int nclouds, uint32_t tiles, float* D, cudaStream_t s);

// rips_scan.cu: exclusive scan of uint32 (in place allowed); returns total in *d_total if non-null
size_t scan_temp_bytes(uint32_t n);
cudaError_t launch_exclusive_scan(const uint32_t* in, uint32_t* out, uint32_t n, void* tmp,
                                  uint32_t* d_total, cudaStream_t s);

// rips_sort.cu: LSD radix sort of 64-bit keys (optionally with uint32 values),
// over bits [0, key_bits).  Result in *out (may alias one of the two buffers).
size_t sort_temp_bytes(uint32_t n);
cudaError_t radix_sort_u64(uint64_t* keys, uint64_t* keys_alt, uint32_t* vals, uint32_t* vals_alt,
                           uint32_t n, int key_bits, void* tmp, size_t tmp_bytes, bool* result_in_alt,
                           cudaStream_t s);

// One dimension of the reduction (rips_dim.cu)
struct DimArgs {
  int d;                           // columns are d-simplices
  int nclouds;
  const CloudInfo* clouds;
  const uint32_t* R;               // rank matrices of all clouds (null for a sparse input)
  const uint32_t* nbr_off;         // neighbour-list CSR over all clouds' vertices (global rows)
  const uint32_t* nbr;             // local vertex ids, decreasing within a row
  const uint32_t* nrank;           // sparse input: rank of the edge to each nbr entry (else null)
  const uint64_t* binom;           // binomial table for n_max, stride bn + 1
  int bn;
  int kmax;                        // rows 0..kmax of the table are staged
  int smem_binom;                  // stage the table in shared memory
  uint32_t p;
  int row_bits;                    // bits of a local (d+1)-simplex index
  int col_bits;                    // bits of a local d-simplex index
  int rank_bits;                   // bits of a diameter rank
  uint32_t rank_max;               // largest diameter rank
  uint32_t* err;
  // zero-persistence apparent pairs (sigma, tau) with sigma a d-simplex, written
  // by the test kernel: a hash table of (key, value) pairs, slot h at amap[2h]
  // and amap[2h + 1] (one 16-byte load reads both), amap_mask + 1 slots; key
  // (cloud << row_bits) | idx(tau), value (ref(sigma) << 4) | position of the
  // vertex tau has beyond sigma, where ref(sigma) is sigma's vertices packed
  // vbits apiece (vertex l at bit l * vbits) when vbits > 0, else its index;
  // null when col_bits > 60 (the index does not fit beside the position)
  uint64_t* amap;
  uint64_t amap_mask;
  int vbits;
  // the same map of dimension d - 1 (keys (cloud << col_bits) | idx(sigma)), or null
  const uint64_t* pmap;
  uint64_t pmap_mask;
  // launch and scheduling parameters (rips_tuning_t)
  uint32_t chain_limit;            // additions a warp makes on one column before a block takes it
  uint32_t merge_max;              // largest run merge one warp makes
  int reduce_blocks_per_sm;        // 0: occupancy limit
  int scan_blocks_per_sm;
  uint32_t opts;                   // RIPS_OPT_* switches (rips_set_options)
};

struct HelpBoard;  // rips_dim.cu
// bytes of the reduction's control block: counters and cursors in the first
// 256, the help board after them (zeroed together before every launch)
constexpr size_t LISTS_BYTES = 16384;

// Reduction state (device pointers) shared by the reduction kernels
struct RedState {
  // columns in processing order
  const uint64_t* col_keys;   // (cloud << (rank_bits + col_bits)) | ((rank_max - rank) << col_bits) | idx
  uint32_t ncols;
  // per-column state
  uint64_t* piv_key;          // row key of the pivot, IDX_NONE for a zero column
  uint32_t* piv_coef;
  uint8_t* reduced;           // 1 once the column has been added to
  // materialised working columns R_j (sorted row keys, nonzero coefficients)
  uint64_t* r_key;
  uint32_t* r_coef;
  unsigned long long* r_off;  // per column; r_len == 0: not materialised
  uint32_t* r_len;
  unsigned long long* r_top;
  unsigned long long r_cap;
  // power of two >= 1 + the largest vertex degree: room for one generated coboundary
  uint32_t scr_slice;
  // pivot table
  uint64_t* t_keys;
  uint32_t* t_vals;
  uint64_t t_mask;
  // work lists
  uint32_t* claim_list;
  uint32_t* reduce_list;
  uint32_t* heavy_list;           // two lists of M entries: columns reduced block-wide, by round parity
  const uint32_t* ncols_dev;      // when set, the column count is read here (ncols is then the capacity)
  unsigned long long* steps;
  unsigned long long* compacted;  // entries read by run compactions (profiling)
  uint32_t* max_chain;            // longest chain of additions (profiling)
  unsigned* heartbeat;            // bumped while chains of additions make progress
  unsigned long long* added;      // entries of the columns added (profiling)
  // board through which a block with a large run merge hands chunks of it to
  // blocks waiting at the grid barrier (zeroed before the launch; null: none),
  // and the number of blocks waiting there
  struct HelpBoard* help;
  const unsigned* idle;
  unsigned long long barrier_ns;  // grid-barrier wait without progress before giving up
  unsigned long long chain_ns;    // one chain of additions before giving up
  uint32_t* err;
};


// from rips_h0.cu
// per-cloud H0 in one block per cloud (every n_c small enough for shared memory)
bool h0_blocks_fit(int n_max);
cudaError_t launch_h0_blocks(const CloudInfo* clouds, int nclouds, int n_max, const uint64_t* sorted_keys,
                             int edge_bits, uint32_t* eu, uint32_t* ev, uint32_t m_total, uint8_t* in_forest,
                             rips_bar_t* bars, uint32_t* nbars, uint32_t bar_cap, unsigned long long* stats,
                             int stats_stride, uint32_t* err, cudaStream_t s);
// one large cloud: Boruvka rounds over the whole GPU, then the elder rule
cudaError_t run_h0_large(int n, const uint64_t* sorted_keys, uint32_t m, int edge_bits, uint32_t* eu, uint32_t* ev,
                         uint32_t* comp, uint32_t* best, uint32_t* parent, uint8_t* in_forest, uint32_t* flags,
                         uint32_t* fpos, void* scan_tmp, uint32_t* d_nf, uint32_t* gtop, rips_bar_t* bars,
                         uint32_t* nbars, uint32_t bar_cap, unsigned long long* stats, uint32_t* err, cudaStream_t s);

// from rips_dim.cu
cudaError_t launch_enumerate(const DimArgs& a, const uint64_t* pidx, const uint32_t* prank, uint32_t np,
                             int prev_col_bits, uint64_t* out_idx, uint32_t* out_rank, unsigned long long* count,
                             unsigned long long cap, cudaStream_t st);
cudaError_t launch_edges_to_simplices(const uint64_t* keys, const uint32_t* erank, uint32_t m, int edge_bits,
                                      int col_bits, uint64_t* sidx, uint32_t* srank, cudaStream_t st);
// stats: per cloud, stats_stride counters; the test writes [4] cofacet, [5] facet, [6] cleared
cudaError_t launch_test(const DimArgs& a, const uint64_t* sidx, const uint32_t* srank, uint32_t ns,
                        const uint8_t* cleared_flag, const uint64_t* prev_keys, uint64_t prev_mask,
                        uint64_t* col_keys, uint32_t* ncols, uint32_t col_cap, unsigned long long* stats,
                        int stats_stride, cudaStream_t st);
// blocks of the cooperative reduction launch (all co-resident), -1 on error
int reduction_blocks(const DimArgs& a, uint32_t ncols);
// ctl: 8 zeroed uint32 (see reduce_persistent_kernel); ctl[6] receives the rounds
cudaError_t launch_reduction(const DimArgs& a, const RedState& s, int blocks, unsigned* ctl, cudaStream_t st);
// stats: [0] pairs, [1] zero pairs, [2] essential, [3] emergent per cloud
cudaError_t launch_readout(const DimArgs& a, const RedState& s, const float* rank_value, rips_bar_t* bars,
                           uint32_t* nbars, uint32_t bar_cap, unsigned long long* stats, int stats_stride,
                           cudaStream_t st);

// from rips_epilogue.cu
cudaError_t launch_bar_order(rips_bar_t* bars, rips_bar_t* bars_alt, uint32_t nb, uint64_t* k0, uint64_t* k1,
                             uint32_t* p0, uint32_t* p1, void* tmp, size_t tmp_bytes, int simplex_bits,
                             int group_bits, cudaStream_t s);
size_t bar_order_temp_bytes(uint32_t nb);

// from rips_backward.cu
cudaError_t launch_backward(const rips_bar_t* bars, uint32_t nb, const float* pts, int k, const int64_t* pt_off,
                            const int64_t* dist_off, const float* gbirth, const float* gdeath, float* gx, float* gd,
                            cudaStream_t s);
// dL/dD only, from each cloud's distance matrix (dists, gdists, ns: DEVICE arrays indexed by cloud)
cudaError_t launch_backward_dist(const rips_bar_t* bars, uint32_t nb, const float* const* dists, float* const* gdists,
                                 const int64_t* ns, const float* gbirth, const float* gdeath, cudaStream_t s);

}  // namespace rips
