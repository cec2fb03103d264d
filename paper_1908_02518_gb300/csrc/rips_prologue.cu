// Prologue of the barcode computation: everything that turns the FP32
// distance matrix into the integer structures the later kernels read.
//
//  * binomial table for the combinatorial number system (Section 2; the table
//    is precomputed as in Section 4, "Vertices and simplices");
//  * validation and the row maxima of the symmetric distance matrix, whose
//    minimum is the enclosing radius used when no threshold is given
//    (Section 4, "Input");
//  * edge keys (FP32 diameter bits above the bit-inverted edge index), whose
//    ascending order is the refined filtration order of the edges (diameter up,
//    then index down, Section 2);
//  * the rank of every edge length among the distinct lengths <= threshold and
//    the symmetric rank matrix R;
//  * per-vertex neighbour lists in decreasing vertex order (the neighbour sets
//    of Section 4, "Enumerating cofacets", restricted to the threshold).
#include <cmath>

#include "rips_internal.cuh"

namespace rips {

namespace {

__global__ void binomial_kernel(uint64_t* __restrict__ tab, int n, int kmax) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i > n) return;
  const int stride = n + 1;
  // C(i, k) = C(i, k-1) * (i - k + 1) / k, exact in 128-bit; saturate at 2^64-1
  unsigned __int128 c = 1;
  bool sat = false;
  tab[i] = 1;
  for (int k = 1; k <= kmax; ++k) {
    if (!sat) {
      if (i - k + 1 <= 0) c = 0;
      else {
        c = c * (unsigned __int128)(i - k + 1) / (unsigned __int128)k;
        if (c > (unsigned __int128)0xFFFFFFFFFFFFFFFFull) sat = true;
      }
    }
    tab[(size_t)k * stride + i] = sat ? ~0ull : (uint64_t)c;
  }
}

constexpr int TILE = 32;

__device__ __forceinline__ void tri_tile(uint32_t b, uint32_t* I, uint32_t* J) {
  // block b -> (I, J), J <= I, row-major over the lower triangle of tiles
  uint32_t i = (uint32_t)((sqrt(8.0 * (double)b + 1.0) - 1.0) * 0.5);
  while ((uint64_t)i * (i + 1) / 2 > b) --i;
  while ((uint64_t)(i + 1) * (i + 2) / 2 <= b) ++i;
  *I = i;
  *J = b - (uint32_t)((uint64_t)i * (i + 1) / 2);
}

// cloud owning block b, given the exclusive prefix off[0..nclouds] of blocks per cloud
__device__ __forceinline__ int cloud_of_block(const uint32_t* __restrict__ off, int nclouds, uint32_t b) {
  int lo = 0, hi = nclouds - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= b) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__global__ void cloud_vertices_kernel(const CloudInfo* __restrict__ clouds, uint32_t* __restrict__ vcloud) {
  const CloudInfo ci = clouds[blockIdx.x];
  for (int i = threadIdx.x; i < ci.n; i += blockDim.x) vcloud[ci.voff + i] = blockIdx.x;
}

// Validates the strict lower triangle of every cloud's matrix and accumulates
// the maximum of each row and column of it (= row maxima of the symmetric
// matrix) as float bits.  One block per 32x32 tile of a lower triangle.
__global__ void __launch_bounds__(TILE * 8) validate_rowmax_kernel(const float* __restrict__ D,
                                                                   const CloudInfo* __restrict__ clouds,
                                                                   const uint32_t* __restrict__ tile_off, int nclouds,
                                                                   uint32_t* __restrict__ rowmax,
                                                                   uint32_t* __restrict__ err) {
  __shared__ uint32_t rmax[TILE][TILE + 1];
  const int c = cloud_of_block(tile_off, nclouds, blockIdx.x);
  const CloudInfo ci = clouds[c];
  const int n = ci.n;
  const float* Dc = D + ci.roff;
  uint32_t* rm = rowmax + ci.voff;
  uint32_t I, J;
  tri_tile(blockIdx.x - tile_off[c], &I, &J);
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int j = J * TILE + tx;
  bool bad = false;
  uint32_t colmax = 0;
  for (int r = ty; r < TILE; r += 8) {
    const int i = I * TILE + r;
    uint32_t bits = 0;
    if (i < n && j < i) {
      float v = Dc[(size_t)i * n + j];
      if (!(v >= 0.0f) || isinf(v)) bad = true;
      else bits = __float_as_uint(v == 0.0f ? 0.0f : v);
    }
    rmax[r][tx] = bits;
    colmax = max(colmax, bits);
  }
  if (bad) set_error(err, ERRF_BAD_INPUT);
  __syncthreads();
  for (int r = ty; r < TILE; r += 8) {
    uint32_t v = rmax[r][tx];
#pragma unroll
    for (int o = 16; o; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int i = I * TILE + r;
    if (tx == 0 && i < n && v) atomicMax(&rm[i], v);
  }
  __syncthreads();
  rmax[ty][tx] = colmax;
  __syncthreads();
  if (ty == 0) {
    uint32_t v = 0;
    for (int r = 0; r < 8; ++r) v = max(v, rmax[r][tx]);
    if (j < n && v) atomicMax(&rm[j], v);
  }
}

// per cloud (one block each): t = threshold, or the enclosing radius
// min_x max_y d(x, y) when the threshold is +inf or NaN
__global__ void threshold_kernel(const uint32_t* __restrict__ rowmax, CloudInfo* __restrict__ clouds, float threshold) {
  __shared__ uint32_t sm[32];
  const CloudInfo ci = clouds[blockIdx.x];
  uint32_t m = 0xFFFFFFFFu;
  for (int i = threadIdx.x; i < ci.n; i += blockDim.x) m = min(m, rowmax[ci.voff + i]);
#pragma unroll
  for (int o = 16; o; o >>= 1) m = min(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = min(m, sm[w]);
    m = min(m, sm[0]);
    float r = ci.n <= 1 ? 0.0f : __uint_as_float(m);
    clouds[blockIdx.x].t_eff = (isnan(threshold) || isinf(threshold)) ? r : threshold;
  }
}

// Edges (i > j) with d(i,j) <= t as keys
//   (cloud << (32 + eb)) | (float bits << eb) | (2^eb - 1 - idx),  idx = C(i,2) + j:
// ascending keys list every cloud's edges contiguously, each cloud in refined
// filtration order (diameter up, then index down).
__global__ void edge_keys_kernel(const float* __restrict__ D, const CloudInfo* __restrict__ clouds,
                                 const uint32_t* __restrict__ vcloud, uint32_t nverts, int eb,
                                 uint64_t* __restrict__ keys, uint32_t* __restrict__ count,
                                 uint32_t* __restrict__ cloud_count, uint32_t cap) {
  const int lane = threadIdx.x & 31;
  const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
  const unsigned lt = (1u << lane) - 1u;
  const uint64_t emask = (1ull << eb) - 1;
  for (uint32_t v = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < nverts; v += warps) {
    const uint32_t c = vcloud[v];
    const CloudInfo ci = clouds[c];
    const int i = (int)(v - ci.voff), n = ci.n;
    const float t = ci.t_eff;
    const float* row = D + ci.roff + (size_t)i * n;
    const uint64_t rowbase = (uint64_t)i * (i - 1) / 2;
    const uint64_t chi = (uint64_t)c << (32 + eb);
    for (int j0 = 0; j0 < i; j0 += 32) {
      const int j = j0 + lane;
      float x = 0.0f;
      bool ok = false;
      if (j < i) {
        x = row[j];
        x = x == 0.0f ? 0.0f : x;
        ok = x <= t;
      }
      unsigned m = __ballot_sync(0xffffffffu, ok);
      if (!m) continue;
      uint32_t base = 0;
      if (lane == 0) {
        base = atomicAdd(count, (uint32_t)__popc(m));
        atomicAdd(&cloud_count[c], (uint32_t)__popc(m));
      }
      base = __shfl_sync(0xffffffffu, base, 0);
      if (ok) {
        uint32_t pos = base + __popc(m & lt);
        if (pos < cap) keys[pos] = chi | ((uint64_t)__float_as_uint(x) << eb) | (emask - (rowbase + j));
      }
    }
  }
}

__global__ void rank_flags_kernel(const uint64_t* __restrict__ keys, uint32_t m, int eb, uint32_t* __restrict__ flags) {
  uint32_t e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m) return;
  flags[e] = (e == 0 || (keys[e] >> eb) != (keys[e - 1] >> eb)) ? 1u : 0u;
}

// rank = index of the run of equal (cloud, length) pairs: increasing with the
// length inside a cloud, so comparing ranks compares lengths exactly
__global__ void rank_finalize_kernel(const uint64_t* __restrict__ keys, uint32_t m, int eb,
                                     const uint32_t* __restrict__ excl, uint32_t* __restrict__ edge_rank,
                                     float* __restrict__ rank_value) {
  uint32_t e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m) return;
  bool first = (e == 0 || (keys[e] >> eb) != (keys[e - 1] >> eb));
  uint32_t r = excl[e] + (first ? 1u : 0u) - 1u;
  edge_rank[e] = r;
  if (first) rank_value[r] = __uint_as_float((uint32_t)(keys[e] >> eb));
}

__device__ __forceinline__ void edge_vertices(uint64_t idx, int* a, int* b) {
  // largest a with a(a-1)/2 <= idx
  int x = (int)((1.0 + sqrt(1.0 + 8.0 * (double)idx)) * 0.5);
  while ((uint64_t)x * (x - 1) / 2 > idx) --x;
  while ((uint64_t)(x + 1) * x / 2 <= idx) ++x;
  *a = x;
  *b = (int)(idx - (uint64_t)x * (x - 1) / 2);
}

__global__ void fill_rank_matrix_kernel(const uint64_t* __restrict__ keys, const uint32_t* __restrict__ edge_rank,
                                        uint32_t m, int eb, const CloudInfo* __restrict__ clouds,
                                        uint32_t* __restrict__ R) {
  uint32_t e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m) return;
  const uint64_t key = keys[e];
  if (key == ~0ull) return;  // padding past the edge count (batch plans)
  const uint64_t emask = (1ull << eb) - 1;
  const uint32_t c = (uint32_t)(key >> (32 + eb));
  const uint64_t idx = emask - (key & emask);
  const CloudInfo ci = clouds[c];
  int a, b;
  edge_vertices(idx, &a, &b);
  const uint32_t r = edge_rank[e];
  uint32_t* Rc = R + ci.roff;
  Rc[(size_t)a * ci.n + b] = r;
  Rc[(size_t)b * ci.n + a] = r;
}

// degree of every vertex: number of u with R[v][u] != INF (one warp per vertex)
__global__ void neighbor_count_kernel(const uint32_t* __restrict__ R, const CloudInfo* __restrict__ clouds,
                                      const uint32_t* __restrict__ vcloud, uint32_t nverts,
                                      uint32_t* __restrict__ deg, uint32_t* __restrict__ max_deg) {
  const int lane = threadIdx.x & 31;
  const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t v = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < nverts; v += warps) {
    const CloudInfo ci = clouds[vcloud[v]];
    const uint32_t* row = R + ci.roff + (size_t)(v - ci.voff) * ci.n;
    uint32_t c = 0;
    for (int u = lane; u < ci.n; u += 32) c += row[u] != RANK_INF;
#pragma unroll
    for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane == 0) {
      deg[v] = c;
      atomicMax(max_deg, c);
    }
  }
}

// neighbour lists (local vertex ids) in decreasing order
__global__ void neighbor_fill_kernel(const uint32_t* __restrict__ R, const CloudInfo* __restrict__ clouds,
                                     const uint32_t* __restrict__ vcloud, uint32_t nverts,
                                     const uint32_t* __restrict__ off, uint32_t* __restrict__ nbr) {
  const int lane = threadIdx.x & 31;
  const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
  const unsigned lt = (1u << lane) - 1u;
  for (uint32_t v = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < nverts; v += warps) {
    const CloudInfo ci = clouds[vcloud[v]];
    const uint32_t* row = R + ci.roff + (size_t)(v - ci.voff) * ci.n;
    uint32_t pos = off[v];
    for (int u0 = ci.n - 1; u0 >= 0; u0 -= 32) {
      int u = u0 - lane;
      bool ok = u >= 0 && row[u] != RANK_INF;
      unsigned m = __ballot_sync(0xffffffffu, ok);
      if (ok) nbr[pos + __popc(m & lt)] = (uint32_t)u;
      pos += __popc(m);
    }
  }
}

// Euclidean distances from FP32 coordinates: float64 squared differences summed
// in coordinate order with separate rounding, correctly rounded sqrt, to FP32.
__global__ void distance_kernel(const float* __restrict__ pts, int n, int k, float* __restrict__ D) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= n || j >= n) return;
  double acc = 0.0;
  for (int c = 0; c < k; ++c) {
    double diff = __dsub_rn((double)pts[(size_t)i * k + c], (double)pts[(size_t)j * k + c]);
    acc = __dadd_rn(acc, __dmul_rn(diff, diff));
  }
  D[(size_t)i * n + j] = __double2float_rn(__dsqrt_rn(acc));
}

// all clouds: one block per 8 rows of a cloud (prefix tile_off over clouds)
__global__ void distance_multi_kernel(const float* __restrict__ pts, int k, const CloudInfo* __restrict__ clouds,
                                      const uint32_t* __restrict__ tile_off, int nclouds, float* __restrict__ D) {
  const int c = cloud_of_block(tile_off, nclouds, blockIdx.x);
  const CloudInfo ci = clouds[c];
  const int n = ci.n;
  const int i = (blockIdx.x - tile_off[c]) * 8 + threadIdx.y;
  if (i >= n) return;
  const float* x = pts + (size_t)ci.voff * k;
  float* Dc = D + ci.roff;
  for (int j = threadIdx.x; j < n; j += 32) {
    double acc = 0.0;
    for (int q = 0; q < k; ++q) {
      double diff = __dsub_rn((double)x[(size_t)i * k + q], (double)x[(size_t)j * k + q]);
      acc = __dadd_rn(acc, __dmul_rn(diff, diff));
    }
    Dc[(size_t)i * n + j] = __double2float_rn(__dsqrt_rn(acc));
  }
}

// ---------------------------------------------------------------- sparse inputs
// A sparse input never forms the n x n matrix: its edges (length <= threshold)
// are listed as keys like edge_keys_kernel's, and the neighbour lists carry the
// rank of each edge (Section 4: sparse distance matrices, where a missing entry
// is an infinite distance).

// one edge key, the same layout as edge_keys_kernel (single cloud)
__device__ __forceinline__ uint64_t edge_key(int i, int j, float x, int eb) {
  const int a = i > j ? i : j, b = i > j ? j : i;
  const uint64_t emask = (1ull << eb) - 1;
  const uint64_t idx = (uint64_t)a * (a - 1) / 2 + (uint64_t)b;
  return ((uint64_t)__float_as_uint(x == 0.0f ? 0.0f : x) << eb) | (emask - idx);
}

// warp-aggregated append of the lanes' keys where `ok` holds
__device__ __forceinline__ void append_key(bool ok, uint64_t key, uint64_t* keys, uint32_t* count, uint32_t cap) {
  const int lane = threadIdx.x & 31;
  const unsigned m = __ballot_sync(0xffffffffu, ok);
  if (!m) return;
  uint32_t base = 0;
  if (lane == 0) base = atomicAdd(count, (uint32_t)__popc(m));
  base = __shfl_sync(0xffffffffu, base, 0);
  if (ok) {
    const uint32_t pos = base + __popc(m & ((1u << lane) - 1u));
    if (pos < cap) keys[pos] = key;
  }
}

// a list of (i, j, length) entries, each unordered pair at most once
__global__ void coo_edge_keys_kernel(const int32_t* __restrict__ ei, const int32_t* __restrict__ ej,
                                     const float* __restrict__ len, uint64_t m, int n, float t, int eb,
                                     uint64_t* __restrict__ keys, uint32_t* __restrict__ count, uint32_t cap,
                                     uint32_t* __restrict__ err) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t first = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (uint64_t e0 = first - (threadIdx.x & 31); e0 < m; e0 += stride) {  // whole warps iterate together
    const uint64_t e = e0 + (threadIdx.x & 31);
    bool ok = false;
    uint64_t key = 0;
    if (e < m) {
      const int i = ei[e], j = ej[e];
      const float x = len[e];
      const bool valid = i >= 0 && i < n && j >= 0 && j < n && i != j && x >= 0.0f && !isinf(x);
      if (!valid) set_error(err, ERRF_BAD_INPUT);
      ok = valid && x <= t;
      if (ok) key = edge_key(i, j, x, eb);
    }
    append_key(ok, key, keys, count, cap);
  }
}

// the edges of a point cloud within the threshold, distances by the rule of
// distance_kernel, one 32 x 32 tile of (i > j) pairs per block (8 rows a warp)
__global__ void point_edges_kernel(const float* __restrict__ pts, int n, int k, float t, int eb,
                                   uint64_t* __restrict__ keys, uint32_t* __restrict__ count, uint32_t cap) {
  uint32_t I, J;  // tile row and column, I >= J
  {
    const uint64_t b = blockIdx.x;
    uint32_t r = (uint32_t)((sqrt(8.0 * (double)b + 1.0) - 1.0) * 0.5);
    while ((uint64_t)r * (r + 1) / 2 > b) --r;
    while ((uint64_t)(r + 1) * (r + 2) / 2 <= b) ++r;
    I = r;
    J = (uint32_t)(b - (uint64_t)r * (r + 1) / 2);
  }
  const int j = (int)(J * 32 + (threadIdx.x & 31));
  for (int rr = threadIdx.x >> 5; rr < 32; rr += blockDim.x >> 5) {
    const int i = (int)(I * 32 + rr);
    bool ok = false;
    float x = 0.0f;
    if (i < n && j < i) {
      double acc = 0.0;
      for (int c = 0; c < k; ++c) {
        const double diff = __dsub_rn((double)pts[(size_t)i * k + c], (double)pts[(size_t)j * k + c]);
        acc = __dadd_rn(acc, __dmul_rn(diff, diff));
      }
      x = __double2float_rn(__dsqrt_rn(acc));
      ok = x <= t;
    }
    append_key(ok, ok ? edge_key(i, j, x, eb) : 0ull, keys, count, cap);
  }
}

// degrees from the sorted edge keys
__global__ void sparse_degree_kernel(const uint64_t* __restrict__ keys, uint32_t m, int eb, uint32_t* __restrict__ deg) {
  const uint32_t e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m) return;
  const uint64_t emask = (1ull << eb) - 1;
  int a, b;
  edge_vertices(emask - (keys[e] & emask), &a, &b);
  atomicAdd(&deg[a], 1u);
  atomicAdd(&deg[b], 1u);
}

// both directions of every edge, keyed (vertex, complement of the neighbour) so
// that one sort leaves each list in decreasing neighbour order, with the rank
__global__ void sparse_fill_kernel(const uint64_t* __restrict__ keys, const uint32_t* __restrict__ erank, uint32_t m,
                                   int eb, const uint32_t* __restrict__ off, uint32_t* __restrict__ cursor,
                                   uint64_t* __restrict__ nkey, uint32_t* __restrict__ nval) {
  const uint32_t e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m) return;
  const uint64_t emask = (1ull << eb) - 1;
  int a, b;
  edge_vertices(emask - (keys[e] & emask), &a, &b);
  const uint32_t r = erank[e];
  const uint32_t pa = off[a] + atomicAdd(&cursor[a], 1u);
  nkey[pa] = ((uint64_t)a << 32) | (0xFFFFFFFFu - (uint32_t)b);
  nval[pa] = r;
  const uint32_t pb = off[b] + atomicAdd(&cursor[b], 1u);
  nkey[pb] = ((uint64_t)b << 32) | (0xFFFFFFFFu - (uint32_t)a);
  nval[pb] = r;
}

__global__ void sparse_unpack_kernel(const uint64_t* __restrict__ nkey, const uint32_t* __restrict__ nval, uint32_t q,
                                     uint32_t* __restrict__ nbr, uint32_t* __restrict__ nrank) {
  const uint32_t e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= q) return;
  nbr[e] = 0xFFFFFFFFu - (uint32_t)(nkey[e] & 0xFFFFFFFFull);
  nrank[e] = nval[e];
}

__global__ void max_kernel(const uint32_t* __restrict__ x, uint32_t n, uint32_t* __restrict__ out) {
  uint32_t m = 0;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) m = max(m, x[i]);
  m = __reduce_max_sync(0xffffffffu, m);
  if ((threadIdx.x & 31) == 0 && m) atomicMax(out, m);
}

}  // namespace

cudaError_t launch_binomial_table(uint64_t* tab, int n, int kmax, cudaStream_t s) {
  binomial_kernel<<<(n + 1 + 255) / 256, 256, 0, s>>>(tab, n, kmax);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_cloud_vertices(const CloudInfo* clouds, int nclouds, uint32_t* vcloud, cudaStream_t s) {
  cloud_vertices_kernel<<<nclouds, 256, 0, s>>>(clouds, vcloud);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_validate_rowmax(const float* D, const CloudInfo* clouds, const uint32_t* tile_off, int nclouds,
                                   uint32_t tiles, uint32_t* rowmax_bits, uint32_t* err, cudaStream_t s) {
  if (tiles == 0) return cudaSuccess;
  validate_rowmax_kernel<<<tiles, TILE * 8, 0, s>>>(D, clouds, tile_off, nclouds, rowmax_bits, err);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_threshold(const uint32_t* rowmax_bits, CloudInfo* clouds, int nclouds, float threshold,
                             cudaStream_t s) {
  threshold_kernel<<<nclouds, 1024, 0, s>>>(rowmax_bits, clouds, threshold);
  note_launch();
  return cudaGetLastError();
}

static int warp_grid(uint64_t items) {
  uint64_t blocks = (items * 32 + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (blocks < 1) blocks = 1;
  return (int)blocks;
}

cudaError_t launch_edge_keys(const float* D, const CloudInfo* clouds, const uint32_t* vcloud, uint32_t nverts,
                             int edge_bits, uint64_t* keys, uint32_t* count, uint32_t* cloud_count, uint32_t cap,
                             cudaStream_t s) {
  edge_keys_kernel<<<warp_grid(nverts), 256, 0, s>>>(D, clouds, vcloud, nverts, edge_bits, keys, count, cloud_count,
                                                    cap);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_assign_ranks(const uint64_t* sorted_keys, uint32_t m, int edge_bits, uint32_t* flags,
                                uint32_t* scan_tmp, uint32_t* edge_rank, float* rank_value, uint32_t* num_ranks,
                                cudaStream_t s) {
  if (m == 0) return cudaMemsetAsync(num_ranks, 0, sizeof(uint32_t), s);
  rank_flags_kernel<<<(m + 255) / 256, 256, 0, s>>>(sorted_keys, m, edge_bits, flags);
  note_launch();
  cudaError_t e = launch_exclusive_scan(flags, flags, m, scan_tmp, num_ranks, s);
  if (e != cudaSuccess) return e;
  rank_finalize_kernel<<<(m + 255) / 256, 256, 0, s>>>(sorted_keys, m, edge_bits, flags, edge_rank, rank_value);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_fill_rank_matrix(const uint64_t* sorted_keys, const uint32_t* edge_rank, uint32_t m,
                                    int edge_bits, const CloudInfo* clouds, uint32_t* R, cudaStream_t s) {
  if (m == 0) return cudaSuccess;
  fill_rank_matrix_kernel<<<(m + 255) / 256, 256, 0, s>>>(sorted_keys, edge_rank, m, edge_bits, clouds, R);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_neighbor_counts(const uint32_t* R, const CloudInfo* clouds, const uint32_t* vcloud,
                                   uint32_t nverts, uint32_t* deg, uint32_t* max_deg, cudaStream_t s) {
  neighbor_count_kernel<<<warp_grid(nverts), 256, 0, s>>>(R, clouds, vcloud, nverts, deg, max_deg);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_neighbor_fill(const uint32_t* R, const CloudInfo* clouds, const uint32_t* vcloud, uint32_t nverts,
                                 const uint32_t* off, uint32_t* nbr, cudaStream_t s) {
  neighbor_fill_kernel<<<warp_grid(nverts), 256, 0, s>>>(R, clouds, vcloud, nverts, off, nbr);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_distance_matrices(const float* pts, int k, const CloudInfo* clouds, const uint32_t* tile_off,
                                     int nclouds, uint32_t tiles, float* D, cudaStream_t s) {
  if (tiles == 0) return cudaSuccess;
  distance_multi_kernel<<<tiles, dim3(32, 8), 0, s>>>(pts, k, clouds, tile_off, nclouds, D);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_distance_matrix(const float* pts, int n, int k, float* D, cudaStream_t s) {
  dim3 blk(32, 8), grd((n + 31) / 32, (n + 7) / 8);
  distance_kernel<<<grd, blk, 0, s>>>(pts, n, k, D);
  note_launch();
  return cudaGetLastError();
}


// Strict triangle of a distance matrix stored packed (row by row) into the
// strict lower triangle of the n x n matrix D: lower layout, entry (i, j) with
// i > j at i(i-1)/2 + j (rows 1 .. n-1 of the lower triangle, each from column
// 0); upper layout, entry (r, c) with r < c at r n - r(r+1)/2 + (c - r - 1)
// (rows 0 .. n-2 of the upper triangle).  Only D[i][j], i > j, is written.
__global__ void unpack_triangle_kernel(const float* __restrict__ packed, int n, int upper, float* __restrict__ D) {
  const int i = blockIdx.y * blockDim.y + threadIdx.y;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || j >= i) return;
  const uint64_t at = upper ? (uint64_t)j * n - (uint64_t)j * (j + 1) / 2 + (uint64_t)(i - j - 1)
                            : (uint64_t)i * (i - 1) / 2 + (uint64_t)j;
  D[(size_t)i * n + j] = packed[at];
}

cudaError_t launch_unpack_triangle(const float* packed, int n, int upper, float* D, cudaStream_t s) {
  if (n < 2) return cudaSuccess;
  dim3 blk(32, 8), grd((n + 31) / 32, (n + 7) / 8);
  unpack_triangle_kernel<<<grd, blk, 0, s>>>(packed, n, upper, D);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_coo_edge_keys(const int32_t* ei, const int32_t* ej, const float* len, uint64_t m, int n, float t,
                                 int eb, uint64_t* keys, uint32_t* count, uint32_t cap, uint32_t* err, cudaStream_t s) {
  if (m == 0) return cudaSuccess;
  uint64_t blocks = (m + 255) / 256;
  if (blocks > 152 * 32) blocks = 152 * 32;
  coo_edge_keys_kernel<<<(unsigned)blocks, 256, 0, s>>>(ei, ej, len, m, n, t, eb, keys, count, cap, err);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_point_edges(const float* pts, int n, int k, float t, int eb, uint64_t* keys, uint32_t* count,
                               uint32_t cap, cudaStream_t s) {
  if (n < 2) return cudaSuccess;
  const uint64_t nb = ((uint64_t)n + 31) / 32;
  point_edges_kernel<<<(unsigned)(nb * (nb + 1) / 2), 256, 0, s>>>(pts, n, k, t, eb, keys, count, cap);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_sparse_degrees(const uint64_t* keys, uint32_t m, int eb, uint32_t* deg, cudaStream_t s) {
  if (m == 0) return cudaSuccess;
  sparse_degree_kernel<<<(m + 255) / 256, 256, 0, s>>>(keys, m, eb, deg);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_sparse_fill(const uint64_t* keys, const uint32_t* erank, uint32_t m, int eb, const uint32_t* off,
                               uint32_t* cursor, uint64_t* nkey, uint32_t* nval, cudaStream_t s) {
  if (m == 0) return cudaSuccess;
  sparse_fill_kernel<<<(m + 255) / 256, 256, 0, s>>>(keys, erank, m, eb, off, cursor, nkey, nval);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_sparse_unpack(const uint64_t* nkey, const uint32_t* nval, uint32_t q, uint32_t* nbr,
                                 uint32_t* nrank, cudaStream_t s) {
  if (q == 0) return cudaSuccess;
  sparse_unpack_kernel<<<(q + 255) / 256, 256, 0, s>>>(nkey, nval, q, nbr, nrank);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_max(const uint32_t* x, uint32_t n, uint32_t* out, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  uint32_t blocks = (n + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  max_kernel<<<blocks, 256, 0, s>>>(x, n, out);
  note_launch();
  return cudaGetLastError();
}

// ---------------------------------------------------------------- batch plans (no host reads)
// Entries [*count, cap) of a key list set to the largest key, so a sort of all
// cap entries leaves the real ones first.
__global__ void pad_past_count_kernel(uint64_t* __restrict__ keys, const uint32_t* __restrict__ count, uint64_t cap) {
  const uint64_t from = *count;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < cap; i += (uint64_t)gridDim.x * blockDim.x)
    if (i >= from) keys[i] = ~0ull;
}

// Each cloud's first edge and edge count in the sorted edge list, from the
// per-cloud counts of the edge-key kernel (one thread: a batch has few clouds).
__global__ void cloud_edge_offsets_kernel(CloudInfo* __restrict__ clouds, const uint32_t* __restrict__ ccounts,
                                          int nclouds) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  uint32_t acc = 0;
  for (int c = 0; c < nclouds; ++c) {
    clouds[c].eoff = acc;
    clouds[c].m = ccounts[c];
    acc += ccounts[c];
  }
}

cudaError_t launch_pad_past_count(uint64_t* keys, const uint32_t* count, uint64_t cap, cudaStream_t s) {
  if (cap == 0) return cudaSuccess;
  uint64_t blocks = (cap + 255) / 256;
  if (blocks > 152 * 32) blocks = 152 * 32;
  pad_past_count_kernel<<<(unsigned)blocks, 256, 0, s>>>(keys, count, cap);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_cloud_edge_offsets(CloudInfo* clouds, const uint32_t* ccounts, int nclouds, cudaStream_t s) {
  cloud_edge_offsets_kernel<<<1, 32, 0, s>>>(clouds, ccounts, nclouds);
  note_launch();
  return cudaGetLastError();
}

}  // namespace rips
