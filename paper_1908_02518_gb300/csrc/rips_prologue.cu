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

// Validates the strict lower triangle and accumulates the maximum of every
// row and column of it (= row maxima of the symmetric matrix) as float bits.
__global__ void __launch_bounds__(TILE * 8) validate_rowmax_kernel(const float* __restrict__ D, int n,
                                                                   uint32_t* __restrict__ rowmax,
                                                                   uint32_t* __restrict__ err) {
  __shared__ uint32_t rmax[TILE][TILE + 1];
  uint32_t I, J;
  tri_tile(blockIdx.x, &I, &J);
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int j = J * TILE + tx;
  bool bad = false;
  uint32_t colmax = 0;
  for (int r = ty; r < TILE; r += 8) {
    const int i = I * TILE + r;
    uint32_t bits = 0;
    if (i < n && j < i) {
      float v = D[(size_t)i * n + j];
      if (!(v >= 0.0f) || isinf(v)) bad = true;
      else bits = __float_as_uint(v == 0.0f ? 0.0f : v);
    }
    rmax[r][tx] = bits;
    colmax = max(colmax, bits);
  }
  if (bad) set_error(err, ERRF_BAD_INPUT);
  __syncthreads();
  // row maxima: warp ty reduces rows ty, ty+8, ...
  for (int r = ty; r < TILE; r += 8) {
    uint32_t v = rmax[r][tx];
#pragma unroll
    for (int o = 16; o; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int i = I * TILE + r;
    if (tx == 0 && i < n && v) atomicMax(&rowmax[i], v);
  }
  __syncthreads();
  rmax[ty][tx] = colmax;
  __syncthreads();
  if (ty == 0) {
    uint32_t v = 0;
    for (int r = 0; r < 8; ++r) v = max(v, rmax[r][tx]);
    if (j < n && v) atomicMax(&rowmax[j], v);
  }
}

__global__ void threshold_kernel(const uint32_t* __restrict__ rowmax, int n, float threshold,
                                 float* __restrict__ t_eff) {
  __shared__ uint32_t sm[32];
  uint32_t m = 0xFFFFFFFFu;
  for (int i = threadIdx.x; i < n; i += blockDim.x) m = min(m, rowmax[i]);
#pragma unroll
  for (int o = 16; o; o >>= 1) m = min(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = min(m, sm[w]);
    m = min(m, sm[0]);
    float r = n <= 1 ? 0.0f : __uint_as_float(m);
    *t_eff = (isnan(threshold) || isinf(threshold)) ? r : threshold;
  }
}

// Edges (i > j) with d(i,j) <= t as keys (float bits << 32) | ~idx, idx = C(i,2)+j.
__global__ void edge_keys_kernel(const float* __restrict__ D, int n, const float* __restrict__ t_eff,
                                 uint64_t* __restrict__ keys, uint32_t* __restrict__ count, uint32_t cap) {
  const float t = *t_eff;
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  const unsigned lt = (1u << lane) - 1u;
  for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += warps) {
    const uint64_t rowbase = (uint64_t)i * (i - 1) / 2;
    for (int j0 = 0; j0 < i; j0 += 32) {
      const int j = j0 + lane;
      float v = 0.0f;
      bool ok = false;
      if (j < i) {
        v = D[(size_t)i * n + j];
        v = v == 0.0f ? 0.0f : v;
        ok = v <= t;
      }
      unsigned m = __ballot_sync(0xffffffffu, ok);
      if (!m) continue;
      uint32_t base = 0;
      if (lane == 0) base = atomicAdd(count, (uint32_t)__popc(m));
      base = __shfl_sync(0xffffffffu, base, 0);
      if (ok) {
        uint32_t pos = base + __popc(m & lt);
        if (pos < cap)
          keys[pos] = ((uint64_t)__float_as_uint(v) << 32) | (uint64_t)(0xFFFFFFFFu - (uint32_t)(rowbase + j));
      }
    }
  }
}

__global__ void rank_flags_kernel(const uint64_t* __restrict__ keys, uint32_t m, uint32_t* __restrict__ flags) {
  uint32_t e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m) return;
  flags[e] = (e == 0 || (keys[e] >> 32) != (keys[e - 1] >> 32)) ? 1u : 0u;
}

__global__ void rank_finalize_kernel(const uint64_t* __restrict__ keys, uint32_t m,
                                     const uint32_t* __restrict__ excl, uint32_t* __restrict__ edge_rank,
                                     float* __restrict__ rank_value) {
  uint32_t e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m) return;
  bool first = (e == 0 || (keys[e] >> 32) != (keys[e - 1] >> 32));
  uint32_t r = excl[e] + (first ? 1u : 0u) - 1u;
  edge_rank[e] = r;
  if (first) rank_value[r] = __uint_as_float((uint32_t)(keys[e] >> 32));
}

__device__ __forceinline__ void edge_vertices(uint32_t idx, int* a, int* b) {
  // largest a with a(a-1)/2 <= idx
  int x = (int)((1.0 + sqrt(1.0 + 8.0 * (double)idx)) * 0.5);
  while ((uint64_t)x * (x - 1) / 2 > idx) --x;
  while ((uint64_t)(x + 1) * x / 2 <= idx) ++x;
  *a = x;
  *b = (int)(idx - (uint32_t)((uint64_t)x * (x - 1) / 2));
}

__global__ void fill_rank_matrix_kernel(const uint64_t* __restrict__ keys, const uint32_t* __restrict__ edge_rank,
                                        uint32_t m, int n, uint32_t* __restrict__ R) {
  uint32_t e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m) return;
  uint32_t idx = 0xFFFFFFFFu - (uint32_t)(keys[e] & 0xFFFFFFFFull);
  int a, b;
  edge_vertices(idx, &a, &b);
  uint32_t r = edge_rank[e];
  R[(size_t)a * n + b] = r;
  R[(size_t)b * n + a] = r;
}

// degree of every vertex: number of u with R[v][u] != INF
__global__ void neighbor_count_kernel(const uint32_t* __restrict__ R, int n, uint32_t* __restrict__ deg) {
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int v = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < n; v += warps) {
    uint32_t c = 0;
    const uint32_t* row = R + (size_t)v * n;
    for (int u = lane; u < n; u += 32) c += row[u] != RANK_INF;
#pragma unroll
    for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane == 0) deg[v] = c;
  }
}

// neighbour lists in decreasing vertex order
__global__ void neighbor_fill_kernel(const uint32_t* __restrict__ R, int n, const uint32_t* __restrict__ off,
                                     uint32_t* __restrict__ nbr) {
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  const unsigned lt = (1u << lane) - 1u;
  for (int v = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < n; v += warps) {
    const uint32_t* row = R + (size_t)v * n;
    uint32_t pos = off[v];
    for (int u0 = n - 1; u0 >= 0; u0 -= 32) {
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

}  // namespace

cudaError_t launch_binomial_table(uint64_t* tab, int n, int kmax, cudaStream_t s) {
  binomial_kernel<<<(n + 1 + 255) / 256, 256, 0, s>>>(tab, n, kmax);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_validate_rowmax(const float* D, int n, uint32_t* rowmax_bits, uint32_t* err, cudaStream_t s) {
  uint32_t nb = (uint32_t)((n + TILE - 1) / TILE);
  uint32_t blocks = nb * (nb + 1) / 2;
  validate_rowmax_kernel<<<blocks, TILE * 8, 0, s>>>(D, n, rowmax_bits, err);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_threshold(const uint32_t* rowmax_bits, int n, float threshold, float* t_eff, cudaStream_t s) {
  threshold_kernel<<<1, 1024, 0, s>>>(rowmax_bits, n, threshold, t_eff);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_edge_keys(const float* D, int n, const float* t_eff, uint64_t* keys, uint32_t* count,
                             uint32_t cap, cudaStream_t s) {
  int blocks = (n * 32 + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (blocks < 1) blocks = 1;
  edge_keys_kernel<<<blocks, 256, 0, s>>>(D, n, t_eff, keys, count, cap);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_assign_ranks(const uint64_t* sorted_keys, uint32_t m, uint32_t* flags, uint32_t* scan_tmp,
                                size_t, uint32_t* edge_rank, float* rank_value, uint32_t* num_ranks,
                                cudaStream_t s) {
  if (m == 0) return cudaMemsetAsync(num_ranks, 0, sizeof(uint32_t), s);
  rank_flags_kernel<<<(m + 255) / 256, 256, 0, s>>>(sorted_keys, m, flags);
  note_launch();
  cudaError_t e = launch_exclusive_scan(flags, flags, m, scan_tmp, num_ranks, s);
  if (e != cudaSuccess) return e;
  rank_finalize_kernel<<<(m + 255) / 256, 256, 0, s>>>(sorted_keys, m, flags, edge_rank, rank_value);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_fill_rank_matrix(const uint64_t* sorted_keys, const uint32_t* edge_rank, uint32_t m, int n,
                                    uint32_t* R, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(R, 0xFF, (size_t)n * n * sizeof(uint32_t), s);
  if (e != cudaSuccess || m == 0) return e;
  fill_rank_matrix_kernel<<<(m + 255) / 256, 256, 0, s>>>(sorted_keys, edge_rank, m, n, R);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_neighbor_counts(const uint32_t* R, int n, uint32_t* deg, cudaStream_t s) {
  int blocks = (n * 32 + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  neighbor_count_kernel<<<blocks, 256, 0, s>>>(R, n, deg);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_neighbor_fill(const uint32_t* R, int n, const uint32_t* off, uint32_t* nbr, cudaStream_t s) {
  int blocks = (n * 32 + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  neighbor_fill_kernel<<<blocks, 256, 0, s>>>(R, n, off, nbr);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_distance_matrix(const float* pts, int n, int k, float* D, cudaStream_t s) {
  dim3 blk(32, 8), grd((n + 31) / 32, (n + 7) / 8);
  distance_kernel<<<grd, blk, 0, s>>>(pts, n, k, D);
  note_launch();
  return cudaGetLastError();
}

}  // namespace rips
