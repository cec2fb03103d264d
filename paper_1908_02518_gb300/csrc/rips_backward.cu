// Backward pass: gradients of a loss on bar endpoints with respect to the point
// coordinates (not part of the paper; the critical-edge map below is the
// standard one for Rips filtrations).
//
// A finite endpoint of a bar is the diameter of its birth or death simplex, i.e.
// the length of one edge of that simplex: the longest one, ties broken towards
// the smallest edge index (the youngest of the tied edges in the refined
// order).  The simplex is decoded from its combinatorial index (the Lemma of
// Section 4 on the largest vertex), its edges are measured from the
// coordinates with the same float64 rule as the forward distances, and
// dL/d(endpoint) is scattered to the two endpoints' coordinates through
// d|x_a - x_b| / dx_a = (x_a - x_b) / |x_a - x_b|.
#include "rips_internal.cuh"

namespace rips {

namespace {

__device__ __forceinline__ uint64_t binom_arith(uint64_t v, int k) {
  if (k < 0 || (uint64_t)k > v) return 0;
  unsigned __int128 c = 1;
  for (int i = 1; i <= k; ++i) c = c * (unsigned __int128)(v - k + i) / (unsigned __int128)i;
  return (uint64_t)c;
}

__device__ void decode_arith(uint64_t N, int d, int n, int* v) {
  int hi = n - 1;
  for (int k = d + 1; k >= 1; --k) {
    int lo = k - 1, h = hi;
    while (lo < h) {
      int mid = (lo + h + 1) >> 1;
      if (binom_arith(mid, k) <= N) lo = mid;
      else h = mid - 1;
    }
    v[d + 1 - k] = lo;
    N -= binom_arith(lo, k);
    hi = lo - 1;
  }
}

__device__ __forceinline__ float dist_rule(const float* __restrict__ x, int k, int a, int b) {
  double acc = 0.0;
  for (int c = 0; c < k; ++c) {
    double diff = __dsub_rn((double)x[(size_t)a * k + c], (double)x[(size_t)b * k + c]);
    acc = __dadd_rn(acc, __dmul_rn(diff, diff));
  }
  return __double2float_rn(__dsqrt_rn(acc));
}

// longest edge (a > b) of the d-simplex with index N; ties: smallest edge index
__device__ void critical_edge(const float* __restrict__ x, int k, int n, uint64_t N, int d, int* ea, int* eb) {
  int v[MAX_DIM + 2];
  decode_arith(N, d, n, v);
  float best = -1.0f;
  uint64_t best_idx = 0;
  *ea = v[0];
  *eb = v[d];
  for (int i = 0; i <= d; ++i)
    for (int j = i + 1; j <= d; ++j) {
      const int a = v[i], b = v[j];  // a > b
      const float w = dist_rule(x, k, a, b);
      const uint64_t eidx = (uint64_t)a * (a - 1) / 2 + b;
      if (w > best || (w == best && eidx < best_idx)) {
        best = w;
        best_idx = eidx;
        *ea = a;
        *eb = b;
      }
    }
}

__device__ void scatter(const float* __restrict__ x, int k, int a, int b, float g, float* __restrict__ gx,
                        float* __restrict__ gd, int n) {
  if (g == 0.0f) return;
  const float w = dist_rule(x, k, a, b);
  if (gd) atomicAdd(&gd[(size_t)a * n + b], g);
  if (!(w > 0.0f)) return;  // the gradient of |x_a - x_b| is undefined at 0
  for (int c = 0; c < k; ++c) {
    const float u = (x[(size_t)a * k + c] - x[(size_t)b * k + c]) / w;
    atomicAdd(&gx[(size_t)a * k + c], g * u);
    atomicAdd(&gx[(size_t)b * k + c], -g * u);
  }
}

__global__ void backward_kernel(const rips_bar_t* __restrict__ bars, uint32_t nb, const float* __restrict__ pts,
                                int k, const int64_t* __restrict__ pt_off, const int64_t* __restrict__ dist_off,
                                const float* __restrict__ gbirth, const float* __restrict__ gdeath,
                                float* __restrict__ gx, float* __restrict__ gd) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nb) return;
  const rips_bar_t b = bars[i];
  const int64_t p0 = pt_off[b.cloud];
  const int n = (int)(pt_off[b.cloud + 1] - p0);
  const float* x = pts + (size_t)p0 * k;
  float* gxc = gx + (size_t)p0 * k;
  float* gdc = gd ? gd + dist_off[b.cloud] : nullptr;
  int ea, eb;
  if (b.dim >= 1 && gbirth) {
    critical_edge(x, k, n, b.birth_simplex, b.dim, &ea, &eb);
    scatter(x, k, ea, eb, gbirth[i], gxc, gdc, n);
  }
  if (isfinite(b.death) && b.death_simplex != ~0ull && gdeath) {
    critical_edge(x, k, n, b.death_simplex, b.dim + 1, &ea, &eb);
    scatter(x, k, ea, eb, gdeath[i], gxc, gdc, n);
  }
}

// Longest edge (a > b) of the d-simplex with index N measured on the FP32
// distance matrix D (n x n, strict lower triangle D[a*n + b]) the forward read;
// ties: smallest edge index, as above.
__device__ void critical_edge_dist(const float* __restrict__ D, int n, uint64_t N, int d, int* ea, int* eb) {
  int v[MAX_DIM + 2];
  decode_arith(N, d, n, v);
  float best = -1.0f;
  uint64_t best_idx = 0;
  *ea = v[0];
  *eb = v[d];
  for (int i = 0; i <= d; ++i)
    for (int j = i + 1; j <= d; ++j) {
      const int a = v[i], b = v[j];  // a > b
      const float w = D[(size_t)a * n + b];
      const uint64_t eidx = (uint64_t)a * (a - 1) / 2 + b;
      if (w > best || (w == best && eidx < best_idx)) {
        best = w;
        best_idx = eidx;
        *ea = a;
        *eb = b;
      }
    }
}

// dL/dD only: every finite endpoint's gradient is added to its critical edge's
// entry of the cloud's gradient matrix
__global__ void backward_dist_kernel(const rips_bar_t* __restrict__ bars, uint32_t nb,
                                     const float* const* __restrict__ dists, float* const* __restrict__ gdists,
                                     const int64_t* __restrict__ ns, const float* __restrict__ gbirth,
                                     const float* __restrict__ gdeath) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nb) return;
  const rips_bar_t b = bars[i];
  const int n = (int)ns[b.cloud];
  const float* D = dists[b.cloud];
  float* G = gdists[b.cloud];
  int ea, eb;
  if (b.dim >= 1 && gbirth && gbirth[i] != 0.0f) {
    critical_edge_dist(D, n, b.birth_simplex, b.dim, &ea, &eb);
    atomicAdd(&G[(size_t)ea * n + eb], gbirth[i]);
  }
  if (isfinite(b.death) && b.death_simplex != ~0ull && gdeath && gdeath[i] != 0.0f) {
    critical_edge_dist(D, n, b.death_simplex, b.dim + 1, &ea, &eb);
    atomicAdd(&G[(size_t)ea * n + eb], gdeath[i]);
  }
}

}  // namespace

cudaError_t launch_backward_dist(const rips_bar_t* bars, uint32_t nb, const float* const* dists, float* const* gdists,
                                 const int64_t* ns, const float* gbirth, const float* gdeath, cudaStream_t s) {
  if (nb == 0) return cudaSuccess;
  backward_dist_kernel<<<(nb + 127) / 128, 128, 0, s>>>(bars, nb, dists, gdists, ns, gbirth, gdeath);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_backward(const rips_bar_t* bars, uint32_t nb, const float* pts, int k, const int64_t* pt_off,
                            const int64_t* dist_off, const float* gbirth, const float* gdeath, float* gx, float* gd,
                            cudaStream_t s) {
  if (nb == 0) return cudaSuccess;
  backward_kernel<<<(nb + 127) / 128, 128, 0, s>>>(bars, nb, pts, k, pt_off, dist_off, gbirth, gdeath, gx, gd);
  note_launch();
  return cudaGetLastError();
}

}  // namespace rips
