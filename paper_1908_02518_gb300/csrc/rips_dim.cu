// One dimension d >= 1 of the cohomology computation (Section 3.3) for every
// cloud of a batch at once: columns are the d-simplices, rows the
// (d+1)-simplices, columns are processed youngest first (diameter down, then
// index up, Section 3.5 "Shortcuts" and Section 4 "Pivot extraction"), and a
// column's pivot is its OLDEST nonzero row (smallest diameter, then largest
// index).  Every work item carries its cloud in the top bits of its key.
//
// Kernels (warp-cooperative; lanes take consecutive entries of a vertex's
// neighbour list, so every cofacet tile is 32 candidates wide):
//
//  enumerate_kernel   all d-simplices <= t, each made once as (j, rho) with
//                     j above the top vertex of a (d-1)-simplex rho (Section 4,
//                     "Assembling column indices").
//  test_kernel        drops a d-simplex if it is cleared (a pivot of the
//                     (d-1)-reduction: Section 3.2 / Algorithm 2), if it has a
//                     zero-persistence apparent cofacet, or a zero-persistence
//                     apparent facet (Proposition in Section 3.5 and the
//                     procedure in its "Shortcuts" paragraph); survivors are
//                     compacted with their processing-order key.
//  reduce_persistent_kernel  one cooperative launch per dimension:
//     first pivots    the cofacets are scanned in decreasing index order and
//                     the first one with the column's own diameter is the pivot
//                     (the emergent-pair shortcut, Section 3.5); only when there
//                     is none is the whole coboundary scanned for its minimum;
//     claim           columns claim their pivot in an open-addressing table by
//                     atomicCAS on the key and atomicMin on the column ordinal:
//                     the earliest column in processing order owns a pivot;
//     reduce          every column whose pivot is owned by an earlier column
//                     adds that column (R_j -= lambda R_k, Algorithm 1) and keeps
//                     going while the new pivot is owned by an earlier column; a
//                     pivot with a zero apparent facet is owned by that facet's
//                     column (Section 4, "Persistence pairs": apparent pairs are
//                     not in the table).  A warp reduces a column while there
//                     are more columns than blocks, for at most DimArgs::chain_limit
//                     additions a round; with fewer, a block takes each column
//                     and adds with a block-wide merge, which is what long
//                     chains of additions need.
//
// The coboundary stays implicit (Section 3.4) for every column that is never
// added to -- apparent, emergent and unreduced owners: their coboundary is
// generated from the combinatorial number system when it is needed.  A column
// that is reduced keeps its working column R_j materialised (sorted row keys,
// nonzero coefficients), so later additions of it cost a merge instead of a
// regeneration; V is not stored since only pairs are reported.
//
// Parallel reduction and correctness.  Claims and reductions alternate in
// rounds separated by grid barriers.  A column only ever adds a column that
// precedes it in processing order (or an apparent facet's column, which
// precedes every column with that pivot), so R = D V with V upper
// unitriangular; pivots only move to younger rows, so the rounds end; at the
// end every nonzero column owns its pivot alone, i.e. R is reduced, and by the
// pivot proposition of Section 3.1 the pairs are exactly those of the
// sequential algorithm (the pairing of a reduced matrix is unique).
#include <mutex>
#include <vector>

#include "rips_internal.cuh"

namespace rips {

namespace {

constexpr int WARPS_PER_BLOCK = 8;
constexpr uint32_t MAX_PIVOT_PASSES = 1u << 30;  // additions in one chain before giving up
constexpr uint8_t HEAVY = 2;                      // flag in RedState::reduced: reduced block-wide

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

struct Binom {
  const uint64_t* t;
  int s;
  __device__ __forceinline__ uint64_t operator()(int i, int k) const { return t[(size_t)k * s + i]; }
};

__device__ __forceinline__ Binom stage_binom(const DimArgs& a, uint64_t* smem) {
  Binom b{a.binom, a.bn + 1};
  if (a.smem_binom) {
    const int total = (a.kmax + 1) * (a.bn + 1);
    for (int i = threadIdx.x; i < total; i += blockDim.x) smem[i] = a.binom[i];
    __syncthreads();
    b.t = smem;
  }
  return b;
}

// ---------------------------------------------------------------- clouds
// A cloud's view: its size, rank matrix and neighbour-list offsets (indexed by
// local vertex) into the shared list array.
// R is null for a sparse input: the rank of an edge then comes from the
// neighbour lists (nrank[q] = rank of the edge to nbr[q]).
struct CV {
  int n;
  const uint32_t* R;
  const uint32_t* off;
  const uint32_t* nbr;
  const uint32_t* nrank;
};

__device__ __forceinline__ CV cloud_view(const DimArgs& a, uint32_t c) {
  const CloudInfo ci = a.clouds[c];
  return CV{ci.n, a.R ? a.R + ci.roff : nullptr, a.nbr_off + ci.voff, a.nbr, a.nrank};
}

// Rank of the edge (x, y), RANK_INF when it is above the threshold or x == y:
// one read of the rank matrix, or with a sparse input a binary search for y in
// x's neighbour list (vertices in decreasing order).
__device__ __forceinline__ uint32_t rank_of(const CV& cv, int x, int y) {
  if (cv.R) return cv.R[(size_t)x * cv.n + y];
  const uint32_t end = cv.off[x + 1];
  uint32_t lo = cv.off[x], hi = end;
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (cv.nbr[mid] > (uint32_t)y) lo = mid + 1;
    else hi = mid;
  }
  return lo < end && cv.nbr[lo] == (uint32_t)y ? cv.nrank[lo] : RANK_INF;
}

__device__ __forceinline__ uint64_t low_mask(int bits) { return bits >= 64 ? ~0ull : ((1ull << bits) - 1); }
__device__ __forceinline__ uint32_t high_part(uint64_t x, int bits) { return bits >= 64 ? 0u : (uint32_t)(x >> bits); }

// ---------------------------------------------------------------- simplex helpers

struct Simplex {
  int v[MAX_DIM + 2];  // vertices, decreasing
  uint64_t idx;
  uint32_t rank;
};

// largest v in [lo, hi] with C(v, k) <= N, by bisection
__device__ __forceinline__ int max_vertex_bisect(const Binom& B, int k, int lo, int hi, uint64_t N) {
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (B(mid, k) <= N) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Largest v in [k-1, hi] with C(v, k) <= N (k >= 2), i.e. the top vertex of the
// k-subset with index N (Section 4, "combinatorial number system").  Since
// C(v, k) is about (v - (k-1)/2)^k / k!, a float root of k! N gives v to within
// one or two; four neighbouring table entries (one or two cache lines) settle
// it, and bisection takes over if the estimate was further off.
__device__ __forceinline__ int max_vertex(const Binom& B, int k, int hi, uint64_t N) {
  float kf = 1.0f;
  for (int i = 2; i <= k; ++i) kf *= (float)i;
  const float est = exp2f(log2f(__ull2float_rn(N) * kf) / (float)k) + 0.5f * (float)(k - 1);
  int v = est >= (float)hi ? hi : (int)est;
  if (v < k - 1) v = k - 1;
  const uint64_t b0 = B(v, k);
  const uint64_t bm = B(v > 0 ? v - 1 : 0, k);
  const uint64_t b1 = B(v + 1 <= hi ? v + 1 : hi, k);
  const uint64_t b2 = B(v + 2 <= hi ? v + 2 : hi, k);
  if (b0 <= N) {
    if (v == hi || b1 > N) return v;
    if (v + 1 == hi || b2 > N) return v + 1;
    return max_vertex_bisect(B, k, v + 2, hi, N);
  }
  // b0 > N implies v >= k, so v - 1 >= k - 1
  if (bm <= N) return v - 1;
  return max_vertex_bisect(B, k, k - 1, v - 2, N);
}

__device__ __forceinline__ void decode(const Binom& B, int n, uint64_t N, int d, int* v) {
  int hi = n - 1;
  for (int k = d + 1; k >= 1; --k) {
    const int x = k == 1 ? (int)N : max_vertex(B, k, hi, N);
    v[d + 1 - k] = x;
    N -= k == 1 ? N : B(x, k);
    hi = x - 1;
  }
}

// Vertices of a d-simplex given by a reference: its index, or (packed) its
// vertices packed vbits apiece as the pair map stores them.
__device__ __forceinline__ void simplex_vertices(const Binom& B, int n, uint64_t ref, bool packed, int vbits, int d,
                                                 int* v) {
  if (!packed) {
    decode(B, n, ref, d, v);
    return;
  }
  const uint64_t m = (1ull << vbits) - 1;
  for (int l = 0; l <= d; ++l) v[l] = (int)((ref >> (l * vbits)) & m);
}

// rank of sigma with vertex v[l] removed, for every l (d >= 1)
__device__ __forceinline__ void ranks_minus_one(const CV& cv, const int* v, int d, uint32_t* out) {
  for (int l = 0; l <= d; ++l) out[l] = 0;
  for (int a = 0; a <= d; ++a)
    for (int b = a + 1; b <= d; ++b) {
      uint32_t r = rank_of(cv, v[a], v[b]);
      for (int l = 0; l <= d; ++l)
        if (l != a && l != b) out[l] = max(out[l], r);
    }
}

// vertex of sigma (index into v) with the shortest neighbour list
__device__ __forceinline__ int min_degree_vertex(const CV& cv, const int* v, int cnt) {
  int best = 0;
  uint32_t bd = cv.off[v[0] + 1] - cv.off[v[0]];
  for (int l = 1; l < cnt; ++l) {
    uint32_t dg = cv.off[v[l] + 1] - cv.off[v[l]];
    if (dg < bd) {
      bd = dg;
      best = l;
    }
  }
  return best;
}

// Cofacet tau = sigma + j of a d-simplex with vertices v (decreasing).  c = number
// of vertices above j.  idx(tau) = above[c] + C(j, d+2-c) + below[c], where
// above[c] = sum_{l<c} C(v[l], d+2-l), below[c] = sum_{l>=c} C(v[l], d+1-l)
// (Section 4, "Enumerating cofacets": the two running partial sums).
struct CofacetSums {
  uint64_t above[MAX_DIM + 2];
  uint64_t below[MAX_DIM + 2];
};

__device__ __forceinline__ void cofacet_sums(const Binom& B, const int* v, int d, CofacetSums& cs) {
  uint64_t acc = 0;
  for (int c = 0; c <= d + 1; ++c) {
    cs.above[c] = acc;
    if (c <= d) acc += B(v[c], d + 2 - c);
  }
  acc = 0;
  for (int c = d + 1; c >= 0; --c) {
    cs.below[c] = acc;
    if (c >= 1) acc += B(v[c - 1], d + 2 - c);
  }
}

// Evaluate candidate j for the cofacets of sigma: returns false if sigma + j is not
// a simplex <= t (including j in sigma).  On success gives rank, index and the
// number c of vertices of sigma above j.
__device__ __forceinline__ bool cofacet_of(const CV& cv, const Binom& B, const int* v, int d, uint32_t srank,
                                           const CofacetSums& cs, int j, uint32_t* rank, uint64_t* idx, int* cpos) {
  uint32_t r = srank;
  int c = 0;
  bool ok = true;
  for (int l = 0; l <= d; ++l) {  // no early exit: the loads are independent
    const uint32_t x = rank_of(cv, v[l], j);
    ok &= x != RANK_INF;
    r = max(r, x);
    c += v[l] > j;
  }
  const uint64_t bj = B(j, d + 2 - c);  // loaded beside the rank lookups, not after them
  if (!ok) return false;
  *rank = r;
  *cpos = c;
  *idx = cs.above[c] + bj + cs.below[c];
  return true;
}

__device__ __forceinline__ uint64_t row_key(const DimArgs& a, uint32_t rank, uint64_t idx) {
  const uint64_t mask = (a.row_bits >= 64) ? ~0ull : ((1ull << a.row_bits) - 1);
  return ((uint64_t)rank << a.row_bits) | (mask - idx);
}
__device__ __forceinline__ uint64_t row_key_idx(const DimArgs& a, uint64_t key) {
  const uint64_t mask = (a.row_bits >= 64) ? ~0ull : ((1ull << a.row_bits) - 1);
  return mask - (key & mask);
}
__device__ __forceinline__ uint32_t row_key_rank(const DimArgs& a, uint64_t key) {
  return (uint32_t)(key >> a.row_bits);
}

// Largest-index cofacet of sigma with the same diameter rank (the candidate tau of
// the Proposition on zero apparent pairs), found by scanning cofacets in
// decreasing index order.  Warp-cooperative; every lane gets the result.
// Returns the vertex j (or -1) and, on the owning lane, fills the ranks of j to
// the vertices of sigma.
__device__ int first_equal_cofacet(const CV& cv, const int* v, int d, uint32_t srank, int lane,
                                   uint32_t* rj /* d+1, valid on the returned lane */, int* hit_lane) {
  int av = v[min_degree_vertex(cv, v, d + 1)];
  const uint32_t beg = cv.off[av], end = cv.off[av + 1];
  for (uint32_t q0 = beg; q0 < end; q0 += 32) {
    const uint32_t q = q0 + lane;
    bool hit = false;
    int j = -1;
    if (q < end) {
      j = (int)cv.nbr[q];
      hit = true;
      for (int l = 0; l <= d; ++l) {
        uint32_t x = rank_of(cv, v[l], j);
        rj[l] = x;
        if (x > srank) hit = false;  // also rejects RANK_INF and j in sigma
      }
    }
    unsigned m = __ballot_sync(0xffffffffu, hit);
    if (m) {
      int src = __ffs(m) - 1;
      *hit_lane = src;
      return __shfl_sync(0xffffffffu, j, src);
    }
  }
  *hit_lane = -1;
  return -1;
}

// Zero apparent facet of a k-simplex tau with vertices w (decreasing) and rank r
// (Section 3.5): rho = the smallest-index facet with the same rank (facets in
// increasing index order drop the largest vertices first); apparent iff tau is
// the largest-index cofacet of rho with that rank, i.e. no vertex u > w[l]
// outside tau gives rank(rho + u) <= r.  Warp-cooperative.  Returns l (the
// dropped vertex position) or -1.
__device__ int zero_apparent_facet(const CV& cv, const int* w, int k, uint32_t r, const uint32_t* minus,
                                   int lane) {
  int l = -1;
  for (int x = 0; x <= k; ++x)
    if (minus[x] == r) {
      l = x;
      break;
    }
  if (l < 0) return -1;
  const int drop = w[l];
  // vertices of rho
  int rv[MAX_DIM + 2];
  int m = 0;
  for (int x = 0; x <= k; ++x)
    if (x != l) rv[m++] = w[x];
  int av = rv[min_degree_vertex(cv, rv, k)];
  const uint32_t beg = cv.off[av], end = cv.off[av + 1];
  for (uint32_t q0 = beg; q0 < end; q0 += 32) {
    const uint32_t q = q0 + lane;
    bool above = false, hit = false;
    if (q < end) {
      int u = (int)cv.nbr[q];
      above = u > drop;
      if (above) {
        hit = true;
        for (int x = 0; x < k; ++x) hit &= rank_of(cv, rv[x], u) <= r;
        // u is not a vertex of tau: the dropped vertex is excluded by u > drop, the
        // others by R = RANK_INF on the diagonal
      }
    }
    if (__any_sync(0xffffffffu, hit)) return -1;
    if (!__all_sync(0xffffffffu, above || q >= end)) break;  // the list went below drop
  }
  return l;
}

// ---------------------------------------------------------------- hash table
__device__ __forceinline__ uint64_t mix(uint64_t x) {
  x ^= x >> 33;
  x *= 0xff51afd7ed558ccdull;
  x ^= x >> 33;
  x *= 0xc4ceb9fe1a85ec53ull;
  x ^= x >> 33;
  return x;
}

// slot of key, inserting it if absent; -1 when the probe limit is hit
__device__ __forceinline__ int64_t table_insert(uint64_t* keys, uint64_t cap_mask, uint64_t key) {
  uint64_t h = mix(key) & cap_mask;
  for (uint64_t probe = 0; probe <= cap_mask; ++probe) {
    uint64_t cur = keys[h];
    if (cur == key) return (int64_t)h;
    if (cur == IDX_NONE) {
      uint64_t old = atomicCAS((unsigned long long*)&keys[h], (unsigned long long)IDX_NONE, (unsigned long long)key);
      if (old == IDX_NONE || old == key) return (int64_t)h;
    }
    h = (h + 1) & cap_mask;
  }
  return -1;
}

// (key, value) pair tables: slot h is kv[2h] (key, IDX_NONE when empty) and
// kv[2h + 1] (value), so a probe reads both in one 16-byte load
__device__ __forceinline__ int64_t pair_insert(uint64_t* kv, uint64_t cap_mask, uint64_t key) {
  uint64_t h = mix(key) & cap_mask;
  for (uint64_t probe = 0; probe <= cap_mask; ++probe) {
    const uint64_t cur = kv[2 * h];
    if (cur == key) return (int64_t)h;
    if (cur == IDX_NONE) {
      const uint64_t old =
          atomicCAS((unsigned long long*)&kv[2 * h], (unsigned long long)IDX_NONE, (unsigned long long)key);
      if (old == IDX_NONE || old == key) return (int64_t)h;
    }
    h = (h + 1) & cap_mask;
  }
  return -1;
}

__device__ __forceinline__ bool pair_find(const uint64_t* kv, uint64_t cap_mask, uint64_t key, uint64_t* val) {
  uint64_t h = mix(key) & cap_mask;
  for (uint64_t probe = 0; probe <= cap_mask; ++probe) {
    const ulonglong2 e = *reinterpret_cast<const ulonglong2*>(kv + 2 * h);
    if (e.x == key) {
      *val = e.y;
      return true;
    }
    if (e.x == IDX_NONE) return false;
    h = (h + 1) & cap_mask;
  }
  return false;
}

__device__ __forceinline__ int64_t table_find(const uint64_t* keys, uint64_t cap_mask, uint64_t key) {
  if (cap_mask == 0 && keys == nullptr) return -1;
  uint64_t h = mix(key) & cap_mask;
  for (uint64_t probe = 0; probe <= cap_mask; ++probe) {
    uint64_t cur = keys[h];
    if (cur == key) return (int64_t)h;
    if (cur == IDX_NONE) return -1;
    h = (h + 1) & cap_mask;
  }
  return -1;
}

}  // namespace

// ====================================================================== enumeration

__global__ void __launch_bounds__(256) enumerate_kernel(DimArgs a, const uint64_t* __restrict__ pidx,
                                                        const uint32_t* __restrict__ prank, uint32_t np, int pbits,
                                                        uint64_t* __restrict__ out_idx, uint32_t* __restrict__ out_rank,
                                                        unsigned long long* __restrict__ count,
                                                        unsigned long long cap) {
  extern __shared__ uint64_t smem[];
  Binom B = stage_binom(a, smem);
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  const int d = a.d;  // new simplices are d-simplices, made from (d-1)-simplices
  const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; s < np; s += warps) {
    const uint64_t g = pidx[s];
    const uint32_t cl = high_part(g, pbits);
    const uint64_t local = g & low_mask(pbits);
    const CV cv = cloud_view(a, cl);
    const uint64_t chi = a.col_bits >= 64 ? 0ull : ((uint64_t)cl << a.col_bits);
    int v[MAX_DIM + 2];
    decode(B, cv.n, local, d - 1, v);
    const uint32_t r0 = prank[s];
    const int top = v[0];
    const int av = v[min_degree_vertex(cv, v, d)];
    const uint32_t beg = cv.off[av], end = cv.off[av + 1];
    for (uint32_t q0 = beg; q0 < end; q0 += 32) {
      const uint32_t q = q0 + lane;
      int j = q < end ? (int)cv.nbr[q] : -1;
      bool ok = j > top;
      uint32_t r = r0;
      if (ok)
        for (int l = 0; l < d; ++l) {
          uint32_t x = rank_of(cv, v[l], j);
          if (x == RANK_INF) {
            ok = false;
            break;
          }
          r = max(r, x);
        }
      unsigned m = __ballot_sync(0xffffffffu, ok);
      if (m) {
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(count, (unsigned long long)__popc(m));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (ok) {
          unsigned long long pos = base + __popc(m & lt);
          if (pos < cap) {
            out_idx[pos] = chi | (local + B(j, d + 1));
            out_rank[pos] = r;
          }
        }
      }
      if (!__all_sync(0xffffffffu, j > top)) break;  // the list went below the top vertex
    }
  }
}

// edges (sorted) -> simplex list of dimension 1
__global__ void edges_to_simplices_kernel(const uint64_t* __restrict__ keys, const uint32_t* __restrict__ erank,
                                          uint32_t m, int eb, int col_bits, uint64_t* __restrict__ sidx,
                                          uint32_t* __restrict__ srank) {
  uint32_t e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m) return;
  const uint64_t key = keys[e];
  if (key == ~0ull) {  // padding past the edge count (batch plans): skipped by the test
    sidx[e] = ~0ull;
    srank[e] = 0;
    return;
  }
  const uint64_t emask = (1ull << eb) - 1;
  const uint64_t c = key >> (32 + eb);
  sidx[e] = (col_bits >= 64 ? 0ull : (c << col_bits)) | (emask - (key & emask));
  srank[e] = erank[e];
}

// ====================================================================== apparent + clearing test

// pivot-table key of a row: (cloud << row_bits) | local row index
__device__ __forceinline__ uint64_t table_key(const DimArgs& a, uint32_t cloud, uint64_t row_idx) {
  return (a.row_bits >= 64 ? 0ull : ((uint64_t)cloud << a.row_bits)) | row_idx;
}

__global__ void __launch_bounds__(256) test_kernel(DimArgs a, const uint64_t* __restrict__ sidx,
                                                   const uint32_t* __restrict__ srank, uint32_t ns,
                                                   const uint8_t* __restrict__ cleared_flag /* d == 1 */,
                                                   const uint64_t* __restrict__ prev_keys, uint64_t prev_mask,
                                                   uint64_t* __restrict__ col_keys, uint32_t* __restrict__ ncols,
                                                   uint32_t col_cap, unsigned long long* __restrict__ st,
                                                   int st_stride) {
  extern __shared__ uint64_t smem[];
  Binom B = stage_binom(a, smem);
  const int lane = threadIdx.x & 31;
  const int d = a.d;
  const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
  // counters are flushed to the cloud's statistics whenever the warp moves to another cloud
  unsigned long long n_cof = 0, n_fac = 0, n_clr = 0;
  uint32_t cur_cloud = 0xFFFFFFFFu;
  auto flush = [&](uint32_t next) {
    if (lane == 0 && cur_cloud != 0xFFFFFFFFu) {
      unsigned long long* q = st + (size_t)cur_cloud * st_stride;
      if (n_cof) atomicAdd(&q[4], n_cof);
      if (n_fac) atomicAdd(&q[5], n_fac);
      if (n_clr) atomicAdd(&q[6], n_clr);
    }
    n_cof = n_fac = n_clr = 0;
    cur_cloud = next;
  };
  for (uint32_t s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; s < ns; s += warps) {
    const uint64_t g = sidx[s];
    if (g == ~0ull) continue;  // padding (batch plans)
    const uint32_t r = srank[s];
    const uint32_t cl = high_part(g, a.col_bits);
    const uint64_t idx = g & low_mask(a.col_bits);
    if (cl != cur_cloud) flush(cl);
    // clearing: pivots of the previous dimension
    bool cleared;
    if (d == 1) cleared = cleared_flag[s] != 0;
    else cleared = prev_keys != nullptr && table_find(prev_keys, prev_mask, g) >= 0;
    if (cleared) {
      ++n_clr;
      continue;
    }
    const CV cv = cloud_view(a, cl);
    int v[MAX_DIM + 2];
    decode(B, cv.n, idx, d, v);
    // cofacet side: (sigma, tau) zero apparent pair?  (not with the apparent-pair
    // shortcut switched off: every simplex that is not cleared is then a column)
    const bool apparent = !(a.opts & RIPS_OPT_NO_APPARENT);
    uint32_t rj[MAX_DIM + 2];
    int hl = -1;
    int j = apparent ? first_equal_cofacet(cv, v, d, r, lane, rj, &hl) : -1;
    if (j >= 0) {
      int app = 0;
      if (lane == hl) {
        uint32_t minus[MAX_DIM + 2];
        ranks_minus_one(cv, v, d, minus);
        app = 1;
        // facets of tau dropping a vertex above j come before sigma in index order
        for (int l = 0; l <= d && v[l] > j; ++l) {
          uint32_t fr = minus[l];
          for (int m2 = 0; m2 <= d; ++m2)
            if (m2 != l) fr = max(fr, rj[m2]);
          if (fr == r) {
            app = 0;
            break;
          }
        }
      }
      app = __shfl_sync(0xffffffffu, app, hl);
      if (app) {
        ++n_cof;
        if (lane == 0 && a.amap) {  // tau -> sigma, for the reduction and the next dimension
          CofacetSums cs;
          cofacet_sums(B, v, d, cs);
          int c = 0;
          for (int l = 0; l <= d; ++l) c += v[l] > j;
          const uint64_t tidx = cs.above[c] + B(j, d + 2 - c) + cs.below[c];
          const int64_t slot = pair_insert(a.amap, a.amap_mask, table_key(a, cl, tidx));
          if (slot < 0) set_error(a.err, ERRF_TABLE_FULL);
          else {
            uint64_t ref = idx;
            if (a.vbits) {
              ref = 0;
              for (int l = 0; l <= d; ++l) ref |= (uint64_t)v[l] << (l * a.vbits);
            }
            a.amap[2 * slot + 1] = (ref << 4) | (uint64_t)c;
          }
        }
        continue;
      }
    }
    // facet side (d >= 2; in dimension 1 such edges are spanning-forest edges):
    // the previous dimension's test recorded every zero apparent pair
    if (apparent && d >= 2) {
      bool fac;
      if (a.pmap) {
        uint64_t unused;
        fac = pair_find(a.pmap, a.pmap_mask, g, &unused);
      } else {
        uint32_t minus[MAX_DIM + 2];
        ranks_minus_one(cv, v, d, minus);
        fac = zero_apparent_facet(cv, v, d, r, minus, lane) >= 0;
      }
      if (fac) {
        ++n_fac;
        continue;
      }
    }
    if (lane == 0) {
      uint32_t pos = atomicAdd(ncols, 1u);
      if (pos < col_cap) {
        const int hb = a.rank_bits + a.col_bits;
        const uint64_t key = (hb >= 64 ? 0ull : ((uint64_t)cl << hb)) |
                             ((uint64_t)(a.rank_max - r) << a.col_bits) | idx;
        col_keys[pos] = key;
      } else {
        set_error(a.err, ERRF_OUT_OVERFLOW);
      }
    }
  }
  flush(0xFFFFFFFFu);
}

// ====================================================================== reduction

namespace {

__device__ __forceinline__ void column_simplex(const DimArgs& a, const RedState& s, uint32_t j, uint64_t* idx,
                                               uint32_t* rank, uint32_t* cloud) {
  const uint64_t key = s.col_keys[j];
  *idx = key & low_mask(a.col_bits);
  *rank = a.rank_max - (uint32_t)((key >> a.col_bits) & low_mask(a.rank_bits));
  *cloud = high_part(key, a.rank_bits + a.col_bits);
}


// Minimum over the cofacet entries of sum_{(s,c) in V} c * delta(s) restricted to
// row keys > after: returns the key (IDX_NONE if none) and the summed
// coefficient at that key (mod p).  Warp-cooperative.
__device__ void min_entry(const DimArgs& a, const CV& cv, const Binom& B, int lane, const uint64_t* vidx,
                          const uint32_t* vrank,
                          const uint32_t* vcoef, uint32_t vlen, uint64_t self_idx, uint32_t self_rank,
                          uint64_t after, bool has_after, uint64_t* out_key, uint32_t* out_coef) {
  const int d = a.d;
  uint64_t best = IDX_NONE;
  uint32_t sum = 0;
  const uint32_t cnt = vlen ? vlen : 1;
  for (uint32_t e = 0; e < cnt; ++e) {
    const uint64_t sidx = vlen ? vidx[e] : self_idx;
    const uint32_t sr = vlen ? vrank[e] : self_rank;
    const uint32_t sc = vlen ? vcoef[e] : 1u;
    int v[MAX_DIM + 2];
    decode(B, cv.n, sidx, d, v);
    CofacetSums cs;
    cofacet_sums(B, v, d, cs);
    const int av = v[min_degree_vertex(cv, v, d + 1)];
    const uint32_t beg = cv.off[av], end = cv.off[av + 1];
    for (uint32_t q = beg + lane; q < end; q += 32) {
      const int j = (int)cv.nbr[q];
      uint32_t r;
      uint64_t tidx;
      int c;
      if (!cofacet_of(cv, B, v, d, sr, cs, j, &r, &tidx, &c)) continue;
      const uint64_t key = row_key(a, r, tidx);
      if (has_after && key <= after) continue;
      // paper's orientation: (-1)^k with k = #vertices below j minus one = d - c
      const uint32_t sgn = ((d - c) & 1) ? a.p - 1 : 1u;
      const uint32_t cf = (uint32_t)(((uint64_t)sgn * sc) % a.p);
      if (key < best) {
        best = key;
        sum = cf;
      } else if (key == best) {
        sum = (sum + cf) % a.p;
      }
    }
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    uint64_t ob = __shfl_xor_sync(0xffffffffu, best, o);
    uint32_t os = __shfl_xor_sync(0xffffffffu, sum, o);
    if (ob < best) {
      best = ob;
      sum = os;
    } else if (ob == best) {
      sum = (sum + os) % a.p;
    }
  }
  *out_key = best;
  *out_coef = best == IDX_NONE ? 0 : sum;
}

// Apparent facet of the pivot row tau (a (d+1)-simplex): returns the facet's
// reference (IDX_NONE if none; packed vertices when the pair map holds them,
// see DimArgs::vbits, else its index), its rank and the coefficient of tau in
// its coboundary.
__device__ uint64_t pivot_apparent_facet(const DimArgs& a, const CV& cv, const Binom& B, int lane, uint32_t cl,
                                         uint64_t key, uint32_t* frank, uint32_t* tcoef) {
  const int k = a.d + 1;
  if (a.amap) {  // recorded by this dimension's test kernel
    uint64_t v;
    if (!pair_find(a.amap, a.amap_mask, table_key(a, cl, row_key_idx(a, key)), &v)) return IDX_NONE;
    *frank = row_key_rank(a, key);
    *tcoef = ((a.d - (int)(v & 15)) & 1) ? a.p - 1 : 1u;
    return v >> 4;
  }
  const uint64_t tidx = row_key_idx(a, key);
  const uint32_t tr = row_key_rank(a, key);
  int w[MAX_DIM + 2];
  decode(B, cv.n, tidx, k, w);
  uint32_t minus[MAX_DIM + 2];
  ranks_minus_one(cv, w, k, minus);
  int l = zero_apparent_facet(cv, w, k, tr, minus, lane);
  if (l < 0) return IDX_NONE;
  // facet index: drop w[l]; vertices above it keep C(w, k+1-pos) -> C(w, k-pos)
  uint64_t fidx = 0;
  int pos = 0;
  for (int x = 0; x <= k; ++x) {
    if (x == l) continue;
    fidx += B(w[x], k - pos);
    ++pos;
  }
  *frank = tr;
  // in the coboundary of the facet, tau = facet + w[l] with c = l vertices above
  const int c = l;
  *tcoef = ((a.d - c) & 1) ? a.p - 1 : 1u;
  return fidx;
}

// Owner of the pivot row `key` of a column of cloud cl: the zero apparent facet
// of the row (Section 4, "Persistence pairs": apparent pairs are not in the
// table; its reference as pivot_apparent_facet gives it), else the table's
// owner (0xFFFFFFFF: none).  With the recorded pair
// map the two lookups run at once on lanes 0 and 1.  Warp-cooperative; every
// lane gets the results.
__device__ __forceinline__ uint64_t pivot_owner(const DimArgs& a, const RedState& s, const CV& cv, const Binom& B,
                                                int lane, uint32_t cl, uint64_t key, uint32_t* frank, uint32_t* tcoef,
                                                uint32_t* owner) {
  const uint64_t tkey = table_key(a, cl, row_key_idx(a, key));
  if (a.opts & RIPS_OPT_NO_APPARENT) {  // apparent pairs are ordinary columns: the table owns every pivot
    const int64_t slot = table_find(s.t_keys, s.t_mask, tkey);
    *owner = slot >= 0 ? s.t_vals[slot] : 0xFFFFFFFFu;
    return IDX_NONE;
  }
  if (a.amap) {
    // lane 0 probes the pair map, lane 1 the pivot table, with the same load
    // instructions, so the two lookups take the time of one
    // (each probe loads the slot's value with its key)
    uint64_t val = 0;
    int found = 0;
    if (lane < 2) {
      const uint64_t mask = lane == 0 ? a.amap_mask : s.t_mask;
      uint64_t h = mix(tkey) & mask;
      for (uint64_t probe = 0; probe <= mask; ++probe) {
        uint64_t cur, cv2;
        if (lane == 0) {
          const ulonglong2 e = *reinterpret_cast<const ulonglong2*>(a.amap + 2 * h);
          cur = e.x;
          cv2 = e.y;
        } else {
          cur = s.t_keys[h];
          cv2 = s.t_vals[h];
        }
        if (cur == tkey) {
          found = 1;
          val = cv2;
          break;
        }
        if (cur == IDX_NONE) break;
        h = (h + 1) & mask;
      }
    }
    const int ffound = __shfl_sync(0xffffffffu, found, 0);
    const uint64_t v = __shfl_sync(0xffffffffu, val, 0);
    const int tfound = __shfl_sync(0xffffffffu, found, 1);
    const uint64_t tv = __shfl_sync(0xffffffffu, val, 1);
    *owner = tfound ? (uint32_t)tv : 0xFFFFFFFFu;
    if (!ffound) return IDX_NONE;
    *frank = row_key_rank(a, key);
    *tcoef = ((a.d - (int)(v & 15)) & 1) ? a.p - 1 : 1u;
    return v >> 4;
  }
  const uint64_t fidx = pivot_apparent_facet(a, cv, B, lane, cl, key, frank, tcoef);
  *owner = 0xFFFFFFFFu;
  if (fidx == IDX_NONE) {
    const int64_t slot = table_find(s.t_keys, s.t_mask, tkey);
    *owner = slot >= 0 ? s.t_vals[slot] : 0xFFFFFFFFu;
  }
  return fidx;
}

// ---------------------------------------------------------------- working columns
// A column that has to be reduced keeps R_j = D V_j materialised in the R arena,
// sorted by row key (oldest row first) with nonzero coefficients: the GPU form of
// the paper's working coboundary (Section 4, "Pivot extraction").  Columns that
// never get reduced (apparent, emergent) never build theirs; the coboundary of an
// unreduced owner or of an apparent facet is generated on the fly into a per-warp
// scratch slice and sorted there.

// all cofacets of the d-simplex (idx, rank) with their paper-orientation signs,
// unsorted, into buf; returns the count (warp-uniform).  idx is a reference as
// simplex_vertices takes it.
__device__ uint32_t gen_coboundary(const DimArgs& a, const CV& cv, const Binom& B, int lane, uint64_t idx,
                                   bool packed, uint32_t rank, uint32_t scale, uint64_t* bkey, uint32_t* bcoef,
                                   uint32_t cap) {
  const int d = a.d;
  const unsigned lt = (1u << lane) - 1u;
  int v[MAX_DIM + 2];
  simplex_vertices(B, cv.n, idx, packed, a.vbits, d, v);
  CofacetSums cs;
  cofacet_sums(B, v, d, cs);
  const int av = v[min_degree_vertex(cv, v, d + 1)];
  const uint32_t beg = cv.off[av], end = cv.off[av + 1];
  uint32_t cnt = 0;
  for (uint32_t q0 = beg; q0 < end; q0 += 32) {
    const uint32_t q = q0 + lane;
    uint32_t r = 0;
    uint64_t tidx = 0;
    int c = 0;
    const bool ok = q < end && cofacet_of(cv, B, v, d, rank, cs, (int)cv.nbr[q], &r, &tidx, &c);
    const unsigned m = __ballot_sync(0xffffffffu, ok);
    if (ok) {
      const uint32_t pos = cnt + __popc(m & lt);
      if (pos < cap) {
        const uint32_t sgn = ((d - c) & 1) ? a.p - 1 : 1u;
        bkey[pos] = row_key(a, r, tidx);
        bcoef[pos] = (uint32_t)(((uint64_t)sgn * scale) % a.p);
      }
    }
    cnt += __popc(m);
  }
  if (cnt > cap) set_error(a.err, ERRF_INTERNAL);
  return cnt < cap ? cnt : cap;
}

// ascending bitonic sort of (key, coef) pairs in a buffer of at least
// next_pow2(n) entries; the padding takes key ~0 (never a row key)
__device__ void warp_sort_pairs(uint64_t* key, uint32_t* coef, uint32_t n, int lane) {
  uint32_t p2 = 1;
  while (p2 < n) p2 <<= 1;
  for (uint32_t i = n + lane; i < p2; i += 32) {
    key[i] = ~0ull;
    coef[i] = 0;
  }
  __syncwarp();
  for (uint32_t k = 2; k <= p2; k <<= 1) {
    for (uint32_t j = k >> 1; j > 0; j >>= 1) {
      for (uint32_t i = lane; i < p2; i += 32) {
        const uint32_t l = i ^ j;
        if (l > i) {
          const uint64_t ki = key[i], kl = key[l];
          const bool up = (i & k) == 0;
          if ((ki > kl) == up) {
            key[i] = kl;
            key[l] = ki;
            const uint32_t t = coef[i];
            coef[i] = coef[l];
            coef[l] = t;
          }
        }
      }
      __syncwarp();
    }
  }
}

// ---------------------------------------------------------------- lazy working column
// During a chain of additions the working column is a sum of sorted runs, one
// per lane (at most 32), each with its own Z/p scale: R_j's own entries and the
// columns added to it.  Adding a column appends a run (no copy of R_j); the
// pivot is the smallest head key whose combined coefficient is nonzero, found by
// warp reductions, and the heads at a key whose coefficients cancel move on:
// the paper's lazily evaluated working coboundary (Section 4, "Pivot
// extraction"), with sorted runs in place of its heap.  Runs are merged size-
// tiered: when four runs (eight short ones) fall in the same size class
// (sizes within a factor of four), they become one, so an entry is merged a
// logarithmic number of times however long the chain; at the end of a chain
// the column is merged into one run, which later columns add.
//
// Each run keeps the RUN_AHEAD entries after its head (key and stored
// coefficient) in registers, loaded that many steps before they are needed.
constexpr int RUN_AHEAD = 1;

struct Run {
  const uint64_t* key;
  const uint32_t* coef;
  uint32_t len, cur, scale;
  uint64_t hk;             // head key, ~0 once the run is used up
  uint32_t hc;             // head coefficient times scale, mod p (1 over Z/2)
  uint64_t nk[RUN_AHEAD];  // the keys after the head (~0 past the end)
  uint32_t nc[RUN_AHEAD];  // and their stored coefficients (not loaded over Z/2)
};

// c * scale mod p; both below p < 2^16, so the product fits in 32 bits
__device__ __forceinline__ uint32_t scaled(uint32_t c, uint32_t scale, uint32_t p) {
  return p == 2 ? 1u : (c * scale) % p;
}

// Remainders mod p of 32-bit numbers by multiplication (Lemire, Kaser and
// Kurz, "Faster remainder by direct computation", 2019): with
// M = floor((2^64 - 1) / p) + 1, a mod p = high 64 bits of (M * a mod 2^64) * p,
// exact for every 32-bit a and p.
struct ModP {
  uint32_t p;
  uint64_t M;
  __device__ __forceinline__ explicit ModP(uint32_t pp) : p(pp), M(~0ull / pp + 1) {}
  __device__ __forceinline__ uint32_t operator()(uint32_t x) const { return (uint32_t)__umul64hi(M * x, p); }
};

// head and look-ahead from the cursor on
__device__ __forceinline__ void run_head(Run& r, uint32_t p) {
  r.hk = r.cur < r.len ? r.key[r.cur] : ~0ull;
  r.hc = r.cur < r.len ? scaled(p == 2 ? 1u : r.coef[r.cur], r.scale, p) : 0u;
#pragma unroll
  for (int i = 0; i < RUN_AHEAD; ++i) {
    const bool in = r.cur + 1 + i < r.len;
    r.nk[i] = in ? r.key[r.cur + 1 + i] : ~0ull;
    r.nc[i] = in && p != 2 ? r.coef[r.cur + 1 + i] : 1u;
  }
}

// move to the next entry, loaded ahead; the entry RUN_AHEAD past it is requested now
__device__ __forceinline__ void run_next(Run& r, uint32_t p) {
  ++r.cur;
  r.hk = r.nk[0];
  r.hc = r.cur < r.len ? scaled(r.nc[0], r.scale, p) : 0u;
#pragma unroll
  for (int i = 0; i + 1 < RUN_AHEAD; ++i) {
    r.nk[i] = r.nk[i + 1];
    r.nc[i] = r.nc[i + 1];
  }
  const bool in = r.cur + RUN_AHEAD < r.len;
  r.nk[RUN_AHEAD - 1] = in ? r.key[r.cur + RUN_AHEAD] : ~0ull;
  r.nc[RUN_AHEAD - 1] = in && p != 2 ? r.coef[r.cur + RUN_AHEAD] : 1u;
}

__device__ __forceinline__ Run empty_run() {
  Run r;
  r.key = nullptr;
  r.coef = nullptr;
  r.len = r.cur = 0;
  r.scale = 1;
  r.hk = ~0ull;
  r.hc = 0;
#pragma unroll
  for (int i = 0; i < RUN_AHEAD; ++i) {
    r.nk[i] = ~0ull;
    r.nc[i] = 1u;
  }
  return r;
}

// A run over n arena entries.  When the block has the first entries in shared
// memory (sk, sc: the same keys and coefficients), the head and look-ahead are
// taken from there instead of waiting for the arena.
__device__ __forceinline__ Run make_run(const uint64_t* k, const uint32_t* c, uint32_t n, uint32_t scale,
                                        uint32_t p, const uint64_t* sk = nullptr, const uint32_t* sc = nullptr) {
  Run r = empty_run();
  r.key = k;
  r.coef = c;
  r.len = n;
  r.scale = scale;
  if (sk) {
    r.hk = n ? sk[0] : ~0ull;
    r.hc = n ? scaled(sc[0], scale, p) : 0u;
#pragma unroll
    for (int i = 0; i < RUN_AHEAD; ++i) {
      const bool in = 1u + i < n;
      r.nk[i] = in ? sk[1 + i] : ~0ull;
      r.nc[i] = in ? sc[1 + i] : 1u;
    }
  } else {
    run_head(r, p);
  }
  return r;
}

// run_next on the lanes where `at` holds, without a divergent branch: every
// lane computes its next state (its loads stay inside its run) and keeps it or not
__device__ __forceinline__ void advance_if(Run& r, bool at, uint32_t p) {
  Run t = r;
  run_next(t, p);
  if (at) r = t;
}

// combined coefficient of the lanes at the current minimum (`at`)
__device__ __forceinline__ uint32_t warp_coef_sum(bool at, uint32_t hc, uint32_t p) {
  if (p == 2) return __popc(__ballot_sync(0xffffffffu, at)) & 1u;
  return __reduce_add_sync(0xffffffffu, at ? hc : 0u) % p;
}

// size class of the run's remaining entries (-1 when used up)
__device__ __forceinline__ int run_tier(const Run& r) {
  const uint32_t n = r.len - r.cur;
  return n ? (31 - __clz(n)) >> 1 : -1;
}

__device__ __forceinline__ uint64_t warp_min_u64(uint64_t x) {
  const uint32_t hi = __reduce_min_sync(0xffffffffu, (uint32_t)(x >> 32));
  const uint32_t lo = __reduce_min_sync(0xffffffffu, (uint32_t)(x >> 32) == hi ? (uint32_t)x : 0xffffffffu);
  return ((uint64_t)hi << 32) | lo;
}

// arena allocation by lane 0, broadcast; false when the arena is full
__device__ __forceinline__ bool arena_alloc(const RedState& s, int lane, unsigned long long count,
                                            unsigned long long* off) {
  unsigned long long o = 0;
  if (lane == 0) o = atomicAdd(s.r_top, count);
  o = __shfl_sync(0xffffffffu, o, 0);
  *off = o;
  return o + count <= s.r_cap;
}

// per-warp shared-memory tile for sorting generated coboundaries
constexpr uint32_t SORT_TILE = 256;
struct SortTile {
  uint64_t* key;
  uint32_t* coef;
};

// coboundary of the d-simplex (idx, rank), generated, sorted (in the warp's
// shared-memory tile when it fits) and stored in the arena
__device__ bool gen_sorted(const DimArgs& a, const RedState& s, const CV& cv, const Binom& B, int lane,
                           const SortTile& tile, uint64_t idx, bool packed, uint32_t rank, const uint64_t** k,
                           const uint32_t** c, uint32_t* n) {
  unsigned long long off;
  if (s.scr_slice <= SORT_TILE) {
    const uint32_t cnt = gen_coboundary(a, cv, B, lane, idx, packed, rank, 1u, tile.key, tile.coef, SORT_TILE);
    __syncwarp();
    warp_sort_pairs(tile.key, tile.coef, cnt, lane);
    if (!arena_alloc(s, lane, cnt ? cnt : 1, &off)) return false;
    for (uint32_t i = lane; i < cnt; i += 32) {
      s.r_key[off + i] = tile.key[i];
      s.r_coef[off + i] = tile.coef[i];
    }
    __syncwarp();
    *k = s.r_key + off;
    *c = s.r_coef + off;
    *n = cnt;
    return true;
  }
  if (!arena_alloc(s, lane, s.scr_slice, &off)) return false;
  uint64_t* kk = s.r_key + off;
  uint32_t* cc = s.r_coef + off;
  const uint32_t cnt = gen_coboundary(a, cv, B, lane, idx, packed, rank, 1u, kk, cc, s.scr_slice);
  __syncwarp();
  warp_sort_pairs(kk, cc, cnt, lane);
  *k = kk;
  *c = cc;
  *n = cnt;
  return true;
}

// Pivot of the run set: the smallest head key with a nonzero combined
// coefficient.  Heads at a key whose coefficients cancel are advanced.
template <bool Z2>
__device__ __forceinline__ uint64_t runs_pivot(Run& rs, uint32_t p, uint32_t* coef_out) {
  Run r = rs;  // the search works on registers; the chain's copy may live in local memory
  for (;;) {
    const uint64_t m = warp_min_u64(r.hk);
    if (m == ~0ull) {
      rs = r;
      *coef_out = 0;
      return IDX_NONE;
    }
    const bool at = r.hk == m;
    const uint32_t c = warp_coef_sum(at, r.hc, Z2 ? 2u : p);
    if (c) {
      rs = r;
      *coef_out = c;
      return m;
    }
    advance_if(r, at, Z2 ? 2u : p);
  }
}

// move the runs that are not used up to lanes 0 .. nr-1
__device__ void runs_pack(Run& r, int lane, int* nr) {
  const unsigned live = __ballot_sync(0xffffffffu, r.hk != ~0ull);
  const int cnt = __popc(live);
  const int src = lane < cnt ? (int)__fns(live, 0, lane + 1) : lane;
  Run t;
  t.key = (const uint64_t*)__shfl_sync(0xffffffffu, (unsigned long long)r.key, src);
  t.coef = (const uint32_t*)__shfl_sync(0xffffffffu, (unsigned long long)r.coef, src);
  t.len = __shfl_sync(0xffffffffu, r.len, src);
  t.cur = __shfl_sync(0xffffffffu, r.cur, src);
  t.scale = __shfl_sync(0xffffffffu, r.scale, src);
  t.hk = __shfl_sync(0xffffffffu, r.hk, src);
  t.hc = __shfl_sync(0xffffffffu, r.hc, src);
#pragma unroll
  for (int i = 0; i < RUN_AHEAD; ++i) {
    t.nk[i] = __shfl_sync(0xffffffffu, r.nk[i], src);
    t.nc[i] = __shfl_sync(0xffffffffu, r.nc[i], src);
  }
  r = lane < cnt ? t : empty_run();
  *nr = cnt;
}

// Runs to merge now: a size class holding MERGE_GROUP runs (MERGE_GROUP_SHORT
// for the classes of runs shorter than 4^(SHORT_TIERS), where a merge costs
// more than the entries it saves), or, when all 32 lanes are taken, the size
// class holding the most runs (the shortest of those); 0 when none.
constexpr int MERGE_GROUP = 4;
constexpr int MERGE_GROUP_SHORT = 8;
constexpr int SHORT_TIERS = 4;  // runs of fewer than 256 entries

__device__ unsigned runs_merge_mask(const Run& r, int lane, int nr) {
  const int t = lane < nr ? run_tier(r) : -1;
  const unsigned grp = __match_any_sync(0xffffffffu, t >= 0 ? t : -2 - lane);
  const unsigned elig =
      __ballot_sync(0xffffffffu, t >= 0 && __popc(grp) >= (t < SHORT_TIERS ? MERGE_GROUP_SHORT : MERGE_GROUP));
  if (elig) return __shfl_sync(0xffffffffu, grp, __ffs(elig) - 1);
  if (nr == 32) {
    const unsigned score = t >= 0 ? ((unsigned)__popc(grp) << 8) | (255u - (unsigned)t) : 0u;
    const unsigned best = __reduce_max_sync(0xffffffffu, score);
    return __shfl_sync(0xffffffffu, grp, __ffs(__ballot_sync(0xffffffffu, score == best)) - 1);
  }
  return 0;
}

// Merges the runs of the lanes in `mask` (from their cursors) into one run in
// the arena, scale 1, held by the lowest of those lanes; the others are used
// up.  One merged entry per step of the warp.  False when the arena is full.
__device__ bool runs_merge_warp(const RedState& s, Run& r, int lane, uint32_t p, unsigned mask) {
  const bool in = (mask >> lane) & 1u;
  const uint32_t rest = __reduce_add_sync(0xffffffffu, in ? r.len - r.cur : 0u);
  unsigned long long off;
  if (!arena_alloc(s, lane, rest ? rest : 1, &off)) return false;
  uint64_t* ok = s.r_key + off;
  uint32_t* oc = s.r_coef + off;
  uint32_t out = 0;
  for (;;) {
    const uint64_t h = in ? r.hk : ~0ull;
    const uint64_t m = warp_min_u64(h);
    if (m == ~0ull) break;
    const bool at = h == m;
    const uint32_t c = warp_coef_sum(at, r.hc, p);
    advance_if(r, at, p);
    if (c) {
      if (lane == 0) {
        ok[out] = m;
        oc[out] = c;
      }
      ++out;
    }
  }
  __syncwarp();
  if (lane == 0) atomicAdd(s.compacted, (unsigned long long)rest);
  if (lane == __ffs(mask) - 1) r = make_run(ok, oc, out, 1, p);
  else if (in) r = empty_run();
  return true;
}

// State of column j's chain of additions, held by the warp that runs it.
struct Chain {
  Run r;          // this lane's run
  int nr;         // lanes in use
  uint32_t step;  // additions so far
  uint64_t key;   // current pivot, IDX_NONE once the column is zero
  uint32_t coef;
  int64_t owner;  // table owner of the pivot, or -1 to look it up
  bool started;   // R_j's own run is in place
  unsigned long long t0;  // globaltimer when the chain passed 255 additions
};

enum : int { CH_DONE = 0, CH_MERGE = 1, CH_ARENA = 2, CH_LONG = 3, CH_INTERNAL = 4, CH_GEN = 5, CH_GEN_SELF = 6,
             CH_HEAVY = 7 };

// work handed from warp 0 to its block: runs to merge, or a coboundary to generate
struct ChainReq {
  unsigned mask;  // CH_MERGE: lanes of the runs
  uint64_t gidx;  // CH_GEN, CH_GEN_SELF: the simplex (a reference as simplex_vertices takes it)
  uint32_t grank;
  bool gpacked;
};

// R_j <- R_j - lambda C, lambda = pivot coefficient ratio (Algorithm 1): the run
// of C joins the set, then the new pivot is found
__device__ __forceinline__ void chain_add(const DimArgs& a, const RedState& s, Chain& ch, int lane,
                                          const uint64_t* wk, const uint32_t* wc, uint32_t wn, uint32_t wcoef,
                                          const uint64_t* sk = nullptr, const uint32_t* sc = nullptr) {
  const uint32_t lam = (uint32_t)(((uint64_t)ch.coef * mod_inv(wcoef, a.p)) % a.p);
  if (lane == ch.nr) ch.r = make_run(wk, wc, wn, (a.p - lam) % a.p, a.p, sk, sc);
  ++ch.nr;
  ++ch.step;
  if (lane == 0) {
    atomicAdd(s.added, (unsigned long long)wn);
    if ((ch.step & 15) == 0) atomicAdd(s.heartbeat, 1u);  // progress, for the grid barrier
  }
  ch.key = a.p == 2 ? runs_pivot<true>(ch.r, a.p, &ch.coef) : runs_pivot<false>(ch.r, a.p, &ch.coef);
  ch.owner = -1;
}

// Column j adds the columns owning its pivot until the pivot is free, owned by
// a later column, or the column is zero (Algorithm 1's inner loop with R = D V,
// Sections 3.1 and 3.4).  Owners found in the table are stable while the
// reduce phase runs (an owner is never on the reduce list), so the chain may
// take several steps in one round.  A pivot with a zero apparent facet is owned
// by that facet's column (Section 4, "Persistence pairs").  In warp mode a
// chain longer than `limit` additions, or one needing a merge of more than
// DimArgs::merge_max entries, stops with CH_HEAVY before anything is written back:
// the column is then reduced block-wide from its last stored state.  The warp
// merges runs and generates coboundaries itself (block mode: chainb_advance).
__device__ int chain_advance(const DimArgs& a, const RedState& s, const CV& cv, const Binom& B, int lane,
                             const SortTile& tile, uint32_t j, uint64_t jidx, uint32_t jrank, uint32_t cl,
                             uint32_t limit, Chain& ch) {
  for (;;) {
    if (ch.nr == 32) runs_pack(ch.r, lane, &ch.nr);  // every lane taken: drop the used-up runs
    const unsigned mm = runs_merge_mask(ch.r, lane, ch.nr);
    if (mm) {
      if (__reduce_add_sync(0xffffffffu, (mm >> lane) & 1u ? ch.r.len - ch.r.cur : 0u) > a.merge_max)
        return CH_HEAVY;
      if (!runs_merge_warp(s, ch.r, lane, a.p, mm)) return CH_ARENA;
      runs_pack(ch.r, lane, &ch.nr);
      continue;
    }
    if (ch.key == IDX_NONE) return CH_DONE;
    if (ch.step > MAX_PIVOT_PASSES) return CH_LONG;
    if ((ch.step & 255) == 255) {  // the chain's wall-clock bound
      const unsigned long long now = __shfl_sync(0xffffffffu, global_ns(), 0);
      if (ch.t0 == 0) ch.t0 = now;
      else if (now - ch.t0 > s.chain_ns) return CH_LONG;
    }
    // the column owning the current pivot: an apparent facet, or the table's owner
    const uint64_t* wk;
    const uint32_t* wc;
    uint32_t wn, wcoef;
    if (ch.owner < 0) {
      uint32_t frank, tcoef, k;
      const uint64_t fidx = pivot_owner(a, s, cv, B, lane, cl, ch.key, &frank, &tcoef, &k);
      if (fidx == IDX_NONE) {
        if (k >= j) return CH_DONE;             // free, or owned by a later column: claim it next round
        if (ch.step >= limit) return CH_HEAVY;  // long chain: a block takes the column over
        ch.owner = k;
        continue;
      }
      if (!gen_sorted(a, s, cv, B, lane, tile, fidx, a.vbits != 0, frank, &wk, &wc, &wn)) return CH_ARENA;
      wcoef = tcoef;
    } else {
      const uint32_t k = (uint32_t)ch.owner;
      // the owner's coefficient, stored run and simplex, read at once
      wcoef = s.piv_coef[k];
      const uint32_t kn = s.r_len[k];
      const unsigned long long ko = s.r_off[k];
      const uint64_t kkey = s.col_keys[k];
      if (kn) {
        wk = s.r_key + ko;
        wc = s.r_coef + ko;
        wn = kn;
      } else {
        const uint64_t kidx = kkey & low_mask(a.col_bits);
        const uint32_t kr = a.rank_max - (uint32_t)((kkey >> a.col_bits) & low_mask(a.rank_bits));
        if (!gen_sorted(a, s, cv, B, lane, tile, kidx, false, kr, &wk, &wc, &wn)) return CH_ARENA;
      }
    }
    // the working column's own entries, on first use
    if (!ch.started) {
      const uint64_t* jk = nullptr;
      const uint32_t* jc = nullptr;
      uint32_t jn = s.r_len[j];
      if (jn) {
        jk = s.r_key + s.r_off[j];
        jc = s.r_coef + s.r_off[j];
      } else if (!gen_sorted(a, s, cv, B, lane, tile, jidx, false, jrank, &jk, &jc, &jn)) {
        return CH_ARENA;
      }
      if (lane == 0) ch.r = make_run(jk, jc, jn, 1, a.p);
      ch.nr = 1;
      ch.started = true;
    }
    chain_add(a, s, ch, lane, wk, wc, wn, wcoef);
  }
}

// Lanes whose runs must be merged before the column is stored as one run (0:
// it already is one run of scale 1).
__device__ __forceinline__ unsigned chain_store_mask(const Chain& ch, int lane) {
  const unsigned live = __ballot_sync(0xffffffffu, lane < ch.nr && ch.r.hk != ~0ull);
  const unsigned scaled = __ballot_sync(0xffffffffu, lane < ch.nr && ch.r.hk != ~0ull && ch.r.scale != 1);
  return (__popc(live) > 1 || scaled) ? live : 0u;
}

// Results of a finished chain: statistics, R_j (lane 0's run after
// chain_store_mask came back 0) when the column changed and is not zero, the
// pivot, and the claim list.
__device__ void chain_finish(const RedState& s, const Chain& ch, int lane, uint32_t j, uint32_t* claim_count) {
  Run r = ch.r;
  const uint32_t src = __ffs(__ballot_sync(0xffffffffu, lane < ch.nr && r.hk != ~0ull)) - 1;
  const unsigned long long off = __shfl_sync(0xffffffffu, (unsigned long long)(r.key + r.cur), src & 31);
  const uint32_t len = __shfl_sync(0xffffffffu, r.len - r.cur, src & 31);
  if (lane != 0) return;
  if (ch.step) {
    s.reduced[j] |= 1;
    atomicAdd(s.steps, (unsigned long long)ch.step);
    atomicMax(s.max_chain, ch.step);
    if (ch.key != IDX_NONE) {
      s.r_off[j] = (unsigned long long)((const uint64_t*)off - s.r_key);
      s.r_len[j] = len;
    }
  }
  s.piv_key[j] = ch.key;
  s.piv_coef[j] = ch.coef;
  if (ch.key != IDX_NONE) s.claim_list[atomicAdd(claim_count, 1u)] = j;
}

// warp mode: run the chain to its end and store the column
__device__ int chain_warp(const DimArgs& a, const RedState& s, const CV& cv, const Binom& B, int lane,
                          const SortTile& tile, uint32_t j, uint64_t jidx, uint32_t jrank, uint32_t cl, uint32_t limit,
                          Chain& ch) {
  int st = chain_advance(a, s, cv, B, lane, tile, j, jidx, jrank, cl, limit, ch);
  if (st != CH_DONE) return st;
  if (ch.step && ch.key != IDX_NONE) {
    const unsigned m = chain_store_mask(ch, lane);
    if (m) {
      if (__reduce_add_sync(0xffffffffu, (m >> lane) & 1u ? ch.r.len - ch.r.cur : 0u) > a.merge_max)
        return CH_HEAVY;
      if (!runs_merge_warp(s, ch.r, lane, a.p, m)) return CH_ARENA;
      runs_pack(ch.r, lane, &ch.nr);
    }
  }
  return CH_DONE;
}

// A warp gives a heavy column up before changing any of its state: the column
// is flagged and queued for a block in the next round.
__device__ __forceinline__ void chain_give_up(const RedState& s, int lane, uint32_t j, uint32_t* heavy_count,
                                              uint32_t* heavy_list) {
  if (lane == 0) {
    s.reduced[j] |= HEAVY;
    heavy_list[atomicAdd(heavy_count, 1u)] = j;
  }
}

__device__ __forceinline__ void chain_error(const DimArgs& a, int st) {
  set_error(a.err, st == CH_ARENA ? ERRF_ARENA : st == CH_LONG ? ERRF_TIMEOUT : ERRF_INTERNAL);
}

// First pivot of column j: the cofacets are scanned in decreasing index order and
// the first with the column's own diameter is the pivot (emergent shortcut,
// Section 3.5); only when there is none is the whole coboundary scanned for its
// oldest entry.  A pivot with a zero apparent facet is eliminated at once.  A
// column with a pivot is appended to the claim list.
__device__ void init_column(const DimArgs& a, const RedState& s, const Binom& B, int lane, const SortTile& tile,
                            uint32_t j, uint32_t* claim_count, uint32_t* heavy_count, uint32_t* heavy_list) {
  const int d = a.d;
  uint64_t idx;
  uint32_t r, cl;
  column_simplex(a, s, j, &idx, &r, &cl);
  const CV cv = cloud_view(a, cl);
  int v[MAX_DIM + 2];
  decode(B, cv.n, idx, d, v);
  uint32_t rj[MAX_DIM + 2];
  int hl;
  // the first cofacet with the column's own diameter is its pivot; with the
  // emergent shortcut switched off the whole coboundary is scanned instead
  const int jv = (a.opts & RIPS_OPT_NO_EMERGENT) ? -1 : first_equal_cofacet(cv, v, d, r, lane, rj, &hl);
  uint64_t key;
  uint32_t coef;
  if (jv >= 0) {
    CofacetSums cs;
    cofacet_sums(B, v, d, cs);
    int c = 0;
    for (int l = 0; l <= d; ++l) c += v[l] > jv;
    const uint64_t tidx = cs.above[c] + B(jv, d + 2 - c) + cs.below[c];
    key = row_key(a, r, tidx);
    coef = ((d - c) & 1) ? a.p - 1 : 1u;
  } else {
    min_entry(a, cv, B, lane, nullptr, nullptr, nullptr, 0, idx, r, 0, false, &key, &coef);
  }
  if (lane == 0) {
    s.r_len[j] = 0;
    s.reduced[j] = 0;
  }
  __syncwarp();
  // during the first phase the table is empty: only apparent facets can own a pivot
  Chain ch{empty_run(), 0, 0, key, coef, -1, false, 0};
  const int st = chain_warp(a, s, cv, B, lane, tile, j, idx, r, cl, ~0u, ch);
  if (st == CH_HEAVY) {  // the block will start over from the first pivot
    if (lane == 0) {
      s.piv_key[j] = key;
      s.piv_coef[j] = coef;
    }
    chain_give_up(s, lane, j, heavy_count, heavy_list);
    return;
  }
  if (st != CH_DONE) {
    chain_error(a, st);  // an arena overflow restarts this dimension with a larger arena
    return;
  }
  chain_finish(s, ch, lane, j, claim_count);
}

// Column j claims its pivot: the smallest ordinal owns it; the loser (j, or the
// displaced former owner) goes to the reduce list.
__device__ __forceinline__ void to_reduce(const RedState& s, uint32_t j, uint32_t* reduce_count, uint32_t* heavy_count,
                                          uint32_t* heavy_list) {
  if (s.reduced[j] & HEAVY) heavy_list[atomicAdd(heavy_count, 1u)] = j;
  else s.reduce_list[atomicAdd(reduce_count, 1u)] = j;
}

__device__ void claim_one(const DimArgs& a, const RedState& s, uint32_t j, uint32_t* reduce_count,
                          uint32_t* heavy_count, uint32_t* heavy_list) {
  const uint64_t key = s.piv_key[j];
  const uint32_t cl = high_part(s.col_keys[j], a.rank_bits + a.col_bits);
  const int64_t slot = table_insert(s.t_keys, s.t_mask, table_key(a, cl, row_key_idx(a, key)));
  if (slot < 0) {
    set_error(a.err, ERRF_TABLE_FULL);
    return;
  }
  const uint32_t old = atomicMin(&s.t_vals[slot], j);
  if (old < j) to_reduce(s, j, reduce_count, heavy_count, heavy_list);
  else if (old != 0xFFFFFFFFu && old != j) to_reduce(s, old, reduce_count, heavy_count, heavy_list);
}

// owner of column j's current pivot in the table, which must precede j
__device__ __forceinline__ int64_t reduce_owner(const DimArgs& a, const RedState& s, uint32_t j, uint32_t cl,
                                                uint64_t key) {
  const int64_t slot = table_find(s.t_keys, s.t_mask, table_key(a, cl, row_key_idx(a, key)));
  const uint32_t k = slot >= 0 ? s.t_vals[slot] : 0xFFFFFFFFu;
  return k < j ? (int64_t)k : -1;
}

// Column j (its pivot owned by an earlier column) reduces as far as it can in
// this round, one warp, at most DimArgs::chain_limit additions, and goes back to
// the claim list unless it became zero.
__device__ void reduce_one(const DimArgs& a, const RedState& s, const Binom& B, int lane, const SortTile& tile,
                           uint32_t j, uint32_t* claim_count, uint32_t* heavy_count, uint32_t* heavy_list) {
  uint64_t jidx;
  uint32_t jr, cl;
  column_simplex(a, s, j, &jidx, &jr, &cl);
  const CV cv = cloud_view(a, cl);
  Chain ch{empty_run(), 0, 0, s.piv_key[j], s.piv_coef[j], -1, false, 0};
  ch.owner = reduce_owner(a, s, j, cl, ch.key);
  if (ch.owner < 0) {
    set_error(a.err, ERRF_INTERNAL);
    return;
  }
  const int st = chain_warp(a, s, cv, B, lane, tile, j, jidx, jr, cl, a.chain_limit, ch);
  if (st == CH_HEAVY) {
    chain_give_up(s, lane, j, heavy_count, heavy_list);
    return;
  }
  if (st != CH_DONE) {
    chain_error(a, st);
    return;
  }
  chain_finish(s, ch, lane, j, claim_count);
}

// ---------------------------------------------------------------- block mode
// When a round has at most one column to reduce per block, each block takes a
// column: warp 0 runs the chain and the pivot search as in warp mode, and the
// merges of runs are done by the whole block, two runs at a time, with a
// block-wide merge of 512 entries per tile.

constexpr uint32_t MERGE_T = 2 * WARPS_PER_BLOCK * 32;  // merged entries per tile, two per thread
constexpr uint32_t FROM_B = 0x80000000u;                // merged entry taken from the second run

struct MergeSmem {
  uint64_t a_key[MERGE_T + 1];
  uint64_t b_key[MERGE_T + 1];
  uint64_t m_key[MERGE_T];
  uint32_t a_coef[MERGE_T + 1];  // coefficients times the run's scale, mod p
  uint32_t b_coef[MERGE_T + 1];
  uint32_t m_val[MERGE_T];  // coefficient, FROM_B set for entries of the second run
  uint32_t warp_sum[WARPS_PER_BLOCK];
  uint32_t split_a, split_b;
};
// the warps' sort tiles, or the block's merge and generation staging area
constexpr size_t RED_SMEM_BYTES = 40 * 1024;
static_assert((size_t)WARPS_PER_BLOCK * SORT_TILE * 12 <= RED_SMEM_BYTES, "sort tiles fit");
static_assert(sizeof(MergeSmem) <= RED_SMEM_BYTES, "merge tile overlays the sort tiles");
static_assert(2 * WARPS_PER_BLOCK * 32 * 24 <= RED_SMEM_BYTES, "small merge fits the sort tiles");

struct RunDesc {
  const uint64_t* key;
  const uint32_t* coef;
  uint32_t len, scale;
};

// a request from warp 0 to the block (see chain_advance), and the block's scratch
struct MergeReq {
  RunDesc d[32];  // runs to merge
  uint32_t n;
  unsigned mask;
  int state;
  uint64_t gidx;  // simplex whose coboundary is to be generated (a reference as simplex_vertices takes it)
  uint32_t grank;
  bool gpacked;
  uint32_t wsum[WARPS_PER_BLOCK];
  uint32_t roff[33];  // run offsets of a merge staged in shared memory
  unsigned long long off;
  uint32_t take;  // the heavy column this block takes next
  // arena slots reserved by this block for generated coboundaries and not yet used
  unsigned long long chunk_off, chunk_left;
  // the simplex whose coboundary the block generates, set up by warp 0
  int gv[MAX_DIM + 2];
  CofacetSums gcs;
  uint32_t gbeg, gend;
};

}  // namespace

// A large run merge shared out (block_merge_helped): the block that owns it
// opens a job in a free slot of the help board, and blocks waiting at the grid
// barrier claim its chunks, first to merge them (phase 1), then to copy their
// merged entries into place (phase 2).  A claim packs the job with the chunk,
// so a claim that succeeds pins the job: it cannot close before that chunk is
// done.  The fields every waiting block polls, the claim counters and the
// completion counters sit in separate cache lines.
constexpr int HELP_SLOTS = 8;
struct alignas(128) HelpSlot {
  unsigned job;              // the open job, 0 when none
  unsigned phase;            // 1 merging, 2 copying out
  unsigned K, n, p;
  const uint32_t* bnd;       // chunk boundaries, (K - 1) x n (see block_merge_chunked)
  uint64_t* tk;              // merged chunks, chunk c from inoff[c]
  uint32_t* tc;
  uint64_t* fk;              // the merged run
  uint32_t* fc;
  uint32_t* inoff;           // per chunk: where its input, and its merged entries, start
  uint32_t* kept;            // per chunk: entries kept
  uint32_t* outoff;          // per chunk: where its entries go in the merged run
  alignas(128) unsigned long long next;  // (job << 32) | next chunk to merge
  unsigned long long next2;              // (job << 32) | next chunk to copy out
  alignas(128) unsigned done;            // chunks merged
  unsigned done2;                        // chunks copied out
  alignas(128) unsigned lock;            // owning block + 1, 0 when free
  unsigned jobs;                         // jobs opened in this slot so far
  RunDesc d[32];                         // the runs
};
struct HelpBoard {
  alignas(128) unsigned active;  // bit i: slot i has an open job
  HelpSlot slot[HELP_SLOTS];
};
static_assert(256 + sizeof(HelpBoard) <= LISTS_BYTES, "the help board fits the control block");

namespace {

// Block mode takes arena slots (for generated coboundaries and merges) from a
// block-local chunk of at least GEN_CHUNK entries, so most requests make no
// global atomic.  Called by one thread; the slots start at q.off.  Whether they
// lie inside the arena is checked by the caller (q.off + want <= r_cap).
constexpr unsigned long long GEN_CHUNK = 4096;

__device__ __forceinline__ void block_reserve(const RedState& s, MergeReq& q, unsigned long long want) {
  if (want > q.chunk_left) {
    const unsigned long long grab = want > GEN_CHUNK ? want : GEN_CHUNK;
    q.chunk_off = atomicAdd(s.r_top, grab);
    q.chunk_left = grab;
  }
  q.off = q.chunk_off;
  q.chunk_off += want;
  q.chunk_left -= want;
}

constexpr uint32_t GEN_SMEM_CAP = (uint32_t)(RED_SMEM_BYTES / 12);  // generated entries sorted in shared memory

// ascending bitonic sort of n2 (a power of two) (key, coef) pairs by the whole block
__device__ void block_bitonic(uint64_t* key, uint32_t* coef, uint32_t n2) {
  for (uint32_t k = 2; k <= n2; k <<= 1) {
    for (uint32_t j = k >> 1; j > 0; j >>= 1) {
      for (uint32_t i = threadIdx.x; i < n2; i += blockDim.x) {
        const uint32_t l = i ^ j;
        if (l > i) {
          const uint64_t ki = key[i], kl = key[l];
          if ((ki > kl) == ((i & k) == 0)) {
            key[i] = kl;
            key[l] = ki;
            const uint32_t t = coef[i];
            coef[i] = coef[l];
            coef[l] = t;
          }
        }
      }
      __syncthreads();
    }
  }
}

// Coboundary of the d-simplex (idx, rank) generated by the whole block: each
// thread tests one neighbour of the simplex's vertex with the fewest
// neighbours and a block scan packs the cofacets into shared memory.  Up to
// blockDim.x cofacets are then placed by rank (each thread counts the smaller
// keys; the keys are distinct) straight into their arena slots, reserved at
// the start; more are sorted by a bitonic network (in an arena buffer past
// GEN_SMEM_CAP) and copied.  *out gets the run (scale 1) and *sk, *sc a
// sorted copy in shared memory (null when the sort ran in the arena).  Called by
// the whole block; false (in every thread) when the arena is full.
__device__ bool block_gen_sorted(const DimArgs& a, const RedState& s, const CV& cv, const Binom& B,
                                 unsigned char* raw, MergeReq& q, uint64_t idx, bool packed, uint32_t rank,
                                 RunDesc* out, const uint64_t** sk, const uint32_t** sc) {
  const uint32_t tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int d = a.d;
  // Warp 0 sets the simplex up in shared memory once for the block (no thread
  // keeps its own copy): lane 0 the vertices, then lane l the two binomials
  // of vertex l that the running sums of the cofacet indices add up (a scan
  // each) and the length of its neighbour list (the shortest is scanned).
  if (wid == 0) {
    if (lane == 0) simplex_vertices(B, cv.n, idx, packed, a.vbits, d, q.gv);
    __syncwarp();
    const bool mine = lane <= (uint32_t)d;
    const int vl = mine ? q.gv[lane] : 0;
    const uint64_t up = mine ? B(vl, d + 2 - (int)lane) : 0ull;  // joins above[c] for c > lane
    const uint64_t dn = mine ? B(vl, d + 1 - (int)lane) : 0ull;  // joins below[c] for c <= lane
    const uint32_t o0 = mine ? cv.off[vl] : 0u, o1 = mine ? cv.off[vl + 1] : 0u;
    uint64_t iu = up, idn = dn;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint64_t tu = __shfl_up_sync(0xffffffffu, iu, o);
      const uint64_t td = __shfl_up_sync(0xffffffffu, idn, o);
      if (lane >= (uint32_t)o) {
        iu += tu;
        idn += td;
      }
    }
    const uint64_t dn_all = __shfl_sync(0xffffffffu, idn, 31);
    if (lane <= (uint32_t)d + 1) {
      q.gcs.above[lane] = iu - up;
      q.gcs.below[lane] = dn_all - (idn - dn);
    }
    const uint32_t dg = mine ? o1 - o0 : 0xFFFFFFFFu;
    const uint32_t mdg = __reduce_min_sync(0xffffffffu, dg);
    const int best = __ffs(__ballot_sync(0xffffffffu, mine && dg == mdg)) - 1;
    const uint32_t b0 = __shfl_sync(0xffffffffu, o0, best), b1 = __shfl_sync(0xffffffffu, o1, best);
    if (lane == 0) {
      q.gbeg = b0;
      q.gend = b1;
    }
  }
  __syncthreads();
  const int* v = q.gv;
  const CofacetSums& cs = q.gcs;
  const uint32_t beg = q.gbeg, end = q.gend;
  const uint32_t deg = end - beg;  // at most this many cofacets
  uint32_t p2 = 1;
  while (p2 < deg) p2 <<= 1;
  const bool in_arena = p2 > GEN_SMEM_CAP;
  // the output slots (and the sort buffer when it does not fit in shared memory)
  const unsigned long long want = in_arena ? p2 : (deg ? deg : 1);
  if (tid == 0) block_reserve(s, q, want);
  uint64_t* bk = (uint64_t*)raw;
  uint32_t* bc = (uint32_t*)(raw + (size_t)GEN_SMEM_CAP * 8);
  if (in_arena) {
    __syncthreads();
    if (q.off + want > s.r_cap) return false;
    bk = s.r_key + q.off;
    bc = s.r_coef + q.off;
  }
  uint32_t cnt = 0;
  for (uint32_t q0 = beg; q0 < end; q0 += blockDim.x) {
    const uint32_t qq = q0 + tid;
    uint32_t r = 0;
    uint64_t tidx = 0;
    int c = 0;
    const bool ok = qq < end && cofacet_of(cv, B, v, d, rank, cs, (int)cv.nbr[qq], &r, &tidx, &c);
    const unsigned m = __ballot_sync(0xffffffffu, ok);
    if (lane == 0) q.wsum[wid] = __popc(m);
    __syncthreads();
    uint32_t base = 0, tot = 0;
    for (uint32_t w = 0; w < WARPS_PER_BLOCK; ++w) {
      const uint32_t t = q.wsum[w];
      if (w < wid) base += t;
      tot += t;
    }
    if (ok) {
      const uint32_t pos = cnt + base + __popc(m & ((1u << lane) - 1u));
      bk[pos] = row_key(a, r, tidx);
      bc[pos] = ((d - c) & 1) ? a.p - 1 : 1u;  // the paper's orientation, as in gen_coboundary
    }
    cnt += tot;
    __syncthreads();  // wsum is reused
  }
  if (beg == end) __syncthreads();  // q.off is read below
  const unsigned long long off = q.off;
  if (off + want > s.r_cap) return false;
  if (!in_arena && cnt <= blockDim.x) {
    static_assert(GEN_SMEM_CAP >= 512, "the sorted copy follows the unsorted entries");
    if (tid < cnt) {  // rank placement, into the arena and into a copy past the first blockDim.x entries
      const uint64_t k = bk[tid];
      const uint32_t cf = bc[tid];
      uint32_t rk = 0;
#pragma unroll 8
      for (uint32_t u = 0; u < cnt; ++u) rk += bk[u] < k;
      s.r_key[off + rk] = k;
      s.r_coef[off + rk] = cf;
      bk[blockDim.x + rk] = k;
      bc[blockDim.x + rk] = cf;
    }
    __syncthreads();
    *out = RunDesc{s.r_key + off, s.r_coef + off, cnt, 1};
    *sk = bk + blockDim.x;
    *sc = bc + blockDim.x;
    return true;
  }
  uint32_t n2 = 1;
  while (n2 < cnt) n2 <<= 1;
  for (uint32_t i = cnt + tid; i < n2; i += blockDim.x) {
    bk[i] = ~0ull;
    bc[i] = 0;
  }
  __syncthreads();
  block_bitonic(bk, bc, n2);
  if (in_arena) {
    *out = RunDesc{bk, bc, cnt, 1};
    *sk = nullptr;
    *sc = nullptr;
    return true;
  }
  *sk = bk;
  *sc = bc;
  for (uint32_t i = tid; i < cnt; i += blockDim.x) {
    s.r_key[off + i] = bk[i];
    s.r_coef[off + i] = bc[i];
  }
  __syncthreads();
  *out = RunDesc{s.r_key + off, s.r_coef + off, cnt, 1};
  return true;
}

// out = sa * A + sb * B over Z/p, A and B sorted with distinct keys each;
// entries whose coefficient vanishes are dropped.  Each tile stages the next
// MERGE_T + 1 entries of both runs in shared memory; thread t finds where
// merged entries 2t and 2t+1 come from by a merge-path search (equal keys: A
// first), an A entry followed by a B entry with the same key takes their sum
// and the B entry is dropped, and a block scan packs the nonzero entries.
// Called by the whole block; returns the output length, the same in every
// thread.
__device__ uint32_t block_axpy(MergeSmem& ms, const RunDesc& A, const RunDesc& Bd, uint32_t p, uint64_t* ok,
                               uint32_t* oc) {
  const uint32_t tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const uint32_t na = A.len, nb = Bd.len;
  uint32_t ia = 0, ib = 0, out = 0;
  uint64_t prev = ~0ull;  // key of the previous tile's last merged entry
  while (ia < na || ib < nb) {
    const uint32_t rest = (na - ia) + (nb - ib);
    const uint32_t nout = rest < MERGE_T ? rest : MERGE_T;
    for (uint32_t i = tid; i <= MERGE_T; i += blockDim.x) {
      const bool ha = i < na - ia, hb = i < nb - ib;
      ms.a_key[i] = ha ? A.key[ia + i] : ~0ull;
      ms.a_coef[i] = ha ? (A.coef[ia + i] * A.scale) % p : 0u;
      ms.b_key[i] = hb ? Bd.key[ib + i] : ~0ull;
      ms.b_coef[i] = hb ? (Bd.coef[ib + i] * Bd.scale) % p : 0u;
    }
    __syncthreads();
    const uint32_t q0 = 2 * tid < nout ? 2 * tid : nout;
    const uint32_t q1 = q0 + 2 < nout ? q0 + 2 : nout;
    // x = number of A entries among the first q0 merged ones
    uint32_t lo = 0, hi = q0;
    while (lo < hi) {
      const uint32_t mid = (lo + hi) >> 1;
      if (ms.a_key[mid] <= ms.b_key[q0 - 1 - mid]) lo = mid + 1;
      else hi = mid;
    }
    uint32_t x = lo, y = q0 - lo;
    for (uint32_t q = q0; q < q1; ++q) {
      const uint64_t ka = ms.a_key[x], kb = ms.b_key[y];
      if (ka <= kb) {
        ms.m_key[q] = ka;
        ms.m_val[q] = ms.a_coef[x++];
      } else {
        ms.m_key[q] = kb;
        ms.m_val[q] = FROM_B | ms.b_coef[y++];
      }
    }
    if (q0 < q1 && q1 == nout) {
      ms.split_a = x;
      ms.split_b = y;
    }
    __syncthreads();
    const uint32_t sa = ms.split_a, sb = ms.split_b;
    // the first entry after this tile, when it comes from B
    const uint64_t nk = ms.b_key[sb] < ms.a_key[sa] ? ms.b_key[sb] : ~0ull;
    const uint32_t nv = ms.b_coef[sb];
    uint64_t kk[2];
    uint32_t vv[2];
    uint32_t cnt = 0;
    for (uint32_t q = q0; q < q1; ++q) {
      const uint64_t k = ms.m_key[q];
      const uint32_t v = ms.m_val[q];
      uint32_t c;
      if (v & FROM_B) {
        c = (q ? ms.m_key[q - 1] : prev) == k ? 0u : (v & ~FROM_B);  // already summed into the A entry
      } else {
        c = v;
        if (q + 1 < nout) {
          if ((ms.m_val[q + 1] & FROM_B) && ms.m_key[q + 1] == k) c = (c + (ms.m_val[q + 1] & ~FROM_B)) % p;
        } else if (nk == k) {
          c = (c + nv) % p;
        }
      }
      if (c) {
        kk[cnt] = k;
        vv[cnt] = c;
        ++cnt;
      }
    }
    uint32_t incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= (uint32_t)o) incl += t;
    }
    if (lane == 31) ms.warp_sum[wid] = incl;
    __syncthreads();
    uint32_t base = 0, total = 0;
    for (uint32_t w = 0; w < WARPS_PER_BLOCK; ++w) {
      const uint32_t t = ms.warp_sum[w];
      if (w < wid) base += t;
      total += t;
    }
    const uint32_t pos = out + base + incl - cnt;
    for (uint32_t e = 0; e < cnt; ++e) {
      ok[pos + e] = kk[e];
      oc[pos + e] = vv[e];
    }
    prev = ms.m_key[nout - 1];
    ia += sa;
    ib += sb;
    out += total;
    __syncthreads();  // the windows and sums are overwritten by the next tile
  }
  return out;
}

// The runs of a merge request, summed two at a time (a tree of block_axpy)
// into q.d[0] with scale 1.  Called by the whole block; false (in every
// thread) when the arena is full.
constexpr uint32_t SMALL_MERGE = 2 * WARPS_PER_BLOCK * 32;  // capacity of the rank-count merge
constexpr uint32_t SMALL_MERGE_USE = 128;  // it counts ranks in O(total^2): used up to this size only

// The request's runs when they hold at most SMALL_MERGE entries together: all
// entries are loaded into shared memory at once, each is placed by its rank
// (smaller keys, then equal keys loaded before it), the first of every group of
// equal keys takes the group's coefficient sum, and a block scan packs the
// nonzero ones into the arena.  One pass instead of a tree of tile merges.
__device__ bool block_merge_small(const RedState& s, unsigned char* raw, MergeReq& q, uint32_t p, uint32_t total) {
  const uint32_t tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  uint64_t* sk = (uint64_t*)raw;                                       // loaded keys
  uint64_t* ok = (uint64_t*)(raw + SMALL_MERGE * 8);                   // sorted keys
  uint32_t* sc = (uint32_t*)(raw + SMALL_MERGE * 16);                  // loaded coefficients (scaled)
  uint32_t* oc = (uint32_t*)(raw + SMALL_MERGE * 16 + SMALL_MERGE * 4);  // sorted coefficients
  if (tid == 0) block_reserve(s, q, total ? total : 1);
  for (uint32_t e = tid; e < total; e += blockDim.x) {
    uint32_t r = 0, pre = 0;
    while (e >= pre + q.d[r].len) pre += q.d[r++].len;
    const RunDesc& R = q.d[r];
    sk[e] = R.key[e - pre];
    sc[e] = R.scale == 1 ? R.coef[e - pre] : (R.coef[e - pre] * R.scale) % p;
  }
  __syncthreads();
  for (uint32_t e = tid; e < total; e += blockDim.x) {
    const uint64_t k = sk[e];
    uint32_t rk = 0;
    for (uint32_t u = 0; u < total; ++u) {
      const uint64_t x = sk[u];
      rk += x < k || (x == k && u < e);
    }
    ok[rk] = k;
    oc[rk] = sc[e];
  }
  __syncthreads();
  uint64_t kk[2];
  uint32_t vv[2];
  uint32_t cnt = 0;
  for (uint32_t x = 2 * tid; x < 2 * tid + 2 && x < total; ++x) {
    if (x > 0 && ok[x - 1] == ok[x]) continue;  // summed into the group's first entry
    uint32_t c = 0;
    for (uint32_t y = x; y < total && ok[y] == ok[x]; ++y) c = (c + oc[y]) % p;
    if (c) {
      kk[cnt] = ok[x];
      vv[cnt] = c;
      ++cnt;
    }
  }
  uint32_t incl = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= (uint32_t)o) incl += t;
  }
  if (lane == 31) q.wsum[wid] = incl;
  __syncthreads();
  uint32_t base = 0, kept = 0;
  for (uint32_t w = 0; w < WARPS_PER_BLOCK; ++w) {
    if (w < wid) base += q.wsum[w];
    kept += q.wsum[w];
  }
  const unsigned long long off = q.off;
  if (off + total > s.r_cap) return false;
  for (uint32_t e = 0; e < cnt; ++e) {
    s.r_key[off + base + incl - cnt + e] = kk[e];
    s.r_coef[off + base + incl - cnt + e] = vv[e];
  }
  __syncthreads();
  if (tid == 0) {
    q.d[0] = RunDesc{s.r_key + off, s.r_coef + off, kept, 1};
    atomicAdd(s.compacted, (unsigned long long)total);
  }
  __syncthreads();
  return true;
}

// Entries of one chunk of a block merge: the staged ranges and their merged
// order both live in the block's shared tile.
constexpr uint32_t MID_MERGE = 1536;
static_assert((size_t)MID_MERGE * 24 <= RED_SMEM_BYTES, "two chunk buffers fit the shared tile");

// first position in the sorted keys k[0, len) whose key is >= x
__device__ __forceinline__ uint32_t lower_bound_u64(const uint64_t* k, uint32_t len, uint64_t x) {
  uint32_t lo = 0, hi = len;
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (k[mid] < x) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

constexpr uint32_t BLOCK_T = WARPS_PER_BLOCK * 32;                // threads of a reduction block
constexpr int CHUNK_PER = (int)((MID_MERGE + BLOCK_T - 1) / BLOCK_T);  // staged entries per thread

// Merge the ranges [lo[r], hi[r]) of the request's runs (at most MID_MERGE
// entries together) and append the nonzero sums to (fk, fc) from position
// `out`; returns how many were appended (the same in every thread).  The ranges
// are staged in shared memory as consecutive segments with scaled
// coefficients (every thread issues all its loads before it stores any), then
// merged two segments at a time, ceil(log2 n) rounds
// between two buffers: every thread emits a fixed share of a round's output,
// starting where a merge-path search on its first output puts it (equal keys:
// the earlier segment first).  In the merged order the entries of one key are
// adjacent (at most one per run); the first of each group takes the group's
// coefficient sum, and a block scan packs the nonzero sums.  Called by the
// whole block.
__device__ uint32_t chunk_merge(MergeReq& q, unsigned char* raw, const uint32_t* lo, const uint32_t* hi, uint32_t n,
                                uint32_t p, uint64_t* fk, uint32_t* fc, uint32_t out) {
  const uint32_t tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const ModP mod(p);
  uint64_t* sk = (uint64_t*)raw;
  uint64_t* dk = sk + MID_MERGE;
  uint32_t* sc = (uint32_t*)(raw + (size_t)MID_MERGE * 16);
  uint32_t* dc = sc + MID_MERGE;
  if (wid == 0) {  // segment offsets: a scan over the n <= 32 range lengths
    const uint32_t len = lane < n ? hi[lane] - lo[lane] : 0u;
    uint32_t incl = len;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= (uint32_t)o) incl += t;
    }
    if (lane == 0) q.roff[0] = 0;
    if (lane < n) q.roff[lane + 1] = incl;
  }
  __syncthreads();
  const uint32_t total = q.roff[n];
  {  // the segment of each entry by a binary search over the offsets; every load before any store
    uint32_t seg[CHUNK_PER];
    uint64_t x[CHUNK_PER];
    uint32_t cf[CHUNK_PER];
#pragma unroll
    for (int k = 0; k < CHUNK_PER; ++k) {
      const uint32_t e = tid + (uint32_t)k * BLOCK_T;
      seg[k] = 0;
      x[k] = 0;
      cf[k] = 1u;
      if (e < total) {
        uint32_t a = 0, b = n;  // roff[a] <= e < roff[b]
        while (b - a > 1) {
          const uint32_t m = (a + b) >> 1;
          if (q.roff[m] <= e) a = m;
          else b = m;
        }
        seg[k] = a;
        const RunDesc& R = q.d[a];
        const uint32_t i = lo[a] + e - q.roff[a];
        x[k] = __ldcg(R.key + i);  // through L2: runs may come from other blocks
        if (p != 2) cf[k] = __ldcg(R.coef + i);
      }
    }
#pragma unroll
    for (int k = 0; k < CHUNK_PER; ++k) {
      const uint32_t e = tid + (uint32_t)k * BLOCK_T;
      if (e < total) {
        const uint32_t scale = q.d[seg[k]].scale;
        sk[e] = x[k];
        sc[e] = (p == 2 || scale == 1) ? cf[k] : mod(cf[k] * scale);
      }
    }
  }
  __syncthreads();
  const uint32_t per = (total + blockDim.x - 1) / blockDim.x;
  const uint32_t e0 = tid * per < total ? tid * per : total;
  const uint32_t e1 = e0 + per < total ? e0 + per : total;
  for (uint32_t nseg = n; nseg > 1; nseg = (nseg + 1) / 2) {
    // segments 2g and 2g+1 become one; a last odd segment is copied
    uint32_t e = e0, g = 0;
    while (e < e1) {
      while (q.roff[2 * g + 2 < nseg ? 2 * g + 2 : nseg] <= e) ++g;
      const uint32_t xs = q.roff[2 * g];
      const uint32_t xe = q.roff[2 * g + 1 < nseg ? 2 * g + 1 : nseg];
      const uint32_t ye = q.roff[2 * g + 2 < nseg ? 2 * g + 2 : nseg];
      const uint32_t a = xe - xs, b = ye - xe, dg = e - xs;
      // i = entries of X among the pair's first dg outputs
      uint32_t ilo = dg > b ? dg - b : 0u, ihi = dg < a ? dg : a;
      while (ilo < ihi) {
        const uint32_t mid = (ilo + ihi) >> 1;
        if (sk[xs + mid] <= sk[xe + dg - mid - 1]) ilo = mid + 1;
        else ihi = mid;
      }
      uint32_t i = ilo, j = dg - ilo;
      const uint32_t stop = e1 < ye ? e1 : ye;
      for (; e < stop; ++e) {
        const bool take_x = j >= b || (i < a && sk[xs + i] <= sk[xe + j]);
        const uint32_t src = take_x ? xs + i : xe + j;
        dk[e] = sk[src];
        dc[e] = sc[src];
        if (take_x) ++i;
        else ++j;
      }
    }
    __syncthreads();
    if (wid == 0) {  // the merged pairs are the next round's segments (at most 16 + 1 offsets)
      const uint32_t m = (nseg + 1) / 2;
      const uint32_t v = lane < m ? q.roff[2 * lane] : total;
      __syncwarp();
      if (lane <= m) q.roff[lane] = v;
    }
    uint64_t* tk = sk;
    sk = dk;
    dk = tk;
    uint32_t* tc = sc;
    sc = dc;
    dc = tc;
    __syncthreads();
  }
  // group sums at the first entry of each key (kept in registers: at most
  // CHUNK_PER entries a thread), then pack the nonzero ones
  uint32_t gsum[CHUNK_PER];
  uint32_t cnt = 0;
#pragma unroll
  for (int k = 0; k < CHUNK_PER; ++k) {
    const uint32_t e = e0 + (uint32_t)k;
    gsum[k] = 0;
    if (e < e1 && (e == 0 || sk[e - 1] != sk[e])) {
      const uint64_t key = sk[e];
      uint32_t c = sc[e];
      for (uint32_t x = e + 1; x < total && sk[x] == key; ++x) c = p == 2 ? c ^ sc[x] : mod(c + sc[x]);
      gsum[k] = c;
      cnt += c != 0;
    }
  }
  uint32_t incl = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= (uint32_t)o) incl += t;
  }
  if (lane == 31) q.wsum[wid] = incl;
  __syncthreads();
  uint32_t base = 0, kept = 0;
  for (uint32_t w = 0; w < WARPS_PER_BLOCK; ++w) {
    const uint32_t t = q.wsum[w];
    if (w < wid) base += t;
    kept += t;
  }
  uint32_t o = out + base + incl - cnt;
#pragma unroll
  for (int k = 0; k < CHUNK_PER; ++k) {
    if (gsum[k]) {
      fk[o] = sk[e0 + (uint32_t)k];
      fc[o] = gsum[k];
      ++o;
    }
  }
  __syncthreads();  // the staging area, offsets and sums are reused
  return kept;
}

// ---------------------------------------------------------------- shared-out merges
constexpr uint32_t HELP_MIN_CHUNKS = 4;  // a merge of fewer chunks stays in its block
constexpr unsigned HELP_MIN_IDLE = 8;    // blocks waiting at the grid barrier before a merge is shared out

// Thread 0: claims a chunk of the slot's open job on the counter of its
// current phase; returns it (and the job and phase) or -1.  The chunk may lie
// past the job's last one (the bound read before the claim is not pinned yet):
// callers check it against the job's chunk count read after the claim.
__device__ int help_claim_slot(HelpSlot* hb, unsigned* job, unsigned* phase) {
  const unsigned jb = *(volatile unsigned*)&hb->job;
  if (!jb) return -1;
  __threadfence();
  const unsigned ph = *(volatile unsigned*)&hb->phase;
  const unsigned K = *(volatile unsigned*)&hb->K;
  unsigned long long* ctr = ph == 2 ? &hb->next2 : &hb->next;
  unsigned long long old = *(volatile unsigned long long*)ctr;
  for (int t = 0; t < 64; ++t) {
    if ((unsigned)(old >> 32) != jb || (unsigned)old >= K) return -1;
    const unsigned long long got = atomicCAS(ctr, old, old + 1);
    if (got == old) {
      *job = jb;
      *phase = ph;
      __threadfence();
      return (int)(unsigned)old;
    }
    old = got;
  }
  return -1;
}

// Thread 0 of a waiting block: a chunk of any open job (slots tried from one
// that depends on the block, so waiting blocks spread over the jobs).
__device__ int help_claim(HelpBoard* B, int* slot, unsigned* phase) {
  const unsigned act = *(volatile unsigned*)&B->active;
  if (!act) return -1;
  for (int k = 0; k < HELP_SLOTS; ++k) {
    const int i = (int)((blockIdx.x + (unsigned)k) % HELP_SLOTS);
    if (!((act >> i) & 1u)) continue;
    unsigned jb = 0;
    const int c = help_claim_slot(&B->slot[i], &jb, phase);
    if (c >= 0) {
      *slot = i;
      return c;
    }
  }
  return -1;
}

// The job's fields, as thread 0 reads them once its claim pins the job
struct HelpView {
  uint32_t K, n, p;
  const uint32_t* bnd;
  uint64_t* tk;
  uint32_t* tc;
  uint64_t* fk;
  uint32_t* fc;
  uint32_t* inoff;
  uint32_t* kept;
  uint32_t* outoff;
  uint32_t in;  // the chunk's inoff
};

// The whole block: chunk c of the job (claimed by thread 0 for `phase`):
// phase 1 merges it into the job's chunk area and records its entries kept,
// phase 2 copies its merged entries to their place in the merged run.  The
// block's own request (q.d) takes the job's runs.
__device__ void help_chunk(HelpSlot* hb, unsigned char* raw, MergeReq& q, int c, unsigned phase) {
  const uint32_t tid = threadIdx.x, lane = tid & 31;
  __shared__ HelpView v;
  __shared__ uint32_t hlo[32], hhi[32];
  __shared__ int valid;
  if (tid == 0) {
    volatile HelpSlot* b = hb;
    v.K = b->K;
    v.n = b->n;
    v.p = b->p;
    v.bnd = b->bnd;
    v.tk = b->tk;
    v.tc = b->tc;
    v.fk = b->fk;
    v.fc = b->fc;
    v.inoff = b->inoff;
    v.kept = b->kept;
    v.outoff = b->outoff;
    valid = (uint32_t)c < v.K;
  }
  __syncthreads();
  if (!valid) {
    __syncthreads();  // v and valid are reused by the next claim
    return;
  }
  const uint32_t n = v.n, K = v.K, uc = (uint32_t)c;
  if (phase == 1) {
    if (tid < n) {
      volatile const RunDesc* src = hb->d + tid;
      q.d[tid] = RunDesc{src->key, src->coef, src->len, src->scale};
    }
    __syncthreads();
    if (tid < 32) {
      const uint32_t lo = tid < n && uc ? __ldcg(v.bnd + (size_t)(uc - 1) * n + tid) : 0u;
      const uint32_t hi = tid < n ? (uc + 1 < K ? __ldcg(v.bnd + (size_t)uc * n + tid) : q.d[tid].len) : 0u;
      if (tid < n) {
        hlo[tid] = lo;
        hhi[tid] = hi;
      }
      const uint32_t in = __reduce_add_sync(0xffffffffu, lo);
      if (lane == 0) v.in = in;
    }
    __syncthreads();
    const uint32_t kept = chunk_merge(q, raw, hlo, hhi, n, v.p, v.tk + v.in, v.tc + v.in, 0);
    __threadfence();
    __syncthreads();
    if (tid == 0) {
      v.inoff[uc] = v.in;
      v.kept[uc] = kept;
      __threadfence();
      atomicAdd(&hb->done, 1u);
    }
  } else {
    const uint32_t cnt = __ldcg(v.kept + uc), src = __ldcg(v.inoff + uc), dst = __ldcg(v.outoff + uc);
    for (uint32_t i = tid; i < cnt; i += blockDim.x) {
      v.fk[dst + i] = __ldcg(v.tk + src + i);
      v.fc[dst + i] = __ldcg(v.tc + src + i);
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) atomicAdd(&hb->done2, 1u);
  }
  __syncthreads();  // v, hlo, hhi and valid are reused by the next claim
}

// Thread 0: waits (bounded by limit_ns) until *ctr reaches K; false on timeout.
__device__ bool help_wait(const unsigned* ctr, unsigned K, unsigned long long limit_ns) {
  const unsigned long long t0 = global_ns();
  while (*(volatile const unsigned*)ctr < K) {
    __nanosleep(64);
    if (global_ns() - t0 > limit_ns) return false;
  }
  __threadfence();
  return true;
}

// A merge of K >= HELP_MIN_CHUNKS chunks (boundaries bnd, output fk/fc) shared
// out through the help board while blocks wait at the grid barrier; this block
// takes chunks like any helper.  Returns 1 when the merged run is in q.d[0], 0
// when the arena is full, -2 when the board is taken (the caller merges alone).
// A helper that does not finish within the barrier's wait limit sets
// ERRF_TIMEOUT and leaves an empty run.
__device__ int block_merge_helped(const RedState& s, unsigned char* raw, MergeReq& q, uint32_t p, uint32_t total,
                                  uint32_t K, const uint32_t* bnd, uint64_t* fk, uint32_t* fc) {
  const uint32_t tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const uint32_t n = q.n;
  __shared__ int st, slot;
  __shared__ uint32_t kept_total;
  if (tid == 0) {  // a free slot
    st = -2;
    for (int k = 0; k < HELP_SLOTS && st != 1; ++k) {
      const int i = (int)((blockIdx.x + (unsigned)k) % HELP_SLOTS);
      if (atomicCAS(&s.help->slot[i].lock, 0u, blockIdx.x + 1u) == 0u) {
        st = 1;
        slot = i;
      }
    }
  }
  __syncthreads();
  if (st != 1) return -2;
  HelpSlot* hb = &s.help->slot[slot];
  // room for the merged chunks and three per-chunk counts
  const unsigned long long want = (unsigned long long)total + 3ull * K;
  if (tid == 0) block_reserve(s, q, want);
  __syncthreads();
  const unsigned long long off = q.off;
  if (off + want > s.r_cap) {
    __syncthreads();
    if (tid == 0) atomicExch(&hb->lock, 0u);
    return 0;
  }
  if (tid == 0) {
    const unsigned job = hb->jobs + 1u;
    hb->jobs = job;
    hb->next = (unsigned long long)job << 32;
    hb->next2 = (unsigned long long)job << 32;
    hb->done = 0;
    hb->done2 = 0;
    __threadfence();  // stale claims on an earlier job fail from here on
    hb->K = K;
    hb->n = n;
    hb->p = p;
    hb->bnd = bnd;
    hb->tk = s.r_key + off;
    hb->tc = s.r_coef + off;
    hb->fk = fk;
    hb->fc = fc;
    hb->inoff = s.r_coef + off + total;
    hb->kept = hb->inoff + K;
    hb->outoff = hb->kept + K;
    hb->phase = 1;
  }
  if (tid < n) hb->d[tid] = q.d[tid];
  __threadfence();
  __syncthreads();
  if (tid == 0) {
    atomicExch(&hb->job, (unsigned)(hb->jobs));
    atomicOr(&s.help->active, 1u << slot);
  }
  for (unsigned phase = 1; phase <= 2; ++phase) {
    __shared__ int hc;
    for (;;) {
      if (tid == 0) {
        unsigned jb = 0, ph = 0;
        hc = help_claim_slot(hb, &jb, &ph);
        if (hc >= 0 && ph != phase) hc = -1;  // cannot happen: the phase changes only below
      }
      __syncthreads();
      const int c = hc;
      __syncthreads();
      if (c < 0) break;
      help_chunk(hb, raw, q, c, phase);
    }
    if (tid == 0 && st == 1 && !help_wait(phase == 1 ? &hb->done : &hb->done2, K, s.barrier_ns)) st = 0;
    __syncthreads();
    if (st != 1) break;
    if (phase == 1) {  // where each chunk's entries go: a scan of the kept counts
      uint32_t* kept = s.r_coef + off + total + K;
      uint32_t* outoff = kept + K;
      const uint32_t per = (K + blockDim.x - 1) / blockDim.x;
      const uint32_t c0 = min(tid * per, K), c1 = min(c0 + per, K);
      uint32_t sum = 0;
      for (uint32_t c = c0; c < c1; ++c) sum += __ldcg(kept + c);
      uint32_t incl = sum;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= (uint32_t)o) incl += t;
      }
      if (lane == 31) q.wsum[wid] = incl;
      __syncthreads();
      uint32_t base = 0, all = 0;
      for (uint32_t w = 0; w < WARPS_PER_BLOCK; ++w) {
        if (w < wid) base += q.wsum[w];
        all += q.wsum[w];
      }
      uint32_t o = base + incl - sum;
      for (uint32_t c = c0; c < c1; ++c) {
        outoff[c] = o;
        o += __ldcg(kept + c);
      }
      if (tid == 0) kept_total = all;
      __threadfence();
      __syncthreads();
      if (tid == 0) atomicExch(&hb->phase, 2u);
    }
  }
  if (tid == 0) {
    if (st == 1) {
      atomicAnd(&s.help->active, ~(1u << slot));
      atomicExch(&hb->job, 0u);
      __threadfence();
      atomicExch(&hb->lock, 0u);
      q.d[0] = RunDesc{fk, fc, kept_total, 1};
      atomicAdd(s.compacted, (unsigned long long)total);
    } else {  // a helper overran the wait: the dimension fails; the job stays open
      set_error(s.err, ERRF_TIMEOUT);
      q.d[0] = RunDesc{fk, fc, 0u, 1};
    }
  }
  __syncthreads();
  return 1;
}

constexpr uint32_t MERGE_CHUNKS = 1u << 16;  // most chunks of one big merge (75 M entries at 3/4 full)

constexpr uint32_t SAMPLE_CAP = 2048;  // splitter samples sorted in shared memory

// Chunk boundaries from samples of every run, for runs whose keys are spread
// too unevenly for splitters from the longest one: every run offers the key at
// every G-th position (G >= total / SAMPLE_CAP), the block sorts the samples,
// and every m-th one is a splitter.  A run that offers s samples inside a
// chunk has at most (s + 1) G entries there, and a chunk takes at most m + n - 1
// samples (its m in sorted order, and up to n - 1 copies of its splitter key
// sorted before it), so it holds at most (m + 2n - 1) G <= MID_MERGE.  Returns 1 with the chunk count and the boundaries
// (in fresh arena slots, laid out as block_merge_chunked's), 0 when the arena
// is full, -1 when no sample gap is small enough.  Called by the whole block.
__device__ int sample_splitters(const RedState& s, unsigned char* raw, MergeReq& q, uint32_t total, uint32_t* Kout,
                                uint32_t** bnd_out) {
  const uint32_t tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const uint32_t n = q.n;
  uint32_t G = (total + SAMPLE_CAP - 1) / SAMPLE_CAP;
  if (G < 16) G = 16;
  if ((2 * n + 1) * G > MID_MERGE) return -1;
  const uint32_t m = MID_MERGE / G - 2 * n + 1;
  uint64_t* sk = (uint64_t*)raw;
  uint32_t* sc = (uint32_t*)(raw + (size_t)SAMPLE_CAP * 8);
  if (wid == 0) {  // samples per run (positions G, 2G, ... below its length) and their offsets
    const uint32_t len = lane < n ? q.d[lane].len : 0u;
    const uint32_t cnt = len ? (len - 1) / G : 0u;
    uint32_t incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= (uint32_t)o) incl += t;
    }
    if (lane == 0) q.roff[0] = 0;
    if (lane < n) q.roff[lane + 1] = incl;
  }
  __syncthreads();
  const uint32_t ns = q.roff[n];  // at most total / G <= SAMPLE_CAP
  uint32_t n2 = 1;
  while (n2 < ns) n2 <<= 1;
  for (uint32_t e = tid; e < n2; e += blockDim.x) {
    uint64_t key = ~0ull;
    if (e < ns) {
      uint32_t a = 0, b = n;  // roff[a] <= e < roff[b]
      while (b - a > 1) {
        const uint32_t mid = (a + b) >> 1;
        if (q.roff[mid] <= e) a = mid;
        else b = mid;
      }
      key = __ldcg(q.d[a].key + (size_t)(e - q.roff[a] + 1) * G);
    }
    sk[e] = key;
    sc[e] = 0u;
  }
  __syncthreads();
  block_bitonic(sk, sc, n2);
  const uint32_t K = ns ? (ns + m - 1) / m : 1u;  // splitters sk[m], sk[2m], ..., sk[(K - 1) m]
  const unsigned long long want = (unsigned long long)(K - 1) * n + 1;
  if (tid == 0) block_reserve(s, q, want);
  __syncthreads();
  const unsigned long long off = q.off;
  if (off + want > s.r_cap) return 0;
  uint32_t* bnd = s.r_coef + off;
  for (uint32_t t = tid; t < (K - 1) * n; t += blockDim.x) {
    const uint32_t c = t / n, r = t % n;
    bnd[t] = lower_bound_u64(q.d[r].key, q.d[r].len, sk[(c + 1) * m]);
  }
  __syncthreads();
  *Kout = K;
  *bnd_out = bnd;
  return 1;
}

// The request's runs merged in one pass into one run of scale 1 in q.d[0], in
// chunks of at most MID_MERGE entries: splitters taken every S entries of the
// longest run cut every run into consecutive ranges (one round of binary
// searches, in parallel), and chunk_merge merges the ranges chunk after chunk
// onto the end of the output.  S is sized so that a chunk holds about 3/4 of
// MID_MERGE entries when the runs' keys are spread alike; when a chunk comes
// out too large S is halved (twice at most), and then splitters come from
// samples of every run (sample_splitters).  The next chunk's ranges are read
// while the current one is merged.  Returns 0 (in every thread) when the arena
// is full, -1 when the runs are too unevenly spread for chunks of that size
// (the caller then merges two runs at a time), 1 on success.
__device__ int block_merge_chunked(const RedState& s, unsigned char* raw, MergeReq& q, uint32_t p, uint32_t total) {
  const uint32_t tid = threadIdx.x;
  const uint32_t n = q.n;
  uint32_t L = 0;
  for (uint32_t i = 1; i < n; ++i)
    if (q.d[i].len > q.d[L].len) L = i;
  const uint32_t lenL = q.d[L].len;
  uint32_t S = (uint32_t)((unsigned long long)(MID_MERGE * 3 / 4) * lenL / (total ? total : 1));
  if (S < 16) S = 16;
  constexpr uint32_t T2 = MID_MERGE * 3 / 4;  // entries of a two-run chunk
  uint32_t Kmax = total <= MID_MERGE ? 1u : (lenL + (S >> 2) - 1) / (S >> 2 ? S >> 2 : 1u);
  if (n == 2) Kmax = max(Kmax, (total + T2 - 1) / T2);
  if (Kmax > 4 * MERGE_CHUNKS) return -1;
  // arena: the output and the chunk boundaries (room for the smallest S tried)
  const unsigned long long want = (unsigned long long)total + (unsigned long long)Kmax * n;
  if (tid == 0) block_reserve(s, q, want);
  __syncthreads();
  const unsigned long long off = q.off;
  if (off + want > s.r_cap) return 0;
  // bnd[c * n + r] = where run r enters chunk c + 1
  uint32_t* bnd = s.r_coef + off + total;
  __shared__ int fits;
  uint32_t K = 1;
  if (n == 2 && total > MID_MERGE) {
    // two runs: splitters at merge-path diagonals, every T2 merged entries (the
    // key there, looked up in both runs, keeps equal keys together), so every
    // chunk holds T2 entries, give or take one
    K = (total + T2 - 1) / T2;
    if (K > MERGE_CHUNKS) return -1;
    const RunDesc A = q.d[0], Bd = q.d[1];
    for (uint32_t c = tid; c + 1 < K; c += blockDim.x) {
      const uint32_t dg = (c + 1) * T2;  // below total
      uint32_t lo = dg > Bd.len ? dg - Bd.len : 0u, hi = min(dg, A.len);
      while (lo < hi) {  // A entries among the first dg merged ones (equal keys: A first)
        const uint32_t mid = (lo + hi) >> 1;
        if (A.key[mid] <= Bd.key[dg - mid - 1]) lo = mid + 1;
        else hi = mid;
      }
      const uint32_t i = lo, j = dg - lo;
      const uint64_t x = j >= Bd.len ? A.key[i] : (i >= A.len ? Bd.key[j] : min(A.key[i], Bd.key[j]));
      bnd[c * 2] = lower_bound_u64(A.key, A.len, x);
      bnd[c * 2 + 1] = lower_bound_u64(Bd.key, Bd.len, x);
    }
    if (tid == 0) fits = 1;
    __syncthreads();
  }
  for (int attempt = 0; attempt < 3 && !(n == 2 && total > MID_MERGE); ++attempt, S >>= 1) {
    K = total <= MID_MERGE ? 1u : (lenL + S - 1) / S;
    if (K > MERGE_CHUNKS) return -1;
    for (uint32_t t = tid; t < (K - 1) * n; t += blockDim.x) {
      const uint32_t c = t / n, r = t % n;
      const uint64_t sp = q.d[L].key[(c + 1) * S];
      bnd[t] = r == L ? (c + 1) * S : lower_bound_u64(q.d[r].key, q.d[r].len, sp);
    }
    if (tid == 0) fits = 1;
    __syncthreads();
    for (uint32_t c = tid; c < K; c += blockDim.x) {
      uint32_t sz = 0;
      for (uint32_t r = 0; r < n; ++r) {
        const uint32_t a0 = c ? bnd[(c - 1) * n + r] : 0u, a1 = c + 1 < K ? bnd[c * n + r] : q.d[r].len;
        sz += a1 - a0;
      }
      if (sz > MID_MERGE) fits = 0;
    }
    __syncthreads();
    if (fits || K == 1) break;
    __syncthreads();  // fits is reset by the next attempt
  }
  if (!fits) {  // splitters from samples of every run
    const int r = sample_splitters(s, raw, q, total, &K, &bnd);
    if (r != 1) return r;
  }
  uint64_t* fk = s.r_key + off;
  uint32_t* fc = s.r_coef + off;
  __shared__ int share;  // read by thread 0 for the whole block: the count changes under other blocks
  if (tid == 0) share = s.help && K >= HELP_MIN_CHUNKS && *(volatile const unsigned*)s.idle >= HELP_MIN_IDLE;
  __syncthreads();
  if (share) {
    const int r = block_merge_helped(s, raw, q, p, total, K, bnd, fk, fc);
    if (r != -2) return r;  // else the board is taken: merge here
  }
  __shared__ uint32_t clo[32], chi[32];
  uint32_t out = 0;
  uint32_t nlo = 0, nhi = 0;  // thread r < n: run r's range in the next chunk
  if (tid < n) {
    nlo = 0;
    nhi = K > 1 ? bnd[tid] : q.d[tid].len;
  }
  for (uint32_t c = 0; c < K; ++c) {
    if (tid < n) {
      clo[tid] = nlo;
      chi[tid] = nhi;
      if (c + 1 < K) {  // read ahead
        nlo = nhi;
        nhi = c + 2 < K ? bnd[(c + 1) * n + tid] : q.d[tid].len;
      }
    }
    __syncthreads();
    out += chunk_merge(q, raw, clo, chi, n, p, fk, fc, out);
  }
  if (tid == 0) {
    q.d[0] = RunDesc{fk, fc, out, 1};
    atomicAdd(s.compacted, (unsigned long long)total);
  }
  __syncthreads();
  return 1;
}

__device__ bool block_merge_runs(const RedState& s, MergeSmem& ms, MergeReq& q, uint32_t p) {
  const RunDesc none{nullptr, nullptr, 0, 1};
  uint32_t n = q.n;
  uint32_t total = 0;
  for (uint32_t i = 0; i < n; ++i) total += q.d[i].len;
  if (total <= SMALL_MERGE_USE) return block_merge_small(s, (unsigned char*)&ms, q, p, total);
  {
    const int r = block_merge_chunked(s, (unsigned char*)&ms, q, p, total);
    if (r >= 0) return r == 1;
  }
  // runs too unevenly spread for one pass: merge them two at a time (two-run
  // chunked merges always fit; the tile merge takes small pairs)
  __shared__ RunDesc tree[32];
  if (threadIdx.x < n) tree[threadIdx.x] = q.d[threadIdx.x];
  __syncthreads();
  while (n > 1 || (n == 1 && tree[0].scale != 1)) {
    const uint32_t h = n > 1 ? n >> 1 : 1;
    for (uint32_t i = 0; i < h; ++i) {
      const RunDesc A = tree[2 * i];
      const RunDesc Bd = n > 1 ? tree[2 * i + 1] : none;
      const unsigned long long want = (unsigned long long)A.len + Bd.len;
      if (n > 1 && want > SMALL_MERGE_USE) {
        __syncthreads();  // every thread has read tree[2i], tree[2i + 1]
        if (threadIdx.x == 0) {
          q.d[0] = A;
          q.d[1] = Bd;
          q.n = 2;
        }
        __syncthreads();
        const int r = block_merge_chunked(s, (unsigned char*)&ms, q, p, (uint32_t)want);
        if (r == 0) return false;
        if (r == 1) {
          if (threadIdx.x == 0) tree[i] = q.d[0];
          __syncthreads();
          continue;
        }
      }
      if (threadIdx.x == 0) block_reserve(s, q, want ? want : 1ull);
      __syncthreads();
      const unsigned long long off = q.off;
      if (off + want > s.r_cap) return false;
      const uint32_t len = block_axpy(ms, A, Bd, p, s.r_key + off, s.r_coef + off);
      if (threadIdx.x == 0) {
        tree[i] = RunDesc{s.r_key + off, s.r_coef + off, len, 1};
        atomicAdd(s.compacted, want);
      }
      __syncthreads();
    }
    if (n > 1 && (n & 1)) {
      if (threadIdx.x == 0) tree[h] = tree[n - 1];
      __syncthreads();
    }
    n = n > 1 ? h + (n & 1) : 1;
  }
  if (threadIdx.x == 0) q.d[0] = tree[0];
  __syncthreads();
  return true;
}

// ---------------------------------------------------------------- block mode: ring runs
// In block mode warp 0 runs the chain as in warp mode, but every run's next
// RING_W entries sit in a ring in shared memory (slot = a ring of the block's
// 32): a step of the pivot search reads its heads from shared memory, and a
// run refills its ring with one coalesced warp-wide load every RING_W entries,
// instead of waiting on a global load at every step.
constexpr uint32_t RING_W = 32;  // entries per ring (one per lane for a refill)

struct Rings {
  uint64_t* k;  // 32 slots of RING_W keys
  uint32_t* c;  // and stored coefficients
};

struct RingRun {
  const uint64_t* key;
  const uint32_t* coef;
  uint32_t len, cur, scale;
  uint64_t hk;    // head key, ~0 once the run is used up
  uint64_t nk;    // the key after the head (~0 past the end)
  uint32_t hc;    // head coefficient times scale, mod p
  uint32_t nc;    // and the next one's
  uint32_t wend;  // the ring holds entries [wend - RING_W, wend) of the run (entry i at i mod RING_W)
  uint32_t slot;
};

__device__ __forceinline__ RingRun ring_empty() {
  RingRun r;
  r.key = nullptr;
  r.coef = nullptr;
  r.len = r.cur = r.wend = 0;
  r.scale = 1;
  r.hk = r.nk = ~0ull;
  r.hc = r.nc = 0;
  r.slot = 0;
  return r;
}

// Warp-wide: lane L's run (its fields set, cursor at cur) loads entries
// [cur, cur + RING_W) into its ring, from the shared-memory copy (sk, sc;
// indexed like the run) when there is one, and takes its head and the entry
// after it.
__device__ __forceinline__ void ring_load(const Rings& R, RingRun& r, int lane, int L, uint32_t p,
                                          const uint64_t* sk = nullptr, const uint32_t* sc = nullptr) {
  const uint64_t* kp = (const uint64_t*)__shfl_sync(0xffffffffu, (unsigned long long)r.key, L);
  const uint32_t* cp = (const uint32_t*)__shfl_sync(0xffffffffu, (unsigned long long)r.coef, L);
  const uint32_t base = __shfl_sync(0xffffffffu, r.cur, L);
  const uint32_t len = __shfl_sync(0xffffffffu, r.len, L);
  const uint32_t slot = __shfl_sync(0xffffffffu, r.slot, L);
  const uint32_t i = base + lane;
  if (i < len) {
    const uint32_t at = slot * RING_W + (i & (RING_W - 1));
    R.k[at] = sk ? sk[i] : __ldcg(kp + i);  // through L2: runs may come from other blocks
    R.c[at] = p == 2 ? 1u : (sc ? sc[i] : __ldcg(cp + i));
  }
  __syncwarp();
  if (lane == L) {
    r.wend = min(base + RING_W, len);
    const uint32_t at = r.slot * RING_W + (r.cur & (RING_W - 1));
    const uint32_t nx = r.slot * RING_W + ((r.cur + 1) & (RING_W - 1));
    r.hk = r.cur < r.len ? R.k[at] : ~0ull;
    r.hc = r.cur < r.len ? scaled(R.c[at], r.scale, p) : 0u;
    r.nk = r.cur + 1 < r.len ? R.k[nx] : ~0ull;
    r.nc = r.cur + 1 < r.len ? scaled(R.c[nx], r.scale, p) : 0u;
  }
}

// Warp-wide: a new run over n entries (scale) at lane L, in a free slot.
__device__ __forceinline__ void ring_new(const Rings& R, RingRun& r, int lane, int L, int nr, const uint64_t* k,
                                         const uint32_t* c, uint32_t n, uint32_t scale, uint32_t p,
                                         const uint64_t* sk = nullptr, const uint32_t* sc = nullptr) {
  const unsigned used = __reduce_or_sync(0xffffffffu, lane < nr && lane != L ? 1u << r.slot : 0u);
  if (lane == L) {
    r.key = k;
    r.coef = c;
    r.len = n;
    r.cur = 0;
    r.scale = scale;
    r.slot = __ffs(~used) - 1;
  }
  ring_load(R, r, lane, L, p, sk, sc);
}

// Pivot of the ring runs: the smallest head key with a nonzero combined
// coefficient; heads at a key whose coefficients cancel move on.  One step is a
// 64-bit warp minimum and one warp sum that carries both the coefficient sum
// (over Z/2, compiled separately, the number) of the heads at the minimum and
// the number of those whose ring runs dry when they move on.  The search is
// pipelined: every lane keeps the entry after its head in registers and reads
// the one after that from its ring at the start of a step, and the next
// minimum, on the assumption that the heads at this one cancel, is taken while
// the sum is still under way, so a step costs about one minimum.
template <bool Z2>
__device__ __forceinline__ uint64_t ring_pivot(const Rings& R, RingRun& rs, int lane, uint32_t p,
                                                uint32_t* coef_out) {
  RingRun r = rs;  // the search works on registers; the chain's copy may live in local memory
  const ModP mod(Z2 ? 2u : p);
  uint64_t m = warp_min_u64(r.hk);
  for (;;) {
    if (m == ~0ull) {
      rs = r;
      *coef_out = 0;
      return IDX_NONE;
    }
    const uint32_t x = r.slot * RING_W + ((r.cur + 2) & (RING_W - 1));
    const uint64_t nn = R.k[x];  // meaningful if it is in the ring (else the ring is refilled below)
    const bool at = r.hk == m;
    const uint32_t c1 = r.cur + 1;    // the head's index once this lane moves on
    const bool more = c1 + 1 < r.len;  // and an entry follows it
    const bool refill = at && more && c1 + 1 >= r.wend;
    const uint32_t sum = Z2 ? __reduce_add_sync(0xffffffffu, at ? 1u + (refill ? 0x10000u : 0u) : 0u)
                            : __reduce_add_sync(0xffffffffu, at ? r.hc + (refill ? 0x1000000u : 0u) : 0u);
    const uint64_t hk2 = at ? r.nk : r.hk;
    const uint64_t m2 = warp_min_u64(hk2);
    const uint64_t nk2 = at ? (more ? nn : ~0ull) : r.nk;
    uint32_t cs;
    if (Z2) {
      cs = sum & 1u;
    } else {
      cs = mod(sum & 0xFFFFFFu);  // at most 32 (p - 1) < 2^21
    }
    if (cs) {
      rs = r;
      *coef_out = cs;
      return m;
    }
    r.cur = at ? c1 : r.cur;  // no divergent branch: every lane selects
    r.hk = hk2;
    r.nk = nk2;
    if (!Z2) {
      const uint32_t nc2 = more ? mod(R.c[x] * r.scale) : 0u;
      r.hc = at ? r.nc : r.hc;
      r.nc = at ? nc2 : r.nc;
    }
    if (sum >> (Z2 ? 16 : 24)) {  // refill the rings that ran dry (the head stays; the entry after it is reloaded)
      unsigned need = __ballot_sync(0xffffffffu, refill);
      while (need) {
        const int L = __ffs(need) - 1;
        need &= need - 1;
        ring_load(R, r, lane, L, Z2 ? 2u : p);
      }
    }
    m = m2;
  }
}

// move the runs that are not used up to lanes 0 .. nr-1 (rings stay in their slots)
__device__ __forceinline__ void ring_pack(RingRun& r, int lane, int* nr) {
  const unsigned live = __ballot_sync(0xffffffffu, lane < *nr && r.hk != ~0ull);
  const int cnt = __popc(live);
  const int src = lane < cnt ? (int)__fns(live, 0, lane + 1) : lane;
  RingRun t;
  t.key = (const uint64_t*)__shfl_sync(0xffffffffu, (unsigned long long)r.key, src);
  t.coef = (const uint32_t*)__shfl_sync(0xffffffffu, (unsigned long long)r.coef, src);
  t.len = __shfl_sync(0xffffffffu, r.len, src);
  t.cur = __shfl_sync(0xffffffffu, r.cur, src);
  t.scale = __shfl_sync(0xffffffffu, r.scale, src);
  t.hk = __shfl_sync(0xffffffffu, r.hk, src);
  t.nk = __shfl_sync(0xffffffffu, r.nk, src);
  t.hc = __shfl_sync(0xffffffffu, r.hc, src);
  t.nc = __shfl_sync(0xffffffffu, r.nc, src);
  t.wend = __shfl_sync(0xffffffffu, r.wend, src);
  t.slot = __shfl_sync(0xffffffffu, r.slot, src);
  r = lane < cnt ? t : ring_empty();
  *nr = cnt;
}

// size class of a ring run's remaining entries (-1 when used up), as run_tier
__device__ __forceinline__ int ring_tier(const RingRun& r) {
  const uint32_t n = r.len - r.cur;
  return r.hk != ~0ull && n ? (31 - __clz(n)) >> 1 : -1;
}

// runs_merge_mask for ring runs
__device__ __forceinline__ unsigned ring_merge_mask(const RingRun& r, int lane, int nr) {
  const int t = lane < nr ? ring_tier(r) : -1;
  const unsigned grp = __match_any_sync(0xffffffffu, t >= 0 ? t : -2 - lane);
  const unsigned elig =
      __ballot_sync(0xffffffffu, t >= 0 && __popc(grp) >= (t < SHORT_TIERS ? MERGE_GROUP_SHORT : MERGE_GROUP));
  if (elig) return __shfl_sync(0xffffffffu, grp, __ffs(elig) - 1);
  if (nr == 32) {
    const unsigned score = t >= 0 ? ((unsigned)__popc(grp) << 8) | (255u - (unsigned)t) : 0u;
    const unsigned best = __reduce_max_sync(0xffffffffu, score);
    return __shfl_sync(0xffffffffu, grp, __ffs(__ballot_sync(0xffffffffu, score == best)) - 1);
  }
  return 0;
}

// State of a heavy column's chain, held by warp 0 of the block that runs it.
struct ChainB {
  RingRun r;
  int nr;
  uint32_t step;
  uint64_t key;
  uint32_t coef;
  int64_t owner;
  bool started;
  uint32_t pcoef;  // pivot coefficient of the column being generated
  unsigned long long t0;
};

// R_j <- R_j - lambda C (Algorithm 1): C joins as a new run, then the new pivot
__device__ __forceinline__ void chainb_add(const DimArgs& a, const RedState& s, const Rings& R, ChainB& ch, int lane,
                                           const uint64_t* wk, const uint32_t* wc, uint32_t wn, uint32_t wcoef,
                                           const uint64_t* sk = nullptr, const uint32_t* sc = nullptr) {
  const uint32_t lam = (uint32_t)(((uint64_t)ch.coef * mod_inv(wcoef, a.p)) % a.p);
  ring_new(R, ch.r, lane, ch.nr, ch.nr, wk, wc, wn, (a.p - lam) % a.p, a.p, sk, sc);
  ++ch.nr;
  ++ch.step;
  if (lane == 0) {
    atomicAdd(s.added, (unsigned long long)wn);
    if ((ch.step & 15) == 0) atomicAdd(s.heartbeat, 1u);  // progress, for the grid barrier
  }
  ch.key = a.p == 2 ? ring_pivot<true>(R, ch.r, lane, a.p, &ch.coef) : ring_pivot<false>(R, ch.r, lane, a.p, &ch.coef);
  ch.owner = -1;
}

// The block-mode chain (see chain_advance, whose block-mode branches it
// follows): merges and generated coboundaries are handed to the block as
// CH_MERGE, CH_GEN and CH_GEN_SELF requests.
__device__ int chainb_advance(const DimArgs& a, const RedState& s, const CV& cv, const Binom& B, const Rings& R,
                              int lane, uint32_t j, uint32_t cl, ChainB& ch, ChainReq* req, uint64_t jidx,
                              uint32_t jrank) {
  for (;;) {
    if (ch.nr == 32) ring_pack(ch.r, lane, &ch.nr);  // every lane taken: drop the used-up runs
    const unsigned mm = ring_merge_mask(ch.r, lane, ch.nr);
    if (mm) {
      req->mask = mm;
      return CH_MERGE;
    }
    if (ch.key == IDX_NONE) return CH_DONE;
    if (ch.step > MAX_PIVOT_PASSES) return CH_LONG;
    if ((ch.step & 255) == 255) {  // the chain's wall-clock bound
      const unsigned long long now = __shfl_sync(0xffffffffu, global_ns(), 0);
      if (ch.t0 == 0) ch.t0 = now;
      else if (now - ch.t0 > s.chain_ns) return CH_LONG;
    }
    if (!ch.started) {
      const uint32_t jn = s.r_len[j];
      if (!jn) {
        req->gidx = jidx;
        req->grank = jrank;
        req->gpacked = false;
        return CH_GEN_SELF;
      }
      ring_new(R, ch.r, lane, 0, 0, s.r_key + s.r_off[j], s.r_coef + s.r_off[j], jn, 1, a.p);
      ch.nr = 1;
      ch.started = true;
    }
    if (ch.owner < 0) {
      uint32_t frank, tcoef, k;
      const uint64_t fidx = pivot_owner(a, s, cv, B, lane, cl, ch.key, &frank, &tcoef, &k);
      if (fidx == IDX_NONE) {
        if (k >= j) return CH_DONE;  // free, or owned by a later column: claim it next round
        ch.owner = k;
        continue;
      }
      req->gidx = fidx;
      req->grank = frank;
      req->gpacked = a.vbits != 0;
      ch.pcoef = tcoef;
      return CH_GEN;
    }
    const uint32_t k = (uint32_t)ch.owner;
    // the owner's coefficient, stored run and simplex, read at once
    const uint32_t wcoef = s.piv_coef[k];
    const uint32_t kn = s.r_len[k];
    const unsigned long long ko = s.r_off[k];
    const uint64_t kkey = s.col_keys[k];
    if (!kn) {
      const uint64_t kidx = kkey & low_mask(a.col_bits);
      const uint32_t kr = a.rank_max - (uint32_t)((kkey >> a.col_bits) & low_mask(a.rank_bits));
      req->gidx = kidx;
      req->grank = kr;
      req->gpacked = false;
      ch.pcoef = wcoef;
      return CH_GEN;
    }
    chainb_add(a, s, R, ch, lane, s.r_key + ko, s.r_coef + ko, kn, wcoef);
  }
}

__device__ __forceinline__ unsigned chainb_store_mask(const ChainB& ch, int lane) {
  const unsigned live = __ballot_sync(0xffffffffu, lane < ch.nr && ch.r.hk != ~0ull);
  const unsigned sc = __ballot_sync(0xffffffffu, lane < ch.nr && ch.r.hk != ~0ull && ch.r.scale != 1);
  return (__popc(live) > 1 || sc) ? live : 0u;
}

__device__ void chainb_finish(const RedState& s, const ChainB& ch, int lane, uint32_t j, uint32_t* claim_count) {
  const RingRun& r = ch.r;
  const uint32_t src = __ffs(__ballot_sync(0xffffffffu, lane < ch.nr && r.hk != ~0ull)) - 1;
  const unsigned long long off = __shfl_sync(0xffffffffu, (unsigned long long)(r.key + r.cur), src & 31);
  const uint32_t len = __shfl_sync(0xffffffffu, r.len - r.cur, src & 31);
  if (lane != 0) return;
  if (ch.step) {
    s.reduced[j] |= 1;
    atomicAdd(s.steps, (unsigned long long)ch.step);
    atomicMax(s.max_chain, ch.step);
    if (ch.key != IDX_NONE) {
      s.r_off[j] = (unsigned long long)((const uint64_t*)off - s.r_key);
      s.r_len[j] = len;
    }
  }
  s.piv_key[j] = ch.key;
  s.piv_coef[j] = ch.coef;
  if (ch.key != IDX_NONE) s.claim_list[atomicAdd(claim_count, 1u)] = j;
}

// Column j, reduced by the whole block (see block mode): warp 0 runs the chain,
// and the block generates coboundaries and merges runs when warp 0 asks for it.
// The chain has no step limit here.  A heavy column given up by a warp may come
// with a pivot nobody owns yet; the chain then ends at once and claims it.
__device__ void reduce_one_block(const DimArgs& a, const RedState& s, const Binom& B, const Rings& R,
                                 unsigned char* raw, MergeReq& q, uint32_t j, uint32_t* claim_count) {
  const uint32_t tid = threadIdx.x;
  const int lane = tid & 31;
  uint64_t jidx;
  uint32_t jr, cl;
  column_simplex(a, s, j, &jidx, &jr, &cl);
  const CV cv = cloud_view(a, cl);
  ChainB ch{ring_empty(), 0, 0, 0, 0, -1, false, 0, 0};  // meaningful in warp 0 only
  bool finishing = false;
  if (tid < 32) {
    ch.key = s.piv_key[j];
    ch.coef = s.piv_coef[j];
    ch.owner = reduce_owner(a, s, j, cl, ch.key);
  }
  int state = CH_DONE;
  for (;;) {
    if (tid < 32) {
      ChainReq cr{0u, 0ull, 0u, false};
      int st = CH_DONE;
      if (!finishing) st = chainb_advance(a, s, cv, B, R, lane, j, cl, ch, &cr, jidx, jr);
      if (st == CH_DONE && !finishing) {  // the chain ended: R_j must become one run
        finishing = true;
        if (ch.step && ch.key != IDX_NONE) {
          cr.mask = chainb_store_mask(ch, lane);
          if (cr.mask) st = CH_MERGE;
        }
      }
      if (st == CH_MERGE) {
        const unsigned mask = cr.mask;
        if ((mask >> lane) & 1u)
          q.d[__popc(mask & ((1u << lane) - 1u))] =
              RunDesc{ch.r.key + ch.r.cur, ch.r.coef + ch.r.cur, ch.r.len - ch.r.cur, ch.r.scale};
        if (lane == 0) {
          q.n = __popc(mask);
          q.mask = mask;
        }
      }
      if (lane == 0) {
        q.state = st;
        q.gidx = cr.gidx;
        q.grank = cr.grank;
        q.gpacked = cr.gpacked;
      }
    }
    __syncthreads();
    state = q.state;
    if (state == CH_MERGE) {
      if (!block_merge_runs(s, *(MergeSmem*)raw, q, a.p)) {
        state = CH_ARENA;
        break;
      }
      if (tid < 32) {  // the merged run replaces the runs it was made of, in the lowest one's slot
        const unsigned mask = q.mask;
        const int L = __ffs(mask) - 1;
        if (lane == L) {
          ch.r.key = q.d[0].key;
          ch.r.coef = q.d[0].coef;
          ch.r.len = q.d[0].len;
          ch.r.cur = 0;
          ch.r.scale = 1;
        } else if ((mask >> lane) & 1u) {
          ch.r = ring_empty();
        }
        ring_load(R, ch.r, lane, L, a.p);
        ring_pack(ch.r, lane, &ch.nr);
      }
    } else if (state == CH_GEN || state == CH_GEN_SELF) {
      RunDesc g;
      const uint64_t* gk;
      const uint32_t* gc;
      if (!block_gen_sorted(a, s, cv, B, raw, q, q.gidx, q.gpacked, q.grank, &g, &gk, &gc)) {
        state = CH_ARENA;
        break;
      }
      if (tid < 32) {
        if (state == CH_GEN_SELF) {
          ring_new(R, ch.r, lane, 0, 0, g.key, g.coef, g.len, 1, a.p, gk, gc);
          ch.nr = 1;
          ch.started = true;
        } else {
          chainb_add(a, s, R, ch, lane, g.key, g.coef, g.len, ch.pcoef, gk, gc);
        }
      }
    } else {
      break;
    }
  }
  if (tid >= 32) return;
  if (state != CH_DONE) {
    if (lane == 0) chain_error(a, state);
    return;
  }
  chainb_finish(s, ch, lane, j, claim_count);
}


// Grid-wide barrier for a cooperative launch (all blocks co-resident).  The
// wait is bounded: when limit_ns pass with no block making progress
// (the heartbeat counter, bumped by long chains of additions, stands still) the
// block records ERRF_TIMEOUT and returns false, and the caller leaves the
// kernel.  While it waits, a block takes chunks of a merge shared out on the
// help board (block_merge_helped), with its own request and staging area.
__device__ bool grid_barrier(unsigned* count, unsigned* gen, const RedState& s, uint32_t* err, unsigned char* raw,
                             MergeReq& q) {
  __shared__ int ok, st, hc, hp, hs;
  enum { WAIT = 0, DONE = 1, HELP = 2 };
  const unsigned* heartbeat = s.heartbeat;
  const unsigned long long limit_ns = s.barrier_ns;
  __syncthreads();
  unsigned g = 0, hb = 0;
  unsigned long long t0 = 0;
  if (threadIdx.x == 0) {
    ok = 1;
    st = WAIT;
    g = *(volatile unsigned*)gen;
    __threadfence();
    if (atomicAdd(count, 1u) == gridDim.x - 1) {
      atomicExch(count, 0u);
      __threadfence();
      atomicAdd(gen, 1u);
      st = DONE;
    } else {
      t0 = global_ns();
      hb = *(volatile const unsigned*)heartbeat;
    }
  }
  for (;;) {
    if (threadIdx.x == 0 && st != DONE) {
      st = WAIT;
      if (*(volatile unsigned*)gen != g) {
        st = DONE;
      } else {
        unsigned ph = 0;
        int sl = 0;
        const int c = s.help ? help_claim(s.help, &sl, &ph) : -1;
        if (c >= 0) {
          st = HELP;
          hc = c;
          hp = (int)ph;
          hs = sl;
          t0 = global_ns();  // helping is progress
        } else {
          __nanosleep(128);
          const unsigned long long now = global_ns();
          if (now - t0 > limit_ns) {
            const unsigned h = *(volatile const unsigned*)heartbeat;
            if (h != hb) {  // another block is still working
              hb = h;
              t0 = now;
            } else {
              set_error(err, ERRF_TIMEOUT);
              ok = 0;
              st = DONE;
            }
          }
        }
      }
    }
    __syncthreads();
    const int now_st = st;
    if (now_st == DONE) break;
    if (now_st == HELP) help_chunk(&s.help->slot[hs], raw, q, hc, (unsigned)hp);
    __syncthreads();
  }
  if (threadIdx.x == 0) __threadfence();
  __syncthreads();
  return ok != 0;
}

}  // namespace

// The whole reduction of one dimension in one cooperative launch: the first
// pivots of all columns, then claim / reduce rounds separated by grid
// barriers, until no column is left to claim or reduce.  The losers of a
// round's claims are reduced in its reduce phase: heavy columns (flagged when a
// warp gave them up) one block each, the others one warp each, both handed out
// by atomic counters; when all fit, every column gets a block.  Work-list
// counters are double buffered by round parity (ctl[0..1] claim, ctl[2..3]
// reduce, ctl[16..17] heavy); ctl[4..5] are the barrier's counter and
// generation, ctl[6] receives the number of rounds, ctl[12] is the progress
// heartbeat and ctl[18..19] the light and heavy work cursors.
__global__ void __launch_bounds__(256, 2) reduce_persistent_kernel(DimArgs a, RedState s, unsigned* ctl) {
  extern __shared__ uint64_t smem[];
  Binom B = stage_binom(a, smem);
  const int lane = threadIdx.x & 31;
  const uint32_t warp_id = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t threads = gridDim.x * blockDim.x;
  // the warps' sort tiles, or one merge tile for the whole block in block mode
  __shared__ __align__(16) unsigned char red_smem[RED_SMEM_BYTES];
  __shared__ MergeReq req;
  // rings of the block-mode chain's runs
  __shared__ uint64_t ring_k[32 * RING_W];
  __shared__ uint32_t ring_c[32 * RING_W];
  const Rings rings{ring_k, ring_c};
  if (threadIdx.x == 0) req.chunk_left = 0;  // visible to the block after the first grid barrier
  const uint32_t w = threadIdx.x >> 5;
  const SortTile tile{(uint64_t*)red_smem + w * SORT_TILE,
                      (uint32_t*)(red_smem + (size_t)WARPS_PER_BLOCK * SORT_TILE * 8) + w * SORT_TILE};
  unsigned* claim_cnt = ctl;
  unsigned* red_cnt = ctl + 2;
  unsigned* bar_count = ctl + 4;
  unsigned* bar_gen = ctl + 5;
  unsigned* heavy_cnt = ctl + 16;
  unsigned* light_next = ctl + 18;
  unsigned* heavy_next = ctl + 19;
  uint32_t* heavy[2] = {s.heavy_list, s.heavy_list + (size_t)s.ncols + 1};
  const uint32_t ncols = s.ncols_dev ? *s.ncols_dev : s.ncols;

  for (uint32_t j = warp_id; j < ncols; j += warps)
    init_column(a, s, B, lane, tile, j, &claim_cnt[0], &heavy_cnt[0], heavy[0]);
  if (!grid_barrier(bar_count, bar_gen, s, a.err, red_smem, req)) return;
  uint32_t r = 0;
  for (;; ++r) {
    const int src = r & 1, dst = src ^ 1;
    const uint32_t nclaim = *(volatile unsigned*)&claim_cnt[src];
    const uint32_t nqueued = *(volatile unsigned*)&heavy_cnt[src];
    // the error word changes under other blocks: thread 0 reads it for the
    // whole block, so its threads leave the loop together
    __shared__ uint32_t errs_seen;
    if (threadIdx.x == 0) errs_seen = *(volatile uint32_t*)a.err;
    __syncthreads();
    const uint32_t errs = errs_seen;
    if ((nclaim == 0 && nqueued == 0) || (errs & (ERRF_ARENA | ERRF_TIMEOUT | ERRF_INTERNAL | ERRF_TABLE_FULL)))
      break;
    for (uint32_t t = tid; t < nclaim; t += threads)
      claim_one(a, s, s.claim_list[t], &red_cnt[src], &heavy_cnt[src], heavy[src]);
    if (tid == 0) {  // the next round's heavy list and this round's cursors start empty
      heavy_cnt[dst] = 0;
      *light_next = 0;
      *heavy_next = 0;
    }
    if (!grid_barrier(bar_count, bar_gen, s, a.err, red_smem, req)) return;
    if (tid == 0) {
      claim_cnt[src] = 0;
      red_cnt[dst] = 0;
    }
    const uint32_t nred = *(volatile unsigned*)&red_cnt[src];
    const uint32_t nheavy = *(volatile unsigned*)&heavy_cnt[src];
    if (nred + nheavy <= gridDim.x) {  // few columns left: one block per column
      const uint32_t t = blockIdx.x;
      if (t < nheavy) reduce_one_block(a, s, B, rings, red_smem, req, heavy[src][t], &claim_cnt[dst]);
      else if (t < nheavy + nred)
        reduce_one_block(a, s, B, rings, red_smem, req, s.reduce_list[t - nheavy], &claim_cnt[dst]);
    } else {
      for (;;) {  // heavy columns: a block each
        if (threadIdx.x == 0) req.take = atomicAdd(heavy_next, 1u);
        __syncthreads();
        const uint32_t t = req.take;
        __syncthreads();
        if (t >= nheavy) break;
        reduce_one_block(a, s, B, rings, red_smem, req, heavy[src][t], &claim_cnt[dst]);
      }
      for (;;) {  // the others: a warp each
        uint32_t t = 0;
        if (lane == 0) t = atomicAdd(light_next, 1u);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= nred) break;
        reduce_one(a, s, B, lane, tile, s.reduce_list[t], &claim_cnt[dst], &heavy_cnt[dst], heavy[dst]);
      }
    }
    if (!grid_barrier(bar_count, bar_gen, s, a.err, red_smem, req)) return;
  }
  if (tid == 0) ctl[6] = r;
}

// bars of this dimension and the statistics
__global__ void readout_kernel(DimArgs a, RedState s, const float* __restrict__ rank_value,
                               rips_bar_t* __restrict__ bars, uint32_t* __restrict__ nbars, uint32_t bar_cap,
                               unsigned long long* __restrict__ stats, int st_stride) {
  const uint32_t ncols = s.ncols_dev ? *s.ncols_dev : s.ncols;
  for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < ncols; j += gridDim.x * blockDim.x) {
    uint64_t idx;
    uint32_t r, cl;
    column_simplex(a, s, j, &idx, &r, &cl);
    // per-cloud counters: [0] pairs, [1] zero pairs, [2] essential, [3] emergent
    unsigned long long* st = stats + (size_t)cl * st_stride;
    const uint64_t key = s.piv_key[j];
    rips_bar_t b;
    b.dim = a.d;
    b.cloud = (int32_t)cl;
    b.birth = rank_value[r];
    b.birth_simplex = idx;
    if (s.reduced[j] == 0 && key != IDX_NONE) atomicAdd(&st[3], 1ull);
    if (key == IDX_NONE) {
      atomicAdd(&st[2], 1ull);
      b.death = __int_as_float(0x7f800000);
      b.death_simplex = ~0ull;
    } else {
      atomicAdd(&st[0], 1ull);
      const uint32_t tr = row_key_rank(a, key);
      if (tr == r) {
        atomicAdd(&st[1], 1ull);
        continue;
      }
      if (tr > a.rank_max) {  // not a row of this filtration: a broken reduction, not a bar
        set_error(a.err, ERRF_INTERNAL);
        continue;
      }
      b.death = rank_value[tr];
      b.death_simplex = row_key_idx(a, key);
    }
    uint32_t pos = atomicAdd(nbars, 1u);
    if (pos < bar_cap) bars[pos] = b;
  }
}

// ---------------------------------------------------------------- host launchers

static int sm_count() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess || sms < 1)
      sms = 152;
  }
  return sms;
}

// one warp per item, at most per_sm blocks on every SM (the rest loop)
static int grid_for_warps(uint64_t items, int per_sm) {
  uint64_t blocks = (items + WARPS_PER_BLOCK - 1) / WARPS_PER_BLOCK;
  const uint64_t cap = (uint64_t)sm_count() * (uint64_t)(per_sm > 0 ? per_sm : 16);
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  return (int)blocks;
}

static size_t binom_smem(const DimArgs& a) {
  return a.smem_binom ? (size_t)(a.kmax + 1) * (a.bn + 1) * sizeof(uint64_t) : 0;
}

// Opt in to more than 48 KB of shared memory when the kernel's static plus
// dynamic shared memory needs it.  The attributes are queried and set once per
// kernel, device and size, so launches that are being captured into a CUDA
// graph make no such calls.
struct PreparedKernel {
  const void* fn;
  int device;
  size_t smem;
};
static std::mutex g_prep_mu;
static std::vector<PreparedKernel> g_prepared;

template <typename K>
static cudaError_t prepare(K kernel, size_t smem) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> g(g_prep_mu);
  for (const PreparedKernel& pk : g_prepared)
    if (pk.fn == (const void*)kernel && pk.device == dev && pk.smem >= smem) return cudaSuccess;
  cudaFuncAttributes fa;
  e = cudaFuncGetAttributes(&fa, kernel);
  if (e != cudaSuccess) return e;
  if (smem + fa.sharedSizeBytes > 48 * 1024)
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) g_prepared.push_back(PreparedKernel{(const void*)kernel, dev, smem});
  return e;
}

cudaError_t launch_enumerate(const DimArgs& a, const uint64_t* pidx, const uint32_t* prank, uint32_t np,
                             int prev_col_bits, uint64_t* out_idx, uint32_t* out_rank, unsigned long long* count,
                             unsigned long long cap, cudaStream_t st) {
  if (np == 0) return cudaSuccess;
  size_t sm = binom_smem(a);
  cudaError_t e = prepare(enumerate_kernel, sm);
  if (e != cudaSuccess) return e;
  enumerate_kernel<<<grid_for_warps(np, a.scan_blocks_per_sm), 256, sm, st>>>(a, pidx, prank, np, prev_col_bits, out_idx, out_rank, count,
                                                        cap);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_edges_to_simplices(const uint64_t* keys, const uint32_t* erank, uint32_t m, int edge_bits,
                                      int col_bits, uint64_t* sidx, uint32_t* srank, cudaStream_t st) {
  if (m == 0) return cudaSuccess;
  edges_to_simplices_kernel<<<(m + 255) / 256, 256, 0, st>>>(keys, erank, m, edge_bits, col_bits, sidx, srank);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_test(const DimArgs& a, const uint64_t* sidx, const uint32_t* srank, uint32_t ns,
                        const uint8_t* cleared_flag, const uint64_t* prev_keys, uint64_t prev_mask,
                        uint64_t* col_keys, uint32_t* ncols, uint32_t col_cap, unsigned long long* stats,
                        int stats_stride, cudaStream_t st) {
  if (ns == 0) return cudaSuccess;
  size_t sm = binom_smem(a);
  cudaError_t e = prepare(test_kernel, sm);
  if (e != cudaSuccess) return e;
  test_kernel<<<grid_for_warps(ns, a.scan_blocks_per_sm), 256, sm, st>>>(a, sidx, srank, ns, cleared_flag, prev_keys, prev_mask, col_keys,
                                                   ncols, col_cap, stats, stats_stride);
  note_launch();
  return cudaGetLastError();
}

int reduction_blocks(const DimArgs& a, uint32_t ncols) {
  const size_t sm = binom_smem(a);
  if (prepare(reduce_persistent_kernel, sm) != cudaSuccess) return -1;
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -1;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, reduce_persistent_kernel, 256, sm) != cudaSuccess)
    return -1;
  if (per_sm < 1) return -1;
  // as many blocks as fit, up to one per column: block mode takes one column per block
  uint64_t want = ncols;
  if (a.reduce_blocks_per_sm > 0 && a.reduce_blocks_per_sm < per_sm) per_sm = a.reduce_blocks_per_sm;
  uint64_t maxb = (uint64_t)sms * per_sm;
  int blocks = (int)(want < maxb ? want : maxb);
  return blocks < 1 ? 1 : blocks;
}

cudaError_t launch_reduction(const DimArgs& a, const RedState& s, int blocks, unsigned* ctl, cudaStream_t st) {
  if (s.ncols == 0) return cudaSuccess;
  if (blocks < 1) return cudaErrorInvalidValue;
  const size_t sm = binom_smem(a);
  cudaError_t e = prepare(reduce_persistent_kernel, sm);
  if (e != cudaSuccess) return e;
  DimArgs aa = a;
  RedState ss = s;
  void* args[] = {&aa, &ss, &ctl};
  e = cudaLaunchCooperativeKernel((const void*)reduce_persistent_kernel, dim3(blocks), dim3(256), args, sm, st);
  note_launch();
  return e;
}

cudaError_t launch_readout(const DimArgs& a, const RedState& s, const float* rank_value, rips_bar_t* bars,
                           uint32_t* nbars, uint32_t bar_cap, unsigned long long* stats, int stats_stride,
                           cudaStream_t st) {
  if (s.ncols == 0) return cudaSuccess;
  int blocks = (int)((s.ncols + 255) / 256);
  if (blocks > 152 * 8) blocks = 152 * 8;
  readout_kernel<<<blocks, 256, 0, st>>>(a, s, rank_value, bars, nbars, bar_cap, stats, stats_stride);
  note_launch();
  return cudaGetLastError();
}

}  // namespace rips
