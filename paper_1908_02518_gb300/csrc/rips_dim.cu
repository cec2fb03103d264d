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
//                     not in the table).
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
#include "rips_internal.cuh"

namespace rips {

namespace {

constexpr int WARPS_PER_BLOCK = 8;
constexpr uint32_t MAX_PIVOT_PASSES = 1u << 18;  // cancellations in a row before giving up

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
struct CV {
  int n;
  const uint32_t* R;
  const uint32_t* off;
  const uint32_t* nbr;
};

__device__ __forceinline__ CV cloud_view(const DimArgs& a, uint32_t c) {
  const CloudInfo ci = a.clouds[c];
  return CV{ci.n, a.R + ci.roff, a.nbr_off + ci.voff, a.nbr};
}

__device__ __forceinline__ uint64_t low_mask(int bits) { return bits >= 64 ? ~0ull : ((1ull << bits) - 1); }
__device__ __forceinline__ uint32_t high_part(uint64_t x, int bits) { return bits >= 64 ? 0u : (uint32_t)(x >> bits); }

// ---------------------------------------------------------------- simplex helpers

struct Simplex {
  int v[MAX_DIM + 2];  // vertices, decreasing
  uint64_t idx;
  uint32_t rank;
};

__device__ __forceinline__ void decode(const Binom& B, int n, uint64_t N, int d, int* v) {
  int hi = n - 1;
  for (int k = d + 1; k >= 1; --k) {
    int lo = k - 1, h = hi;
    while (lo < h) {
      int mid = (lo + h + 1) >> 1;
      if (B(mid, k) <= N) lo = mid;
      else h = mid - 1;
    }
    v[d + 1 - k] = lo;
    N -= B(lo, k);
    hi = lo - 1;
  }
}

// rank of sigma with vertex v[l] removed, for every l (d >= 1)
__device__ __forceinline__ void ranks_minus_one(const uint32_t* __restrict__ R, int n, const int* v, int d,
                                                uint32_t* out) {
  for (int l = 0; l <= d; ++l) out[l] = 0;
  for (int a = 0; a <= d; ++a)
    for (int b = a + 1; b <= d; ++b) {
      uint32_t r = R[(size_t)v[a] * n + v[b]];
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
  for (int l = 0; l <= d; ++l) {
    uint32_t x = cv.R[(size_t)v[l] * cv.n + j];
    if (x == RANK_INF) return false;
    r = max(r, x);
    c += v[l] > j;
  }
  *rank = r;
  *cpos = c;
  *idx = cs.above[c] + B(j, d + 2 - c) + cs.below[c];
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
        uint32_t x = cv.R[(size_t)v[l] * cv.n + j];
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
        for (int x = 0; x < k; ++x) {
          uint32_t y = cv.R[(size_t)rv[x] * cv.n + u];
          if (y > r) {
            hit = false;
            break;
          }
        }
        // u must not be a vertex of tau (the dropped vertex is excluded by u > drop)
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
          uint32_t x = cv.R[(size_t)v[l] * cv.n + j];
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
  const uint64_t emask = (1ull << eb) - 1;
  const uint64_t c = key >> (32 + eb);
  sidx[e] = (col_bits >= 64 ? 0ull : (c << col_bits)) | (emask - (key & emask));
  srank[e] = erank[e];
}

// ====================================================================== apparent + clearing test

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
    // cofacet side: (sigma, tau) zero apparent pair?
    uint32_t rj[MAX_DIM + 2];
    int hl;
    int j = first_equal_cofacet(cv, v, d, r, lane, rj, &hl);
    if (j >= 0) {
      int app = 0;
      if (lane == hl) {
        uint32_t minus[MAX_DIM + 2];
        ranks_minus_one(cv.R, cv.n, v, d, minus);
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
        continue;
      }
    }
    // facet side (d >= 2; in dimension 1 such edges are spanning-forest edges)
    if (d >= 2) {
      uint32_t minus[MAX_DIM + 2];
      ranks_minus_one(cv.R, cv.n, v, d, minus);
      if (zero_apparent_facet(cv, v, d, r, minus, lane) >= 0) {
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

// pivot-table key of a row: (cloud << row_bits) | local row index
__device__ __forceinline__ uint64_t table_key(const DimArgs& a, uint32_t cloud, uint64_t row_idx) {
  return (a.row_bits >= 64 ? 0ull : ((uint64_t)cloud << a.row_bits)) | row_idx;
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

// Apparent facet of the pivot row tau (a (d+1)-simplex): returns the facet index
// (IDX_NONE if none), its rank and the coefficient of tau in its coboundary.
__device__ uint64_t pivot_apparent_facet(const DimArgs& a, const CV& cv, const Binom& B, int lane, uint64_t key,
                                         uint32_t* frank, uint32_t* tcoef) {
  const int k = a.d + 1;
  const uint64_t tidx = row_key_idx(a, key);
  const uint32_t tr = row_key_rank(a, key);
  int w[MAX_DIM + 2];
  decode(B, cv.n, tidx, k, w);
  uint32_t minus[MAX_DIM + 2];
  ranks_minus_one(cv.R, cv.n, w, k, minus);
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

// ---------------------------------------------------------------- working columns
// A column that has to be reduced keeps R_j = D V_j materialised in the R arena,
// sorted by row key (oldest row first) with nonzero coefficients: the GPU form of
// the paper's working coboundary (Section 4, "Pivot extraction").  Columns that
// never get reduced (apparent, emergent) never build theirs; the coboundary of an
// unreduced owner or of an apparent facet is generated on the fly into a per-warp
// scratch slice and sorted there.

// all cofacets of the d-simplex (idx, rank) with their paper-orientation signs,
// unsorted, into buf; returns the count (warp-uniform)
__device__ uint32_t gen_coboundary(const DimArgs& a, const CV& cv, const Binom& B, int lane, uint64_t idx,
                                   uint32_t rank, uint32_t scale, uint64_t* bkey, uint32_t* bcoef, uint32_t cap) {
  const int d = a.d;
  const unsigned lt = (1u << lane) - 1u;
  int v[MAX_DIM + 2];
  decode(B, cv.n, idx, d, v);
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
// During a chain of additions the working column is a sum of up to 32 sorted
// runs, one per lane, each with its own Z/p scale: R_j's own entries and the
// columns added to it.  Adding a column appends a run (no copy of R_j); the
// pivot is the smallest head key whose combined coefficient is nonzero, found by
// a warp min-reduction, with the heads at a cancelled key advanced (the paper's
// lazily evaluated heap, Section 4 "Pivot extraction").  When all 32 lanes hold
// runs they are merged into one, and at the end of a chain the column is
// written back as a single run so later columns can add it.
struct Run {
  const uint64_t* key;
  const uint32_t* coef;
  uint32_t len, cur, scale;
};

__device__ __forceinline__ uint64_t warp_min_u64(uint64_t x) {
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    const uint64_t y = __shfl_xor_sync(0xffffffffu, x, o);
    x = y < x ? y : x;
  }
  return x;
}

__device__ __forceinline__ uint32_t warp_sum_mod(uint32_t x, uint32_t p) {
#pragma unroll
  for (int o = 16; o; o >>= 1) x = (x + __shfl_xor_sync(0xffffffffu, x, o)) % p;
  return x;
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
                           const SortTile& tile, uint64_t idx, uint32_t rank, const uint64_t** k, const uint32_t** c,
                           uint32_t* n) {
  unsigned long long off;
  if (s.scr_slice <= SORT_TILE) {
    const uint32_t cnt = gen_coboundary(a, cv, B, lane, idx, rank, 1u, tile.key, tile.coef, SORT_TILE);
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
  const uint32_t cnt = gen_coboundary(a, cv, B, lane, idx, rank, 1u, kk, cc, s.scr_slice);
  __syncwarp();
  warp_sort_pairs(kk, cc, cnt, lane);
  *k = kk;
  *c = cc;
  *n = cnt;
  return true;
}

// Pivot of the run set: the smallest head key with a nonzero combined
// coefficient.  Heads at a key whose coefficients cancel are advanced.
__device__ uint64_t runs_pivot(Run& r, uint32_t p, uint32_t* coef_out) {
  for (;;) {
    const uint64_t h = r.cur < r.len ? r.key[r.cur] : ~0ull;
    const uint64_t m = warp_min_u64(h);
    if (m == ~0ull) {
      *coef_out = 0;
      return IDX_NONE;
    }
    const uint32_t mine = h == m ? (uint32_t)(((uint64_t)r.coef[r.cur] * r.scale) % p) : 0u;
    const uint32_t c = warp_sum_mod(mine, p);
    if (c != 0) {
      *coef_out = c;
      return m;
    }
    if (h == m) ++r.cur;  // the key cancels: every run holding it moves on
  }
}

// Merge every run (from its cursor) into one sorted run in the arena; run 0
// becomes that run and the other lanes are emptied.  False when the arena is full.
__device__ bool runs_compact(const RedState& s, Run& r, int lane, uint32_t p, unsigned long long* out_off,
                             uint32_t* out_len) {
  uint32_t rest = r.len - r.cur;
#pragma unroll
  for (int o = 16; o; o >>= 1) rest += __shfl_xor_sync(0xffffffffu, rest, o);
  unsigned long long off;
  if (!arena_alloc(s, lane, rest ? rest : 1, &off)) return false;
  uint64_t* ok = s.r_key + off;
  uint32_t* oc = s.r_coef + off;
  uint32_t out = 0;
  for (;;) {
    const uint64_t h = r.cur < r.len ? r.key[r.cur] : ~0ull;
    const uint64_t m = warp_min_u64(h);
    if (m == ~0ull) break;
    const uint32_t mine = h == m ? (uint32_t)(((uint64_t)r.coef[r.cur] * r.scale) % p) : 0u;
    const uint32_t c = warp_sum_mod(mine, p);
    if (h == m) ++r.cur;
    if (c != 0) {
      if (lane == 0) {
        ok[out] = m;
        oc[out] = c;
      }
      ++out;
    }
  }
  __syncwarp();
  if (lane == 0) atomicAdd(s.compacted, (unsigned long long)rest);
  r.key = ok;
  r.coef = oc;
  r.len = lane == 0 ? out : 0;
  r.cur = 0;
  r.scale = 1;
  *out_off = off;
  *out_len = out;
  return true;
}

// Column j adds the columns owning its pivot until the pivot is free, owned by
// a later column, or the column is zero (Algorithm 1's inner loop with R = D V,
// Sections 3.1 and 3.4).  Owners found in the table are stable while the
// reduce phase runs (an owner is never on the reduce list), so the chain may
// take several steps in one round.  A pivot with a zero apparent facet is owned
// by that facet's column (Section 4, "Persistence pairs").  `owner` is the table
// owner of the current pivot, or -1 to look it up (apparent facets first).
// Returns false on arena overflow.
__device__ bool reduce_chain(const DimArgs& a, const RedState& s, const CV& cv, const Binom& B, int lane,
                             const SortTile& tile, uint32_t j, uint64_t jidx, uint32_t jrank, uint32_t cl,
                             int64_t owner, uint64_t* key, uint32_t* coef) {
  Run r{nullptr, nullptr, 0, 0, 1};
  int nr = 0;  // runs in use (lanes 0 .. nr-1)
  bool changed = false;
  uint32_t step = 0;
  for (; *key != IDX_NONE; ++step) {
    if (step > MAX_PIVOT_PASSES) {
      set_error(a.err, ERRF_TIMEOUT);
      return true;
    }
    // the column owning the current pivot: an apparent facet, or the table's owner
    const uint64_t* wk;
    const uint32_t* wc;
    uint32_t wn, wcoef;
    if (owner < 0) {
      uint32_t frank, tcoef;
      const uint64_t fidx = pivot_apparent_facet(a, cv, B, lane, *key, &frank, &tcoef);
      if (fidx == IDX_NONE) {
        const int64_t slot = table_find(s.t_keys, s.t_mask, table_key(a, cl, row_key_idx(a, *key)));
        const uint32_t k = slot >= 0 ? s.t_vals[slot] : 0xFFFFFFFFu;
        if (k >= j) break;  // free, or owned by a later column: claim it next round
        owner = k;
        continue;
      }
      if (!gen_sorted(a, s, cv, B, lane, tile, fidx, frank, &wk, &wc, &wn)) return false;
      wcoef = tcoef;
    } else {
      const uint32_t k = (uint32_t)owner;
      wcoef = s.piv_coef[k];
      if (s.r_len[k]) {
        wk = s.r_key + s.r_off[k];
        wc = s.r_coef + s.r_off[k];
        wn = s.r_len[k];
      } else {
        uint64_t kidx;
        uint32_t kr, kcl;
        column_simplex(a, s, k, &kidx, &kr, &kcl);
        if (!gen_sorted(a, s, cv, B, lane, tile, kidx, kr, &wk, &wc, &wn)) return false;
      }
    }
    // the working column's own entries, on first use
    if (nr == 0) {
      const uint64_t* jk;
      const uint32_t* jc;
      uint32_t jn;
      if (s.r_len[j]) {
        jk = s.r_key + s.r_off[j];
        jc = s.r_coef + s.r_off[j];
        jn = s.r_len[j];
      } else if (!gen_sorted(a, s, cv, B, lane, tile, jidx, jrank, &jk, &jc, &jn)) {
        return false;
      }
      if (lane == 0) r = Run{jk, jc, jn, 0, 1};
      nr = 1;
    }
    if (nr == 32) {
      unsigned long long o;
      uint32_t l;
      if (!runs_compact(s, r, lane, a.p, &o, &l)) return false;
      nr = 1;
    }
    // R_j <- R_j - lambda R_owner, lambda = pivot coefficient ratio (Algorithm 1)
    const uint32_t lam = (uint32_t)(((uint64_t)(*coef) * mod_inv(wcoef, a.p)) % a.p);
    if (lane == nr) r = Run{wk, wc, wn, 0, (a.p - lam) % a.p};
    ++nr;
    changed = true;
    if (lane == 0) {
      s.reduced[j] = 1;
      atomicAdd(s.steps, 1ull);
    }
    *key = runs_pivot(r, a.p, coef);
    owner = -1;
  }
  if (lane == 0 && step) atomicMax(s.max_chain, step);
  // write the working column back as one run so later columns can add it
  if (changed && *key != IDX_NONE) {
    unsigned long long o;
    uint32_t l;
    if (!runs_compact(s, r, lane, a.p, &o, &l)) return false;
    if (lane == 0) {
      s.r_off[j] = o;
      s.r_len[j] = l;
    }
    __syncwarp();
  }
  return true;
}

// First pivot of column j: the cofacets are scanned in decreasing index order and
// the first with the column's own diameter is the pivot (emergent shortcut,
// Section 3.5); only when there is none is the whole coboundary scanned for its
// oldest entry.  A pivot with a zero apparent facet is eliminated at once.  A
// column with a pivot is appended to the claim list.
__device__ void init_column(const DimArgs& a, const RedState& s, const Binom& B, int lane, const SortTile& tile,
                            uint32_t j, uint32_t* claim_count) {
  const int d = a.d;
  uint64_t idx;
  uint32_t r, cl;
  column_simplex(a, s, j, &idx, &r, &cl);
  const CV cv = cloud_view(a, cl);
  int v[MAX_DIM + 2];
  decode(B, cv.n, idx, d, v);
  uint32_t rj[MAX_DIM + 2];
  int hl;
  const int jv = first_equal_cofacet(cv, v, d, r, lane, rj, &hl);
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
  if (key != IDX_NONE && !reduce_chain(a, s, cv, B, lane, tile, j, idx, r, cl, -1, &key, &coef)) {
    set_error(a.err, ERRF_ARENA);  // the host restarts this dimension with a larger arena
    key = IDX_NONE;
  }
  if (lane == 0) {
    s.piv_key[j] = key;
    s.piv_coef[j] = coef;
    if (key != IDX_NONE) s.claim_list[atomicAdd(claim_count, 1u)] = j;
  }
}

// Column j claims its pivot: the smallest ordinal owns it; the loser (j, or the
// displaced former owner) goes to the reduce list.
__device__ void claim_one(const DimArgs& a, const RedState& s, uint32_t j, uint32_t* reduce_count) {
  const uint64_t key = s.piv_key[j];
  const uint32_t cl = high_part(s.col_keys[j], a.rank_bits + a.col_bits);
  const int64_t slot = table_insert(s.t_keys, s.t_mask, table_key(a, cl, row_key_idx(a, key)));
  if (slot < 0) {
    set_error(a.err, ERRF_TABLE_FULL);
    return;
  }
  const uint32_t old = atomicMin(&s.t_vals[slot], j);
  if (old < j) s.reduce_list[atomicAdd(reduce_count, 1u)] = j;
  else if (old != 0xFFFFFFFFu && old != j) s.reduce_list[atomicAdd(reduce_count, 1u)] = old;
}

// Column j (its pivot owned by an earlier column) reduces as far as it can in
// this round and goes back to the claim list unless it became zero.
__device__ void reduce_one(const DimArgs& a, const RedState& s, const Binom& B, int lane, const SortTile& tile,
                           uint32_t j, uint32_t* claim_count) {
  uint64_t jidx;
  uint32_t jr, cl;
  column_simplex(a, s, j, &jidx, &jr, &cl);
  const CV cv = cloud_view(a, cl);
  uint64_t key = s.piv_key[j];
  uint32_t coef = s.piv_coef[j];
  const int64_t slot = table_find(s.t_keys, s.t_mask, table_key(a, cl, row_key_idx(a, key)));
  if (slot < 0) {
    set_error(a.err, ERRF_INTERNAL);
    return;
  }
  const uint32_t k = s.t_vals[slot];
  if (k >= j) {
    set_error(a.err, ERRF_INTERNAL);
    return;
  }
  if (!reduce_chain(a, s, cv, B, lane, tile, j, jidx, jr, cl, (int64_t)k, &key, &coef)) {
    set_error(a.err, ERRF_ARENA);
    return;
  }
  if (lane == 0) {
    s.piv_key[j] = key;
    s.piv_coef[j] = coef;
    if (key != IDX_NONE) s.claim_list[atomicAdd(claim_count, 1u)] = j;
  }
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

constexpr unsigned long long BARRIER_LIMIT_NS = 30ull * 1000 * 1000 * 1000;  // 30 s

// Grid-wide barrier for a cooperative launch (all blocks co-resident).  The
// wait is bounded: past BARRIER_LIMIT_NS the block records ERRF_TIMEOUT and
// returns false, and the caller leaves the kernel.
__device__ bool grid_barrier(unsigned* count, unsigned* gen, uint32_t* err) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    const unsigned g = *(volatile unsigned*)gen;
    __threadfence();
    if (atomicAdd(count, 1u) == gridDim.x - 1) {
      atomicExch(count, 0u);
      __threadfence();
      atomicAdd(gen, 1u);
    } else {
      const unsigned long long t0 = global_ns();
      while (*(volatile unsigned*)gen == g) {
        __nanosleep(128);
        if (global_ns() - t0 > BARRIER_LIMIT_NS) {
          set_error(err, ERRF_TIMEOUT);
          ok = 0;
          break;
        }
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

}  // namespace

// The whole reduction of one dimension in one cooperative launch: the first
// pivots of all columns, then claim / reduce rounds separated by grid
// barriers, until no column is left to claim.  Work-list counters are double
// buffered by round parity (ctl[0..1] claim, ctl[2..3] reduce); ctl[4..5] are
// the barrier's counter and generation, ctl[6] receives the number of rounds.
__global__ void __launch_bounds__(256) reduce_persistent_kernel(DimArgs a, RedState s, unsigned* ctl) {
  extern __shared__ uint64_t smem[];
  Binom B = stage_binom(a, smem);
  const int lane = threadIdx.x & 31;
  const uint32_t warp_id = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t threads = gridDim.x * blockDim.x;
  __shared__ uint64_t tile_key[WARPS_PER_BLOCK][SORT_TILE];
  __shared__ uint32_t tile_coef[WARPS_PER_BLOCK][SORT_TILE];
  const SortTile tile{tile_key[threadIdx.x >> 5], tile_coef[threadIdx.x >> 5]};
  unsigned* claim_cnt = ctl;
  unsigned* red_cnt = ctl + 2;
  unsigned* bar_count = ctl + 4;
  unsigned* bar_gen = ctl + 5;

  for (uint32_t j = warp_id; j < s.ncols; j += warps) init_column(a, s, B, lane, tile, j, &claim_cnt[0]);
  if (!grid_barrier(bar_count, bar_gen, a.err)) return;
  uint32_t r = 0;
  for (;; ++r) {
    const int src = r & 1, dst = src ^ 1;
    const uint32_t nclaim = *(volatile unsigned*)&claim_cnt[src];
    const uint32_t errs = *(volatile uint32_t*)a.err;
    if (nclaim == 0 || (errs & (ERRF_ARENA | ERRF_TIMEOUT | ERRF_INTERNAL | ERRF_TABLE_FULL))) break;
    for (uint32_t t = tid; t < nclaim; t += threads) claim_one(a, s, s.claim_list[t], &red_cnt[src]);
    if (!grid_barrier(bar_count, bar_gen, a.err)) return;
    if (tid == 0) {
      claim_cnt[src] = 0;
      red_cnt[dst] = 0;
    }
    const uint32_t nred = *(volatile unsigned*)&red_cnt[src];
    for (uint32_t t = warp_id; t < nred; t += warps)
      reduce_one(a, s, B, lane, tile, s.reduce_list[t], &claim_cnt[dst]);
    if (!grid_barrier(bar_count, bar_gen, a.err)) return;
  }
  if (tid == 0) ctl[6] = r;
}

// bars of this dimension and the statistics
__global__ void readout_kernel(DimArgs a, RedState s, const float* __restrict__ rank_value,
                               rips_bar_t* __restrict__ bars, uint32_t* __restrict__ nbars, uint32_t bar_cap,
                               unsigned long long* __restrict__ stats, int st_stride) {
  for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < s.ncols; j += gridDim.x * blockDim.x) {
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
    if (!s.reduced[j] && key != IDX_NONE) atomicAdd(&st[3], 1ull);
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
      b.death = rank_value[tr];
      b.death_simplex = row_key_idx(a, key);
    }
    uint32_t pos = atomicAdd(nbars, 1u);
    if (pos < bar_cap) bars[pos] = b;
  }
}

// ---------------------------------------------------------------- host launchers

static int grid_for_warps(uint64_t items) {
  uint64_t blocks = (items + WARPS_PER_BLOCK - 1) / WARPS_PER_BLOCK;
  if (blocks > 152ull * 16) blocks = 152ull * 16;
  if (blocks < 1) blocks = 1;
  return (int)blocks;
}

static size_t binom_smem(const DimArgs& a) {
  return a.smem_binom ? (size_t)(a.kmax + 1) * (a.bn + 1) * sizeof(uint64_t) : 0;
}

// Opt in to more than 48 KB of shared memory when the kernel's static plus
// dynamic shared memory needs it.
template <typename K>
static cudaError_t prepare(K kernel, size_t smem) {
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
  if (e != cudaSuccess) return e;
  if (smem + fa.sharedSizeBytes > 48 * 1024)
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  return cudaSuccess;
}

cudaError_t launch_enumerate(const DimArgs& a, const uint64_t* pidx, const uint32_t* prank, uint32_t np,
                             int prev_col_bits, uint64_t* out_idx, uint32_t* out_rank, unsigned long long* count,
                             unsigned long long cap, cudaStream_t st) {
  if (np == 0) return cudaSuccess;
  size_t sm = binom_smem(a);
  cudaError_t e = prepare(enumerate_kernel, sm);
  if (e != cudaSuccess) return e;
  enumerate_kernel<<<grid_for_warps(np), 256, sm, st>>>(a, pidx, prank, np, prev_col_bits, out_idx, out_rank, count,
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
  test_kernel<<<grid_for_warps(ns), 256, sm, st>>>(a, sidx, srank, ns, cleared_flag, prev_keys, prev_mask, col_keys,
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
  uint64_t want = ((uint64_t)ncols + WARPS_PER_BLOCK - 1) / WARPS_PER_BLOCK;
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
