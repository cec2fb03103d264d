// One dimension d >= 1 of the cohomology computation (Section 3.3): columns are
// the d-simplices, rows the (d+1)-simplices, columns are processed youngest
// first (diameter down, then index up, Section 3.5 "Shortcuts" and Section 4
// "Pivot extraction"), and a column's pivot is its OLDEST nonzero row (smallest
// diameter, then largest index).
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
//  init_kernel        first pivot of every column.  The cofacets are scanned in
//                     decreasing index order and the first one with the
//                     column's own diameter is the pivot (the emergent-pair
//                     shortcut, Section 3.5); only when there is none is the
//                     whole coboundary scanned for its minimum.
//  claim_kernel       columns claim their pivot in an open-addressing table by
//                     atomicCAS on the key and atomicMin on the column ordinal:
//                     the earliest column in processing order owns a pivot.
//  reduce_kernel      every column whose pivot is owned by an earlier column
//                     adds that column (R_j -= lambda D V_k, V_j -= lambda V_k:
//                     Algorithm 1 with implicit R = D V, Section 3.4) and finds
//                     its next pivot; a pivot with a zero apparent facet is owned
//                     by that facet's implicit column and eliminated at once
//                     (Section 4, "Persistence pairs": apparent pairs are not in
//                     the table).
//
// Parallel reduction and correctness.  Claims and reductions alternate in
// rounds.  A column only ever adds a column that precedes it in processing
// order, so V stays upper unitriangular; pivots only move to younger rows, so
// the rounds end; at the end every nonzero column owns its pivot alone, i.e.
// R = D V is reduced, and by the pivot proposition of Section 3.1 the pairs are
// exactly those of the sequential algorithm (the pairing of a reduced matrix is
// unique).
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
  Binom b{a.binom, a.n + 1};
  if (a.smem_binom) {
    const int total = (a.kmax + 1) * (a.n + 1);
    for (int i = threadIdx.x; i < total; i += blockDim.x) smem[i] = a.binom[i];
    __syncthreads();
    b.t = smem;
  }
  return b;
}

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
__device__ __forceinline__ int min_degree_vertex(const DimArgs& a, const int* v, int cnt) {
  int best = 0;
  uint32_t bd = a.nbr_off[v[0] + 1] - a.nbr_off[v[0]];
  for (int l = 1; l < cnt; ++l) {
    uint32_t dg = a.nbr_off[v[l] + 1] - a.nbr_off[v[l]];
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
__device__ __forceinline__ bool cofacet_of(const DimArgs& a, const Binom& B, const int* v, int d, uint32_t srank,
                                           const CofacetSums& cs, int j, uint32_t* rank, uint64_t* idx, int* cpos) {
  uint32_t r = srank;
  int c = 0;
  for (int l = 0; l <= d; ++l) {
    uint32_t x = a.R[(size_t)v[l] * a.n + j];
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
__device__ int first_equal_cofacet(const DimArgs& a, const int* v, int d, uint32_t srank, int lane,
                                   uint32_t* rj /* d+1, valid on the returned lane */, int* hit_lane) {
  int av = v[min_degree_vertex(a, v, d + 1)];
  const uint32_t beg = a.nbr_off[av], end = a.nbr_off[av + 1];
  for (uint32_t q0 = beg; q0 < end; q0 += 32) {
    const uint32_t q = q0 + lane;
    bool hit = false;
    int j = -1;
    if (q < end) {
      j = (int)a.nbr[q];
      hit = true;
      for (int l = 0; l <= d; ++l) {
        uint32_t x = a.R[(size_t)v[l] * a.n + j];
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
__device__ int zero_apparent_facet(const DimArgs& a, const int* w, int k, uint32_t r, const uint32_t* minus,
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
  int av = rv[min_degree_vertex(a, rv, k)];
  const uint32_t beg = a.nbr_off[av], end = a.nbr_off[av + 1];
  for (uint32_t q0 = beg; q0 < end; q0 += 32) {
    const uint32_t q = q0 + lane;
    bool above = false, hit = false;
    if (q < end) {
      int u = (int)a.nbr[q];
      above = u > drop;
      if (above) {
        hit = true;
        for (int x = 0; x < k; ++x) {
          uint32_t y = a.R[(size_t)rv[x] * a.n + u];
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
                                                        const uint32_t* __restrict__ prank, uint32_t np,
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
    int v[MAX_DIM + 2];
    decode(B, a.n, pidx[s], d - 1, v);
    const uint32_t r0 = prank[s];
    const int top = v[0];
    const int av = v[min_degree_vertex(a, v, d)];
    const uint32_t beg = a.nbr_off[av], end = a.nbr_off[av + 1];
    for (uint32_t q0 = beg; q0 < end; q0 += 32) {
      const uint32_t q = q0 + lane;
      int j = q < end ? (int)a.nbr[q] : -1;
      bool ok = j > top;
      uint32_t r = r0;
      if (ok)
        for (int l = 0; l < d; ++l) {
          uint32_t x = a.R[(size_t)v[l] * a.n + j];
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
            out_idx[pos] = pidx[s] + B(j, d + 1);
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
                                          uint32_t m, uint64_t* __restrict__ sidx, uint32_t* __restrict__ srank) {
  uint32_t e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m) return;
  sidx[e] = 0xFFFFFFFFu - (uint32_t)(keys[e] & 0xFFFFFFFFull);
  srank[e] = erank[e];
}

// ====================================================================== apparent + clearing test

__global__ void __launch_bounds__(256) test_kernel(DimArgs a, const uint64_t* __restrict__ sidx,
                                                   const uint32_t* __restrict__ srank, uint32_t ns,
                                                   const uint8_t* __restrict__ cleared_flag /* d == 1 */,
                                                   const uint64_t* __restrict__ prev_keys, uint64_t prev_mask,
                                                   uint64_t* __restrict__ col_keys, uint32_t* __restrict__ ncols,
                                                   uint32_t col_cap, unsigned long long* __restrict__ st) {
  extern __shared__ uint64_t smem[];
  Binom B = stage_binom(a, smem);
  const int lane = threadIdx.x & 31;
  const int d = a.d;
  const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
  unsigned long long n_cof = 0, n_fac = 0, n_clr = 0;
  for (uint32_t s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; s < ns; s += warps) {
    const uint64_t idx = sidx[s];
    const uint32_t r = srank[s];
    // clearing: pivots of the previous dimension
    bool cleared;
    if (d == 1) cleared = cleared_flag[s] != 0;
    else cleared = prev_keys != nullptr && table_find(prev_keys, prev_mask, idx) >= 0;
    if (cleared) {
      ++n_clr;
      continue;
    }
    int v[MAX_DIM + 2];
    decode(B, a.n, idx, d, v);
    // cofacet side: (sigma, tau) zero apparent pair?
    uint32_t rj[MAX_DIM + 2];
    int hl;
    int j = first_equal_cofacet(a, v, d, r, lane, rj, &hl);
    if (j >= 0) {
      int app = 0;
      if (lane == hl) {
        uint32_t minus[MAX_DIM + 2];
        ranks_minus_one(a.R, a.n, v, d, minus);
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
      ranks_minus_one(a.R, a.n, v, d, minus);
      if (zero_apparent_facet(a, v, d, r, minus, lane) >= 0) {
        ++n_fac;
        continue;
      }
    }
    if (lane == 0) {
      uint32_t pos = atomicAdd(ncols, 1u);
      if (pos < col_cap) {
        const uint64_t key = ((uint64_t)(a.rank_max - r) << a.col_bits) | idx;
        col_keys[pos] = key;
      } else {
        set_error(a.err, ERRF_OUT_OVERFLOW);
      }
    }
  }
  if (lane == 0) {
    if (n_cof) atomicAdd(&st[0], n_cof);
    if (n_fac) atomicAdd(&st[1], n_fac);
    if (n_clr) atomicAdd(&st[2], n_clr);
  }
}

// ====================================================================== reduction

namespace {

__device__ __forceinline__ void column_simplex(const DimArgs& a, const RedState& s, uint32_t j, uint64_t* idx,
                                               uint32_t* rank) {
  const uint64_t key = s.col_keys[j];
  const uint64_t mask = (1ull << a.col_bits) - 1;
  *idx = key & mask;
  *rank = a.rank_max - (uint32_t)(key >> a.col_bits);
}

// Minimum over the cofacet entries of sum_{(s,c) in V} c * delta(s) restricted to
// row keys > after: returns the key (IDX_NONE if none) and the summed
// coefficient at that key (mod p).  Warp-cooperative.
__device__ void min_entry(const DimArgs& a, const Binom& B, int lane, const uint64_t* vidx, const uint32_t* vrank,
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
    decode(B, a.n, sidx, d, v);
    CofacetSums cs;
    cofacet_sums(B, v, d, cs);
    const int av = v[min_degree_vertex(a, v, d + 1)];
    const uint32_t beg = a.nbr_off[av], end = a.nbr_off[av + 1];
    for (uint32_t q = beg + lane; q < end; q += 32) {
      const int j = (int)a.nbr[q];
      uint32_t r;
      uint64_t tidx;
      int c;
      if (!cofacet_of(a, B, v, d, sr, cs, j, &r, &tidx, &c)) continue;
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
__device__ uint64_t pivot_apparent_facet(const DimArgs& a, const Binom& B, int lane, uint64_t key, uint32_t* frank,
                                         uint32_t* tcoef) {
  const int k = a.d + 1;
  const uint64_t tidx = row_key_idx(a, key);
  const uint32_t tr = row_key_rank(a, key);
  int w[MAX_DIM + 2];
  decode(B, a.n, tidx, k, w);
  uint32_t minus[MAX_DIM + 2];
  ranks_minus_one(a.R, a.n, w, k, minus);
  int l = zero_apparent_facet(a, w, k, tr, minus, lane);
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

// V_j <- V_j + lam * W (both sorted by index; e_j / single entries given inline).
// Lane 0 merges into a fresh arena block.  Returns false when the arena is full.
__device__ bool v_axpy(const RedState& s, int lane, uint32_t j, uint64_t jidx, uint32_t jrank, const uint64_t* widx,
                       const uint32_t* wrank, const uint32_t* wcoef, uint32_t wlen, uint32_t lam, uint32_t p) {
  uint32_t ok = 1;
  if (lane == 0) {
    const uint32_t alen = s.v_len[j];
    const uint64_t* aidx = alen ? s.v_idx + s.v_off[j] : &jidx;
    const uint32_t* arank = alen ? s.v_rank + s.v_off[j] : &jrank;
    const uint32_t one = 1;
    const uint32_t* acoef = alen ? s.v_coef + s.v_off[j] : &one;
    const uint32_t na = alen ? alen : 1;
    const unsigned long long need = na + wlen;
    const unsigned long long off = atomicAdd(s.v_top, need);
    if (off + need > s.v_cap) {
      ok = 0;
    } else {
      uint32_t x = 0, y = 0, m = 0;
      while (x < na || y < wlen) {
        uint64_t ii;
        uint32_t rr, cc;
        if (y >= wlen || (x < na && aidx[x] < widx[y])) {
          ii = aidx[x];
          rr = arank[x];
          cc = acoef[x];
          ++x;
        } else if (x >= na || widx[y] < aidx[x]) {
          ii = widx[y];
          rr = wrank[y];
          cc = (uint32_t)(((uint64_t)wcoef[y] * lam) % p);
          ++y;
        } else {
          ii = aidx[x];
          rr = arank[x];
          cc = (uint32_t)((acoef[x] + (uint64_t)wcoef[y] * lam) % p);
          ++x;
          ++y;
        }
        if (cc) {
          s.v_idx[off + m] = ii;
          s.v_rank[off + m] = rr;
          s.v_coef[off + m] = cc;
          ++m;
        }
      }
      __threadfence();
      if (m == 0) {
        // V_j always keeps its diagonal entry; an empty result is a bug
        set_error(s.err, ERRF_INTERNAL);
      } else {
        s.v_off[j] = (uint32_t)off;
        s.v_len[j] = m;
      }
    }
  }
  ok = __shfl_sync(0xffffffffu, ok, 0);
  __syncwarp();
  return ok != 0;
}

// Eliminate the current pivot of column j with the implicit column of a pivot's
// apparent facet as long as there is one, then find the next pivot.  On entry
// *key/*coef hold the current pivot.  Returns 0 normally, 1 on arena overflow.
__device__ int settle_apparent(const DimArgs& a, const RedState& s, const Binom& B, int lane, uint32_t j,
                               uint64_t jidx, uint32_t jrank, uint64_t* key, uint32_t* coef) {
  for (uint32_t pass = 0; *key != IDX_NONE; ++pass) {
    if (pass > MAX_PIVOT_PASSES) {
      set_error(a.err, ERRF_TIMEOUT);
      return 0;
    }
    uint32_t frank, tcoef;
    const uint64_t fidx = pivot_apparent_facet(a, B, lane, *key, &frank, &tcoef);
    if (fidx == IDX_NONE) return 0;
    // R_j -= lam * delta(facet), V_j -= lam * e_facet
    const uint32_t lam = (uint32_t)(((uint64_t)(*coef) * mod_inv(tcoef, a.p)) % a.p);
    const uint32_t neg = (a.p - lam) % a.p;
    const uint32_t one = 1;
    if (!v_axpy(s, lane, j, jidx, jrank, &fidx, &frank, &one, 1, neg, a.p)) return 1;
    if (lane == 0) s.reduced[j] = 1;
    // next pivot: smallest key above the eliminated one with nonzero coefficient
    uint64_t after = *key;
    for (uint32_t it = 0;; ++it) {
      if (it > MAX_PIVOT_PASSES) {
        set_error(a.err, ERRF_TIMEOUT);
        return 0;
      }
      const uint32_t vl = s.v_len[j];
      uint64_t k2;
      uint32_t c2;
      min_entry(a, B, lane, s.v_idx + s.v_off[j], s.v_rank + s.v_off[j], s.v_coef + s.v_off[j], vl, jidx, jrank,
                after, true, &k2, &c2);
      if (k2 == IDX_NONE || c2 != 0) {
        *key = k2;
        *coef = c2;
        break;
      }
      after = k2;
    }
  }
  return 0;
}

}  // namespace

// first pivot of every column (emergent shortcut first), then elimination of
// apparent-facet pivots; columns with a pivot go to the claim list
__global__ void __launch_bounds__(256) init_kernel(DimArgs a, RedState s) {
  extern __shared__ uint64_t smem[];
  Binom B = stage_binom(a, smem);
  const int lane = threadIdx.x & 31;
  const int d = a.d;
  const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; j < s.ncols; j += warps) {
    uint64_t idx;
    uint32_t r;
    column_simplex(a, s, j, &idx, &r);
    int v[MAX_DIM + 2];
    decode(B, a.n, idx, d, v);
    uint32_t rj[MAX_DIM + 2];
    int hl;
    int jv = first_equal_cofacet(a, v, d, r, lane, rj, &hl);
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
      min_entry(a, B, lane, nullptr, nullptr, nullptr, 0, idx, r, 0, false, &key, &coef);
    }
    if (lane == 0) {
      s.v_len[j] = 0;
      s.reduced[j] = 0;
    }
    __syncwarp();
    if (settle_apparent(a, s, B, lane, j, idx, r, &key, &coef)) {
      set_error(a.err, ERRF_ARENA);
      key = IDX_NONE;  // the host aborts this dimension and retries with a larger arena
    }
    if (lane == 0) {
      s.piv_key[j] = key;
      s.piv_coef[j] = coef;
      if (key != IDX_NONE) s.claim_list[atomicAdd(s.claim_count, 1u)] = j;
    }
  }
}

__global__ void claim_kernel(DimArgs a, RedState s, uint32_t count) {
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < count; t += gridDim.x * blockDim.x) {
    const uint32_t j = s.claim_list[t];
    const uint64_t key = s.piv_key[j];
    const int64_t slot = table_insert(s.t_keys, s.t_mask, row_key_idx(a, key));
    if (slot < 0) {
      set_error(a.err, ERRF_TABLE_FULL);
      continue;
    }
    const uint32_t old = atomicMin(&s.t_vals[slot], j);
    if (old < j) s.reduce_list[atomicAdd(s.reduce_count, 1u)] = j;
    else if (old != 0xFFFFFFFFu && old != j) s.reduce_list[atomicAdd(s.reduce_count, 1u)] = old;
  }
}

__global__ void __launch_bounds__(256) reduce_kernel(DimArgs a, RedState s, uint32_t count) {
  extern __shared__ uint64_t smem[];
  Binom B = stage_binom(a, smem);
  const int lane = threadIdx.x & 31;
  const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < count; t += warps) {
    const uint32_t j = s.reduce_list[t];
    uint64_t jidx;
    uint32_t jr;
    column_simplex(a, s, j, &jidx, &jr);
    uint64_t key = s.piv_key[j];
    uint32_t coef = s.piv_coef[j];
    const int64_t slot = table_find(s.t_keys, s.t_mask, row_key_idx(a, key));
    if (slot < 0) {
      set_error(a.err, ERRF_INTERNAL);
      continue;
    }
    const uint32_t k = s.t_vals[slot];
    if (k >= j) {
      set_error(a.err, ERRF_INTERNAL);
      continue;
    }
    // R_j -= lam * D V_k, V_j -= lam * V_k
    const uint32_t lam = (uint32_t)(((uint64_t)coef * mod_inv(s.piv_coef[k], a.p)) % a.p);
    const uint32_t neg = (a.p - lam) % a.p;
    uint64_t kidx;
    uint32_t kr;
    column_simplex(a, s, k, &kidx, &kr);
    const uint32_t kl = s.v_len[k];
    const uint32_t one = 1;
    const uint64_t* wi = kl ? s.v_idx + s.v_off[k] : &kidx;
    const uint32_t* wr = kl ? s.v_rank + s.v_off[k] : &kr;
    const uint32_t* wc = kl ? s.v_coef + s.v_off[k] : &one;
    if (!v_axpy(s, lane, j, jidx, jr, wi, wr, wc, kl ? kl : 1, neg, a.p)) {
      set_error(a.err, ERRF_ARENA);
      if (lane == 0) s.claim_list[atomicAdd(s.claim_count, 1u)] = j;  // unchanged; retried after growth
      continue;
    }
    if (lane == 0) {
      s.reduced[j] = 1;
      atomicAdd(s.steps, 1ull);
    }
    // next pivot after the eliminated row
    uint64_t after = key;
    for (uint32_t it = 0;; ++it) {
      if (it > MAX_PIVOT_PASSES) {
        set_error(a.err, ERRF_TIMEOUT);
        key = IDX_NONE;
        break;
      }
      uint64_t k2;
      uint32_t c2;
      min_entry(a, B, lane, s.v_idx + s.v_off[j], s.v_rank + s.v_off[j], s.v_coef + s.v_off[j], s.v_len[j], jidx,
                jr, after, true, &k2, &c2);
      if (k2 == IDX_NONE || c2 != 0) {
        key = k2;
        coef = c2;
        break;
      }
      after = k2;
    }
    if (settle_apparent(a, s, B, lane, j, jidx, jr, &key, &coef)) {
      set_error(a.err, ERRF_ARENA);
      key = IDX_NONE;
    }
    if (lane == 0) {
      s.piv_key[j] = key;
      s.piv_coef[j] = coef;
      if (key != IDX_NONE) s.claim_list[atomicAdd(s.claim_count, 1u)] = j;
    }
  }
}

// bars of this dimension and the statistics
__global__ void readout_kernel(DimArgs a, RedState s, const float* __restrict__ rank_value, int cloud,
                               rips_bar_t* __restrict__ bars, uint32_t* __restrict__ nbars, uint32_t bar_cap,
                               unsigned long long* __restrict__ st /* pairs, zero, essential, emergent */) {
  for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < s.ncols; j += gridDim.x * blockDim.x) {
    uint64_t idx;
    uint32_t r;
    column_simplex(a, s, j, &idx, &r);
    const uint64_t key = s.piv_key[j];
    rips_bar_t b;
    b.dim = a.d;
    b.cloud = cloud;
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
  return a.smem_binom ? (size_t)(a.kmax + 1) * (a.n + 1) * sizeof(uint64_t) : 0;
}

template <typename K>
static cudaError_t prepare(K kernel, size_t smem) {
  if (smem > 48 * 1024) return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  return cudaSuccess;
}

cudaError_t launch_enumerate(const DimArgs& a, const uint64_t* pidx, const uint32_t* prank, uint32_t np,
                             uint64_t* out_idx, uint32_t* out_rank, unsigned long long* count,
                             unsigned long long cap, cudaStream_t st) {
  if (np == 0) return cudaSuccess;
  size_t sm = binom_smem(a);
  cudaError_t e = prepare(enumerate_kernel, sm);
  if (e != cudaSuccess) return e;
  enumerate_kernel<<<grid_for_warps(np), 256, sm, st>>>(a, pidx, prank, np, out_idx, out_rank, count, cap);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_edges_to_simplices(const uint64_t* keys, const uint32_t* erank, uint32_t m, uint64_t* sidx,
                                      uint32_t* srank, cudaStream_t st) {
  if (m == 0) return cudaSuccess;
  edges_to_simplices_kernel<<<(m + 255) / 256, 256, 0, st>>>(keys, erank, m, sidx, srank);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_test(const DimArgs& a, const uint64_t* sidx, const uint32_t* srank, uint32_t ns,
                        const uint8_t* cleared_flag, const uint64_t* prev_keys, uint64_t prev_mask,
                        uint64_t* col_keys, uint32_t* ncols, uint32_t col_cap, unsigned long long* stats,
                        cudaStream_t st) {
  if (ns == 0) return cudaSuccess;
  size_t sm = binom_smem(a);
  cudaError_t e = prepare(test_kernel, sm);
  if (e != cudaSuccess) return e;
  test_kernel<<<grid_for_warps(ns), 256, sm, st>>>(a, sidx, srank, ns, cleared_flag, prev_keys, prev_mask, col_keys,
                                                   ncols, col_cap, stats);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_init(const DimArgs& a, const RedState& s, cudaStream_t st) {
  if (s.ncols == 0) return cudaSuccess;
  size_t sm = binom_smem(a);
  cudaError_t e = prepare(init_kernel, sm);
  if (e != cudaSuccess) return e;
  init_kernel<<<grid_for_warps(s.ncols), 256, sm, st>>>(a, s);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_claim(const DimArgs& a, const RedState& s, uint32_t count, cudaStream_t st) {
  if (count == 0) return cudaSuccess;
  int blocks = (int)((count + 255) / 256);
  if (blocks > 152 * 8) blocks = 152 * 8;
  claim_kernel<<<blocks, 256, 0, st>>>(a, s, count);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_reduce(const DimArgs& a, const RedState& s, uint32_t count, cudaStream_t st) {
  if (count == 0) return cudaSuccess;
  size_t sm = binom_smem(a);
  cudaError_t e = prepare(reduce_kernel, sm);
  if (e != cudaSuccess) return e;
  reduce_kernel<<<grid_for_warps(count), 256, sm, st>>>(a, s, count);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_readout(const DimArgs& a, const RedState& s, const float* rank_value, int cloud,
                           rips_bar_t* bars, uint32_t* nbars, uint32_t bar_cap, unsigned long long* stats,
                           cudaStream_t st) {
  if (s.ncols == 0) return cudaSuccess;
  int blocks = (int)((s.ncols + 255) / 256);
  if (blocks > 152 * 8) blocks = 152 * 8;
  readout_kernel<<<blocks, 256, 0, st>>>(a, s, rank_value, cloud, bars, nbars, bar_cap, stats);
  note_launch();
  return cudaGetLastError();
}

}  // namespace rips
