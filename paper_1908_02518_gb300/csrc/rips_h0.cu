// Dimension 0 (Section 4, "Persistence pairs": the paper uses Kruskal's
// algorithm with union-find).  The persistence pairs of dimension 0 are the
// edges of the minimum spanning forest of the threshold graph under the refined
// filtration order, each paired with the vertex whose component dies (elder
// rule: of the two merging components, the one whose oldest vertex -- the
// largest index, Section 2 -- is younger dies).
//
// GB300 design: after the edge sort each cloud's edges are contiguous and in
// filtration order, so an edge's position is a unique weight realising the
// total order.  The spanning forest comes from Borůvka rounds (parallel over
// edges and components, at most ceil(log2 n)+1 rounds); only the n-1 forest
// edges then go through the sequential elder rule, with the union-find in
// shared memory.  Small clouds run one block each (all clouds of a batch in
// one launch); a single large cloud uses grid-wide rounds.
#include "rips_internal.cuh"

namespace rips {

namespace {

constexpr int H0_BLOCK_MAX_N = 12800;  // 16 bytes of shared memory per vertex

__device__ __forceinline__ void edge_vertices_u32(uint64_t idx, uint32_t* a, uint32_t* b) {
  uint32_t x = (uint32_t)((1.0 + sqrt(1.0 + 8.0 * (double)idx)) * 0.5);
  while ((uint64_t)x * (x - 1) / 2 > idx) --x;
  while ((uint64_t)(x + 1) * x / 2 <= idx) ++x;
  *a = x;
  *b = (uint32_t)(idx - (uint64_t)x * (x - 1) / 2);
}

__device__ __forceinline__ uint64_t key_edge_index(uint64_t key, int eb) {
  const uint64_t emask = (1ull << eb) - 1;
  return emask - (key & emask);
}
__device__ __forceinline__ float key_length(uint64_t key, int eb) {
  return __uint_as_float((uint32_t)(key >> eb));
}

__device__ void emit_bar(rips_bar_t* bars, uint32_t* nbars, uint32_t cap, int cloud, float death, uint64_t birth_v,
                         uint64_t death_s) {
  const uint32_t pos = atomicAdd(nbars, 1u);
  if (pos < cap) {
    rips_bar_t b;
    b.dim = 0;
    b.birth = 0.0f;
    b.death = death;
    b.cloud = cloud;
    b.birth_simplex = birth_v;
    b.death_simplex = death_s;
    bars[pos] = b;
  }
}

// Elder rule over the forest edges fpos[0..nf) (increasing positions) of one
// cloud, by the calling thread, with parent/top already initialised.
__device__ void elder_rule(const uint64_t* __restrict__ keys, int eb, const uint32_t* __restrict__ eu,
                           const uint32_t* __restrict__ ev, const uint32_t* __restrict__ fpos, uint32_t nf, int n,
                           uint32_t* parent, uint32_t* top, int cloud, rips_bar_t* bars, uint32_t* nbars,
                           uint32_t cap, unsigned long long* st) {
  unsigned long long zero = 0;
  for (uint32_t q = 0; q < nf; ++q) {
    const uint32_t e = fpos[q];
    uint32_t ru = eu[e], rv = ev[e];
    while (parent[ru] != ru) {
      parent[ru] = parent[parent[ru]];
      ru = parent[ru];
    }
    while (parent[rv] != rv) {
      parent[rv] = parent[parent[rv]];
      rv = parent[rv];
    }
    if (ru == rv) continue;  // cannot happen on a forest edge
    const uint32_t die = min(top[ru], top[rv]);
    const uint32_t live = max(top[ru], top[rv]);
    parent[ru] = rv;
    top[rv] = live;
    const float death = key_length(keys[e], eb);
    if (death == 0.0f) {
      ++zero;
      continue;
    }
    emit_bar(bars, nbars, cap, cloud, death, die, key_edge_index(keys[e], eb));
  }
  unsigned long long ess = 0;
  for (int v = 0; v < n; ++v)
    if (parent[v] == (uint32_t)v) {
      emit_bar(bars, nbars, cap, cloud, __int_as_float(0x7f800000), top[v], ~0ull);
      ++ess;
    }
  st[0] = nf;
  st[1] = zero;
  st[2] = ess;
}

// local endpoints of every sorted edge
__global__ void edge_endpoints_kernel(const uint64_t* __restrict__ keys, uint32_t m, int eb, uint32_t* __restrict__ eu,
                                      uint32_t* __restrict__ ev) {
  uint32_t e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m) return;
  uint32_t a, b;
  edge_vertices_u32(key_edge_index(keys[e], eb), &a, &b);
  eu[e] = a;
  ev[e] = b;
}

// One cloud per block: Borůvka rounds with __syncthreads as the barrier,
// block-wide compaction of the forest edges, then the elder rule by one thread.
__global__ void __launch_bounds__(1024) h0_block_kernel(const CloudInfo* __restrict__ clouds,
                                                        const uint64_t* __restrict__ keys, int eb,
                                                        const uint32_t* __restrict__ eu_all,
                                                        const uint32_t* __restrict__ ev_all,
                                                        uint8_t* __restrict__ in_forest_all,
                                                        rips_bar_t* __restrict__ bars, uint32_t* __restrict__ nbars,
                                                        uint32_t bar_cap, unsigned long long* __restrict__ stats,
                                                        int stats_stride, uint32_t* __restrict__ err) {
  extern __shared__ uint32_t sm[];
  const int cloud = blockIdx.x;
  const CloudInfo ci = clouds[cloud];
  const int n = ci.n;
  const uint32_t m = ci.m;
  const uint64_t* ek = keys + ci.eoff;
  const uint32_t* eu = eu_all + ci.eoff;
  const uint32_t* ev = ev_all + ci.eoff;
  uint8_t* in_forest = in_forest_all + ci.eoff;
  uint32_t* comp = sm;
  uint32_t* best = sm + n;
  uint32_t* parent = sm + 2 * n;
  uint32_t* top = sm + 3 * n;
  __shared__ int hooked;
  __shared__ uint32_t warp_tot[32];
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int v = tid; v < n; v += nt) {
    comp[v] = v;
    best[v] = 0xFFFFFFFFu;
  }
  for (uint32_t e = tid; e < m; e += nt) in_forest[e] = 0;
  __syncthreads();
  for (int round = 0; round < 64; ++round) {
    for (uint32_t e = tid; e < m; e += nt) {
      const uint32_t cu = comp[eu[e]], cv = comp[ev[e]];
      if (cu != cv) {
        atomicMin(&best[cu], e);
        atomicMin(&best[cv], e);
      }
    }
    if (tid == 0) hooked = 0;
    __syncthreads();
    for (int c = tid; c < n; c += nt) {
      parent[c] = c;
      if (comp[c] != (uint32_t)c) continue;
      const uint32_t e = best[c];
      if (e == 0xFFFFFFFFu) continue;
      const uint32_t a = comp[eu[e]], b = comp[ev[e]];
      const uint32_t other = (a == (uint32_t)c) ? b : a;
      if (best[other] == e && (uint32_t)c < other) continue;
      parent[c] = other;
      in_forest[e] = 1;
      hooked = 1;
    }
    __syncthreads();
    if (!hooked) break;
    for (int v = tid; v < n; v += nt) {
      uint32_t x = comp[v];
      for (int guard = 0; parent[x] != x; ++guard) {
        x = parent[x];
        if (guard > n) {
          set_error(err, ERRF_TIMEOUT);
          break;
        }
      }
      comp[v] = x;
      best[v] = 0xFFFFFFFFu;
    }
    __syncthreads();
  }
  __syncthreads();
  // forest edge positions in increasing order into best[] (at most n-1 of them)
  uint32_t* fpos = best;
  uint32_t base = 0;
  const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  for (uint32_t e0 = 0; e0 < m; e0 += nt) {
    const uint32_t e = e0 + tid;
    const bool f = e < m && in_forest[e];
    const unsigned bal = __ballot_sync(0xffffffffu, f);
    if (lane == 0) warp_tot[warp] = __popc(bal);
    __syncthreads();
    uint32_t off = base;
    for (int w = 0; w < warp; ++w) off += warp_tot[w];
    if (f) fpos[off + __popc(bal & ((1u << lane) - 1u))] = e;
    uint32_t tot = 0;
    for (int w = 0; w < nw; ++w) tot += warp_tot[w];
    base += tot;
    __syncthreads();
  }
  for (int v = tid; v < n; v += nt) {
    parent[v] = v;
    top[v] = v;
  }
  __syncthreads();
  if (tid == 0)
    elder_rule(ek, eb, eu, ev, fpos, base, n, parent, top, cloud, bars, nbars, bar_cap,
               stats + (size_t)cloud * stats_stride);
}

// ---------------------------------------------------------------- one large cloud

__global__ void init_components_kernel(int n, uint32_t* __restrict__ comp, uint32_t* __restrict__ best) {
  int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  comp[v] = v;
  best[v] = 0xFFFFFFFFu;
}

__global__ void boruvka_min_edge_kernel(const uint32_t* __restrict__ eu, const uint32_t* __restrict__ ev,
                                        uint32_t m, const uint32_t* __restrict__ comp, uint32_t* __restrict__ best) {
  for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < m; e += gridDim.x * blockDim.x) {
    uint32_t cu = comp[eu[e]], cv = comp[ev[e]];
    if (cu != cv) {
      atomicMin(&best[cu], e);
      atomicMin(&best[cv], e);
    }
  }
}

// every root hooks onto the component across its cheapest edge; of two
// components that chose the same edge, the larger label hooks
__global__ void boruvka_hook_kernel(int n, const uint32_t* __restrict__ eu, const uint32_t* __restrict__ ev,
                                    const uint32_t* __restrict__ comp, const uint32_t* __restrict__ best,
                                    uint32_t* __restrict__ parent, uint8_t* __restrict__ in_forest) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n || comp[c] != (uint32_t)c) return;
  uint32_t e = best[c];
  if (e == 0xFFFFFFFFu) {
    parent[c] = c;
    return;
  }
  uint32_t a = comp[eu[e]], b = comp[ev[e]];
  uint32_t other = (a == (uint32_t)c) ? b : a;
  if (best[other] == e && (uint32_t)c < other) {
    parent[c] = c;
  } else {
    parent[c] = other;
    in_forest[e] = 1;
  }
}

__global__ void boruvka_jump_kernel(int n, uint32_t* __restrict__ comp, const uint32_t* __restrict__ parent,
                                    uint32_t* __restrict__ best, uint32_t* __restrict__ err) {
  int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  uint32_t x = comp[v];
  int guard = 0;
  while (parent[x] != x) {
    x = parent[x];
    if (++guard > n) {
      set_error(err, ERRF_TIMEOUT);
      break;
    }
  }
  comp[v] = x;
  best[v] = 0xFFFFFFFFu;
}

__global__ void elder_rule_kernel(int n, const uint32_t* __restrict__ fpos, const uint32_t* __restrict__ nf,
                                  const uint32_t* __restrict__ eu, const uint32_t* __restrict__ ev,
                                  const uint64_t* __restrict__ keys, int eb, uint32_t* __restrict__ parent,
                                  uint32_t* __restrict__ top, rips_bar_t* __restrict__ bars,
                                  uint32_t* __restrict__ nbars, uint32_t bar_cap, unsigned long long* __restrict__ st) {
  for (int v = threadIdx.x; v < n; v += blockDim.x) {
    parent[v] = v;
    top[v] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) elder_rule(keys, eb, eu, ev, fpos, *nf, n, parent, top, 0, bars, nbars, bar_cap, st);
}

__global__ void flags_from_bytes_kernel(const uint8_t* __restrict__ b, uint32_t m, uint32_t* __restrict__ f) {
  uint32_t e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < m) f[e] = b[e];
}

__global__ void compact_positions_kernel(const uint8_t* __restrict__ in_forest, const uint32_t* __restrict__ excl,
                                         uint32_t m, uint32_t* __restrict__ out) {
  uint32_t e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < m && in_forest[e]) out[excl[e]] = e;
}

}  // namespace

bool h0_blocks_fit(int n_max) { return n_max <= H0_BLOCK_MAX_N; }

cudaError_t launch_h0_blocks(const CloudInfo* clouds, int nclouds, int n_max, const uint64_t* sorted_keys,
                             int edge_bits, uint32_t* eu, uint32_t* ev, uint32_t m_total, uint8_t* in_forest,
                             rips_bar_t* bars, uint32_t* nbars, uint32_t bar_cap, unsigned long long* stats,
                             int stats_stride, uint32_t* err, cudaStream_t s) {
  cudaError_t e;
  if (m_total) {
    edge_endpoints_kernel<<<(m_total + 255) / 256, 256, 0, s>>>(sorted_keys, m_total, edge_bits, eu, ev);
    note_launch();
  }
  const size_t smem = (size_t)4 * (n_max > 0 ? n_max : 1) * sizeof(uint32_t);
  if (smem > 48 * 1024 &&
      (e = cudaFuncSetAttribute(h0_block_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
          cudaSuccess)
    return e;
  h0_block_kernel<<<nclouds, 1024, smem, s>>>(clouds, sorted_keys, edge_bits, eu, ev, in_forest, bars, nbars, bar_cap,
                                              stats, stats_stride, err);
  note_launch();
  return cudaGetLastError();
}

cudaError_t run_h0_large(int n, const uint64_t* sorted_keys, uint32_t m, int edge_bits, uint32_t* eu, uint32_t* ev,
                         uint32_t* comp, uint32_t* best, uint32_t* parent, uint8_t* in_forest, uint32_t* flags,
                         uint32_t* fpos, void* scan_tmp, uint32_t* d_nf, uint32_t* gtop, rips_bar_t* bars,
                         uint32_t* nbars, uint32_t bar_cap, unsigned long long* stats, uint32_t* err, cudaStream_t s) {
  cudaError_t e;
  if ((e = cudaMemsetAsync(in_forest, 0, m ? m : 1, s)) != cudaSuccess) return e;
  if (m) {
    edge_endpoints_kernel<<<(m + 255) / 256, 256, 0, s>>>(sorted_keys, m, edge_bits, eu, ev);
    note_launch();
  }
  init_components_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, comp, best);
  note_launch();
  int rounds = 1;
  while ((1 << (rounds - 1)) < n) ++rounds;
  int eblocks = (int)((m + 255) / 256);
  if (eblocks > 152 * 8) eblocks = 152 * 8;
  if (eblocks < 1) eblocks = 1;
  for (int r = 0; m && r < rounds; ++r) {
    boruvka_min_edge_kernel<<<eblocks, 256, 0, s>>>(eu, ev, m, comp, best);
    note_launch();
    boruvka_hook_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, eu, ev, comp, best, parent, in_forest);
    note_launch();
    boruvka_jump_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, comp, parent, best, err);
    note_launch();
  }
  if (m) {
    flags_from_bytes_kernel<<<(m + 255) / 256, 256, 0, s>>>(in_forest, m, flags);
    note_launch();
    if ((e = launch_exclusive_scan(flags, flags, m, scan_tmp, d_nf, s)) != cudaSuccess) return e;
    compact_positions_kernel<<<(m + 255) / 256, 256, 0, s>>>(in_forest, flags, m, fpos);
    note_launch();
  } else {
    if ((e = cudaMemsetAsync(d_nf, 0, sizeof(uint32_t), s)) != cudaSuccess) return e;
  }
  // the forest has at most n - 1 edges; the elder rule reads the count on the device
  elder_rule_kernel<<<1, 256, 0, s>>>(n, fpos, d_nf, eu, ev, sorted_keys, edge_bits, parent, gtop, bars, nbars, bar_cap,
                                      stats);
  note_launch();
  return cudaGetLastError();
}

}  // namespace rips
