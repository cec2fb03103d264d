// Dimension 0 (Section 4, "Persistence pairs": the paper uses Kruskal's
// algorithm with union-find).  The persistence pairs of dimension 0 are the
// edges of the minimum spanning forest of the threshold graph under the refined
// filtration order, each paired with the vertex whose component dies (elder
// rule: among the two merging components, the one whose oldest vertex -- the
// largest index, Section 2 -- is younger dies).
//
// GB300 design: the edges arrive sorted, so an edge's position is a unique
// weight that realises the total order.  The spanning forest is found with
// Borůvka rounds (parallel over edges and components, at most ceil(log2 n)+1
// rounds); only the n-1 forest edges then go through the sequential elder rule,
// with the union-find held in shared memory.
#include "rips_internal.cuh"

namespace rips {

namespace {

__device__ __forceinline__ void edge_vertices_u32(uint32_t idx, uint32_t* a, uint32_t* b) {
  uint32_t x = (uint32_t)((1.0 + sqrt(1.0 + 8.0 * (double)idx)) * 0.5);
  while ((uint64_t)x * (x - 1) / 2 > idx) --x;
  while ((uint64_t)(x + 1) * x / 2 <= idx) ++x;
  *a = x;
  *b = idx - (uint32_t)((uint64_t)x * (x - 1) / 2);
}

__global__ void edge_endpoints_kernel(const uint64_t* __restrict__ keys, uint32_t m, uint32_t* __restrict__ eu,
                                      uint32_t* __restrict__ ev) {
  uint32_t e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m) return;
  uint32_t idx = 0xFFFFFFFFu - (uint32_t)(keys[e] & 0xFFFFFFFFull);
  uint32_t a, b;
  edge_vertices_u32(idx, &a, &b);
  eu[e] = a;
  ev[e] = b;
}

__global__ void init_components_kernel(int n, uint32_t* __restrict__ comp, uint32_t* __restrict__ best) {
  int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  comp[v] = v;
  best[v] = 0xFFFFFFFFu;
}

// cheapest (smallest position) edge leaving every component
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

// Elder rule over the forest edges in filtration order (one thread; the
// union-find lives in shared memory when it fits).  Writes the H0 bars and
// marks each forest edge's position for clearing in dimension 1.
__global__ void elder_rule_kernel(int n, const uint8_t* __restrict__ in_forest, const uint32_t* __restrict__ fpos,
                                  uint32_t nf, const uint32_t* __restrict__ eu, const uint32_t* __restrict__ ev,
                                  const uint64_t* __restrict__ keys, uint32_t* __restrict__ gparent,
                                  uint32_t* __restrict__ gtop, int use_smem, rips_bar_t* __restrict__ bars,
                                  uint32_t* __restrict__ nbars, uint32_t bar_cap, int cloud,
                                  unsigned long long* __restrict__ stats /* pairs, zero, essential */) {
  extern __shared__ uint32_t sm[];
  uint32_t* parent = use_smem ? sm : gparent;
  uint32_t* top = use_smem ? sm + n : gtop;
  for (int v = threadIdx.x; v < n; v += blockDim.x) {
    parent[v] = v;
    top[v] = v;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  uint32_t nb = *nbars;
  unsigned long long zero = 0;
  for (uint32_t q = 0; q < nf; ++q) {
    uint32_t e = fpos[q];
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
    uint32_t die = min(top[ru], top[rv]);
    uint32_t live = max(top[ru], top[rv]);
    parent[ru] = rv;
    top[rv] = live;
    float death = __uint_as_float((uint32_t)(keys[e] >> 32));
    if (death == 0.0f) {
      ++zero;
      continue;
    }
    if (nb < bar_cap) {
      rips_bar_t b;
      b.dim = 0;
      b.birth = 0.0f;
      b.death = death;
      b.cloud = cloud;
      b.birth_simplex = die;
      b.death_simplex = 0xFFFFFFFFu - (uint32_t)(keys[e] & 0xFFFFFFFFull);
      bars[nb] = b;
    }
    ++nb;
  }
  unsigned long long ess = 0;
  for (int v = 0; v < n; ++v)
    if (parent[v] == (uint32_t)v) {
      if (nb < bar_cap) {
        rips_bar_t b;
        b.dim = 0;
        b.birth = 0.0f;
        b.death = __int_as_float(0x7f800000);
        b.cloud = cloud;
        b.birth_simplex = top[v];
        b.death_simplex = ~0ull;
        bars[nb] = b;
      }
      ++nb;
      ++ess;
    }
  *nbars = nb;
  stats[0] = nf;
  stats[1] = zero;
  stats[2] = ess;
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

// H0 driver: returns the number of forest edges in *h_nf (host), after a sync.
cudaError_t run_h0(int n, const uint64_t* sorted_keys, uint32_t m, uint32_t* eu, uint32_t* ev, uint32_t* comp,
                   uint32_t* best, uint32_t* parent, uint8_t* in_forest, uint32_t* flags, uint32_t* fpos,
                   void* scan_tmp, uint32_t* d_nf, uint32_t* gtop, rips_bar_t* bars, uint32_t* nbars,
                   uint32_t bar_cap, int cloud, unsigned long long* stats, uint32_t* err, cudaStream_t s) {
  cudaError_t e;
  if ((e = cudaMemsetAsync(in_forest, 0, m ? m : 1, s)) != cudaSuccess) return e;
  if (m) {
    edge_endpoints_kernel<<<(m + 255) / 256, 256, 0, s>>>(sorted_keys, m, eu, ev);
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
  uint32_t h_nf = 0;
  if ((e = cudaMemcpyAsync(&h_nf, d_nf, sizeof(uint32_t), cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
  size_t smem = (size_t)2 * n * sizeof(uint32_t);
  int use_smem = smem <= 96 * 1024;
  if (use_smem && smem > 48 * 1024) {
    if ((e = cudaFuncSetAttribute(elder_rule_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
        cudaSuccess)
      return e;
  }
  elder_rule_kernel<<<1, 256, use_smem ? smem : 0, s>>>(n, in_forest, fpos, h_nf, eu, ev, sorted_keys, parent, gtop,
                                                       use_smem, bars, nbars, bar_cap, cloud, stats);
  note_launch();
  return cudaGetLastError();
}

}  // namespace rips
