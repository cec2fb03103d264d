// Canonical order of the output bars: by cloud and dimension, then birth, then
// death, then birth simplex index.  Up to SMALL_BARS bars: one comparison sort
// in shared memory.  Beyond that: three stable LSD radix sorts of a permutation
// (least significant key first), then one gather.
#include <atomic>

#include "rips_internal.cuh"

namespace rips {

namespace {

__global__ void iota_kernel(uint32_t* __restrict__ p, uint32_t n) {
  uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = i;
}

// key of bar perm[i] for pass `which`
__global__ void bar_key_kernel(const rips_bar_t* __restrict__ bars, const uint32_t* __restrict__ perm, uint32_t n,
                               int which, uint64_t* __restrict__ keys) {
  uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const rips_bar_t b = bars[perm[i]];
  uint64_t k;
  if (which == 0) k = b.birth_simplex;
  else if (which == 1) k = ((uint64_t)__float_as_uint(b.birth) << 32) | __float_as_uint(b.death);
  else k = ((uint64_t)(uint32_t)b.cloud << 8) | (uint32_t)b.dim;
  keys[i] = k;
}

// Up to SMALL_BARS bars: one block sorts their indices by the same three keys
// (group, birth and death, birth simplex; no two bars share all three) with a
// bitonic network in shared memory and gathers them, in one launch.
constexpr uint32_t SMALL_BARS = 2048;

__global__ void __launch_bounds__(1024) bar_order_small_kernel(const rips_bar_t* __restrict__ bars, uint32_t n,
                                                                uint32_t n2, rips_bar_t* __restrict__ out) {
  extern __shared__ uint64_t sm[];
  uint64_t* k2 = sm;           // cloud and dimension
  uint64_t* k1 = sm + n2;      // birth and death bits
  uint64_t* k0 = sm + 2 * n2;  // birth simplex
  uint32_t* perm = (uint32_t*)(sm + 3 * n2);
  for (uint32_t i = threadIdx.x; i < n2; i += blockDim.x) {
    perm[i] = i;
    if (i < n) {
      const rips_bar_t b = bars[i];
      k2[i] = ((uint64_t)(uint32_t)b.cloud << 8) | (uint32_t)b.dim;
      k1[i] = ((uint64_t)__float_as_uint(b.birth) << 32) | __float_as_uint(b.death);
      k0[i] = b.birth_simplex;
    } else {  // padding sorts last
      k2[i] = ~0ull;
      k1[i] = ~0ull;
      k0[i] = ~0ull;
    }
  }
  __syncthreads();
  for (uint32_t size = 2; size <= n2; size <<= 1) {
    for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
      for (uint32_t i = threadIdx.x; i < n2; i += blockDim.x) {
        const uint32_t l = i ^ stride;
        if (l > i) {
          const uint32_t a = perm[i], b = perm[l];
          const bool gt = k2[a] != k2[b] ? k2[a] > k2[b] : k1[a] != k1[b] ? k1[a] > k1[b] : k0[a] > k0[b];
          if (gt == ((i & size) == 0)) {
            perm[i] = b;
            perm[l] = a;
          }
        }
      }
      __syncthreads();
    }
  }
  for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) out[i] = bars[perm[i]];
}

__global__ void gather_bars_kernel(const rips_bar_t* __restrict__ in, const uint32_t* __restrict__ perm, uint32_t n,
                                   rips_bar_t* __restrict__ out) {
  uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = in[perm[i]];
}

}  // namespace

size_t bar_order_temp_bytes(uint32_t nb) { return sort_temp_bytes(nb); }

cudaError_t launch_bar_order(rips_bar_t* bars, rips_bar_t* bars_alt, uint32_t nb, uint64_t* k0, uint64_t* k1,
                             uint32_t* p0, uint32_t* p1, void* tmp, size_t tmp_bytes, int simplex_bits,
                             int group_bits, cudaStream_t s) {
  if (nb == 0) return cudaSuccess;
  if (nb <= SMALL_BARS) {
    uint32_t n2 = 2;
    while (n2 < nb) n2 <<= 1;
    const size_t smem = (size_t)n2 * 28;
    static std::atomic<bool> opted[64];  // once per device (any thread)
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64 || !opted[dev].load(std::memory_order_acquire)) {
      e = cudaFuncSetAttribute(bar_order_small_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)(SMALL_BARS * 28));
      if (e != cudaSuccess) return e;
      if (dev >= 0 && dev < 64) opted[dev].store(true, std::memory_order_release);
    }
    bar_order_small_kernel<<<1, 1024, smem, s>>>(bars, nb, n2, bars_alt);
    note_launch();
    return cudaGetLastError();
  }
  const int blocks = (int)((nb + 255) / 256);
  iota_kernel<<<blocks, 256, 0, s>>>(p0, nb);
  note_launch();
  uint32_t* perm = p0;
  uint32_t* perm_alt = p1;
  const int bits[3] = {simplex_bits, 64, 8 + group_bits};
  for (int which = 0; which < 3; ++which) {
    bar_key_kernel<<<blocks, 256, 0, s>>>(bars, perm, nb, which, k0);
    note_launch();
    bool alt = false;
    cudaError_t e = radix_sort_u64(k0, k1, perm, perm_alt, nb, bits[which], tmp, tmp_bytes, &alt, s);
    if (e != cudaSuccess) return e;
    if (alt) {
      uint32_t* t = perm;
      perm = perm_alt;
      perm_alt = t;
    }
  }
  gather_bars_kernel<<<blocks, 256, 0, s>>>(bars, perm, nb, bars_alt);
  note_launch();
  return cudaGetLastError();
}

}  // namespace rips
