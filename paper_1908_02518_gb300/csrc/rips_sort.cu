// Exclusive scan and LSD radix sort on 64-bit keys (filtration order, Section 2:
// keys pack the diameter rank above the simplex index, so one unsigned sort
// realises "diameter, then index").
//
// Radix sort: 8-bit digits, one pass per digit.  Each pass is
//   (1) tile histograms      hist[digit][tile]   (digit-major),
//   (2) per-digit scan over tiles plus digit totals,
//   (3) stable scatter: every warp ranks its 32-key steps with
//       __match_any_sync, warps are ordered by a shared-memory prefix, so keys
//       with equal digits keep their relative order (LSD correctness).

#include <atomic>

#include "rips_internal.cuh"

namespace rips {

// ============================================================ scan
namespace {
constexpr int SCAN_THREADS = 1024;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += y;
  }
  return v;
}

// block-wide exclusive scan of one value per thread; returns total in *total
__device__ uint32_t block_excl_scan(uint32_t v, uint32_t* smem, uint32_t* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  uint32_t inc = warp_incl_scan(v);
  if (lane == 31) smem[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = lane < nw ? smem[lane] : 0;
    uint32_t wi = warp_incl_scan(w);
    if (lane < nw) smem[lane] = wi - w;
    if (lane == nw - 1) smem[32] = wi;
  }
  __syncthreads();
  uint32_t r = smem[warp] + inc - v;
  *total = smem[32];
  __syncthreads();
  return r;
}

__global__ void scan_reduce_kernel(const uint32_t* __restrict__ in, uint32_t n, uint32_t* __restrict__ sums) {
  __shared__ uint32_t sm[33];
  size_t base = (size_t)blockIdx.x * SCAN_TILE;
  uint32_t s = 0;
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    size_t idx = base + (size_t)threadIdx.x * SCAN_ITEMS + i;
    if (idx < n) s += in[idx];
  }
  uint32_t tot;
  block_excl_scan(s, sm, &tot);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void scan_sums_kernel(uint32_t* __restrict__ sums, uint32_t nb, uint32_t* __restrict__ total) {
  __shared__ uint32_t sm[33];
  uint32_t carry = 0;
  for (uint32_t base = 0; base < nb; base += blockDim.x) {
    uint32_t idx = base + threadIdx.x;
    uint32_t v = idx < nb ? sums[idx] : 0;
    uint32_t tot;
    uint32_t e = block_excl_scan(v, sm, &tot);
    if (idx < nb) sums[idx] = carry + e;
    carry += tot;
  }
  if (threadIdx.x == 0 && total) *total = carry;
}

__global__ void scan_apply_kernel(const uint32_t* __restrict__ in, uint32_t* __restrict__ out, uint32_t n,
                                  const uint32_t* __restrict__ sums) {
  __shared__ uint32_t sm[33];
  size_t base = (size_t)blockIdx.x * SCAN_TILE;
  uint32_t v[SCAN_ITEMS];
  uint32_t s = 0;
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    size_t idx = base + (size_t)threadIdx.x * SCAN_ITEMS + i;
    v[i] = idx < n ? in[idx] : 0;
    s += v[i];
  }
  uint32_t tot;
  uint32_t e = block_excl_scan(s, sm, &tot) + sums[blockIdx.x];
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    size_t idx = base + (size_t)threadIdx.x * SCAN_ITEMS + i;
    if (idx < n) out[idx] = e;
    e += v[i];
  }
}
}  // namespace

size_t scan_temp_bytes(uint32_t n) {
  size_t nb = ((size_t)n + SCAN_TILE - 1) / SCAN_TILE;
  return (nb + 1) * sizeof(uint32_t);
}

cudaError_t launch_exclusive_scan(const uint32_t* in, uint32_t* out, uint32_t n, void* tmp,
                                  uint32_t* d_total, cudaStream_t s) {
  uint32_t nb = (uint32_t)(((size_t)n + SCAN_TILE - 1) / SCAN_TILE);
  if (nb == 0) nb = 1;
  uint32_t* sums = (uint32_t*)tmp;
  scan_reduce_kernel<<<nb, SCAN_THREADS, 0, s>>>(in, n, sums);
  note_launch();
  scan_sums_kernel<<<1, SCAN_THREADS, 0, s>>>(sums, nb, d_total);
  note_launch();
  scan_apply_kernel<<<nb, SCAN_THREADS, 0, s>>>(in, out, n, sums);
  note_launch();
  return cudaGetLastError();
}

// ============================================================ radix sort
namespace {
constexpr int RS_THREADS = 256;   // 8 warps
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_STEPS = 16;      // 32-key steps per warp
constexpr int RS_TILE = RS_WARPS * RS_STEPS * 32;  // 4096 keys per tile
constexpr int RADIX = 256;

__global__ void __launch_bounds__(RS_THREADS) rs_hist_kernel(const uint64_t* __restrict__ keys, uint32_t n,
                                                             int shift, uint32_t* __restrict__ hist,
                                                             uint32_t tiles) {
  __shared__ uint32_t h[RADIX];
  for (int i = threadIdx.x; i < RADIX; i += RS_THREADS) h[i] = 0;
  __syncthreads();
  size_t base = (size_t)blockIdx.x * RS_TILE;
  for (int i = threadIdx.x; i < RS_TILE; i += RS_THREADS) {
    size_t idx = base + i;
    if (idx < n) atomicAdd(&h[(uint32_t)(keys[idx] >> shift) & 0xFFu], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < RADIX; i += RS_THREADS) hist[(size_t)i * tiles + blockIdx.x] = h[i];
}

// one block per digit: exclusive scan of hist[digit][0..tiles) and digit total
__global__ void rs_tile_scan_kernel(uint32_t* __restrict__ hist, uint32_t tiles, uint32_t* __restrict__ totals) {
  __shared__ uint32_t sm[33];
  uint32_t* row = hist + (size_t)blockIdx.x * tiles;
  uint32_t carry = 0;
  for (uint32_t b = 0; b < tiles; b += blockDim.x) {
    uint32_t idx = b + threadIdx.x;
    uint32_t v = idx < tiles ? row[idx] : 0;
    uint32_t tot;
    uint32_t e = block_excl_scan(v, sm, &tot);
    if (idx < tiles) row[idx] = carry + e;
    carry += tot;
  }
  if (threadIdx.x == 0) totals[blockIdx.x] = carry;
}

template <bool HAS_VALS>
__global__ void __launch_bounds__(RS_THREADS) rs_scatter_kernel(
    const uint64_t* __restrict__ keys, uint64_t* __restrict__ keys_out, const uint32_t* __restrict__ vals,
    uint32_t* __restrict__ vals_out, uint32_t n, int shift, const uint32_t* __restrict__ hist, uint32_t tiles,
    const uint32_t* __restrict__ totals) {
  __shared__ uint32_t digit_base[RADIX];          // global start of each digit
  __shared__ uint32_t warp_cnt[RS_WARPS][RADIX];  // per-warp digit counts -> running positions
  __shared__ uint32_t sm[33];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned lt_mask = (1u << lane) - 1u;

  // digit starts: exclusive scan of the digit totals
  {
    uint32_t v = threadIdx.x < RADIX ? totals[threadIdx.x] : 0;
    uint32_t tot;
    uint32_t e = block_excl_scan(v, sm, &tot);
    if (threadIdx.x < RADIX) digit_base[threadIdx.x] = e + hist[(size_t)threadIdx.x * tiles + blockIdx.x];
  }
  for (int i = threadIdx.x; i < RS_WARPS * RADIX; i += RS_THREADS) (&warp_cnt[0][0])[i] = 0;
  __syncthreads();

  const size_t base = (size_t)blockIdx.x * RS_TILE + (size_t)warp * RS_STEPS * 32;
  uint64_t k[RS_STEPS];
#pragma unroll
  for (int st = 0; st < RS_STEPS; ++st) {
    size_t idx = base + st * 32 + lane;
    k[st] = idx < n ? keys[idx] : ~0ull;
  }
  // (A) per-warp digit counts
#pragma unroll
  for (int st = 0; st < RS_STEPS; ++st) {
    size_t idx = base + st * 32 + lane;
    bool valid = idx < n;
    uint32_t dg = (uint32_t)(k[st] >> shift) & 0xFFu;
    unsigned act = __ballot_sync(0xffffffffu, valid);
    if (valid) {
      unsigned peers = __match_any_sync(act, dg);
      if ((peers & lt_mask) == 0) warp_cnt[warp][dg] += __popc(peers);
    }
    __syncwarp();
  }
  __syncthreads();
  // (B) exclusive prefix across warps, per digit
  for (int dg = threadIdx.x; dg < RADIX; dg += RS_THREADS) {
    uint32_t run = digit_base[dg];
    for (int w = 0; w < RS_WARPS; ++w) {
      uint32_t c = warp_cnt[w][dg];
      warp_cnt[w][dg] = run;
      run += c;
    }
  }
  __syncthreads();
  // (C) stable ranks and scatter
#pragma unroll
  for (int st = 0; st < RS_STEPS; ++st) {
    size_t idx = base + st * 32 + lane;
    bool valid = idx < n;
    uint32_t dg = (uint32_t)(k[st] >> shift) & 0xFFu;
    unsigned act = __ballot_sync(0xffffffffu, valid);
    if (valid) {
      unsigned peers = __match_any_sync(act, dg);
      uint32_t pos = warp_cnt[warp][dg] + __popc(peers & lt_mask);
      keys_out[pos] = k[st];
      if (HAS_VALS) vals_out[pos] = vals[idx];
      __syncwarp(act);
      if ((peers & lt_mask) == 0) warp_cnt[warp][dg] += __popc(peers);
    }
    __syncwarp();
  }
}
}  // namespace

size_t sort_temp_bytes(uint32_t n) {
  size_t tiles = ((size_t)n + RS_TILE - 1) / RS_TILE;
  if (tiles == 0) tiles = 1;
  return (tiles * RADIX + RADIX) * sizeof(uint32_t);
}

// Up to SMALL_SORT keys without values: one block sorts them in shared memory
// with a bitonic network, in one launch instead of three per radix digit.
// Without values the order of equal keys does not show, so the result is the
// radix sort's.
constexpr uint32_t SMALL_SORT = 8192;

__global__ void __launch_bounds__(1024) sort_small_kernel(uint64_t* __restrict__ keys, uint32_t n, uint32_t n2) {
  extern __shared__ uint64_t k[];
  for (uint32_t i = threadIdx.x; i < n2; i += blockDim.x) k[i] = i < n ? keys[i] : ~0ull;
  __syncthreads();
  for (uint32_t size = 2; size <= n2; size <<= 1) {
    for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
      for (uint32_t i = threadIdx.x; i < n2; i += blockDim.x) {
        const uint32_t l = i ^ stride;
        if (l > i) {
          const uint64_t a = k[i], b = k[l];
          if ((a > b) == ((i & size) == 0)) {
            k[i] = b;
            k[l] = a;
          }
        }
      }
      __syncthreads();
    }
  }
  for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) keys[i] = k[i];
}

cudaError_t radix_sort_u64(uint64_t* keys, uint64_t* keys_alt, uint32_t* vals, uint32_t* vals_alt, uint32_t n,
                           int key_bits, void* tmp, size_t tmp_bytes, bool* result_in_alt, cudaStream_t s) {
  *result_in_alt = false;
  if (n <= 1 || key_bits <= 0) return cudaSuccess;
  if (!vals && n <= SMALL_SORT) {
    uint32_t n2 = 2;
    while (n2 < n) n2 <<= 1;
    const size_t smem = (size_t)n2 * 8;
    if (smem > 48 * 1024) {
      static std::atomic<bool> opted[64];  // once per device (any thread)
      int dev = 0;
      cudaError_t e = cudaGetDevice(&dev);
      if (e != cudaSuccess) return e;
      if (dev < 0 || dev >= 64 || !opted[dev].load(std::memory_order_acquire)) {
        e = cudaFuncSetAttribute(sort_small_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(SMALL_SORT * 8));
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) opted[dev].store(true, std::memory_order_release);
      }
    }
    sort_small_kernel<<<1, 1024, smem, s>>>(keys, n, n2);
    note_launch();
    return cudaGetLastError();
  }
  uint32_t tiles = (uint32_t)(((size_t)n + RS_TILE - 1) / RS_TILE);
  if (tmp_bytes < sort_temp_bytes(n)) return cudaErrorInvalidValue;
  uint32_t* hist = (uint32_t*)tmp;
  uint32_t* totals = hist + (size_t)tiles * RADIX;
  uint64_t* kin = keys;
  uint64_t* kout = keys_alt;
  uint32_t* vin = vals;
  uint32_t* vout = vals_alt;
  bool alt = false;
  for (int shift = 0; shift < key_bits; shift += 8) {
    rs_hist_kernel<<<tiles, RS_THREADS, 0, s>>>(kin, n, shift, hist, tiles);
    note_launch();
    rs_tile_scan_kernel<<<RADIX, 256, 0, s>>>(hist, tiles, totals);
    note_launch();
    if (vals)
      rs_scatter_kernel<true><<<tiles, RS_THREADS, 0, s>>>(kin, kout, vin, vout, n, shift, hist, tiles, totals);
    else
      rs_scatter_kernel<false><<<tiles, RS_THREADS, 0, s>>>(kin, kout, nullptr, nullptr, n, shift, hist, tiles,
                                                            totals);
    note_launch();
    uint64_t* t = kin;
    kin = kout;
    kout = t;
    uint32_t* tv = vin;
    vin = vout;
    vout = tv;
    alt = !alt;
  }
  *result_in_alt = alt;
  return cudaGetLastError();
}

}  // namespace rips
