// Allocation-free H0 barcode entry point.
//
// Some callers cannot allocate device memory at the moment they need a
// barcode: a serving process whose memory pool already owns every byte of the
// device (a cudaMalloc would fail, or take memory the pool has promised
// elsewhere), or a real-time loop that must not stall on the allocator
// (cudaMalloc and cudaFree may synchronise the device and take unbounded
// time).  For them, rips_h0_barcode_noalloc computes the dimension-0 barcode
// of one distance matrix of at most RIPS_NOALLOC_MAX_N points without any
// allocation: every intermediate buffer lives in one file-scope device array
// of fixed size (NOALLOC_BYTES below, about 3.3 MB), which every GPU that
// loads the library holds until the process exits.  The caller passes the
// matrix and the output buffers.
//
// Because every call shares that array, calls that overlap on the GPU (on
// different streams, or from different host threads) race and must not be
// issued.  Each call clears what has to start at zero; the array otherwise
// keeps the last call's contents.  The first call on a device looks up the
// array's device address (cudaGetSymbolAddress, with that device current) and
// keeps it for later calls; make that first call before any stream capture
// begins.  After cudaDeviceReset the kept address belongs to a destroyed
// context: do not call this entry point again in that process.  The call
// waits for its stream before it returns (it reads the error word back).
#include <cmath>
#include <mutex>

#include "rips_internal.cuh"

namespace rips {

namespace {

constexpr int NA_MAX_N = RIPS_NOALLOC_MAX_N;
constexpr uint64_t NA_MAX_EDGES = (uint64_t)NA_MAX_N * (NA_MAX_N - 1) / 2;
constexpr int NA_EDGE_BITS = 17;  // C(512, 2) - 1 < 2^17
static_assert(NA_MAX_EDGES < (1ull << NA_EDGE_BITS), "edge index bits");

// layout of the scratch array (byte offsets, each 256-aligned)
constexpr size_t al(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t OFF_KEYS = 0;
constexpr size_t OFF_KEYS_ALT = OFF_KEYS + al(NA_MAX_EDGES * 8);
constexpr size_t OFF_EU = OFF_KEYS_ALT + al(NA_MAX_EDGES * 8);
constexpr size_t OFF_EV = OFF_EU + al(NA_MAX_EDGES * 4);
constexpr size_t OFF_FOREST = OFF_EV + al(NA_MAX_EDGES * 4);
constexpr size_t OFF_ROWMAX = OFF_FOREST + al(NA_MAX_EDGES);
constexpr size_t OFF_VCLOUD = OFF_ROWMAX + al(NA_MAX_N * 4);
constexpr size_t OFF_CLOUD = OFF_VCLOUD + al(NA_MAX_N * 4);
constexpr size_t OFF_TILEOFF = OFF_CLOUD + al(sizeof(CloudInfo));
constexpr size_t OFF_COUNTS = OFF_TILEOFF + al(2 * 4);   // [0] edges, [1] error flags, [2] per-cloud edges
constexpr size_t OFF_STATS = OFF_COUNTS + al(4 * 4);
constexpr size_t OFF_SORT = OFF_STATS + al(16 * 8);
constexpr size_t SORT_TMP_BYTES = ((NA_MAX_EDGES + 4095) / 4096 * 256 + 256) * 4;
constexpr size_t NOALLOC_BYTES = OFF_SORT + al(SORT_TMP_BYTES);

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

std::mutex g_na_mu;
unsigned char* g_na_ptr[64] = {};

// pad every unused edge slot with the largest key so that it sorts last
__global__ void na_pad_keys_kernel(uint64_t* keys, uint64_t cap) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < cap; i += (uint64_t)gridDim.x * blockDim.x)
    keys[i] = ~0ull;
}

// the cloud table and tile offsets of the single cloud, written on the device
// (no host buffer is involved)
__global__ void na_init_kernel(CloudInfo* ci, uint32_t* tile_off, int n, uint32_t tiles) {
  *ci = CloudInfo{n, 0u, 0ull, 0u, 0u, 0.0f, 0u};
  tile_off[0] = 0u;
  tile_off[1] = tiles;
}

// device error flags -> status: a bounded wait that ran out, a capacity limit,
// anything else an internal failure
int na_status(uint32_t err) {
  if (err & ERRF_BAD_INPUT) return RIPS_ERR_BAD_ARG;
  if (err & ERRF_TIMEOUT) return RIPS_ERR_DEVICE_TIMEOUT;
  if (err & (ERRF_TABLE_FULL | ERRF_OUT_OVERFLOW | ERRF_ARENA)) return RIPS_ERR_OOM;
  if (err) return RIPS_ERR_INTERNAL;
  return RIPS_OK;
}

// cloud table of the single cloud once the edge count is known (on the device)
__global__ void na_cloud_kernel(CloudInfo* ci, const uint32_t* counts) {
  ci->eoff = 0;
  ci->m = counts[0] < (uint32_t)NA_MAX_EDGES ? counts[0] : (uint32_t)NA_MAX_EDGES;
}

}  // namespace

// Address of the scratch array on the current device, looked up once per device.
static unsigned char* noalloc_scratch(int dev) {
  std::lock_guard<std::mutex> g(g_na_mu);
  if (dev < 0 || dev >= 64) return nullptr;
  if (!g_na_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    g_na_ptr[dev] = (unsigned char*)p;
  }
  return g_na_ptr[dev];
}

}  // namespace rips

using namespace rips;

extern "C" RIPS_API int rips_h0_barcode_noalloc(const float* d_dist, int64_t n, float threshold, rips_bar_t* d_bars,
                                                uint32_t* d_nbars, void* cuda_stream) {
  if (!d_dist || !d_bars || !d_nbars || n < 1) return RIPS_ERR_BAD_ARG;
  if (n > NA_MAX_N) return RIPS_ERR_BAD_ARG;  // larger than the fixed scratch array allows
  if (!std::isnan(threshold) && threshold < 0.0f) return RIPS_ERR_BAD_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return RIPS_ERR_CUDA;
  }
  unsigned char* base = noalloc_scratch(dev);
  if (!base) return RIPS_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  uint64_t* keys = (uint64_t*)(base + OFF_KEYS);
  uint64_t* keys_alt = (uint64_t*)(base + OFF_KEYS_ALT);
  uint32_t* eu = (uint32_t*)(base + OFF_EU);
  uint32_t* ev = (uint32_t*)(base + OFF_EV);
  uint8_t* forest = base + OFF_FOREST;
  uint32_t* rowmax = (uint32_t*)(base + OFF_ROWMAX);
  uint32_t* vcloud = (uint32_t*)(base + OFF_VCLOUD);
  CloudInfo* cloud = (CloudInfo*)(base + OFF_CLOUD);
  uint32_t* tile_off = (uint32_t*)(base + OFF_TILEOFF);
  uint32_t* counts = (uint32_t*)(base + OFF_COUNTS);
  unsigned long long* stats = (unsigned long long*)(base + OFF_STATS);
  void* sort_tmp = base + OFF_SORT;

  const uint64_t m_cap = (uint64_t)n * (n - 1) / 2;
  const uint32_t nb = (uint32_t)((n + 31) / 32);
  const uint32_t tiles = nb * (nb + 1) / 2;
  cudaError_t e = cudaSuccess;
  // everything that must start at zero (or at its initial value) is reset here
  na_init_kernel<<<1, 1, 0, s>>>(cloud, tile_off, (int)n, tiles);
  note_launch();
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemsetAsync(rowmax, 0, (size_t)n * 4, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(counts, 0, 4 * 4, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(stats, 0, 16 * 8, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_nbars, 0, 4, s);
  if (e == cudaSuccess && m_cap) {
    na_pad_keys_kernel<<<(unsigned)((m_cap + 255) / 256 < 1024 ? (m_cap + 255) / 256 : 1024), 256, 0, s>>>(keys, m_cap);
    note_launch();
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = launch_cloud_vertices(cloud, 1, vcloud, s);
  if (e == cudaSuccess && n > 1) e = launch_validate_rowmax(d_dist, cloud, tile_off, 1, tiles, rowmax, counts + 1, s);
  if (e == cudaSuccess) e = launch_threshold(rowmax, cloud, 1, threshold, s);
  if (e == cudaSuccess && n > 1)
    e = launch_edge_keys(d_dist, cloud, vcloud, (uint32_t)n, NA_EDGE_BITS, keys, counts, counts + 2,
                         (uint32_t)m_cap, s);
  bool alt = false;
  if (e == cudaSuccess && m_cap > 1)
    e = radix_sort_u64(keys, keys_alt, nullptr, nullptr, (uint32_t)m_cap, 32 + NA_EDGE_BITS, sort_tmp,
                       SORT_TMP_BYTES, &alt, s);
  const uint64_t* sorted = alt ? keys_alt : keys;
  if (e == cudaSuccess) {
    na_cloud_kernel<<<1, 1, 0, s>>>(cloud, counts);
    note_launch();
    e = cudaGetLastError();
  }
  if (e == cudaSuccess)
    e = launch_h0_blocks(cloud, 1, (int)n, sorted, NA_EDGE_BITS, eu, ev, (uint32_t)m_cap, forest, d_bars, d_nbars,
                         (uint32_t)n, stats, 16, counts + 1, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return RIPS_ERR_CUDA;
  }
  // invalid distances are reported by the validation kernel through the error word
  uint32_t err = 0;
  if (cudaMemcpyAsync(&err, counts + 1, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return RIPS_ERR_CUDA;
  }
  return na_status(err);
}
