// C ABI of librips: orchestration of the barcode pipeline on one GPU.
//
// Per call (one cloud):
//   prologue   validate the matrix, enclosing radius, edge keys, edge sort,
//              diameter ranks, rank matrix R, neighbour lists, binomial table;
//   H0         spanning forest + elder rule (rips_h0.cu);
//   d = 1..dim_max:
//              d-simplices (edges, or enumeration from the (d-1)-simplices),
//              apparent/clearing test and compaction, radix sort into
//              processing order, parallel reduction, bar readout
//              (rips_dim.cu);
//   epilogue   canonical order of the bars on the device, copy to the host.
//
// Device memory lives in a per-device workspace of grow-only buffers, reused
// across calls; calls on one device are serialised by a mutex.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "rips_internal.cuh"

namespace rips {

// ------------------------------------------------------------------ launch counter
static thread_local long long g_launches = 0;
void note_launch() { ++g_launches; }

// ------------------------------------------------------------------ buffers
struct Buf {
  void* p = nullptr;
  size_t cap = 0;
};

static int ensure(Buf& b, size_t bytes) {
  if (bytes == 0) bytes = 8;
  if (bytes <= b.cap) return RIPS_OK;
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.cap = 0;
  size_t want = bytes + bytes / 4;
  if (cudaMalloc(&b.p, want) != cudaSuccess) {
    cudaGetLastError();
    if (cudaMalloc(&b.p, bytes) != cudaSuccess) {
      cudaGetLastError();
      b.p = nullptr;
      return RIPS_ERR_OOM;
    }
    want = bytes;
  }
  b.cap = want;
  return RIPS_OK;
}

// grow keeping the first `keep` bytes
static int grow_keep(Buf& b, size_t bytes, size_t keep, cudaStream_t s) {
  if (bytes <= b.cap) return RIPS_OK;
  void* np = nullptr;
  size_t want = bytes * 2;
  if (cudaMalloc(&np, want) != cudaSuccess) {
    cudaGetLastError();
    return RIPS_ERR_OOM;
  }
  if (keep && b.p) {
    if (cudaMemcpyAsync(np, b.p, keep, cudaMemcpyDeviceToDevice, s) != cudaSuccess) return RIPS_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return RIPS_ERR_CUDA;
  }
  if (b.p) cudaFree(b.p);
  b.p = np;
  b.cap = want;
  return RIPS_OK;
}

template <typename T>
static T* P(Buf& b) {
  return (T*)b.p;
}

struct HostPinned {
  uint32_t u32[16];
  unsigned long long u64[16 * (MAX_DIM + 1)];
  float f32[4];
};

struct Workspace {
  std::mutex mu;
  int device = -1;
  Buf dist, binom, rowmax, teff, err, ecount;
  Buf ekeys, ekeys_alt, eflags, escan, erank, rvalue, R, deg, nbr;
  Buf eu, ev, comp, best, parent, gtop, inforest, fpos, nf;
  Buf sidx[2], srank[2], scount;
  Buf ckeys, ckeys_alt, ccount, sorttmp;
  Buf piv_key, piv_coef, r_off, r_len, reduced, claim, reduce, heavy, lists;
  Buf r_key, r_coef, r_top;
  Buf tkeys[2], tvals[2];
  Buf amk[2];  // apparent-pair maps of dimensions d and d - 1 ((key, value) pairs)
  Buf bars, bars_alt, bk0, bk1, bp0, bp1, bartmp, nbars;
  Buf stats, bwd_bars, bwd_off, cdist, clouds, tileoff, vcloud, ccounts;
  Buf nrank, nkey, nkey_alt, nval, nval_alt, cursor;  // neighbour lists of a sparse input
  size_t r_cap = 0;
  HostPinned* pinned = nullptr;
  cudaEvent_t tev[16] = {};
  bool events = false;
  // per-kernel-class timing (enabled by rips_set_kernel_timing)
  std::vector<cudaEvent_t> kev;       // pool of events, used in (start, stop) pairs
  std::vector<int> kev_class;         // class of each pair
  size_t kev_used = 0;                // pairs in use for the current call
};

static bool g_kernel_timing = false;

// Records a (start, stop) event pair around the launches of one kernel class.
struct KTimer {
  Workspace& w;
  cudaStream_t s;
  size_t pair = (size_t)-1;
  KTimer(Workspace& w_, int cls, cudaStream_t s_) : w(w_), s(s_) {
    if (!g_kernel_timing) return;
    if (w.kev_used * 2 + 2 > w.kev.size()) {
      for (int i = 0; i < 64; ++i) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) {
          cudaGetLastError();
          return;
        }
        w.kev.push_back(e);
      }
      w.kev_class.resize(w.kev.size() / 2);
    }
    pair = w.kev_used++;
    w.kev_class[pair] = cls;
    cudaEventRecord(w.kev[2 * pair], s);
  }
  ~KTimer() {
    if (pair != (size_t)-1) cudaEventRecord(w.kev[2 * pair + 1], s);
  }
};

static std::mutex g_ws_mu;
static Workspace* g_ws[64] = {};

static Workspace* workspace(int dev) {
  std::lock_guard<std::mutex> g(g_ws_mu);
  if (dev < 0 || dev >= 64) return nullptr;
  if (!g_ws[dev]) {
    Workspace* w = new (std::nothrow) Workspace();
    if (!w) return nullptr;
    w->device = dev;
    if (cudaMallocHost((void**)&w->pinned, sizeof(HostPinned)) != cudaSuccess) {
      cudaGetLastError();
      delete w;
      return nullptr;
    }
    for (auto& e : w->tev)
      if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        delete w;
        return nullptr;
      }
    w->events = true;
    g_ws[dev] = w;
  }
  return g_ws[dev];
}

}  // namespace rips

// ------------------------------------------------------------------ result object
struct rips_result {
  float kernel_ms[RIPS_KERNEL_CLASSES] = {};
  int64_t kernel_launches[RIPS_KERNEL_CLASSES] = {};
  int32_t clouds = 1;
  int32_t dim_max = 0;
  std::vector<rips_bar_t> bars;             // cloud, then dim, then canonical order
  std::vector<int64_t> offsets;             // (clouds * (dim_max+1) + 1) offsets into bars
  std::vector<float> thresholds;            // per cloud
  std::vector<rips_stats_t> stats;          // clouds * (dim_max+1)
  std::vector<int64_t> npoints;             // per cloud
  std::vector<int64_t> point_offsets;       // per cloud (batched): first point
  int32_t k = 0;                            // coordinates per point (batched)
  std::vector<float> phase_ms;
};

using namespace rips;

// ------------------------------------------------------------------ tuning table
// Launch and scheduling parameters per (dimension, largest cloud size), set by
// the autotuner or the caller; the defaults are the values that serve the test
// workloads well.
namespace {
struct TuneEntry {
  int32_t dim;
  int64_t lo, hi;
  rips_tuning_t t;
};
std::mutex g_tune_mu;
std::vector<TuneEntry> g_tune;
constexpr rips_tuning_t TUNE_DEFAULT{32, 2048, 0, 16};

std::mutex g_limits_mu;
rips_limits_t g_limits{0, 0, 0, 0};
uint32_t g_options = 0;  // RIPS_OPT_* (guarded by g_limits_mu)

uint32_t current_options() {
  std::lock_guard<std::mutex> g(g_limits_mu);
  return g_options;
}

rips_limits_t current_limits() {
  std::lock_guard<std::mutex> g(g_limits_mu);
  return g_limits;
}

rips_tuning_t tuning_for(int dim, int64_t n) {
  std::lock_guard<std::mutex> g(g_tune_mu);
  for (auto it = g_tune.rbegin(); it != g_tune.rend(); ++it)
    if (it->dim == dim && n >= it->lo && n <= it->hi) return it->t;
  return TUNE_DEFAULT;
}
}  // namespace

namespace {

#define CK(x)                                      \
  do {                                             \
    cudaError_t _e = (x);                          \
    if (_e != cudaSuccess) {                       \
      cudaGetLastError();                          \
      return _e == cudaErrorMemoryAllocation ? RIPS_ERR_OOM : RIPS_ERR_CUDA; \
    }                                              \
  } while (0)
#define CR(x)                  \
  do {                         \
    int _r = (x);              \
    if (_r != RIPS_OK) return _r; \
  } while (0)

// Bits per vertex when the d + 1 vertices of a d-simplex of a cloud of at most
// n_max points fit in 60 bits (the pair map's values then carry them, so the
// reduction need not decode the facet's index), else 0.
int packed_vertex_bits(int n_max, int d) {
  int b = 1;
  while (b < 31 && (1ll << b) < (long long)n_max) ++b;
  return (d + 1) * b <= 60 ? b : 0;
}

bool is_prime(uint32_t p) {
  if (p < 2) return false;
  for (uint32_t q = 2; (uint64_t)q * q <= p; ++q)
    if (p % q == 0) return false;
  return true;
}

// C(n, k) exactly, saturating at 2^64 - 1
uint64_t host_binom(uint64_t n, int k) {
  if (k < 0 || (uint64_t)k > n) return 0;
  unsigned __int128 c = 1;
  for (int i = 1; i <= k; ++i) {
    c = c * (unsigned __int128)(n - k + i) / (unsigned __int128)i;
    if (c > (unsigned __int128)~0ull) return ~0ull;
  }
  return (uint64_t)c;
}

int check_args(int64_t n, int32_t dim_max, float threshold, uint32_t p) {
  if (n < 1 || n > 46340 || dim_max < 0 || dim_max > MAX_DIM - 1) return RIPS_ERR_BAD_ARG;
  if (!std::isnan(threshold) && threshold < 0.0f) return RIPS_ERR_BAD_ARG;
  if (!is_prime(p) || p >= 65536) return RIPS_ERR_BAD_MODULUS;
  if (host_binom((uint64_t)n, dim_max + 2) >= (1ull << 63)) return RIPS_ERR_OVERFLOW;
  return RIPS_OK;
}

int map_device_error(uint32_t e) {
  if (e & ERRF_BAD_INPUT) return RIPS_ERR_BAD_ARG;
  if (e & ERRF_TIMEOUT) return RIPS_ERR_DEVICE_TIMEOUT;
  if (e & ERRF_TABLE_FULL) return RIPS_ERR_OOM;  // the cause; lookups that then miss also flag INTERNAL
  if (e & ERRF_INTERNAL) return RIPS_ERR_INTERNAL;
  return RIPS_OK;
}

uint32_t pow2_at_least(uint64_t x) {
  uint64_t c = 16;
  while (c < x) c <<= 1;
  return (uint32_t)c;
}

// One cloud on the device: appends its bars (device) at *nbars and writes stats.
// Everything one call produces besides the bars (which stay on the device).
struct BatchOut {
  std::vector<float> t_eff;                 // per cloud
  std::vector<rips_stats_t> stats;          // clouds * (dim_max + 1)
  std::vector<float> phase_ms;
  float kernel_ms[RIPS_KERNEL_CLASSES] = {};
  int64_t kernel_regions[RIPS_KERNEL_CLASSES] = {};
  uint32_t nbars = 0;
};

int sync_read(Workspace& w, cudaStream_t s) {
  (void)w;
  CK(cudaStreamSynchronize(s));
  return RIPS_OK;
}

int bits_of_count(uint64_t count) { return std::max(1, bit_width64(count ? count - 1 : 0)); }

// One cloud given by its edges only (no n x n matrix): a list of (i, j,
// length) entries, or a point cloud whose pairs within the threshold are found
// on the device.
struct SparseIn {
  const int32_t* ei = nullptr;
  const int32_t* ej = nullptr;
  const float* len = nullptr;
  uint64_t m = 0;
  const float* pts = nullptr;
  int k = 0;
};

// The whole barcode pipeline for a batch of clouds whose n_c x n_c distance
// matrices lie back to back at dD -- or, with `sp`, for one cloud given by its
// edges, which never forms an n x n array.  Bars are left in w.bars (device),
// with the statistics, thresholds and timings in `out`.
int run_batch(Workspace& w, const float* dD, const std::vector<int64_t>& ns, int dim_max, float threshold,
              uint32_t p, cudaStream_t s, BatchOut& out, const SparseIn* sp = nullptr) {
  HostPinned* hp = w.pinned;
  const int C = (int)ns.size();
  const int kmax = dim_max + 2;
  const int SPC = (dim_max + 1) * 16;  // statistics counters per cloud
  w.kev_used = 0;
  if (w.events) CK(cudaEventRecord(w.tev[0], s));

  // ---------------- cloud table
  int n_max = 1;
  uint64_t N = 0, RR = 0, e_cap = 0, tiles = 0;
  std::vector<CloudInfo> ci(C);
  std::vector<uint32_t> tile_off(C + 1, 0);
  for (int c = 0; c < C; ++c) {
    const int n = (int)ns[c];
    n_max = std::max(n_max, n);
    ci[c].n = n;
    ci[c].voff = (uint32_t)N;
    ci[c].roff = RR;
    ci[c].eoff = 0;
    ci[c].m = 0;
    ci[c].t_eff = 0;
    ci[c].pad = 0;
    N += n;
    RR += (uint64_t)n * n;
    e_cap += (uint64_t)n * (n - 1) / 2;
    const uint64_t nb = (n + 31) / 32;
    tile_off[c] = (uint32_t)tiles;
    tiles += nb * (nb + 1) / 2;
  }
  tile_off[C] = (uint32_t)tiles;
  if (sp) {  // a sparse input: no matrix, and the edge list's room is what the input needs
    if (C != 1) return RIPS_ERR_BAD_ARG;
    RR = 0;
    tiles = 0;
    e_cap = sp->pts ? std::min<uint64_t>(e_cap, 64ull * (uint64_t)n_max + 1024) : std::max<uint64_t>(sp->m, 1);
    const float t = (std::isnan(threshold) || std::isinf(threshold)) ? INFINITY : threshold;
    ci[0].t_eff = t;
  }
  if (N > 0xFFFFFFF0ull || e_cap > 0xFFFFFFF0ull || tiles > 0x7FFFFFFFull) return RIPS_ERR_OVERFLOW;
  const int cb = C > 1 ? bit_width64((uint64_t)C - 1) : 0;
  const int eb = bits_of_count(host_binom(n_max, 2));
  if (cb + 32 + eb > 64) return RIPS_ERR_OVERFLOW;
  CR(ensure(w.clouds, (size_t)C * sizeof(CloudInfo)));
  CR(ensure(w.tileoff, (size_t)(C + 1) * 4));
  CR(ensure(w.vcloud, (size_t)N * 4));
  CR(ensure(w.ccounts, (size_t)(C + 1) * 4));
  CloudInfo* dclouds = P<CloudInfo>(w.clouds);
  CK(cudaMemcpyAsync(dclouds, ci.data(), (size_t)C * sizeof(CloudInfo), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(w.tileoff.p, tile_off.data(), (size_t)(C + 1) * 4, cudaMemcpyHostToDevice, s));

  // ---------------- prologue
  CR(ensure(w.rowmax, (size_t)N * 4));
  CR(ensure(w.teff, 16));
  CR(ensure(w.err, 16));
  CR(ensure(w.ecount, 16));
  CR(ensure(w.ekeys, e_cap * 8));
  CR(ensure(w.ekeys_alt, e_cap * 8));
  CK(cudaMemsetAsync(w.rowmax.p, 0, (size_t)N * 4, s));
  CK(cudaMemsetAsync(w.err.p, 0, 16, s));
  CK(cudaMemsetAsync(w.ecount.p, 0, 16, s));
  CK(cudaMemsetAsync(w.ccounts.p, 0, (size_t)(C + 1) * 4, s));
  std::vector<uint32_t> ccount(C);
  if (!sp) {
    {
      KTimer kt(w, RIPS_K_PROLOGUE, s);
      CK(launch_cloud_vertices(dclouds, C, P<uint32_t>(w.vcloud), s));
      CK(launch_validate_rowmax(dD, dclouds, P<uint32_t>(w.tileoff), C, (uint32_t)tiles, P<uint32_t>(w.rowmax),
                                P<uint32_t>(w.err), s));
      CK(launch_threshold(P<uint32_t>(w.rowmax), dclouds, C, threshold, s));
      CK(launch_edge_keys(dD, dclouds, P<uint32_t>(w.vcloud), (uint32_t)N, eb, P<uint64_t>(w.ekeys),
                          P<uint32_t>(w.ecount), P<uint32_t>(w.ccounts), (uint32_t)e_cap, s));
    }
    CK(cudaMemcpyAsync(&hp->u32[0], w.ecount.p, 4, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(&hp->u32[1], w.err.p, 4, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(ccount.data(), w.ccounts.p, (size_t)C * 4, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(ci.data(), dclouds, (size_t)C * sizeof(CloudInfo), cudaMemcpyDeviceToHost, s));
    CR(sync_read(w, s));
  } else {
    // the edges within the threshold, grown and listed again if the room was short
    for (int attempt = 0; attempt < 8; ++attempt) {
      {
        KTimer kt(w, RIPS_K_PROLOGUE, s);
        CK(launch_cloud_vertices(dclouds, C, P<uint32_t>(w.vcloud), s));
        if (sp->pts)
          CK(launch_point_edges(sp->pts, n_max, sp->k, ci[0].t_eff, eb, P<uint64_t>(w.ekeys), P<uint32_t>(w.ecount),
                                (uint32_t)e_cap, s));
        else
          CK(launch_coo_edge_keys(sp->ei, sp->ej, sp->len, sp->m, n_max, ci[0].t_eff, eb, P<uint64_t>(w.ekeys),
                                  P<uint32_t>(w.ecount), (uint32_t)e_cap, P<uint32_t>(w.err), s));
      }
      CK(cudaMemcpyAsync(&hp->u32[0], w.ecount.p, 4, cudaMemcpyDeviceToHost, s));
      CK(cudaMemcpyAsync(&hp->u32[1], w.err.p, 4, cudaMemcpyDeviceToHost, s));
      CR(sync_read(w, s));
      if (hp->u32[1] & ERRF_BAD_INPUT) return RIPS_ERR_BAD_ARG;
      if (hp->u32[0] <= e_cap) break;
      e_cap = hp->u32[0];
      CR(ensure(w.ekeys, e_cap * 8));
      CR(ensure(w.ekeys_alt, e_cap * 8));
      CK(cudaMemsetAsync(w.ecount.p, 0, 16, s));
    }
    if (hp->u32[0] > e_cap) return RIPS_ERR_INTERNAL;
    ccount[0] = hp->u32[0];
  }
  if (hp->u32[1] & ERRF_BAD_INPUT) return RIPS_ERR_BAD_ARG;
  const uint32_t m = hp->u32[0];
  out.t_eff.resize(C);
  {
    uint32_t acc = 0;
    for (int c = 0; c < C; ++c) {
      ci[c].eoff = acc;
      ci[c].m = ccount[c];
      acc += ccount[c];
      out.t_eff[c] = ci[c].t_eff;
    }
  }
  CK(cudaMemcpyAsync(dclouds, ci.data(), (size_t)C * sizeof(CloudInfo), cudaMemcpyHostToDevice, s));

  // sort edges: (cloud, length bits, inverted index) ascending = each cloud's filtration order
  CR(ensure(w.sorttmp, std::max(sort_temp_bytes(m), scan_temp_bytes((uint32_t)std::max<uint64_t>(m, N + 1)))));
  bool alt = false;
  {
    KTimer kt(w, RIPS_K_EDGE_SORT, s);
    CK(radix_sort_u64(P<uint64_t>(w.ekeys), P<uint64_t>(w.ekeys_alt), nullptr, nullptr, m, cb + 32 + eb,
                      w.sorttmp.p, w.sorttmp.cap, &alt, s));
  }
  const uint64_t* keys = alt ? P<uint64_t>(w.ekeys_alt) : P<uint64_t>(w.ekeys);

  CR(ensure(w.eflags, (size_t)(m + 1) * 4));
  CR(ensure(w.erank, (size_t)(m + 1) * 4));
  CR(ensure(w.rvalue, (size_t)(m + 1) * 4));
  if (!sp) CR(ensure(w.R, RR * 4));
  CR(ensure(w.deg, (size_t)(N + 2) * 4));
  {
    KTimer kt(w, RIPS_K_PROLOGUE, s);
    CK(launch_assign_ranks(keys, m, eb, P<uint32_t>(w.eflags), (uint32_t*)w.sorttmp.p, P<uint32_t>(w.erank),
                           P<float>(w.rvalue), &P<uint32_t>(w.ecount)[1], s));
    CK(cudaMemsetAsync(w.deg.p, 0, (size_t)(N + 2) * 4, s));
    if (!sp) {
      CK(cudaMemsetAsync(w.R.p, 0xFF, RR * 4, s));
      CK(launch_fill_rank_matrix(keys, P<uint32_t>(w.erank), m, eb, dclouds, P<uint32_t>(w.R), s));
      CK(launch_neighbor_counts(P<uint32_t>(w.R), dclouds, P<uint32_t>(w.vcloud), (uint32_t)N, P<uint32_t>(w.deg),
                                &P<uint32_t>(w.ecount)[3], s));
    } else {
      CK(cudaMemsetAsync((char*)w.ecount.p + 12, 0, 4, s));
      CK(launch_sparse_degrees(keys, m, eb, P<uint32_t>(w.deg), s));
      CK(launch_max(P<uint32_t>(w.deg), (uint32_t)N, &P<uint32_t>(w.ecount)[3], s));
    }
    CK(launch_exclusive_scan(P<uint32_t>(w.deg), P<uint32_t>(w.deg), (uint32_t)N + 1, w.sorttmp.p,
                             &P<uint32_t>(w.ecount)[2], s));
  }
  CK(cudaMemcpyAsync(&hp->u32[2], (char*)w.ecount.p + 4, 12, cudaMemcpyDeviceToHost, s));
  CR(sync_read(w, s));
  const uint32_t num_ranks = hp->u32[2];
  const uint32_t nbr_total = hp->u32[3];
  const uint32_t max_deg = hp->u32[4];
  CR(ensure(w.nbr, (size_t)nbr_total * 4 + 4));
  CR(ensure(w.binom, (size_t)(kmax + 1) * (n_max + 1) * 8));
  if (sp) {  // both directions of every edge with its rank, sorted into decreasing neighbour order
    const uint32_t q = nbr_total;
    CR(ensure(w.nrank, (size_t)q * 4 + 4));
    CR(ensure(w.nkey, (size_t)q * 8 + 8));
    CR(ensure(w.nkey_alt, (size_t)q * 8 + 8));
    CR(ensure(w.nval, (size_t)q * 4 + 4));
    CR(ensure(w.nval_alt, (size_t)q * 4 + 4));
    CR(ensure(w.cursor, (size_t)N * 4 + 4));
    CR(ensure(w.sorttmp, std::max(w.sorttmp.cap, sort_temp_bytes(q))));
    KTimer kt(w, RIPS_K_PROLOGUE, s);
    CK(cudaMemsetAsync(w.cursor.p, 0, (size_t)N * 4, s));
    CK(launch_sparse_fill(keys, P<uint32_t>(w.erank), m, eb, P<uint32_t>(w.deg), P<uint32_t>(w.cursor),
                          P<uint64_t>(w.nkey), P<uint32_t>(w.nval), s));
    bool nalt = false;
    CK(radix_sort_u64(P<uint64_t>(w.nkey), P<uint64_t>(w.nkey_alt), P<uint32_t>(w.nval), P<uint32_t>(w.nval_alt), q,
                      32 + bit_width64((uint64_t)n_max), w.sorttmp.p, w.sorttmp.cap, &nalt, s));
    CK(launch_sparse_unpack(nalt ? P<uint64_t>(w.nkey_alt) : P<uint64_t>(w.nkey),
                            nalt ? P<uint32_t>(w.nval_alt) : P<uint32_t>(w.nval), q, P<uint32_t>(w.nbr),
                            P<uint32_t>(w.nrank), s));
    CK(launch_binomial_table(P<uint64_t>(w.binom), n_max, kmax, s));
  } else {
    KTimer kt(w, RIPS_K_PROLOGUE, s);
    CK(launch_neighbor_fill(P<uint32_t>(w.R), dclouds, P<uint32_t>(w.vcloud), (uint32_t)N, P<uint32_t>(w.deg),
                            P<uint32_t>(w.nbr), s));
    CK(launch_binomial_table(P<uint64_t>(w.binom), n_max, kmax, s));
  }

  // ---------------- H0
  CR(grow_keep(w.bars, ((size_t)N + 16) * sizeof(rips_bar_t), 0, s));
  CR(ensure(w.eu, (size_t)(m + 1) * 4));
  CR(ensure(w.ev, (size_t)(m + 1) * 4));
  CR(ensure(w.inforest, (size_t)m + 1));
  CR(ensure(w.nbars, 16));
  CR(ensure(w.stats, (size_t)C * SPC * 8));
  CK(cudaMemsetAsync(w.stats.p, 0, (size_t)C * SPC * 8, s));
  CK(cudaMemsetAsync(w.nbars.p, 0, 4, s));
  unsigned long long* dstats = P<unsigned long long>(w.stats);
  {
    KTimer kt(w, RIPS_K_H0, s);
    if (h0_blocks_fit(n_max)) {
      CK(launch_h0_blocks(dclouds, C, n_max, keys, eb, P<uint32_t>(w.eu), P<uint32_t>(w.ev), m,
                          P<uint8_t>(w.inforest), P<rips_bar_t>(w.bars), P<uint32_t>(w.nbars),
                          (uint32_t)(w.bars.cap / sizeof(rips_bar_t)), dstats, SPC, P<uint32_t>(w.err), s));
    } else {
      if (C != 1) return RIPS_ERR_BAD_ARG;
      const int n = n_max;
      CR(ensure(w.comp, (size_t)n * 4));
      CR(ensure(w.best, (size_t)n * 4));
      CR(ensure(w.parent, (size_t)n * 4));
      CR(ensure(w.gtop, (size_t)n * 4));
      CR(ensure(w.fpos, (size_t)n * 4));
      CR(ensure(w.nf, 16));
      CK(run_h0_large(n, keys, m, eb, P<uint32_t>(w.eu), P<uint32_t>(w.ev), P<uint32_t>(w.comp), P<uint32_t>(w.best),
                      P<uint32_t>(w.parent), P<uint8_t>(w.inforest), P<uint32_t>(w.eflags), P<uint32_t>(w.fpos),
                      w.sorttmp.p, P<uint32_t>(w.nf), P<uint32_t>(w.gtop), P<rips_bar_t>(w.bars),
                      P<uint32_t>(w.nbars), (uint32_t)(w.bars.cap / sizeof(rips_bar_t)), dstats, P<uint32_t>(w.err),
                      s));
    }
  }
  if (w.events) CK(cudaEventRecord(w.tev[1], s));

  // ---------------- dimensions 1..dim_max
  const int rank_bits = bit_width64(num_ranks ? num_ranks - 1 : 0);
  uint32_t ns_prev = 0;  // size of the (d-1)-simplex list in sidx[cur^1]
  int prev_col_bits = 0;
  int cur = 0;
  uint64_t* prev_tkeys = nullptr;
  uint64_t prev_tmask = 0;
  const uint64_t* prev_amap = nullptr;
  uint64_t prev_amask = 0;
  for (int d = 1; d <= dim_max; ++d) {
    DimArgs a;
    a.d = d;
    a.nclouds = C;
    a.clouds = dclouds;
    a.R = sp ? nullptr : P<uint32_t>(w.R);
    a.nbr_off = P<uint32_t>(w.deg);
    a.nbr = P<uint32_t>(w.nbr);
    a.nrank = sp ? P<uint32_t>(w.nrank) : nullptr;
    a.binom = P<uint64_t>(w.binom);
    a.bn = n_max;
    a.kmax = kmax;
    a.smem_binom = (size_t)(kmax + 1) * (n_max + 1) * 8 <= 48 * 1024;
    a.p = p;
    a.col_bits = bits_of_count(host_binom(n_max, d + 1));
    a.row_bits = bits_of_count(host_binom(n_max, d + 2));
    a.rank_bits = rank_bits;
    a.rank_max = num_ranks ? num_ranks - 1 : 0;
    a.err = P<uint32_t>(w.err);
    a.amap = nullptr;
    a.amap_mask = 0;
    a.vbits = 0;
    a.pmap = prev_amap;
    a.pmap_mask = prev_amask;
    {
      const rips_tuning_t tu = tuning_for(d, n_max);
      a.chain_limit = (uint32_t)tu.warp_chain_limit;
      a.merge_max = (uint32_t)tu.warp_merge_max;
      a.reduce_blocks_per_sm = tu.reduce_blocks_per_sm;
      a.scan_blocks_per_sm = tu.scan_blocks_per_sm;
    }
    a.opts = current_options();
    if (rank_bits + a.row_bits > 63 || cb + rank_bits + a.col_bits > 64 || cb + a.row_bits > 64)
      return RIPS_ERR_OVERFLOW;
    unsigned long long* st = dstats + d * 16;  // cloud c: st + c * SPC

    // d-simplices
    uint32_t nsd = 0;
    if (d == 1) {
      nsd = m;
      CR(ensure(w.sidx[cur], (size_t)(m + 1) * 8));
      CR(ensure(w.srank[cur], (size_t)(m + 1) * 4));
      CK(launch_edges_to_simplices(keys, P<uint32_t>(w.erank), m, eb, a.col_bits, P<uint64_t>(w.sidx[cur]),
                                   P<uint32_t>(w.srank[cur]), s));
    } else {
      CR(ensure(w.scount, 16));
      const int pv = cur ^ 1;
      for (int attempt = 0; attempt < 2; ++attempt) {
        unsigned long long cap = w.sidx[cur].cap / 8;
        if (w.srank[cur].cap / 4 < cap) cap = w.srank[cur].cap / 4;
        CK(cudaMemsetAsync(w.scount.p, 0, 8, s));
        {
          KTimer kt(w, RIPS_K_ENUMERATE, s);
          CK(launch_enumerate(a, P<uint64_t>(w.sidx[pv]), P<uint32_t>(w.srank[pv]), ns_prev, prev_col_bits,
                              P<uint64_t>(w.sidx[cur]), P<uint32_t>(w.srank[cur]),
                              P<unsigned long long>(w.scount), cap, s));
        }
        CK(cudaMemcpyAsync(&hp->u64[0], w.scount.p, 8, cudaMemcpyDeviceToHost, s));
        CR(sync_read(w, s));
        const unsigned long long got = hp->u64[0];
        if (got > 0xFFFFFFF0ull) return RIPS_ERR_OVERFLOW;
        if (got <= cap) {
          nsd = (uint32_t)got;
          break;
        }
        CR(ensure(w.sidx[cur], got * 8));
        CR(ensure(w.srank[cur], got * 4));
      }
    }

    // apparent pairs, clearing, compaction
    CR(ensure(w.ckeys, (size_t)(nsd + 1) * 8));
    CR(ensure(w.ckeys_alt, (size_t)(nsd + 1) * 8));
    CR(ensure(w.ccount, 16));
    CK(cudaMemsetAsync(w.ccount.p, 0, 16, s));
    // map of this dimension's zero apparent pairs (at most one per tested simplex)
    uint64_t acap = 16;
    while (acap < 2ull * nsd + 16) acap <<= 1;
    if (!(a.opts & RIPS_OPT_NO_APPARENT) && a.col_bits <= 60 &&
        acap * 16 <= (16ull << 30)) {  // else the test and reduction scan instead
      CR(ensure(w.amk[cur], (size_t)acap * 16));
      CK(cudaMemsetAsync(w.amk[cur].p, 0xFF, (size_t)acap * 16, s));
      a.amap = P<uint64_t>(w.amk[cur]);
      a.amap_mask = acap - 1;
      a.vbits = packed_vertex_bits(n_max, d);
    }
    {
      KTimer kt(w, RIPS_K_APPARENT, s);
      CK(launch_test(a, P<uint64_t>(w.sidx[cur]), P<uint32_t>(w.srank[cur]), nsd, P<uint8_t>(w.inforest), prev_tkeys,
                     prev_tmask, P<uint64_t>(w.ckeys), P<uint32_t>(w.ccount), nsd + 1, st, SPC, s));
    }
    CK(cudaMemcpyAsync(&hp->u32[5], w.ccount.p, 4, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(&hp->u32[10], w.nbars.p, 4, cudaMemcpyDeviceToHost, s));
    CR(sync_read(w, s));
    const uint32_t M = hp->u32[5];
    // processing order
    CR(ensure(w.sorttmp, std::max(w.sorttmp.cap, sort_temp_bytes(M + 1))));
    bool calt = false;
    {
      KTimer kt(w, RIPS_K_COL_SORT, s);
      CK(radix_sort_u64(P<uint64_t>(w.ckeys), P<uint64_t>(w.ckeys_alt), nullptr, nullptr, M,
                        cb + rank_bits + a.col_bits, w.sorttmp.p, w.sorttmp.cap, &calt, s));
    }
    const uint64_t* ckeys = calt ? P<uint64_t>(w.ckeys_alt) : P<uint64_t>(w.ckeys);
    // bars of this dimension are appended after the current count
    CR(grow_keep(w.bars, ((size_t)hp->u32[10] + M + 16) * sizeof(rips_bar_t),
                 (size_t)hp->u32[10] * sizeof(rips_bar_t), s));

    // reduction
    const int tb = cur;  // table for this dimension (the other one holds d-1)
    const rips_limits_t lim = current_limits();
    const uint32_t tcap = lim.table_slots ? (uint32_t)lim.table_slots : pow2_at_least(2ull * M + 16);
    CR(ensure(w.tkeys[tb], (size_t)tcap * 8));
    CR(ensure(w.tvals[tb], (size_t)tcap * 4));
    CR(ensure(w.piv_key, (size_t)(M + 1) * 8));
    CR(ensure(w.piv_coef, (size_t)(M + 1) * 4));
    CR(ensure(w.r_off, (size_t)(M + 1) * 8));
    CR(ensure(w.r_len, (size_t)(M + 1) * 4));
    CR(ensure(w.reduced, (size_t)(M + 1)));
    CR(ensure(w.claim, (size_t)(M + 1) * 4));
    CR(ensure(w.reduce, (size_t)(M + 1) * 4));
    CR(ensure(w.heavy, (size_t)(M + 1) * 8));
    CR(ensure(w.lists, LISTS_BYTES));
    CR(ensure(w.r_top, 16));
    // a generated coboundary holds at most max_deg entries (sorted in a power-of-two buffer)
    const int blocks = M ? reduction_blocks(a, M) : 1;
    if (blocks < 1) return RIPS_ERR_CUDA;
    uint32_t slice = 32;
    while (slice < max_deg + 1) slice <<= 1;
    // The arena holds every run a reduction writes (generated coboundaries,
    // merges, stored columns), which long chains make large; an arena that
    // proves too small costs a rerun of the dimension with 8x the room, so a
    // first call starts at up to 2^30 entries (12 GB) when the device has 16x
    // that free (the workspace keeps it for later calls).
    size_t rcap = lim.arena_entries ? (size_t)lim.arena_entries
                                    : std::max<size_t>(w.r_cap, std::max<size_t>(16 * (size_t)M, (size_t)1 << 22));
    if (!lim.arena_entries && M > 4096) {
      size_t free_b = 0, total_b = 0;
      if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess) {
        const size_t roomy = std::min<size_t>((size_t)1 << 30, free_b / 16 / 12);
        rcap = std::max(rcap, roomy);
      } else {
        cudaGetLastError();
      }
    }
    bool done = false;
    for (int attempt = 0; attempt < 6 && !done; ++attempt) {
      CR(ensure(w.r_key, rcap * 8));
      CR(ensure(w.r_coef, rcap * 4));
      w.r_cap = rcap;
      CK(cudaMemsetAsync(w.tkeys[tb].p, 0xFF, (size_t)tcap * 8, s));
      CK(cudaMemsetAsync(w.tvals[tb].p, 0xFF, (size_t)tcap * 4, s));
      CK(cudaMemsetAsync(w.lists.p, 0, LISTS_BYTES, s));
      CK(cudaMemsetAsync(w.r_top.p, 0, 16, s));
      uint32_t* counts = P<uint32_t>(w.lists);
      RedState rs;
      rs.col_keys = ckeys;
      rs.ncols = M;
      rs.piv_key = P<uint64_t>(w.piv_key);
      rs.piv_coef = P<uint32_t>(w.piv_coef);
      rs.reduced = P<uint8_t>(w.reduced);
      rs.r_key = P<uint64_t>(w.r_key);
      rs.r_coef = P<uint32_t>(w.r_coef);
      rs.r_off = P<unsigned long long>(w.r_off);
      rs.r_len = P<uint32_t>(w.r_len);
      rs.r_top = P<unsigned long long>(w.r_top);
      rs.r_cap = rcap;
      rs.scr_slice = slice;
      rs.t_keys = P<uint64_t>(w.tkeys[tb]);
      rs.t_vals = P<uint32_t>(w.tvals[tb]);
      rs.t_mask = tcap - 1;
      rs.claim_list = P<uint32_t>(w.claim);
      rs.reduce_list = P<uint32_t>(w.reduce);
      rs.heavy_list = P<uint32_t>(w.heavy);
      rs.ncols_dev = nullptr;
      rs.steps = P<unsigned long long>(w.lists) + 4;
      rs.compacted = P<unsigned long long>(w.lists) + 5;
      rs.max_chain = counts + 7;
      rs.heartbeat = counts + 12;
      rs.added = P<unsigned long long>(w.lists) + 7;
      rs.help = (HelpBoard*)(P<unsigned char>(w.lists) + 256);
      rs.idle = counts + 4;
      rs.barrier_ns = lim.barrier_wait_ns ? lim.barrier_wait_ns : 30ull * 1000 * 1000 * 1000;
      rs.chain_ns = lim.chain_ns ? lim.chain_ns : 600ull * 1000 * 1000 * 1000;
      rs.err = P<uint32_t>(w.err);
      {
        KTimer kt(w, RIPS_K_REDUCE, s);
        CK(launch_reduction(a, rs, blocks, counts, s));
      }
      CK(cudaMemcpyAsync(&hp->u32[6], counts + 6, 4, cudaMemcpyDeviceToHost, s));
      CK(cudaMemcpyAsync(&hp->u32[8], w.err.p, 4, cudaMemcpyDeviceToHost, s));
      CK(cudaMemcpyAsync(&hp->u64[1], rs.steps, 16, cudaMemcpyDeviceToHost, s));
      CK(cudaMemcpyAsync(&hp->u64[3], rs.added, 8, cudaMemcpyDeviceToHost, s));
      CK(cudaMemcpyAsync(&hp->u32[9], counts + 7, 4, cudaMemcpyDeviceToHost, s));
      CR(sync_read(w, s));
      if (hp->u32[8] & ERRF_ARENA) {
        // start this dimension's reduction over with a larger arena
        CK(cudaMemsetAsync(w.err.p, 0, 4, s));
        rcap *= 8;
        continue;
      }
      if (int e = map_device_error(hp->u32[8])) return e;
      out.stats.resize((size_t)C * (dim_max + 1));
      // rounds and steps are properties of the whole batch's reduction
      for (int c = 0; c < C; ++c) {
        out.stats[(size_t)c * (dim_max + 1) + d].rounds = hp->u32[6];
        out.stats[(size_t)c * (dim_max + 1) + d].reduction_steps = (int64_t)hp->u64[1];
        out.stats[(size_t)c * (dim_max + 1) + d].longest_chain = hp->u32[9];
        out.stats[(size_t)c * (dim_max + 1) + d].compacted_entries = (int64_t)hp->u64[2];
        out.stats[(size_t)c * (dim_max + 1) + d].added_entries = (int64_t)hp->u64[3];
      }
      {
        KTimer kt(w, RIPS_K_READOUT, s);
        CK(launch_readout(a, rs, P<float>(w.rvalue), P<rips_bar_t>(w.bars), P<uint32_t>(w.nbars),
                          (uint32_t)(w.bars.cap / sizeof(rips_bar_t)), st, SPC, s));
      }
      done = true;
    }
    if (!done) return RIPS_ERR_OOM;
    prev_tkeys = P<uint64_t>(w.tkeys[tb]);
    prev_amap = a.amap;
    prev_amask = a.amap_mask;
    prev_tmask = tcap - 1;
    ns_prev = nsd;
    prev_col_bits = a.col_bits;
    cur ^= 1;
    if (w.events && d + 1 < 16) CK(cudaEventRecord(w.tev[d + 1], s));
  }

  // statistics and bar count
  std::vector<unsigned long long> hstats((size_t)C * SPC);
  CK(cudaMemcpyAsync(hstats.data(), dstats, (size_t)C * SPC * 8, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(&hp->u32[11], w.nbars.p, 4, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(&hp->u32[12], w.err.p, 4, cudaMemcpyDeviceToHost, s));
  CR(sync_read(w, s));
  if (int e = map_device_error(hp->u32[12])) return e;
  out.nbars = hp->u32[11];
  out.stats.resize((size_t)C * (dim_max + 1));
  for (int c = 0; c < C; ++c) {
    const unsigned long long* q0 = hstats.data() + (size_t)c * SPC;
    rips_stats_t& s0 = out.stats[(size_t)c * (dim_max + 1)];
    s0.simplices = ns[c];
    s0.columns = ns[c];
    s0.pairs = (int64_t)q0[0];
    s0.zero_pairs = (int64_t)q0[1];
    s0.essential = (int64_t)q0[2];
    for (int d = 1; d <= dim_max; ++d) {
      const unsigned long long* q = q0 + d * 16;
      rips_stats_t& sd = out.stats[(size_t)c * (dim_max + 1) + d];
      sd.pairs = (int64_t)q[0];
      sd.zero_pairs = (int64_t)q[1];
      sd.essential = (int64_t)q[2];
      sd.emergent = (int64_t)q[3];
      sd.apparent_cofacet = (int64_t)q[4];
      sd.apparent_facet = (int64_t)q[5];
      sd.cleared = (int64_t)q[6];
      // columns = pairs found by the reduction + essential classes; simplices = all four categories
      sd.columns = sd.pairs + sd.essential;
      sd.simplices = sd.apparent_cofacet + sd.apparent_facet + sd.cleared + sd.columns;
    }
  }
  for (size_t q = 0; q < w.kev_used; ++q) {
    float ms = 0;
    if (cudaEventElapsedTime(&ms, w.kev[2 * q], w.kev[2 * q + 1]) == cudaSuccess) {
      out.kernel_ms[w.kev_class[q]] += ms;
      out.kernel_regions[w.kev_class[q]] += 1;
    } else {
      cudaGetLastError();
    }
  }
  w.kev_used = 0;
  if (w.events) {
    out.phase_ms.clear();
    for (int d = 0; d <= dim_max && d + 1 < 16; ++d) {
      float ms = 0;
      cudaEventElapsedTime(&ms, w.tev[d], w.tev[d + 1]);
      out.phase_ms.push_back(ms);
    }
  }
  return RIPS_OK;
}

// canonical order on the device and copy to the host
int finish_bars(Workspace& w, uint32_t nb, int simplex_bits, int group_bits, cudaStream_t s,
                std::vector<rips_bar_t>& host) {
  host.resize(nb);
  if (nb == 0) return RIPS_OK;
  CR(ensure(w.bars_alt, (size_t)nb * sizeof(rips_bar_t)));
  CR(ensure(w.bk0, (size_t)nb * 8));
  CR(ensure(w.bk1, (size_t)nb * 8));
  CR(ensure(w.bp0, (size_t)nb * 4));
  CR(ensure(w.bp1, (size_t)nb * 4));
  CR(ensure(w.bartmp, bar_order_temp_bytes(nb)));
  CK(launch_bar_order(P<rips_bar_t>(w.bars), P<rips_bar_t>(w.bars_alt), nb, P<uint64_t>(w.bk0), P<uint64_t>(w.bk1),
                      P<uint32_t>(w.bp0), P<uint32_t>(w.bp1), w.bartmp.p, w.bartmp.cap, simplex_bits, group_bits, s));
  CK(cudaMemcpyAsync(host.data(), w.bars_alt.p, (size_t)nb * sizeof(rips_bar_t), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return RIPS_OK;
}

void index_result(rips_result* r) {
  const int D = r->dim_max + 1;
  r->offsets.assign((size_t)r->clouds * D + 1, 0);
  std::vector<int64_t> cnt((size_t)r->clouds * D, 0);
  for (const auto& b : r->bars) ++cnt[(size_t)b.cloud * D + b.dim];
  for (size_t i = 0; i < cnt.size(); ++i) r->offsets[i + 1] = r->offsets[i] + cnt[i];
}

void fill_result(rips_result* r, const BatchOut& bo) {
  r->thresholds = bo.t_eff;
  r->stats = bo.stats;
  r->phase_ms = bo.phase_ms;
  for (int q = 0; q < RIPS_KERNEL_CLASSES; ++q) {
    r->kernel_ms[q] = bo.kernel_ms[q];
    r->kernel_launches[q] = bo.kernel_regions[q];
  }
}

// caller holds w.mu
int barcodes_locked(Workspace& w, const float* dD, int64_t n, int32_t dim_max, float threshold, uint32_t p,
                    cudaStream_t s, rips_result_t** out) {
  rips_result* r = new (std::nothrow) rips_result();
  if (!r) return RIPS_ERR_OOM;
  r->clouds = 1;
  r->dim_max = dim_max;
  BatchOut bo;
  std::vector<int64_t> ns{n};
  int rc = run_batch(w, dD, ns, dim_max, threshold, p, s, bo);
  if (rc == RIPS_OK) {
    const int sbits = std::max(1, bit_width64(host_binom((uint64_t)n, dim_max + 1)));
    rc = finish_bars(w, bo.nbars, sbits, 0, s, r->bars);
  }
  if (rc != RIPS_OK) {
    delete r;
    return rc;
  }
  fill_result(r, bo);
  r->npoints.push_back(n);
  r->point_offsets = {0, n};
  index_result(r);
  *out = r;
  return RIPS_OK;
}

// one cloud given by its edges (SparseIn): the barcode without an n x n array
int sparse_locked(Workspace& w, const SparseIn& sp, int64_t n, int32_t dim_max, float threshold, uint32_t p,
                  cudaStream_t s, rips_result_t** out) {
  rips_result* r = new (std::nothrow) rips_result();
  if (!r) return RIPS_ERR_OOM;
  r->clouds = 1;
  r->dim_max = dim_max;
  r->k = sp.pts ? sp.k : 0;
  BatchOut bo;
  std::vector<int64_t> ns{n};
  int rc = run_batch(w, nullptr, ns, dim_max, threshold, p, s, bo, &sp);
  if (rc == RIPS_OK) {
    const int sbits = std::max(1, bit_width64(host_binom((uint64_t)n, dim_max + 1)));
    rc = finish_bars(w, bo.nbars, sbits, 0, s, r->bars);
  }
  if (rc != RIPS_OK) {
    delete r;
    return rc;
  }
  fill_result(r, bo);
  r->npoints.push_back(n);
  r->point_offsets = {0, n};
  index_result(r);
  *out = r;
  return RIPS_OK;
}

// sparse inputs: vertex ids and edge indices stay within 32 and 64 bits
int check_sparse_args(int64_t n, int32_t dim_max, float threshold, uint32_t p) {
  if (n < 1 || n > 92681 || dim_max < 0 || dim_max > MAX_DIM - 1) return RIPS_ERR_BAD_ARG;
  if (!std::isnan(threshold) && threshold < 0.0f) return RIPS_ERR_BAD_ARG;
  if (!is_prime(p) || p >= 65536) return RIPS_ERR_BAD_MODULUS;
  if (host_binom((uint64_t)n, dim_max + 2) >= (1ull << 63)) return RIPS_ERR_OVERFLOW;
  return RIPS_OK;
}

Workspace* current_workspace() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return workspace(dev);
}

// all clouds' distance matrices in one launch, then one pipeline for the batch
int batched_locked(Workspace& w, const float* d_points, const int64_t* offsets, int32_t batch, int32_t k,
                   int32_t dim_max, float threshold, uint32_t p, cudaStream_t s, rips_result_t** out) {
  rips_result* r = new (std::nothrow) rips_result();
  if (!r) return RIPS_ERR_OOM;
  r->clouds = batch;
  r->dim_max = dim_max;
  r->k = k;
  std::vector<int64_t> ns(batch);
  std::vector<CloudInfo> ci(batch);
  std::vector<uint32_t> row_off(batch + 1, 0);
  uint64_t RR = 0, rows = 0;
  int64_t nmax = 1;
  for (int32_t c = 0; c < batch; ++c) {
    ns[c] = offsets[c + 1] - offsets[c];
    nmax = std::max<int64_t>(nmax, ns[c]);
    ci[c] = CloudInfo{(int)ns[c], (uint32_t)offsets[c], RR, 0, 0, 0.0f, 0};
    RR += (uint64_t)ns[c] * ns[c];
    row_off[c] = (uint32_t)rows;
    rows += (ns[c] + 7) / 8;
  }
  row_off[batch] = (uint32_t)rows;
  int rc = ensure(w.cdist, RR * 4);
  if (rc == RIPS_OK) rc = ensure(w.clouds, (size_t)batch * sizeof(CloudInfo));
  if (rc == RIPS_OK) rc = ensure(w.tileoff, (size_t)(batch + 1) * 4);
  if (rc == RIPS_OK) {
    if (cudaMemcpyAsync(w.clouds.p, ci.data(), (size_t)batch * sizeof(CloudInfo), cudaMemcpyHostToDevice, s) !=
            cudaSuccess ||
        cudaMemcpyAsync(w.tileoff.p, row_off.data(), (size_t)(batch + 1) * 4, cudaMemcpyHostToDevice, s) !=
            cudaSuccess ||
        launch_distance_matrices(d_points, k, P<CloudInfo>(w.clouds), P<uint32_t>(w.tileoff), batch, (uint32_t)rows,
                                 P<float>(w.cdist), s) != cudaSuccess) {
      cudaGetLastError();
      rc = RIPS_ERR_CUDA;
    }
  }
  BatchOut bo;
  if (rc == RIPS_OK) rc = run_batch(w, P<float>(w.cdist), ns, dim_max, threshold, p, s, bo);
  if (rc == RIPS_OK) {
    const int sbits = std::max(1, bit_width64(host_binom((uint64_t)nmax, dim_max + 1)));
    rc = finish_bars(w, bo.nbars, sbits, std::max(1, bit_width64((uint64_t)batch)), s, r->bars);
  }
  if (rc != RIPS_OK) {
    delete r;
    return rc;
  }
  fill_result(r, bo);
  r->npoints = ns;
  r->point_offsets.assign(offsets, offsets + batch + 1);
  index_result(r);
  *out = r;
  return RIPS_OK;
}

int backward_locked(Workspace& w, const rips_result* r, const float* d_points, int32_t k, const float* gb,
                    const float* gd, float* gx, float* gdist, cudaStream_t s) {
  const uint32_t nb = (uint32_t)r->bars.size();
  if (nb == 0) return RIPS_OK;
  const int C = r->clouds;
  std::vector<int64_t> off(2 * (size_t)C + 2, 0);
  for (int c = 0; c <= C; ++c) off[c] = r->point_offsets[c];
  int64_t acc = 0;
  for (int c = 0; c < C; ++c) {
    off[C + 1 + c] = acc;
    acc += r->npoints[c] * r->npoints[c];
  }
  CR(ensure(w.bwd_bars, (size_t)nb * sizeof(rips_bar_t)));
  CR(ensure(w.bwd_off, off.size() * 8));
  CK(cudaMemcpyAsync(w.bwd_bars.p, r->bars.data(), (size_t)nb * sizeof(rips_bar_t), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(w.bwd_off.p, off.data(), off.size() * 8, cudaMemcpyHostToDevice, s));
  CK(launch_backward(P<rips_bar_t>(w.bwd_bars), nb, d_points, k, P<int64_t>(w.bwd_off),
                     P<int64_t>(w.bwd_off) + C + 1, gb, gd, gx, gdist, s));
  CK(cudaStreamSynchronize(s));  // the host-side copies above must finish before returning
  return RIPS_OK;
}


// batched over distance matrices: the clouds' matrices are gathered back to
// back into the workspace, then one pipeline runs for the batch
int batched_dists_locked(Workspace& w, const float* const* d_dists, const int64_t* ns_in, int32_t batch,
                         int32_t dim_max, float threshold, uint32_t p, cudaStream_t s, rips_result_t** out) {
  rips_result* r = new (std::nothrow) rips_result();
  if (!r) return RIPS_ERR_OOM;
  r->clouds = batch;
  r->dim_max = dim_max;
  std::vector<int64_t> ns(ns_in, ns_in + batch);
  std::vector<int64_t> poff(batch + 1, 0);
  uint64_t RR = 0;
  int64_t nmax = 1;
  for (int32_t c = 0; c < batch; ++c) {
    nmax = std::max<int64_t>(nmax, ns[c]);
    poff[c + 1] = poff[c] + ns[c];
    RR += (uint64_t)ns[c] * ns[c];
  }
  int rc = ensure(w.cdist, RR * 4);
  uint64_t at = 0;
  for (int32_t c = 0; c < batch && rc == RIPS_OK; ++c) {
    const size_t bytes = (size_t)ns[c] * ns[c] * 4;
    if (cudaMemcpyAsync(P<float>(w.cdist) + at, d_dists[c], bytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
      cudaGetLastError();
      rc = RIPS_ERR_CUDA;
    }
    at += (uint64_t)ns[c] * ns[c];
  }
  BatchOut bo;
  if (rc == RIPS_OK) rc = run_batch(w, P<float>(w.cdist), ns, dim_max, threshold, p, s, bo);
  if (rc == RIPS_OK) {
    const int sbits = std::max(1, bit_width64(host_binom((uint64_t)nmax, dim_max + 1)));
    rc = finish_bars(w, bo.nbars, sbits, std::max(1, bit_width64((uint64_t)batch)), s, r->bars);
  }
  if (rc != RIPS_OK) {
    delete r;
    return rc;
  }
  fill_result(r, bo);
  r->npoints = ns;
  r->point_offsets = poff;
  index_result(r);
  *out = r;
  return RIPS_OK;
}

// dL/dD of every cloud of a result from the matrices it was computed from
int backward_dist_locked(Workspace& w, const rips_result* r, const float* const* d_dists, const float* gb,
                         const float* gd, float* const* d_grad, cudaStream_t s) {
  const uint32_t nb = (uint32_t)r->bars.size();
  if (nb == 0) return RIPS_OK;
  const int C = r->clouds;
  // one table: C matrix pointers, C gradient pointers, C sizes (8 bytes each)
  std::vector<uint64_t> tab(3 * (size_t)C);
  for (int c = 0; c < C; ++c) {
    tab[c] = (uint64_t)(uintptr_t)d_dists[c];
    tab[C + c] = (uint64_t)(uintptr_t)d_grad[c];
    tab[2 * C + c] = (uint64_t)r->npoints[c];
  }
  CR(ensure(w.bwd_bars, (size_t)nb * sizeof(rips_bar_t)));
  CR(ensure(w.bwd_off, tab.size() * 8));
  CK(cudaMemcpyAsync(w.bwd_bars.p, r->bars.data(), (size_t)nb * sizeof(rips_bar_t), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(w.bwd_off.p, tab.data(), tab.size() * 8, cudaMemcpyHostToDevice, s));
  uint64_t* dt = P<uint64_t>(w.bwd_off);
  CK(launch_backward_dist(P<rips_bar_t>(w.bwd_bars), nb, (const float* const*)dt, (float* const*)(dt + C),
                          (const int64_t*)(dt + 2 * C), gb, gd, s));
  CK(cudaStreamSynchronize(s));  // the host-side copies above must finish before returning
  return RIPS_OK;
}

// ------------------------------------------------------------------ batch plans
// A batch plan fixes the clouds' sizes (and k, threshold, p; dimensions 0 and
// 1) and sizes every buffer from the worst case at creation: all C(n, 2)
// edges of every cloud, all of them columns.  Lists then have a fixed
// capacity, the parts past their device-side counts are padded with the
// largest key (sorted last, skipped by the kernels), and nothing between two
// kernels needs a count on the host.  plan_run therefore only enqueues device
// work and can be captured into a CUDA graph; plan_result reads everything back
// afterwards.
struct PlanState {
  Workspace w;
  int32_t C = 0, k = 0;
  float threshold = 0.0f;
  uint32_t p = 2;
  int n_max = 1;
  std::vector<int64_t> ns, offsets;
  uint64_t N = 0, RR = 0, e_cap = 0, drows = 0, vtiles = 0;
  int eb = 0, cb = 0;
  DimArgs a{};
  uint32_t tcap = 0;
  uint64_t acap = 0;
  size_t arena = 0;
  int blocks = 0;
  uint32_t slice = 0;
  Buf clouds0, dtile;
};

constexpr int PLAN_SPC = 32;  // statistics counters per cloud (dimensions 0 and 1)

void release(Buf& b) {
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.cap = 0;
}

void release_plan(PlanState& pl) {
  Workspace& w = pl.w;
  Buf* all[] = {&w.dist, &w.binom, &w.rowmax, &w.teff, &w.err, &w.ecount, &w.ekeys, &w.ekeys_alt, &w.eflags,
                &w.escan, &w.erank, &w.rvalue, &w.R, &w.deg, &w.nbr, &w.eu, &w.ev, &w.comp, &w.best, &w.parent,
                &w.gtop, &w.inforest, &w.fpos, &w.nf, &w.sidx[0], &w.sidx[1], &w.srank[0], &w.srank[1],
                &w.scount, &w.ckeys, &w.ckeys_alt, &w.ccount, &w.sorttmp, &w.piv_key, &w.piv_coef, &w.r_off,
                &w.r_len, &w.reduced, &w.claim, &w.reduce, &w.heavy, &w.lists, &w.r_key, &w.r_coef, &w.r_top,
                &w.tkeys[0], &w.tkeys[1], &w.tvals[0], &w.tvals[1], &w.amk[0], &w.amk[1],
                &w.bars, &w.bars_alt, &w.bk0, &w.bk1, &w.bp0, &w.bp1, &w.bartmp, &w.nbars, &w.stats,
                &w.bwd_bars, &w.bwd_off, &w.cdist, &w.clouds, &w.tileoff, &w.vcloud, &w.ccounts, &pl.clouds0,
                &pl.dtile};
  for (Buf* b : all) release(*b);
}

int plan_create(PlanState& pl, const int64_t* offsets, int32_t batch, int32_t k, float threshold, uint32_t p,
                int64_t arena_entries) {
  if (!offsets || batch < 1 || k < 1 || offsets[0] < 0 || arena_entries < 0) return RIPS_ERR_BAD_ARG;
  if (!is_prime(p) || p >= 65536) return RIPS_ERR_BAD_MODULUS;
  if (!std::isnan(threshold) && threshold < 0.0f) return RIPS_ERR_BAD_ARG;
  pl.C = batch;
  pl.k = k;
  pl.threshold = threshold;
  pl.p = p;
  pl.offsets.assign(offsets, offsets + batch + 1);
  pl.ns.resize(batch);
  std::vector<CloudInfo> ci(batch);
  std::vector<uint32_t> dtile(batch + 1), vtile(batch + 1);
  for (int32_t c = 0; c < batch; ++c) {
    const int64_t n = offsets[c + 1] - offsets[c];
    if (n < 1 || n > 46340) return RIPS_ERR_BAD_ARG;
    pl.ns[c] = n;
    pl.n_max = std::max<int>(pl.n_max, (int)n);
    ci[c] = CloudInfo{(int)n, (uint32_t)(offsets[c] - offsets[0]), pl.RR, 0, 0, 0.0f, 0};
    dtile[c] = (uint32_t)pl.drows;
    vtile[c] = (uint32_t)pl.vtiles;
    const uint64_t nb = ((uint64_t)n + 31) / 32;
    pl.N += (uint64_t)n;
    pl.RR += (uint64_t)n * (uint64_t)n;
    pl.e_cap += (uint64_t)n * (uint64_t)(n - 1) / 2;
    pl.drows += ((uint64_t)n + 7) / 8;
    pl.vtiles += nb * (nb + 1) / 2;
  }
  dtile[batch] = (uint32_t)pl.drows;
  vtile[batch] = (uint32_t)pl.vtiles;
  if (pl.e_cap == 0 || !h0_blocks_fit(pl.n_max)) return RIPS_ERR_BAD_ARG;
  if (pl.N > 0xFFFFFFF0ull || pl.e_cap > 0x7FFFFFF0ull || pl.vtiles > 0x7FFFFFFFull || pl.drows > 0x7FFFFFFFull)
    return RIPS_ERR_OVERFLOW;
  pl.cb = batch > 1 ? bit_width64((uint64_t)batch - 1) : 0;
  pl.eb = bits_of_count(host_binom((uint64_t)pl.n_max, 2));
  if (pl.cb + 32 + pl.eb > 64) return RIPS_ERR_OVERFLOW;
  const int kmax = 3;
  DimArgs& a = pl.a;
  a.d = 1;
  a.nclouds = batch;
  a.bn = pl.n_max;
  a.kmax = kmax;
  a.smem_binom = (size_t)(kmax + 1) * (pl.n_max + 1) * 8 <= 48 * 1024;
  a.p = p;
  a.col_bits = bits_of_count(host_binom((uint64_t)pl.n_max, 2));
  a.row_bits = bits_of_count(host_binom((uint64_t)pl.n_max, 3));
  a.rank_bits = bit_width64(pl.e_cap) + 1;  // every rank is below e_cap, the padding's included
  a.rank_max = (uint32_t)pl.e_cap;
  if (a.rank_bits + a.row_bits > 63 || pl.cb + a.rank_bits + a.col_bits > 64 || pl.cb + a.row_bits > 64)
    return RIPS_ERR_OVERFLOW;
  {
    const rips_tuning_t tu = tuning_for(1, pl.n_max);
    a.chain_limit = (uint32_t)tu.warp_chain_limit;
    a.merge_max = (uint32_t)tu.warp_merge_max;
    a.reduce_blocks_per_sm = tu.reduce_blocks_per_sm;
    a.scan_blocks_per_sm = tu.scan_blocks_per_sm;
  }
  a.pmap = nullptr;
  a.pmap_mask = 0;
  a.opts = 0;  // batch plans always take both shortcuts
  pl.tcap = pow2_at_least(2ull * pl.e_cap + 16);
  pl.acap = pow2_at_least(2ull * pl.e_cap + 16);
  if (arena_entries) {
    pl.arena = (size_t)arena_entries;
  } else {  // every merge and generated coboundary takes new arena space: 384 entries per edge, within 40 % of free memory
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
      cudaGetLastError();
      free_b = (size_t)16 << 30;
    }
    pl.arena = std::max<size_t>(std::min<size_t>(384 * (size_t)pl.e_cap, free_b / 12 * 2 / 5), (size_t)1 << 22);
  }
  pl.slice = 32;
  while (pl.slice < (uint32_t)pl.n_max + 1) pl.slice <<= 1;
  Workspace& w = pl.w;
  const uint64_t E = pl.e_cap, N = pl.N;
  const size_t SPCB = (size_t)batch * PLAN_SPC * 8;
  CR(ensure(w.clouds, (size_t)batch * sizeof(CloudInfo)));
  CR(ensure(pl.clouds0, (size_t)batch * sizeof(CloudInfo)));
  CR(ensure(pl.dtile, (size_t)(batch + 1) * 4));
  CR(ensure(w.tileoff, (size_t)(batch + 1) * 4));
  CR(ensure(w.vcloud, N * 4));
  CR(ensure(w.ccounts, (size_t)(batch + 1) * 4));
  CR(ensure(w.rowmax, N * 4));
  CR(ensure(w.err, 16));
  CR(ensure(w.ecount, 16));
  CR(ensure(w.ekeys, E * 8));
  CR(ensure(w.ekeys_alt, E * 8));
  CR(ensure(w.sorttmp, std::max(sort_temp_bytes((uint32_t)E), scan_temp_bytes((uint32_t)std::max<uint64_t>(E, N + 1)))));
  CR(ensure(w.eflags, (E + 1) * 4));
  CR(ensure(w.erank, (E + 1) * 4));
  CR(ensure(w.rvalue, (E + 1) * 4));
  CR(ensure(w.R, pl.RR * 4));
  CR(ensure(w.deg, (N + 2) * 4));
  CR(ensure(w.nbr, 2 * E * 4));
  CR(ensure(w.binom, (size_t)(kmax + 1) * (pl.n_max + 1) * 8));
  CR(ensure(w.cdist, pl.RR * 4));
  CR(ensure(w.bars, (N + E + 16) * sizeof(rips_bar_t)));
  CR(ensure(w.eu, (E + 1) * 4));
  CR(ensure(w.ev, (E + 1) * 4));
  CR(ensure(w.inforest, E + 1));
  CR(ensure(w.nbars, 16));
  CR(ensure(w.stats, SPCB));
  CR(ensure(w.sidx[0], (E + 1) * 8));
  CR(ensure(w.srank[0], (E + 1) * 4));
  CR(ensure(w.ckeys, (E + 1) * 8));
  CR(ensure(w.ckeys_alt, (E + 1) * 8));
  CR(ensure(w.ccount, 16));
  CR(ensure(w.amk[0], pl.acap * 16));
  CR(ensure(w.tkeys[0], (size_t)pl.tcap * 8));
  CR(ensure(w.tvals[0], (size_t)pl.tcap * 4));
  CR(ensure(w.piv_key, (E + 1) * 8));
  CR(ensure(w.piv_coef, (E + 1) * 4));
  CR(ensure(w.r_off, (E + 1) * 8));
  CR(ensure(w.r_len, (E + 1) * 4));
  CR(ensure(w.reduced, E + 1));
  CR(ensure(w.claim, (E + 1) * 4));
  CR(ensure(w.reduce, (E + 1) * 4));
  CR(ensure(w.heavy, (E + 1) * 8));
  CR(ensure(w.lists, LISTS_BYTES));
  CR(ensure(w.r_top, 16));
  CR(ensure(w.r_key, pl.arena * 8));
  CR(ensure(w.r_coef, pl.arena * 4));
  w.r_cap = pl.arena;
  if (cudaMemcpy(pl.clouds0.p, ci.data(), (size_t)batch * sizeof(CloudInfo), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(pl.dtile.p, dtile.data(), (size_t)(batch + 1) * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(w.tileoff.p, vtile.data(), (size_t)(batch + 1) * 4, cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaGetLastError();
    return RIPS_ERR_CUDA;
  }
  a.clouds = P<CloudInfo>(w.clouds);
  a.R = P<uint32_t>(w.R);
  a.nbr_off = P<uint32_t>(w.deg);
  a.nbr = P<uint32_t>(w.nbr);
  a.nrank = nullptr;
  a.binom = P<uint64_t>(w.binom);
  a.err = P<uint32_t>(w.err);
  a.amap = P<uint64_t>(w.amk[0]);
  a.amap_mask = pl.acap - 1;
  a.vbits = packed_vertex_bits(pl.n_max, 1);
  pl.blocks = reduction_blocks(a, (uint32_t)E);
  if (pl.blocks < 1) return RIPS_ERR_CUDA;
  return RIPS_OK;
}

// Enqueues the whole forward of a plan on stream s; no host synchronisation,
// no allocation.
int plan_run(PlanState& pl, const float* d_points, cudaStream_t s) {
  Workspace& w = pl.w;
  const int C = pl.C;
  const uint64_t E = pl.e_cap, N = pl.N;
  CloudInfo* dclouds = P<CloudInfo>(w.clouds);
  unsigned long long* dstats = P<unsigned long long>(w.stats);
  const float* pts = d_points + (size_t)pl.offsets[0] * pl.k;
  CK(cudaMemcpyAsync(dclouds, pl.clouds0.p, (size_t)C * sizeof(CloudInfo), cudaMemcpyDeviceToDevice, s));
  CK(cudaMemsetAsync(w.rowmax.p, 0, N * 4, s));
  CK(cudaMemsetAsync(w.err.p, 0, 16, s));
  CK(cudaMemsetAsync(w.ecount.p, 0, 16, s));
  CK(cudaMemsetAsync(w.ccounts.p, 0, (size_t)(C + 1) * 4, s));
  CK(cudaMemsetAsync(w.stats.p, 0, (size_t)C * PLAN_SPC * 8, s));
  CK(cudaMemsetAsync(w.nbars.p, 0, 16, s));
  CK(launch_distance_matrices(pts, pl.k, dclouds, P<uint32_t>(pl.dtile), C, (uint32_t)pl.drows, P<float>(w.cdist), s));
  const float* dD = P<float>(w.cdist);
  // prologue
  CK(launch_cloud_vertices(dclouds, C, P<uint32_t>(w.vcloud), s));
  CK(launch_validate_rowmax(dD, dclouds, P<uint32_t>(w.tileoff), C, (uint32_t)pl.vtiles, P<uint32_t>(w.rowmax),
                            P<uint32_t>(w.err), s));
  CK(launch_threshold(P<uint32_t>(w.rowmax), dclouds, C, pl.threshold, s));
  CK(launch_edge_keys(dD, dclouds, P<uint32_t>(w.vcloud), (uint32_t)N, pl.eb, P<uint64_t>(w.ekeys),
                      P<uint32_t>(w.ecount), P<uint32_t>(w.ccounts), (uint32_t)E, s));
  CK(launch_cloud_edge_offsets(dclouds, P<uint32_t>(w.ccounts), C, s));
  CK(launch_pad_past_count(P<uint64_t>(w.ekeys), P<uint32_t>(w.ecount), E, s));
  bool alt = false;
  CK(radix_sort_u64(P<uint64_t>(w.ekeys), P<uint64_t>(w.ekeys_alt), nullptr, nullptr, (uint32_t)E,
                    pl.cb + 32 + pl.eb, w.sorttmp.p, w.sorttmp.cap, &alt, s));
  const uint64_t* keys = alt ? P<uint64_t>(w.ekeys_alt) : P<uint64_t>(w.ekeys);
  CK(launch_assign_ranks(keys, (uint32_t)E, pl.eb, P<uint32_t>(w.eflags), (uint32_t*)w.sorttmp.p,
                         P<uint32_t>(w.erank), P<float>(w.rvalue), &P<uint32_t>(w.ecount)[1], s));
  CK(cudaMemsetAsync(w.R.p, 0xFF, pl.RR * 4, s));
  CK(launch_fill_rank_matrix(keys, P<uint32_t>(w.erank), (uint32_t)E, pl.eb, dclouds, P<uint32_t>(w.R), s));
  CK(cudaMemsetAsync(w.deg.p, 0, (N + 2) * 4, s));
  CK(launch_neighbor_counts(P<uint32_t>(w.R), dclouds, P<uint32_t>(w.vcloud), (uint32_t)N, P<uint32_t>(w.deg),
                            &P<uint32_t>(w.ecount)[3], s));
  CK(launch_exclusive_scan(P<uint32_t>(w.deg), P<uint32_t>(w.deg), (uint32_t)N + 1, w.sorttmp.p,
                           &P<uint32_t>(w.ecount)[2], s));
  CK(launch_neighbor_fill(P<uint32_t>(w.R), dclouds, P<uint32_t>(w.vcloud), (uint32_t)N, P<uint32_t>(w.deg),
                          P<uint32_t>(w.nbr), s));
  CK(launch_binomial_table(P<uint64_t>(w.binom), pl.n_max, 3, s));
  // H0, one block per cloud (edges at the cloud table's offsets, set on the device)
  const uint32_t bar_cap = (uint32_t)(w.bars.cap / sizeof(rips_bar_t));
  CK(launch_h0_blocks(dclouds, C, pl.n_max, keys, pl.eb, P<uint32_t>(w.eu), P<uint32_t>(w.ev), (uint32_t)E,
                      P<uint8_t>(w.inforest), P<rips_bar_t>(w.bars), P<uint32_t>(w.nbars), bar_cap, dstats, PLAN_SPC,
                      P<uint32_t>(w.err), s));
  // dimension 1 over all E slots (the padding is skipped)
  const DimArgs& a = pl.a;
  unsigned long long* st = dstats + 16;
  CK(launch_edges_to_simplices(keys, P<uint32_t>(w.erank), (uint32_t)E, pl.eb, a.col_bits, P<uint64_t>(w.sidx[0]),
                               P<uint32_t>(w.srank[0]), s));
  CK(cudaMemsetAsync(w.ccount.p, 0, 16, s));
  CK(cudaMemsetAsync(w.amk[0].p, 0xFF, pl.acap * 16, s));
  CK(launch_test(a, P<uint64_t>(w.sidx[0]), P<uint32_t>(w.srank[0]), (uint32_t)E, P<uint8_t>(w.inforest), nullptr, 0,
                 P<uint64_t>(w.ckeys), P<uint32_t>(w.ccount), (uint32_t)E + 1, st, PLAN_SPC, s));
  CK(launch_pad_past_count(P<uint64_t>(w.ckeys), P<uint32_t>(w.ccount), E, s));
  bool calt = false;
  CK(radix_sort_u64(P<uint64_t>(w.ckeys), P<uint64_t>(w.ckeys_alt), nullptr, nullptr, (uint32_t)E,
                    pl.cb + a.rank_bits + a.col_bits, w.sorttmp.p, w.sorttmp.cap, &calt, s));
  CK(cudaMemsetAsync(w.tkeys[0].p, 0xFF, (size_t)pl.tcap * 8, s));
  CK(cudaMemsetAsync(w.tvals[0].p, 0xFF, (size_t)pl.tcap * 4, s));
  CK(cudaMemsetAsync(w.lists.p, 0, LISTS_BYTES, s));
  CK(cudaMemsetAsync(w.r_top.p, 0, 16, s));
  uint32_t* counts = P<uint32_t>(w.lists);
  RedState rs;
  rs.col_keys = calt ? P<uint64_t>(w.ckeys_alt) : P<uint64_t>(w.ckeys);
  rs.ncols = (uint32_t)E;
  rs.ncols_dev = P<uint32_t>(w.ccount);
  rs.piv_key = P<uint64_t>(w.piv_key);
  rs.piv_coef = P<uint32_t>(w.piv_coef);
  rs.reduced = P<uint8_t>(w.reduced);
  rs.r_key = P<uint64_t>(w.r_key);
  rs.r_coef = P<uint32_t>(w.r_coef);
  rs.r_off = P<unsigned long long>(w.r_off);
  rs.r_len = P<uint32_t>(w.r_len);
  rs.r_top = P<unsigned long long>(w.r_top);
  rs.r_cap = pl.arena;
  rs.scr_slice = pl.slice;
  rs.t_keys = P<uint64_t>(w.tkeys[0]);
  rs.t_vals = P<uint32_t>(w.tvals[0]);
  rs.t_mask = pl.tcap - 1;
  rs.claim_list = P<uint32_t>(w.claim);
  rs.reduce_list = P<uint32_t>(w.reduce);
  rs.heavy_list = P<uint32_t>(w.heavy);
  rs.steps = P<unsigned long long>(w.lists) + 4;
  rs.compacted = P<unsigned long long>(w.lists) + 5;
  rs.max_chain = counts + 7;
  rs.heartbeat = counts + 12;
  rs.added = P<unsigned long long>(w.lists) + 7;
  rs.help = (HelpBoard*)(P<unsigned char>(w.lists) + 256);
  rs.idle = counts + 4;
  const rips_limits_t lim = current_limits();
  rs.barrier_ns = lim.barrier_wait_ns ? lim.barrier_wait_ns : 30ull * 1000 * 1000 * 1000;
  rs.chain_ns = lim.chain_ns ? lim.chain_ns : 600ull * 1000 * 1000 * 1000;
  rs.err = P<uint32_t>(w.err);
  CK(launch_reduction(a, rs, pl.blocks, counts, s));
  CK(launch_readout(a, rs, P<float>(w.rvalue), P<rips_bar_t>(w.bars), P<uint32_t>(w.nbars), bar_cap, st, PLAN_SPC,
                    s));
  return RIPS_OK;
}

// Waits for stream s, then reads the plan's last run back as a result.
int plan_result(PlanState& pl, cudaStream_t s, rips_result_t** out) {
  Workspace& w = pl.w;
  const int C = pl.C;
  CK(cudaStreamSynchronize(s));
  uint32_t err = 0, nbars = 0, counts[32] = {};
  unsigned long long lists[16] = {};
  std::vector<unsigned long long> hst((size_t)C * PLAN_SPC);
  std::vector<CloudInfo> ci(C);
  CK(cudaMemcpy(&err, w.err.p, 4, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(&nbars, w.nbars.p, 4, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(counts, w.lists.p, 128, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(lists, w.lists.p, 128, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(hst.data(), w.stats.p, hst.size() * 8, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(ci.data(), w.clouds.p, (size_t)C * sizeof(CloudInfo), cudaMemcpyDeviceToHost));
  if (err & ERRF_ARENA) return RIPS_ERR_OOM;  // the plan's arena is fixed: make the plan with a larger one
  if (int e = map_device_error(err)) return e;
  rips_result* r = new (std::nothrow) rips_result();
  if (!r) return RIPS_ERR_OOM;
  r->clouds = C;
  r->dim_max = 1;
  r->k = pl.k;
  r->npoints = pl.ns;
  r->point_offsets = pl.offsets;
  r->thresholds.resize(C);
  r->stats.resize((size_t)C * 2);
  for (int c = 0; c < C; ++c) {
    r->thresholds[c] = ci[c].t_eff;
    const unsigned long long* q0 = hst.data() + (size_t)c * PLAN_SPC;
    rips_stats_t& s0 = r->stats[(size_t)c * 2];
    s0.simplices = pl.ns[c];
    s0.columns = pl.ns[c];
    s0.pairs = (int64_t)q0[0];
    s0.zero_pairs = (int64_t)q0[1];
    s0.essential = (int64_t)q0[2];
    const unsigned long long* q = q0 + 16;
    rips_stats_t& sd = r->stats[(size_t)c * 2 + 1];
    sd.pairs = (int64_t)q[0];
    sd.zero_pairs = (int64_t)q[1];
    sd.essential = (int64_t)q[2];
    sd.emergent = (int64_t)q[3];
    sd.apparent_cofacet = (int64_t)q[4];
    sd.apparent_facet = (int64_t)q[5];
    sd.cleared = (int64_t)q[6];
    sd.columns = sd.pairs + sd.essential;
    sd.simplices = sd.apparent_cofacet + sd.apparent_facet + sd.cleared + sd.columns;
    sd.rounds = counts[6];
    sd.reduction_steps = (int64_t)lists[4];
    sd.longest_chain = counts[7];
    sd.compacted_entries = (int64_t)lists[5];
    sd.added_entries = (int64_t)lists[7];
  }
  const int sbits = std::max(1, bit_width64(host_binom((uint64_t)pl.n_max, 2)));
  const int rc = finish_bars(w, nbars, sbits, std::max(1, bit_width64((uint64_t)C)), s, r->bars);
  if (rc != RIPS_OK) {
    delete r;
    return rc;
  }
  index_result(r);
  *out = r;
  return RIPS_OK;
}

}  // namespace

// ------------------------------------------------------------------ exported API
extern "C" {

RIPS_API int rips_barcodes_device(const float* d_dist, int64_t n, int32_t dim_max, float threshold, uint32_t p,
                                  void* cuda_stream, rips_result_t** out) {
  if (!out) return RIPS_ERR_BAD_ARG;
  *out = nullptr;
  if (!d_dist) return RIPS_ERR_BAD_ARG;
  int rc = check_args(n, dim_max, threshold, p);
  if (rc != RIPS_OK) return rc;
  try {
    Workspace* w = current_workspace();
    if (!w) return RIPS_ERR_OOM;
    std::lock_guard<std::mutex> g(w->mu);
    return barcodes_locked(*w, d_dist, n, dim_max, threshold, p, (cudaStream_t)cuda_stream, out);
  } catch (...) {
    return RIPS_ERR_INTERNAL;
  }
}

RIPS_API int rips_barcodes(const float* dist, int64_t n, int32_t dim_max, float threshold, uint32_t p,
                           rips_result_t** out) {
  if (!out) return RIPS_ERR_BAD_ARG;
  *out = nullptr;
  if (!dist) return RIPS_ERR_BAD_ARG;
  int rc = check_args(n, dim_max, threshold, p);
  if (rc != RIPS_OK) return rc;
  try {
    Workspace* w = current_workspace();
    if (!w) return RIPS_ERR_OOM;
    std::lock_guard<std::mutex> g(w->mu);
    CR(ensure(w->dist, (size_t)n * n * 4));
    CK(cudaMemcpyAsync(w->dist.p, dist, (size_t)n * n * 4, cudaMemcpyHostToDevice, 0));
    return barcodes_locked(*w, P<float>(w->dist), n, dim_max, threshold, p, 0, out);
  } catch (...) {
    return RIPS_ERR_INTERNAL;
  }
}

RIPS_API int rips_barcodes_packed(const float* d_packed, int64_t n, int32_t layout, int32_t dim_max,
                                  float threshold, uint32_t p, void* cuda_stream, rips_result_t** out) {
  if (!out) return RIPS_ERR_BAD_ARG;
  *out = nullptr;
  if ((!d_packed && n > 1) || (layout != RIPS_LOWER_TRIANGLE && layout != RIPS_UPPER_TRIANGLE))
    return RIPS_ERR_BAD_ARG;
  int rc = check_args(n, dim_max, threshold, p);
  if (rc != RIPS_OK) return rc;
  try {
    Workspace* w = current_workspace();
    if (!w) return RIPS_ERR_OOM;
    std::lock_guard<std::mutex> g(w->mu);
    const cudaStream_t s = (cudaStream_t)cuda_stream;
    CR(ensure(w->dist, (size_t)n * n * 4));
    CK(launch_unpack_triangle(d_packed, (int)n, layout == RIPS_UPPER_TRIANGLE, P<float>(w->dist), s));
    return barcodes_locked(*w, P<float>(w->dist), n, dim_max, threshold, p, s, out);
  } catch (...) {
    return RIPS_ERR_INTERNAL;
  }
}

RIPS_API int rips_barcodes_sparse(const int32_t* d_i, const int32_t* d_j, const float* d_len, int64_t m, int64_t n,
                                  int32_t dim_max, float threshold, uint32_t p, void* cuda_stream,
                                  rips_result_t** out) {
  if (!out) return RIPS_ERR_BAD_ARG;
  *out = nullptr;
  if (m < 0 || (m > 0 && (!d_i || !d_j || !d_len)) || (uint64_t)m > 0xFFFFFFF0ull) return RIPS_ERR_BAD_ARG;
  int rc = check_sparse_args(n, dim_max, threshold, p);
  if (rc != RIPS_OK) return rc;
  try {
    Workspace* w = current_workspace();
    if (!w) return RIPS_ERR_OOM;
    std::lock_guard<std::mutex> g(w->mu);
    SparseIn sp;
    sp.ei = d_i;
    sp.ej = d_j;
    sp.len = d_len;
    sp.m = (uint64_t)m;
    return sparse_locked(*w, sp, n, dim_max, threshold, p, (cudaStream_t)cuda_stream, out);
  } catch (...) {
    return RIPS_ERR_INTERNAL;
  }
}

RIPS_API int rips_barcodes_sparse_points(const float* d_points, int64_t n, int32_t k, int32_t dim_max,
                                         float threshold, uint32_t p, void* cuda_stream, rips_result_t** out) {
  if (!out) return RIPS_ERR_BAD_ARG;
  *out = nullptr;
  if (!d_points || k < 1 || !(threshold >= 0.0f) || std::isinf(threshold)) return RIPS_ERR_BAD_ARG;
  int rc = check_sparse_args(n, dim_max, threshold, p);
  if (rc != RIPS_OK) return rc;
  try {
    Workspace* w = current_workspace();
    if (!w) return RIPS_ERR_OOM;
    std::lock_guard<std::mutex> g(w->mu);
    SparseIn sp;
    sp.pts = d_points;
    sp.k = k;
    return sparse_locked(*w, sp, n, dim_max, threshold, p, (cudaStream_t)cuda_stream, out);
  } catch (...) {
    return RIPS_ERR_INTERNAL;
  }
}

RIPS_API int rips_distance_matrix_device(const float* d_points, int64_t n, int32_t k, float* d_dist,
                                         void* cuda_stream) {
  if (!d_points || !d_dist || n < 1 || n > 46340 || k < 1) return RIPS_ERR_BAD_ARG;
  CK(launch_distance_matrix(d_points, (int)n, k, d_dist, (cudaStream_t)cuda_stream));
  return RIPS_OK;
}

RIPS_API int64_t rips_result_num_bars(const rips_result_t* r, int32_t cloud, int32_t dim) {
  if (!r || cloud < -1 || cloud >= r->clouds || dim < -1 || dim > r->dim_max) return RIPS_ERR_BAD_ARG;
  const int D = r->dim_max + 1;
  if (cloud == -1 && dim == -1) return (int64_t)r->bars.size();
  if (cloud == -1) {
    int64_t c = 0;
    for (int q = 0; q < r->clouds; ++q) c += r->offsets[(size_t)q * D + dim + 1] - r->offsets[(size_t)q * D + dim];
    return c;
  }
  if (dim == -1) return r->offsets[(size_t)(cloud + 1) * D] - r->offsets[(size_t)cloud * D];
  return r->offsets[(size_t)cloud * D + dim + 1] - r->offsets[(size_t)cloud * D + dim];
}

RIPS_API const rips_bar_t* rips_result_bars(const rips_result_t* r, int32_t cloud, int32_t dim) {
  if (!r || cloud < -1 || cloud >= r->clouds || dim < -1 || dim > r->dim_max || r->bars.empty()) return nullptr;
  const int D = r->dim_max + 1;
  if (cloud == -1) return dim == -1 ? r->bars.data() : nullptr;
  const int64_t off = r->offsets[(size_t)cloud * D + (dim == -1 ? 0 : dim)];
  return r->bars.data() + off;
}

RIPS_API int32_t rips_result_num_clouds(const rips_result_t* r) { return r ? r->clouds : RIPS_ERR_BAD_ARG; }
RIPS_API int32_t rips_result_dim_max(const rips_result_t* r) { return r ? r->dim_max : RIPS_ERR_BAD_ARG; }
RIPS_API float rips_result_threshold(const rips_result_t* r, int32_t cloud) {
  if (!r || cloud < 0 || cloud >= r->clouds) return NAN;
  return r->thresholds[cloud];
}

RIPS_API int rips_result_stats(const rips_result_t* r, int32_t cloud, int32_t dim, rips_stats_t* out) {
  if (!r || !out || cloud < 0 || cloud >= r->clouds || dim < 0 || dim > r->dim_max) return RIPS_ERR_BAD_ARG;
  *out = r->stats[(size_t)cloud * (r->dim_max + 1) + dim];
  return RIPS_OK;
}

RIPS_API int32_t rips_result_phase_ms(const rips_result_t* r, float* out, int32_t cap) {
  if (!r || (!out && cap > 0)) return RIPS_ERR_BAD_ARG;
  int32_t k = 0;
  for (; k < cap && k < (int32_t)r->phase_ms.size(); ++k) out[k] = r->phase_ms[k];
  return k;
}

RIPS_API void rips_result_free(rips_result_t* r) { delete r; }

RIPS_API int rips_set_kernel_timing(int enable) {
  const int prev = g_kernel_timing ? 1 : 0;
  g_kernel_timing = enable != 0;
  return prev;
}

RIPS_API int rips_result_kernel_ms(const rips_result_t* r, int32_t cls, float* ms, int64_t* regions) {
  if (!r || cls < 0 || cls >= RIPS_KERNEL_CLASSES) return RIPS_ERR_BAD_ARG;
  if (ms) *ms = r->kernel_ms[cls];
  if (regions) *regions = r->kernel_launches[cls];
  return RIPS_OK;
}

RIPS_API const char* rips_status_string(int status) {
  switch (status) {
    case RIPS_OK: return "ok";
    case RIPS_ERR_BAD_ARG: return "bad argument";
    case RIPS_ERR_BAD_MODULUS: return "modulus is not a prime below 65536";
    case RIPS_ERR_OVERFLOW: return "simplex index or filtration key exceeds 64 bits";
    case RIPS_ERR_OOM: return "out of memory";
    case RIPS_ERR_CUDA: return "CUDA runtime error";
    case RIPS_ERR_DEVICE_TIMEOUT: return "device loop hit its iteration limit";
    case RIPS_ERR_INTERNAL: return "internal consistency check failed";
    default: return "unknown status";
  }
}

RIPS_API int64_t rips_kernel_launch_count(int reset) {
  long long v = g_launches;
  if (reset) g_launches = 0;
  return v;
}

RIPS_API int rips_set_tuning(int32_t dim, int64_t n_lo, int64_t n_hi, const rips_tuning_t* t) {
  if (!t || dim < 1 || dim > 7 || n_lo < 1 || n_hi < n_lo) return RIPS_ERR_BAD_ARG;
  if (t->warp_chain_limit < 1 || t->warp_merge_max < 1 || t->reduce_blocks_per_sm < 0 ||
      t->scan_blocks_per_sm < 1 || t->scan_blocks_per_sm > 64)
    return RIPS_ERR_BAD_ARG;
  std::lock_guard<std::mutex> g(g_tune_mu);
  g_tune.push_back(TuneEntry{dim, n_lo, n_hi, *t});
  return RIPS_OK;
}

RIPS_API int rips_get_tuning(int32_t dim, int64_t n, rips_tuning_t* out) {
  if (!out || dim < 1 || dim > 7 || n < 1) return RIPS_ERR_BAD_ARG;
  *out = tuning_for(dim, n);
  return RIPS_OK;
}

RIPS_API void rips_clear_tuning(void) {
  std::lock_guard<std::mutex> g(g_tune_mu);
  g_tune.clear();
}

RIPS_API int rips_set_limits(const rips_limits_t* limits) {
  if (!limits) return RIPS_ERR_BAD_ARG;
  const uint64_t t = limits->table_slots;
  if (t && (t & (t - 1))) return RIPS_ERR_BAD_ARG;
  if (t > (1ull << 31)) return RIPS_ERR_BAD_ARG;
  std::lock_guard<std::mutex> g(g_limits_mu);
  g_limits = *limits;
  return RIPS_OK;
}

RIPS_API int rips_set_options(uint32_t flags) {
  if (flags & ~(uint32_t)(RIPS_OPT_NO_APPARENT | RIPS_OPT_NO_EMERGENT)) return RIPS_ERR_BAD_ARG;
  std::lock_guard<std::mutex> g(g_limits_mu);
  g_options = flags;
  return RIPS_OK;
}

RIPS_API uint32_t rips_get_options(void) { return current_options(); }

RIPS_API int rips_get_limits(rips_limits_t* out) {
  if (!out) return RIPS_ERR_BAD_ARG;
  *out = current_limits();
  return RIPS_OK;
}

RIPS_API int rips_barcodes_batched(const float* d_points, const int64_t* offsets, int32_t batch, int32_t k,
                                   int32_t dim_max, float threshold, uint32_t p, void* cuda_stream,
                                   rips_result_t** out) {
  if (!out) return RIPS_ERR_BAD_ARG;
  *out = nullptr;
  if (!d_points || !offsets || batch < 1 || k < 1) return RIPS_ERR_BAD_ARG;
  if (offsets[0] != 0) return RIPS_ERR_BAD_ARG;
  for (int32_t c = 0; c < batch; ++c) {
    int rc = check_args(offsets[c + 1] - offsets[c], dim_max, threshold, p);
    if (rc != RIPS_OK) return rc;
  }
  try {
    Workspace* w = current_workspace();
    if (!w) return RIPS_ERR_OOM;
    std::lock_guard<std::mutex> g(w->mu);
    return batched_locked(*w, d_points, offsets, batch, k, dim_max, threshold, p, (cudaStream_t)cuda_stream, out);
  } catch (...) {
    return RIPS_ERR_INTERNAL;
  }
}

RIPS_API int rips_barcodes_backward(const rips_result_t* res, const float* d_points, int32_t k,
                                    const float* grad_birth, const float* grad_death, float* d_grad_points,
                                    float* d_grad_dist, void* cuda_stream) {
  if (!res || !d_points || k < 1 || !d_grad_points) return RIPS_ERR_BAD_ARG;
  if (res->k && res->k != k) return RIPS_ERR_BAD_ARG;
  try {
    Workspace* w = current_workspace();
    if (!w) return RIPS_ERR_OOM;
    std::lock_guard<std::mutex> g(w->mu);
    return backward_locked(*w, res, d_points, k, grad_birth, grad_death, d_grad_points, d_grad_dist,
                           (cudaStream_t)cuda_stream);
  } catch (...) {
    return RIPS_ERR_INTERNAL;
  }
}


RIPS_API int rips_barcodes_batched_dists(const float* const* d_dists, const int64_t* ns, int32_t batch,
                                         int32_t dim_max, float threshold, uint32_t p, void* cuda_stream,
                                         rips_result_t** out) {
  if (!out) return RIPS_ERR_BAD_ARG;
  *out = nullptr;
  if (!d_dists || !ns || batch < 1) return RIPS_ERR_BAD_ARG;
  for (int32_t c = 0; c < batch; ++c) {
    if (!d_dists[c]) return RIPS_ERR_BAD_ARG;
    int rc = check_args(ns[c], dim_max, threshold, p);
    if (rc != RIPS_OK) return rc;
  }
  try {
    Workspace* w = current_workspace();
    if (!w) return RIPS_ERR_OOM;
    std::lock_guard<std::mutex> g(w->mu);
    return batched_dists_locked(*w, d_dists, ns, batch, dim_max, threshold, p, (cudaStream_t)cuda_stream, out);
  } catch (...) {
    return RIPS_ERR_INTERNAL;
  }
}

RIPS_API int rips_barcodes_backward_dist(const rips_result_t* res, const float* const* d_dists,
                                         const float* grad_birth, const float* grad_death, float* const* d_grad_dists,
                                         void* cuda_stream) {
  if (!res || !d_dists || !d_grad_dists) return RIPS_ERR_BAD_ARG;
  for (int32_t c = 0; c < res->clouds; ++c)
    if (!d_dists[c] || !d_grad_dists[c]) return RIPS_ERR_BAD_ARG;
  try {
    Workspace* w = current_workspace();
    if (!w) return RIPS_ERR_OOM;
    std::lock_guard<std::mutex> g(w->mu);
    return backward_dist_locked(*w, res, d_dists, grad_birth, grad_death, d_grad_dists, (cudaStream_t)cuda_stream);
  } catch (...) {
    return RIPS_ERR_INTERNAL;
  }
}


struct rips_batch_plan {
  PlanState st;
  int device = -1;
};

RIPS_API int rips_batch_plan_create(const int64_t* offsets, int32_t batch, int32_t k, float threshold, uint32_t p,
                                    int64_t arena_entries, rips_batch_plan_t** out) {
  if (!out) return RIPS_ERR_BAD_ARG;
  *out = nullptr;
  try {
    rips_batch_plan* b = new (std::nothrow) rips_batch_plan();
    if (!b) return RIPS_ERR_OOM;
    if (cudaGetDevice(&b->device) != cudaSuccess) {
      cudaGetLastError();
      delete b;
      return RIPS_ERR_CUDA;
    }
    const int rc = plan_create(b->st, offsets, batch, k, threshold, p, arena_entries);
    if (rc != RIPS_OK) {
      release_plan(b->st);
      delete b;
      return rc;
    }
    *out = b;
    return RIPS_OK;
  } catch (...) {
    return RIPS_ERR_INTERNAL;
  }
}

RIPS_API int rips_batch_plan_run(rips_batch_plan_t* plan, const float* d_points, void* cuda_stream) {
  if (!plan || !d_points) return RIPS_ERR_BAD_ARG;
  try {
    std::lock_guard<std::mutex> g(plan->st.w.mu);
    return plan_run(plan->st, d_points, (cudaStream_t)cuda_stream);
  } catch (...) {
    return RIPS_ERR_INTERNAL;
  }
}

RIPS_API int rips_batch_plan_result(rips_batch_plan_t* plan, void* cuda_stream, rips_result_t** out) {
  if (!plan || !out) return RIPS_ERR_BAD_ARG;
  *out = nullptr;
  try {
    std::lock_guard<std::mutex> g(plan->st.w.mu);
    return plan_result(plan->st, (cudaStream_t)cuda_stream, out);
  } catch (...) {
    return RIPS_ERR_INTERNAL;
  }
}

RIPS_API void rips_batch_plan_free(rips_batch_plan_t* plan) {
  if (!plan) return;
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess) cudaGetLastError();
  if (plan->device >= 0 && cur != plan->device) cudaSetDevice(plan->device);
  release_plan(plan->st);
  if (cur >= 0 && cur != plan->device) cudaSetDevice(cur);
  delete plan;
}

}  // extern "C"
