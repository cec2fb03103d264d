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
  Buf piv_key, piv_coef, v_off, v_len, reduced, claim, reduce, lists;
  Buf v_idx, v_rank, v_coef, v_top;
  Buf tkeys[2], tvals[2];
  Buf bars, bars_alt, bk0, bk1, bp0, bp1, bartmp, nbars;
  Buf stats, bwd_bars, bwd_off, cdist;
  size_t v_cap = 0;
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
  if (e & (ERRF_INTERNAL | ERRF_TABLE_FULL)) return RIPS_ERR_INTERNAL;
  return RIPS_OK;
}

uint32_t pow2_at_least(uint64_t x) {
  uint64_t c = 16;
  while (c < x) c <<= 1;
  return (uint32_t)c;
}

// One cloud on the device: appends its bars (device) at *nbars and writes stats.
struct CloudOut {
  float kernel_ms[RIPS_KERNEL_CLASSES] = {};
  int64_t kernel_regions[RIPS_KERNEL_CLASSES] = {};
  float t_eff = 0;
  std::vector<rips_stats_t> stats;
  std::vector<float> phase_ms;
};

int sync_read(Workspace& w, cudaStream_t s) {
  CK(cudaStreamSynchronize(s));
  return RIPS_OK;
}

int run_cloud(Workspace& w, const float* dD, int n, int dim_max, float threshold, uint32_t p, int cloud,
              cudaStream_t s, uint32_t* h_nbars_io, CloudOut& out) {
  HostPinned* hp = w.pinned;
  const int kmax = dim_max + 2;
  w.kev_used = 0;
  out.stats.assign(dim_max + 1, rips_stats_t{});
  if (w.events) CK(cudaEventRecord(w.tev[0], s));

  // ---------------- prologue
  const uint64_t e_cap = (uint64_t)n * (n - 1) / 2;
  CR(ensure(w.rowmax, (size_t)n * 4));
  CR(ensure(w.teff, 16));
  CR(ensure(w.err, 16));
  CR(ensure(w.ecount, 16));
  CR(ensure(w.ekeys, e_cap * 8));
  CR(ensure(w.ekeys_alt, e_cap * 8));
  CK(cudaMemsetAsync(w.rowmax.p, 0, (size_t)n * 4, s));
  CK(cudaMemsetAsync(w.err.p, 0, 16, s));
  CK(cudaMemsetAsync(w.ecount.p, 0, 16, s));
  {
    KTimer kt(w, RIPS_K_PROLOGUE, s);
    if (n > 1) CK(launch_validate_rowmax(dD, n, P<uint32_t>(w.rowmax), P<uint32_t>(w.err), s));
    CK(launch_threshold(P<uint32_t>(w.rowmax), n, threshold, P<float>(w.teff), s));
    if (n > 1)
      CK(launch_edge_keys(dD, n, P<float>(w.teff), P<uint64_t>(w.ekeys), P<uint32_t>(w.ecount), (uint32_t)e_cap, s));
  }
  CK(cudaMemcpyAsync(&hp->u32[0], w.ecount.p, 4, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(&hp->u32[1], w.err.p, 4, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(&hp->f32[0], w.teff.p, 4, cudaMemcpyDeviceToHost, s));
  CR(sync_read(w, s));
  if (hp->u32[1] & ERRF_BAD_INPUT) return RIPS_ERR_BAD_ARG;
  const uint32_t m = hp->u32[0];
  out.t_eff = hp->f32[0];

  // sort edges: (diameter bits, inverted index) ascending = filtration order
  CR(ensure(w.sorttmp, std::max(sort_temp_bytes(m), scan_temp_bytes(m > (uint32_t)n + 1 ? m : n + 1))));
  bool alt = false;
  {
    KTimer kt(w, RIPS_K_EDGE_SORT, s);
    CK(radix_sort_u64(P<uint64_t>(w.ekeys), P<uint64_t>(w.ekeys_alt), nullptr, nullptr, m, 64, w.sorttmp.p,
                      w.sorttmp.cap, &alt, s));
  }
  const uint64_t* keys = alt ? P<uint64_t>(w.ekeys_alt) : P<uint64_t>(w.ekeys);
  uint64_t* keys_other = alt ? P<uint64_t>(w.ekeys) : P<uint64_t>(w.ekeys_alt);

  CR(ensure(w.eflags, (size_t)(m + 1) * 4));
  CR(ensure(w.erank, (size_t)(m + 1) * 4));
  CR(ensure(w.rvalue, (size_t)(m + 1) * 4));
  KTimer* kt_pro = new KTimer(w, RIPS_K_PROLOGUE, s);
  CK(launch_assign_ranks(keys, m, P<uint32_t>(w.eflags), (uint32_t*)w.sorttmp.p, w.sorttmp.cap,
                         P<uint32_t>(w.erank), P<float>(w.rvalue), &P<uint32_t>(w.ecount)[1], s));
  CR(ensure(w.R, (size_t)n * n * 4));
  CK(launch_fill_rank_matrix(keys, P<uint32_t>(w.erank), m, n, P<uint32_t>(w.R), s));
  CR(ensure(w.deg, (size_t)(n + 2) * 4));
  CK(cudaMemsetAsync(w.deg.p, 0, (size_t)(n + 2) * 4, s));
  CK(launch_neighbor_counts(P<uint32_t>(w.R), n, P<uint32_t>(w.deg), s));
  CK(launch_exclusive_scan(P<uint32_t>(w.deg), P<uint32_t>(w.deg), (uint32_t)n + 1, w.sorttmp.p,
                           &P<uint32_t>(w.ecount)[2], s));
  delete kt_pro;
  CK(cudaMemcpyAsync(&hp->u32[2], (char*)w.ecount.p + 4, 8, cudaMemcpyDeviceToHost, s));
  CR(sync_read(w, s));
  const uint32_t num_ranks = hp->u32[2];
  const uint32_t nbr_total = hp->u32[3];
  CR(ensure(w.nbr, (size_t)nbr_total * 4));
  CR(ensure(w.binom, (size_t)(kmax + 1) * (n + 1) * 8));
  {
    KTimer kt(w, RIPS_K_PROLOGUE, s);
    CK(launch_neighbor_fill(P<uint32_t>(w.R), n, P<uint32_t>(w.deg), P<uint32_t>(w.nbr), s));
    CK(launch_binomial_table(P<uint64_t>(w.binom), n, kmax, s));
  }

  // ---------------- H0
  const uint64_t bar_need = (uint64_t)*h_nbars_io + (uint64_t)n + 16;
  CR(grow_keep(w.bars, bar_need * sizeof(rips_bar_t), (size_t)*h_nbars_io * sizeof(rips_bar_t), s));
  CR(ensure(w.eu, (size_t)(m + 1) * 4));
  CR(ensure(w.ev, (size_t)(m + 1) * 4));
  CR(ensure(w.comp, (size_t)n * 4));
  CR(ensure(w.best, (size_t)n * 4));
  CR(ensure(w.parent, (size_t)n * 4));
  CR(ensure(w.gtop, (size_t)n * 4));
  CR(ensure(w.inforest, (size_t)m + 1));
  CR(ensure(w.fpos, (size_t)n * 4));
  CR(ensure(w.nf, 16));
  CR(ensure(w.nbars, 16));
  CR(ensure(w.stats, (size_t)(dim_max + 1) * 16 * 8));
  CK(cudaMemsetAsync(w.stats.p, 0, (size_t)(dim_max + 1) * 16 * 8, s));
  hp->u32[4] = *h_nbars_io;
  CK(cudaMemcpyAsync(w.nbars.p, &hp->u32[4], 4, cudaMemcpyHostToDevice, s));
  unsigned long long* dstats = P<unsigned long long>(w.stats);
  KTimer* kt_h0 = new KTimer(w, RIPS_K_H0, s);
  CK(run_h0(n, keys, m, P<uint32_t>(w.eu), P<uint32_t>(w.ev), P<uint32_t>(w.comp), P<uint32_t>(w.best),
            P<uint32_t>(w.parent), P<uint8_t>(w.inforest), P<uint32_t>(w.eflags), P<uint32_t>(w.fpos), w.sorttmp.p,
            P<uint32_t>(w.nf), P<uint32_t>(w.gtop), P<rips_bar_t>(w.bars), P<uint32_t>(w.nbars),
            (uint32_t)(w.bars.cap / sizeof(rips_bar_t)), cloud, dstats, P<uint32_t>(w.err), s));
  delete kt_h0;
  if (w.events) CK(cudaEventRecord(w.tev[1], s));

  // ---------------- dimensions 1..dim_max
  const int rank_bits = bit_width64(num_ranks ? num_ranks - 1 : 0);
  uint32_t ns_prev = 0;  // size of the (d-1)-simplex list in sidx[cur^1]
  int cur = 0;
  uint64_t* prev_tkeys = nullptr;
  uint64_t prev_tmask = 0;
  for (int d = 1; d <= dim_max; ++d) {
    DimArgs a;
    a.n = n;
    a.d = d;
    a.R = P<uint32_t>(w.R);
    a.nbr_off = P<uint32_t>(w.deg);
    a.nbr = P<uint32_t>(w.nbr);
    a.binom = P<uint64_t>(w.binom);
    a.kmax = kmax;
    a.smem_binom = (size_t)(kmax + 1) * (n + 1) * 8 <= 48 * 1024;
    a.p = p;
    a.col_bits = std::max(1, bit_width64(host_binom(n, d + 1) ? host_binom(n, d + 1) - 1 : 0));
    a.row_bits = std::max(1, bit_width64(host_binom(n, d + 2) ? host_binom(n, d + 2) - 1 : 0));
    a.rank_max = num_ranks ? num_ranks - 1 : 0;
    a.err = P<uint32_t>(w.err);
    if (rank_bits + a.row_bits > 64 || rank_bits + a.col_bits > 64) return RIPS_ERR_OVERFLOW;
    unsigned long long* st = dstats + d * 16;

    // d-simplices
    uint32_t ns = 0;
    if (d == 1) {
      ns = m;
      CR(ensure(w.sidx[cur], (size_t)(m + 1) * 8));
      CR(ensure(w.srank[cur], (size_t)(m + 1) * 4));
      CK(launch_edges_to_simplices(keys, P<uint32_t>(w.erank), m, P<uint64_t>(w.sidx[cur]), P<uint32_t>(w.srank[cur]),
                                   s));
    } else {
      CR(ensure(w.scount, 16));
      const int pv = cur ^ 1;
      for (int attempt = 0; attempt < 2; ++attempt) {
        unsigned long long cap = w.sidx[cur].cap / 8;
        if (w.srank[cur].cap / 4 < cap) cap = w.srank[cur].cap / 4;
        CK(cudaMemsetAsync(w.scount.p, 0, 8, s));
        KTimer kt(w, RIPS_K_ENUMERATE, s);
        CK(launch_enumerate(a, P<uint64_t>(w.sidx[pv]), P<uint32_t>(w.srank[pv]), ns_prev, P<uint64_t>(w.sidx[cur]),
                            P<uint32_t>(w.srank[cur]), P<unsigned long long>(w.scount), cap, s));
        CK(cudaMemcpyAsync(&hp->u64[0], w.scount.p, 8, cudaMemcpyDeviceToHost, s));
        CR(sync_read(w, s));
        const unsigned long long got = hp->u64[0];
        if (got > 0xFFFFFFF0ull) return RIPS_ERR_OVERFLOW;
        if (got <= cap) {
          ns = (uint32_t)got;
          break;
        }
        CR(ensure(w.sidx[cur], got * 8));
        CR(ensure(w.srank[cur], got * 4));
      }
    }
    out.stats[d].simplices = ns;

    // apparent pairs, clearing, compaction
    CR(ensure(w.ckeys, (size_t)(ns + 1) * 8));
    CR(ensure(w.ckeys_alt, (size_t)(ns + 1) * 8));
    CR(ensure(w.ccount, 16));
    CK(cudaMemsetAsync(w.ccount.p, 0, 16, s));
    {
      KTimer kt(w, RIPS_K_APPARENT, s);
      CK(launch_test(a, P<uint64_t>(w.sidx[cur]), P<uint32_t>(w.srank[cur]), ns, P<uint8_t>(w.inforest), prev_tkeys,
                     prev_tmask, P<uint64_t>(w.ckeys), P<uint32_t>(w.ccount), ns + 1, st + 4, s));
    }
    CK(cudaMemcpyAsync(&hp->u32[5], w.ccount.p, 4, cudaMemcpyDeviceToHost, s));
    CR(sync_read(w, s));
    const uint32_t M = hp->u32[5];
    // processing order
    CR(ensure(w.sorttmp, std::max(w.sorttmp.cap, sort_temp_bytes(M + 1))));
    bool calt = false;
    KTimer* kt_cs = new KTimer(w, RIPS_K_COL_SORT, s);
    CK(radix_sort_u64(P<uint64_t>(w.ckeys), P<uint64_t>(w.ckeys_alt), nullptr, nullptr, M, rank_bits + a.col_bits,
                      w.sorttmp.p, w.sorttmp.cap, &calt, s));
    delete kt_cs;
    const uint64_t* ckeys = calt ? P<uint64_t>(w.ckeys_alt) : P<uint64_t>(w.ckeys);

    // reduction
    const int tb = cur;  // table for this dimension (the other one holds d-1)
    const uint32_t tcap = pow2_at_least(2ull * M + 16);
    CR(ensure(w.tkeys[tb], (size_t)tcap * 8));
    CR(ensure(w.tvals[tb], (size_t)tcap * 4));
    CR(ensure(w.piv_key, (size_t)(M + 1) * 8));
    CR(ensure(w.piv_coef, (size_t)(M + 1) * 4));
    CR(ensure(w.v_off, (size_t)(M + 1) * 4));
    CR(ensure(w.v_len, (size_t)(M + 1) * 4));
    CR(ensure(w.reduced, (size_t)(M + 1)));
    CR(ensure(w.claim, (size_t)(M + 1) * 4));
    CR(ensure(w.reduce, (size_t)(M + 1) * 4));
    CR(ensure(w.lists, 64));
    CR(ensure(w.v_top, 16));
    size_t vcap = std::max<size_t>(w.v_cap, 4 * (size_t)M + 4096);
    int red_rc = RIPS_OK;
    for (int attempt = 0; attempt < 6; ++attempt) {
      CR(ensure(w.v_idx, vcap * 8));
      CR(ensure(w.v_rank, vcap * 4));
      CR(ensure(w.v_coef, vcap * 4));
      w.v_cap = vcap;
      CK(cudaMemsetAsync(w.tkeys[tb].p, 0xFF, (size_t)tcap * 8, s));
      CK(cudaMemsetAsync(w.tvals[tb].p, 0xFF, (size_t)tcap * 4, s));
      CK(cudaMemsetAsync(w.lists.p, 0, 64, s));
      CK(cudaMemsetAsync(w.v_top.p, 0, 16, s));
      CK(cudaMemsetAsync(st + 9, 0, 8, s));
      uint32_t* counts = P<uint32_t>(w.lists);
      RedState rs;
      rs.col_keys = ckeys;
      rs.ncols = M;
      rs.piv_key = P<uint64_t>(w.piv_key);
      rs.piv_coef = P<uint32_t>(w.piv_coef);
      rs.v_off = P<uint32_t>(w.v_off);
      rs.v_len = P<uint32_t>(w.v_len);
      rs.reduced = P<uint8_t>(w.reduced);
      rs.v_idx = P<uint64_t>(w.v_idx);
      rs.v_rank = P<uint32_t>(w.v_rank);
      rs.v_coef = P<uint32_t>(w.v_coef);
      rs.v_top = P<unsigned long long>(w.v_top);
      rs.v_cap = vcap;
      rs.t_keys = P<uint64_t>(w.tkeys[tb]);
      rs.t_vals = P<uint32_t>(w.tvals[tb]);
      rs.t_mask = tcap - 1;
      rs.claim_list = P<uint32_t>(w.claim);
      rs.reduce_list = P<uint32_t>(w.reduce);
      rs.steps = st + 9;
      rs.err = P<uint32_t>(w.err);
      // claim counter at counts[0], reduce counter at counts[1]
      rs.claim_count = counts + 0;
      rs.reduce_count = counts + 1;
      {
        KTimer kt(w, RIPS_K_PIVOT_INIT, s);
        CK(launch_init(a, rs, s));
      }
      uint32_t rounds = 0;
      bool arena_full = false;
      for (;;) {
        CK(cudaMemcpyAsync(&hp->u32[6], w.lists.p, 8, cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(&hp->u32[8], w.err.p, 4, cudaMemcpyDeviceToHost, s));
        CR(sync_read(w, s));
        if (hp->u32[8] & ERRF_ARENA) {
          arena_full = true;
          break;
        }
        if (int e = map_device_error(hp->u32[8])) return e;
        const uint32_t nclaim = hp->u32[6];
        if (nclaim == 0) break;
        if (++rounds > 1000000u) return RIPS_ERR_DEVICE_TIMEOUT;
        // claims: claim list -> reduce list
        CK(cudaMemsetAsync(counts + 1, 0, 4, s));
        {
          KTimer kt(w, RIPS_K_REDUCE, s);
          CK(launch_claim(a, rs, nclaim, s));
        }
        CK(cudaMemsetAsync(counts + 0, 0, 4, s));
        CK(cudaMemcpyAsync(&hp->u32[7], counts + 1, 4, cudaMemcpyDeviceToHost, s));
        CR(sync_read(w, s));
        const uint32_t nred = hp->u32[7];
        // reductions: reduce list -> claim list
        {
          KTimer kt(w, RIPS_K_REDUCE, s);
          CK(launch_reduce(a, rs, nred, s));
        }
      }
      if (arena_full) {
        // start this dimension's reduction over with a larger arena
        hp->u32[9] = 0;
        CK(cudaMemsetAsync(w.err.p, 0, 4, s));
        vcap *= 4;
        continue;
      }
      out.stats[d].rounds = rounds;
      // bars are appended after the current count: make sure room exists
      {
        CK(cudaMemcpyAsync(&hp->u32[10], w.nbars.p, 4, cudaMemcpyDeviceToHost, s));
        CR(sync_read(w, s));
        const size_t need = ((size_t)hp->u32[10] + M + 16) * sizeof(rips_bar_t);
        CR(grow_keep(w.bars, need, (size_t)hp->u32[10] * sizeof(rips_bar_t), s));
      }
      {
        KTimer kt(w, RIPS_K_READOUT, s);
        CK(launch_readout(a, rs, P<float>(w.rvalue), cloud, P<rips_bar_t>(w.bars), P<uint32_t>(w.nbars),
                          (uint32_t)(w.bars.cap / sizeof(rips_bar_t)), st, s));
      }
      red_rc = RIPS_OK;
      break;
    }
    CR(red_rc);
    out.stats[d].columns = M;
    prev_tkeys = P<uint64_t>(w.tkeys[tb]);
    prev_tmask = tcap - 1;
    ns_prev = ns;
    cur ^= 1;
    if (w.events && d + 1 < 16) CK(cudaEventRecord(w.tev[d + 1], s));
  }

  // statistics and bar count
  CK(cudaMemcpyAsync(hp->u64, dstats, (size_t)(dim_max + 1) * 16 * 8, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(&hp->u32[11], w.nbars.p, 4, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(&hp->u32[12], w.err.p, 4, cudaMemcpyDeviceToHost, s));
  CR(sync_read(w, s));
  if (int e = map_device_error(hp->u32[12])) return e;
  *h_nbars_io = hp->u32[11];
  // dimension 0 statistics from the H0 kernel (pairs, zero, essential)
  out.stats[0].simplices = n;
  out.stats[0].columns = n;
  out.stats[0].pairs = (int64_t)hp->u64[0];
  out.stats[0].zero_pairs = (int64_t)hp->u64[1];
  out.stats[0].essential = (int64_t)hp->u64[2];
  out.stats[0].emergent = 0;
  for (int d = 1; d <= dim_max; ++d) {
    const unsigned long long* q = hp->u64 + d * 16;
    out.stats[d].pairs = (int64_t)q[0];
    out.stats[d].zero_pairs = (int64_t)q[1];
    out.stats[d].essential = (int64_t)q[2];
    out.stats[d].emergent = (int64_t)q[3];
    out.stats[d].apparent_cofacet = (int64_t)q[4];
    out.stats[d].apparent_facet = (int64_t)q[5];
    out.stats[d].cleared = (int64_t)q[6];
    out.stats[d].reduction_steps = (int64_t)q[9];
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

// caller holds w.mu
int barcodes_locked(Workspace& w, const float* dD, int64_t n, int32_t dim_max, float threshold, uint32_t p,
                    cudaStream_t s, rips_result_t** out) {
  rips_result* r = new (std::nothrow) rips_result();
  if (!r) return RIPS_ERR_OOM;
  r->clouds = 1;
  r->dim_max = dim_max;
  uint32_t nb = 0;
  CloudOut co;
  int rc = run_cloud(w, dD, (int)n, dim_max, threshold, p, 0, s, &nb, co);
  if (rc == RIPS_OK) {
    const int sbits = std::max(1, bit_width64(host_binom((uint64_t)n, dim_max + 1)));
    rc = finish_bars(w, nb, sbits, 0, s, r->bars);
  }
  if (rc != RIPS_OK) {
    delete r;
    return rc;
  }
  r->thresholds.push_back(co.t_eff);
  r->stats = co.stats;
  r->phase_ms = co.phase_ms;
  for (int q = 0; q < RIPS_KERNEL_CLASSES; ++q) {
    r->kernel_ms[q] = co.kernel_ms[q];
    r->kernel_launches[q] = co.kernel_regions[q];
  }
  r->npoints.push_back(n);
  r->point_offsets = {0, n};
  index_result(r);
  *out = r;
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

int batched_locked(Workspace& w, const float* d_points, const int64_t* offsets, int32_t batch, int32_t k,
                   int32_t dim_max, float threshold, uint32_t p, cudaStream_t s, rips_result_t** out) {
  rips_result* r = new (std::nothrow) rips_result();
  if (!r) return RIPS_ERR_OOM;
  r->clouds = batch;
  r->dim_max = dim_max;
  r->k = k;
  uint32_t nb = 0;
  int rc = RIPS_OK;
  int64_t nmax = 1;
  for (int32_t c = 0; c < batch; ++c) nmax = std::max<int64_t>(nmax, offsets[c + 1] - offsets[c]);
  rc = ensure(w.cdist, (size_t)nmax * nmax * 4);
  for (int32_t c = 0; rc == RIPS_OK && c < batch; ++c) {
    const int64_t n = offsets[c + 1] - offsets[c];
    if (launch_distance_matrix(d_points + (size_t)offsets[c] * k, (int)n, k, P<float>(w.cdist), s) != cudaSuccess) {
      cudaGetLastError();
      rc = RIPS_ERR_CUDA;
      break;
    }
    CloudOut co;
    rc = run_cloud(w, P<float>(w.cdist), (int)n, dim_max, threshold, p, c, s, &nb, co);
    if (rc != RIPS_OK) break;
    r->thresholds.push_back(co.t_eff);
    r->stats.insert(r->stats.end(), co.stats.begin(), co.stats.end());
    for (int q = 0; q < RIPS_KERNEL_CLASSES; ++q) {
      r->kernel_ms[q] += co.kernel_ms[q];
      r->kernel_launches[q] += co.kernel_regions[q];
    }
    r->npoints.push_back(n);
  }
  if (rc == RIPS_OK) {
    const int sbits = std::max(1, bit_width64(host_binom((uint64_t)nmax, dim_max + 1)));
    rc = finish_bars(w, nb, sbits, std::max(1, bit_width64((uint64_t)batch)), s, r->bars);
  }
  if (rc != RIPS_OK) {
    delete r;
    return rc;
  }
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

}  // extern "C"
