/*
 * CPU oracle for Vietoris–Rips persistence barcodes -- TEST INFRASTRUCTURE.
 *
 * Plain, slow and single-threaded on purpose.  Only the tests, the smoke check
 * and the benchmark's CPU-baseline leg may call it.  It shares no code with the
 * CUDA library.  See rips_oracle.h for the two methods it implements.
 *
 * Conventions (all from Section 2 of the paper):
 *  - a d-simplex is a set of d+1 vertices; its index in the combinatorial number
 *    system is sum_l C(a_l, l+1) over its vertices a_0 < a_1 < ... < a_d;
 *  - its diameter is the largest pairwise distance (0 for a vertex);
 *  - the lexicographically refined Rips filtration orders simplices by diameter,
 *    then dimension, then reverse colexicographic order (larger index = older);
 *  - boundary coefficients are the standard orientation signs: removing the
 *    vertex at position q (increasing order) gives the facet with sign (-1)^q.
 */
#include "rips_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------- */
/* small utilities                                                           */

typedef struct {
  void* p;
  int64_t n, cap;
  size_t elem;
} vec;

static int vec_push(vec* v, const void* x) {
  if (v->n == v->cap) {
    int64_t nc = v->cap ? 2 * v->cap : 64;
    void* np = realloc(v->p, (size_t)nc * v->elem);
    if (!np) return -3;
    v->p = np;
    v->cap = nc;
  }
  memcpy((char*)v->p + (size_t)v->n * v->elem, x, v->elem);
  v->n++;
  return 0;
}
static void vec_free(vec* v) { free(v->p); v->p = NULL; v->n = v->cap = 0; }
#define VEC(T) {NULL, 0, 0, sizeof(T)}
#define AT(v, T, i) (((T*)(v).p)[i])

static float dget(const float* D, int64_t n, int64_t i, int64_t j) {
  /* strict lower triangle only */
  if (i == j) return 0.0f;
  return i > j ? D[i * n + j] : D[j * n + i];
}

/* binomial table C(i, k) for i <= n, k <= kmax, saturating at INT64_MAX */
typedef struct {
  int64_t n;
  int32_t kmax;
  int64_t* t;
} binom_t;

static int binom_init(binom_t* b, int64_t n, int32_t kmax) {
  b->n = n;
  b->kmax = kmax;
  b->t = (int64_t*)calloc((size_t)(n + 1) * (size_t)(kmax + 1), sizeof(int64_t));
  if (!b->t) return -3;
  for (int64_t i = 0; i <= n; i++) {
    for (int32_t k = 0; k <= kmax; k++) {
      int64_t v;
      if (k == 0) v = 1;
      else if (i == 0) v = 0;
      else {
        int64_t a = b->t[(i - 1) * (kmax + 1) + k - 1];
        int64_t c = b->t[(i - 1) * (kmax + 1) + k];
        v = (a > INT64_MAX - c) ? INT64_MAX : a + c;
      }
      b->t[i * (kmax + 1) + k] = v;
    }
  }
  return 0;
}
static int64_t C(const binom_t* b, int64_t i, int32_t k) {
  if (k < 0 || i < k) return 0;
  return b->t[i * (b->kmax + 1) + k];
}
static void binom_free(binom_t* b) { free(b->t); b->t = NULL; }

/* index of the simplex on ascending vertices a[0..d] */
static int64_t index_of(const binom_t* b, const int64_t* a, int32_t d) {
  int64_t s = 0;
  for (int32_t l = 0; l <= d; l++) s += C(b, a[l], l + 1);
  return s;
}

/* vertices (ascending) of the d-simplex with the given index: repeatedly take
 * the largest v with C(v, k) <= index (the Lemma of Section 4) */
static void vertices_of(const binom_t* b, int64_t idx, int32_t d, int64_t n, int64_t* a) {
  int64_t hi = n - 1;
  for (int32_t k = d + 1; k >= 1; k--) {
    int64_t v = hi;
    while (v >= 0 && C(b, v, k) > idx) v--;
    a[k - 1] = v;
    idx -= C(b, v, k);
    hi = v - 1;
  }
}

static uint32_t modinv(uint32_t a, uint32_t p) {
  /* Fermat: a^(p-2) mod p, p prime */
  uint64_t r = 1, base = a % p;
  uint32_t e = p - 2;
  while (e) {
    if (e & 1) r = (r * base) % p;
    base = (base * base) % p;
    e >>= 1;
  }
  return (uint32_t)r;
}

static int is_prime(uint32_t p) {
  if (p < 2) return 0;
  for (uint32_t q = 2; (uint64_t)q * q <= p; q++)
    if (p % q == 0) return 0;
  return 1;
}

float oracle_enclosing_radius(const float* D, int64_t n) {
  if (n <= 1) return 0.0f;
  float best = INFINITY;
  for (int64_t i = 0; i < n; i++) {
    float m = 0.0f;
    for (int64_t j = 0; j < n; j++)
      if (j != i) {
        float v = dget(D, n, i, j);
        if (v > m) m = v;
      }
    if (m < best) best = m;
  }
  return best;
}

static int check_input(const float* D, int64_t n, float threshold, float* t_eff) {
  if (!D || n < 1) return -1;
  for (int64_t i = 0; i < n; i++)
    for (int64_t j = 0; j < i; j++) {
      float v = D[i * n + j];
      if (!(v >= 0.0f) || isinf(v)) return -1;
    }
  if (isnan(threshold) || isinf(threshold)) *t_eff = oracle_enclosing_radius(D, n);
  else if (threshold < 0.0f) return -1;
  else *t_eff = threshold;
  return 0;
}

/* ------------------------------------------------------------------------- */
/* simplex lists                                                             */

typedef struct {
  int64_t idx;
  float diam;
} simp;

/* neighbour lists: nbr[v] = ascending list of u != v with d(u, v) <= t */
typedef struct {
  int64_t* off;
  int64_t* adj;
} nbrs_t;

static int nbrs_init(nbrs_t* g, const float* D, int64_t n, float t) {
  g->off = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  if (!g->off) return -3;
  for (int64_t v = 0; v < n; v++) {
    int64_t c = 0;
    for (int64_t u = 0; u < n; u++)
      if (u != v && dget(D, n, u, v) <= t) c++;
    g->off[v + 1] = g->off[v] + c;
  }
  g->adj = (int64_t*)malloc((size_t)(g->off[n] ? g->off[n] : 1) * sizeof(int64_t));
  if (!g->adj) return -3;
  for (int64_t v = 0; v < n; v++) {
    int64_t c = g->off[v];
    for (int64_t u = 0; u < n; u++)
      if (u != v && dget(D, n, u, v) <= t) g->adj[c++] = u;
  }
  return 0;
}
static void nbrs_free(nbrs_t* g) { free(g->off); free(g->adj); }

/* all d-simplices with diameter <= t, each formed as (u, rho) with u above the
 * largest vertex of a (d-1)-simplex rho (Section 4, assembling columns) */
static int next_simplices(const binom_t* b, const float* D, int64_t n, float t,
                          const nbrs_t* g, const vec* prev, int32_t d, vec* out) {
  int64_t a[64];
  for (int64_t s = 0; s < prev->n; s++) {
    simp r = AT(*prev, simp, s);
    vertices_of(b, r.idx, d - 1, n, a);
    int64_t top = a[d - 1];
    for (int64_t q = g->off[top]; q < g->off[top + 1]; q++) {
      int64_t u = g->adj[q];
      if (u <= top) continue;
      float m = r.diam;
      int ok = 1;
      for (int32_t l = 0; l < d; l++) {
        float v = dget(D, n, u, a[l]);
        if (v > t) { ok = 0; break; }
        if (v > m) m = v;
      }
      if (!ok) continue;
      simp x = {r.idx + C(b, u, d + 1), m};
      if (vec_push(out, &x)) return -3;
    }
  }
  return 0;
}

static int vertex_list(int64_t n, vec* out) {
  for (int64_t v = 0; v < n; v++) {
    simp x = {v, 0.0f};
    if (vec_push(out, &x)) return -3;
  }
  return 0;
}

/* ------------------------------------------------------------------------- */
/* result object                                                             */

/* where a bar's representative cocycle lies in the result's entry pool */
typedef struct {
  int64_t off, len;
} cospan;

struct oracle_result {
  vec bars;
  vec cospans; /* one per bar (len 0: none recorded) */
  vec copool;  /* oracle_cocycle_entry */
  float t;
  int32_t dim_max;
  int32_t keep_zero; /* also list zero-persistence pairs as bars */
  oracle_dim_stats stats[64];
};

static int add_bar(oracle_result* r, int32_t dim, float b, float dth, int64_t bs, int64_t ds) {
  oracle_bar x = {dim, b, dth, bs, ds};
  cospan none = {0, 0};
  if (vec_push(&r->bars, &x)) return -3;
  return vec_push(&r->cospans, &none);
}

int64_t oracle_result_num_bars(const oracle_result* r) { return r ? r->bars.n : -1; }
const oracle_bar* oracle_result_bars(const oracle_result* r) { return r ? (const oracle_bar*)r->bars.p : NULL; }
float oracle_result_threshold(const oracle_result* r) { return r ? r->t : NAN; }
int oracle_result_stats(const oracle_result* r, int32_t dim, oracle_dim_stats* out) {
  if (!r || dim < 0 || dim > r->dim_max + 1 || !out) return -1;
  *out = r->stats[dim];
  return 0;
}
void oracle_result_free(oracle_result* r) {
  if (!r) return;
  vec_free(&r->bars);
  vec_free(&r->cospans);
  vec_free(&r->copool);
  free(r);
}

int64_t oracle_result_cocycle(const oracle_result* r, int64_t bar, int64_t* idx_out, uint32_t* coef_out,
                              int64_t cap) {
  if (!r || bar < 0 || bar >= r->cospans.n || cap < 0 || (cap > 0 && (!idx_out || !coef_out))) return -1;
  const cospan sp = ((const cospan*)r->cospans.p)[bar];
  const oracle_cocycle_entry* e = (const oracle_cocycle_entry*)r->copool.p + sp.off;
  for (int64_t q = 0; q < sp.len && q < cap; q++) {
    idx_out[q] = e[q].idx;
    coef_out[q] = e[q].c;
  }
  return sp.len;
}

int64_t oracle_simplex_index(const int64_t* verts, int32_t d) {
  int64_t a[64];
  if (d < 0 || d > 60) return -1;
  memcpy(a, verts, sizeof(int64_t) * (size_t)(d + 1));
  for (int32_t x = 1; x <= d; x++) /* insertion sort, ascending */
    for (int32_t y = x; y > 0 && a[y - 1] > a[y]; y--) {
      int64_t tmp = a[y];
      a[y] = a[y - 1];
      a[y - 1] = tmp;
    }
  int64_t mx = a[d];
  binom_t b;
  if (binom_init(&b, mx + 1, d + 1)) return -1;
  int64_t s = index_of(&b, a, d);
  binom_free(&b);
  return s;
}

int oracle_simplex_vertices(int64_t index, int32_t d, int64_t n, int64_t* verts_out) {
  if (d < 0 || d > 60 || n < d + 1) return -1;
  binom_t b;
  if (binom_init(&b, n, d + 1)) return -3;
  if (index < 0 || index >= C(&b, n, d + 1)) { binom_free(&b); return -1; }
  int64_t a[64];
  vertices_of(&b, index, d, n, a);
  for (int32_t l = 0; l <= d; l++) verts_out[l] = a[d - l];
  binom_free(&b);
  return 0;
}

/* ========================================================================= */
/* ORACLE_DEF: explicit filtration boundary matrix + Algorithm 1              */

typedef struct {
  int32_t dim;
  int64_t idx;
  float diam;
} fsimp;

static int fsimp_cmp(const void* x, const void* y) {
  const fsimp* a = (const fsimp*)x;
  const fsimp* b = (const fsimp*)y;
  if (a->diam != b->diam) return a->diam < b->diam ? -1 : 1;
  if (a->dim != b->dim) return a->dim < b->dim ? -1 : 1;
  if (a->idx != b->idx) return a->idx > b->idx ? -1 : 1; /* reverse colex */
  return 0;
}

/* the maxdim-skeleton of Rips_t in filtration order */
static int build_filtration(const float* D, int64_t n, int32_t maxdim, float t,
                            const binom_t* b, vec* out /* fsimp */) {
  nbrs_t g;
  if (nbrs_init(&g, D, n, t)) return -3;
  vec cur = VEC(simp);
  int rc = vertex_list(n, &cur);
  for (int32_t d = 0; !rc && d <= maxdim; d++) {
    if (d > 0) {
      vec nx = VEC(simp);
      rc = next_simplices(b, D, n, t, &g, &cur, d, &nx);
      vec_free(&cur);
      cur = nx;
      if (rc) break;
    }
    for (int64_t s = 0; s < cur.n && !rc; s++) {
      fsimp x = {d, AT(cur, simp, s).idx, AT(cur, simp, s).diam};
      rc = vec_push(out, &x);
    }
  }
  vec_free(&cur);
  nbrs_free(&g);
  if (rc) return rc;
  qsort(out->p, (size_t)out->n, sizeof(fsimp), fsimp_cmp);
  return 0;
}

/* position lookup: per dimension, (idx, pos) sorted by idx */
typedef struct {
  int64_t idx, pos;
} ipos;
static int ipos_cmp(const void* x, const void* y) {
  int64_t a = ((const ipos*)x)->idx, b = ((const ipos*)y)->idx;
  return a < b ? -1 : (a > b ? 1 : 0);
}
typedef struct {
  ipos* tab[64];
  int64_t cnt[64];
} posmap;

static int posmap_init(posmap* m, const vec* filt, int32_t maxdim) {
  memset(m, 0, sizeof(*m));
  for (int64_t s = 0; s < filt->n; s++) m->cnt[AT(*filt, fsimp, s).dim]++;
  for (int32_t d = 0; d <= maxdim; d++) {
    m->tab[d] = (ipos*)malloc((size_t)(m->cnt[d] ? m->cnt[d] : 1) * sizeof(ipos));
    if (!m->tab[d]) return -3;
    m->cnt[d] = 0;
  }
  for (int64_t s = 0; s < filt->n; s++) {
    fsimp f = AT(*filt, fsimp, s);
    ipos e = {f.idx, s};
    m->tab[f.dim][m->cnt[f.dim]++] = e;
  }
  for (int32_t d = 0; d <= maxdim; d++) qsort(m->tab[d], (size_t)m->cnt[d], sizeof(ipos), ipos_cmp);
  return 0;
}
static int64_t posmap_get(const posmap* m, int32_t d, int64_t idx) {
  int64_t lo = 0, hi = m->cnt[d] - 1;
  while (lo <= hi) {
    int64_t mid = (lo + hi) / 2;
    if (m->tab[d][mid].idx == idx) return m->tab[d][mid].pos;
    if (m->tab[d][mid].idx < idx) lo = mid + 1;
    else hi = mid - 1;
  }
  return -1;
}
static void posmap_free(posmap* m) {
  for (int32_t d = 0; d < 64; d++) free(m->tab[d]);
}

/* sparse column: entries sorted by row position ascending, coefficients != 0 */
typedef struct {
  int64_t row;
  uint32_t c;
} ent;
static int ent_cmp(const void* x, const void* y) {
  int64_t a = ((const ent*)x)->row, b = ((const ent*)y)->row;
  return a < b ? -1 : (a > b ? 1 : 0);
}

/* boundary column of the simplex at filtration position j */
static int boundary_column(const vec* filt, const posmap* pm, const binom_t* b, int64_t n,
                           int64_t j, uint32_t p, ent* out, int32_t* len) {
  fsimp f = AT(*filt, fsimp, j);
  *len = 0;
  if (f.dim == 0) return 0;
  int64_t a[64], fa[64];
  vertices_of(b, f.idx, f.dim, n, a);
  for (int32_t q = 0; q <= f.dim; q++) {
    int32_t m = 0;
    for (int32_t l = 0; l <= f.dim; l++)
      if (l != q) fa[m++] = a[l];
    int64_t fi = index_of(b, fa, f.dim - 1);
    int64_t row = posmap_get(pm, f.dim - 1, fi);
    if (row < 0) return -1; /* a facet must be in the complex */
    ent e = {row, (q % 2 == 0) ? 1u % p : p - 1};
    out[(*len)++] = e;
  }
  qsort(out, (size_t)*len, sizeof(ent), ent_cmp);
  return 0;
}

/* r <- r - lam * s over Z/p, both sorted by row */
static int col_axpy(ent** r, int32_t* rl, int32_t* rcap, const ent* s, int32_t sl,
                    uint32_t lam, uint32_t p) {
  ent* out = (ent*)malloc(sizeof(ent) * (size_t)(*rl + sl + 1));
  if (!out) return -3;
  int32_t i = 0, k = 0, m = 0;
  uint32_t neg = (p - lam % p) % p;
  while (i < *rl || k < sl) {
    if (k >= sl || (i < *rl && (*r)[i].row < s[k].row)) out[m++] = (*r)[i++];
    else if (i >= *rl || s[k].row < (*r)[i].row) {
      uint32_t c = (uint32_t)(((uint64_t)s[k].c * neg) % p);
      if (c) { out[m].row = s[k].row; out[m].c = c; m++; }
      k++;
    } else {
      uint32_t c = (uint32_t)(((*r)[i].c + (uint64_t)s[k].c * neg) % p);
      if (c) { out[m].row = s[k].row; out[m].c = c; m++; }
      i++;
      k++;
    }
  }
  free(*r);
  *r = out;
  *rl = m;
  *rcap = *rl + sl + 1;
  return 0;
}

static int oracle_def(const float* D, int64_t n, int32_t dim_max, float t, uint32_t p,
                      oracle_result* res) {
  int32_t maxdim = dim_max + 1;
  binom_t b;
  if (binom_init(&b, n, maxdim + 1)) return -3;
  if (C(&b, n, maxdim + 1) == INT64_MAX) { binom_free(&b); return -2; }
  vec filt = VEC(fsimp);
  int rc = build_filtration(D, n, maxdim, t, &b, &filt);
  posmap pm;
  if (!rc) rc = posmap_init(&pm, &filt, maxdim);
  int64_t N = filt.n;
  ent** R = NULL;
  int32_t* Rl = NULL;
  int64_t* owner = NULL;
  if (!rc) {
    R = (ent**)calloc((size_t)N + 1, sizeof(ent*));
    Rl = (int32_t*)calloc((size_t)N + 1, sizeof(int32_t));
    owner = (int64_t*)malloc(sizeof(int64_t) * ((size_t)N + 1));
    if (!R || !Rl || !owner) rc = -3;
  }
  for (int64_t i = 0; !rc && i < N; i++) owner[i] = -1;
  /* Algorithm 1: columns in increasing order; reduce while an earlier column
   * has the same pivot (largest row index). */
  for (int64_t j = 0; !rc && j < N; j++) {
    ent tmp[64];
    int32_t len;
    rc = boundary_column(&filt, &pm, &b, n, j, p, tmp, &len);
    if (rc) break;
    int32_t cap = len + 1;
    R[j] = (ent*)malloc(sizeof(ent) * (size_t)cap);
    if (!R[j]) { rc = -3; break; }
    memcpy(R[j], tmp, sizeof(ent) * (size_t)len);
    Rl[j] = len;
    while (Rl[j] > 0) {
      int64_t piv = R[j][Rl[j] - 1].row;
      int64_t k = owner[piv];
      if (k < 0) break;
      uint32_t lam = (uint32_t)(((uint64_t)R[j][Rl[j] - 1].c * modinv(R[k][Rl[k] - 1].c, p)) % p);
      res->stats[AT(filt, fsimp, j).dim < 63 ? AT(filt, fsimp, j).dim : 63].additions++;
      rc = col_axpy(&R[j], &Rl[j], &cap, R[k], Rl[k], lam, p);
      if (rc) break;
    }
    if (!rc && Rl[j] > 0) owner[R[j][Rl[j] - 1].row] = j;
  }
  /* pairs (pivot R_j, j) and essential indices (R_i = 0, i not a pivot) */
  if (!rc) {
    for (int64_t j = 0; j < N; j++) {
      fsimp fj = AT(filt, fsimp, j);
      if (fj.dim <= dim_max) res->stats[fj.dim].simplices++;
      if (Rl[j] > 0) {
        int64_t i = R[j][Rl[j] - 1].row;
        fsimp fi = AT(filt, fsimp, i);
        res->stats[fi.dim].pairs++;
        if (fi.diam == fj.diam) res->stats[fi.dim].zero_pairs++;
        if ((fi.diam != fj.diam || res->keep_zero) &&
            (rc = add_bar(res, fi.dim, fi.diam, fj.diam, fi.idx, fj.idx)))
          break;
      }
    }
    for (int64_t i = 0; !rc && i < N; i++) {
      fsimp fi = AT(filt, fsimp, i);
      if (fi.dim > dim_max) continue;
      if (Rl[i] == 0 && owner[i] < 0) {
        res->stats[fi.dim].essential++;
        rc = add_bar(res, fi.dim, fi.diam, INFINITY, fi.idx, -1);
      }
    }
    for (int32_t d = 0; d <= dim_max; d++) res->stats[d].columns = res->stats[d].simplices;
  }
  /* zero-persistence apparent pairs, for the statistics */
  if (!rc) {
    int64_t* mincof = (int64_t*)malloc(sizeof(int64_t) * ((size_t)N + 1));
    if (!mincof) rc = -3;
    for (int64_t i = 0; !rc && i < N; i++) mincof[i] = -1;
    for (int64_t j = 0; !rc && j < N; j++) {
      ent tmp[64];
      int32_t len;
      rc = boundary_column(&filt, &pm, &b, n, j, p, tmp, &len);
      for (int32_t q = 0; !rc && q < len; q++)
        if (mincof[tmp[q].row] < 0) mincof[tmp[q].row] = j; /* j increasing */
    }
    for (int64_t j = 0; !rc && j < N; j++) {
      ent tmp[64];
      int32_t len;
      rc = boundary_column(&filt, &pm, &b, n, j, p, tmp, &len);
      if (rc || len == 0) continue;
      int64_t s = tmp[len - 1].row; /* youngest facet */
      if (mincof[s] == j && AT(filt, fsimp, s).diam == AT(filt, fsimp, j).diam) {
        int32_t d = AT(filt, fsimp, s).dim;
        if (d <= dim_max) res->stats[d].apparent_zero++;
      }
    }
    free(mincof);
  }
  if (R)
    for (int64_t j = 0; j < N; j++) free(R[j]);
  free(R);
  free(Rl);
  free(owner);
  if (filt.p) posmap_free(&pm);
  vec_free(&filt);
  binom_free(&b);
  return rc;
}

int64_t oracle_filtration(const float* D, int64_t n, int32_t maxdim, float threshold,
                          int32_t* out_dim, int64_t* out_index, float* out_diam, int64_t cap) {
  float t;
  if (check_input(D, n, threshold, &t) || maxdim < 0 || maxdim > 60) return -1;
  binom_t b;
  if (binom_init(&b, n, maxdim + 1)) return -3;
  vec filt = VEC(fsimp);
  int rc = build_filtration(D, n, maxdim, t, &b, &filt);
  int64_t N = filt.n;
  for (int64_t s = 0; !rc && s < N && s < cap; s++) {
    fsimp f = AT(filt, fsimp, s);
    if (out_dim) out_dim[s] = f.dim;
    if (out_index) out_index[s] = f.idx;
    if (out_diam) out_diam[s] = f.diam;
  }
  vec_free(&filt);
  binom_free(&b);
  return rc ? rc : N;
}

int64_t oracle_boundary_matrix(const float* D, int64_t n, int32_t maxdim, float threshold,
                               uint32_t p, int64_t* out_row, int64_t* out_col,
                               uint32_t* out_coeff, int64_t cap) {
  float t;
  if (check_input(D, n, threshold, &t) || maxdim < 0 || maxdim > 60 || !is_prime(p)) return -1;
  binom_t b;
  if (binom_init(&b, n, maxdim + 1)) return -3;
  vec filt = VEC(fsimp);
  int rc = build_filtration(D, n, maxdim, t, &b, &filt);
  posmap pm;
  if (!rc) rc = posmap_init(&pm, &filt, maxdim);
  int64_t cnt = 0;
  for (int64_t j = 0; !rc && j < filt.n; j++) {
    ent tmp[64];
    int32_t len;
    rc = boundary_column(&filt, &pm, &b, n, j, p, tmp, &len);
    for (int32_t q = 0; !rc && q < len; q++) {
      if (cnt < cap) {
        out_row[cnt] = tmp[q].row;
        out_col[cnt] = j;
        out_coeff[cnt] = tmp[q].c;
      }
      cnt++;
    }
  }
  if (filt.p) posmap_free(&pm);
  vec_free(&filt);
  binom_free(&b);
  return rc ? rc : cnt;
}

int64_t oracle_apparent_pairs(const float* D, int64_t n, int32_t maxdim, float threshold,
                              int64_t* out_sigma, int64_t* out_tau, int64_t cap) {
  float t;
  if (check_input(D, n, threshold, &t) || maxdim < 0 || maxdim > 60) return -1;
  binom_t b;
  if (binom_init(&b, n, maxdim + 1)) return -3;
  vec filt = VEC(fsimp);
  int rc = build_filtration(D, n, maxdim, t, &b, &filt);
  posmap pm;
  if (!rc) rc = posmap_init(&pm, &filt, maxdim);
  int64_t N = filt.n, cnt = 0;
  int64_t* mincof = rc ? NULL : (int64_t*)malloc(sizeof(int64_t) * ((size_t)N + 1));
  if (!rc && !mincof) rc = -3;
  for (int64_t i = 0; !rc && i < N; i++) mincof[i] = -1;
  /* oldest cofacet of sigma = cofacet with the smallest filtration position */
  for (int64_t j = 0; !rc && j < N; j++) {
    ent tmp[64];
    int32_t len;
    rc = boundary_column(&filt, &pm, &b, n, j, 2, tmp, &len);
    for (int32_t q = 0; !rc && q < len; q++)
      if (mincof[tmp[q].row] < 0) mincof[tmp[q].row] = j;
  }
  /* (sigma, tau) apparent iff sigma is the youngest facet of tau and tau is the
   * oldest cofacet of sigma */
  for (int64_t j = 0; !rc && j < N; j++) {
    ent tmp[64];
    int32_t len;
    rc = boundary_column(&filt, &pm, &b, n, j, 2, tmp, &len);
    if (rc || len == 0) continue;
    int64_t s = tmp[len - 1].row;
    if (mincof[s] == j) {
      if (cnt < cap) {
        out_sigma[cnt] = s;
        out_tau[cnt] = j;
      }
      cnt++;
    }
  }
  free(mincof);
  if (filt.p) posmap_free(&pm);
  vec_free(&filt);
  binom_free(&b);
  return rc ? rc : cnt;
}

int64_t oracle_count_simplices(const float* D, int64_t n, int32_t d, float threshold) {
  float t;
  if (check_input(D, n, threshold, &t) || d < 0 || d > 60) return -1;
  if (d == 0) return n;
  binom_t b;
  if (binom_init(&b, n, d + 1)) return -3;
  nbrs_t g;
  if (nbrs_init(&g, D, n, t)) { binom_free(&b); return -3; }
  vec cur = VEC(simp);
  int rc = vertex_list(n, &cur);
  for (int32_t k = 1; !rc && k <= d; k++) {
    vec nx = VEC(simp);
    rc = next_simplices(&b, D, n, t, &g, &cur, k, &nx);
    vec_free(&cur);
    cur = nx;
  }
  int64_t cnt = cur.n;
  vec_free(&cur);
  nbrs_free(&g);
  binom_free(&b);
  return rc ? rc : cnt;
}

/* ========================================================================= */
/* ORACLE_COH: cohomology with clearing, implicit coboundary columns          */

/* a coboundary entry: a (d+1)-simplex with its diameter and coefficient */
typedef struct {
  float diam;
  int64_t idx;
  uint32_t c;
} cent;

/* filtration order on rows: older first = smaller diameter, then larger index */
static int older(float da, int64_t ia, float db, int64_t ib) {
  return da < db || (da == db && ia > ib);
}
/* column processing order: reverse filtration = larger diameter, then smaller index */
static int col_cmp(const void* x, const void* y) {
  const simp* a = (const simp*)x;
  const simp* b = (const simp*)y;
  if (a->diam != b->diam) return a->diam > b->diam ? -1 : 1;
  if (a->idx != b->idx) return a->idx < b->idx ? -1 : 1;
  return 0;
}
/* filtration order on simplices of one dimension: diameter up, then index down */
static int edge_filtration_cmp(const void* x, const void* y) {
  const simp* a = (const simp*)x;
  const simp* b = (const simp*)y;
  if (a->diam != b->diam) return a->diam < b->diam ? -1 : 1;
  if (a->idx != b->idx) return a->idx > b->idx ? -1 : 1;
  return 0;
}
static int simp_idx_cmp(const void* x, const void* y) {
  int64_t a = ((const simp*)x)->idx, b = ((const simp*)y)->idx;
  return a < b ? -1 : (a > b ? 1 : 0);
}

/* open-addressing map int64 -> int64 */
typedef struct {
  int64_t* keys;
  int64_t* vals;
  int64_t cap, cnt;
} hmap;
static uint64_t mix64(uint64_t x) {
  x ^= x >> 33;
  x *= 0xff51afd7ed558ccdULL;
  x ^= x >> 33;
  x *= 0xc4ceb9fe1a85ec53ULL;
  x ^= x >> 33;
  return x;
}
static int hmap_init(hmap* h, int64_t cap) {
  h->cap = 16;
  while (h->cap < 2 * cap) h->cap *= 2;
  h->cnt = 0;
  h->keys = (int64_t*)malloc(sizeof(int64_t) * (size_t)h->cap);
  h->vals = (int64_t*)malloc(sizeof(int64_t) * (size_t)h->cap);
  if (!h->keys || !h->vals) return -3;
  for (int64_t i = 0; i < h->cap; i++) h->keys[i] = -1;
  return 0;
}
static int64_t* hmap_slot(const hmap* h, int64_t key) {
  uint64_t i = mix64((uint64_t)key) & (uint64_t)(h->cap - 1);
  while (h->keys[i] != -1 && h->keys[i] != key) i = (i + 1) & (uint64_t)(h->cap - 1);
  return &h->keys[i];
}
static int64_t hmap_get(const hmap* h, int64_t key) {
  int64_t* s = hmap_slot(h, key);
  return *s == key ? h->vals[s - h->keys] : -1;
}
static int hmap_put(hmap* h, int64_t key, int64_t val) {
  if (2 * (h->cnt + 1) > h->cap) {
    hmap g;
    if (hmap_init(&g, h->cap)) return -3;
    for (int64_t i = 0; i < h->cap; i++)
      if (h->keys[i] != -1) {
        int64_t* s = hmap_slot(&g, h->keys[i]);
        *s = h->keys[i];
        g.vals[s - g.keys] = h->vals[i];
        g.cnt++;
      }
    free(h->keys);
    free(h->vals);
    *h = g;
  }
  int64_t* s = hmap_slot(h, key);
  if (*s != key) { *s = key; h->cnt++; }
  h->vals[s - h->keys] = val;
  return 0;
}
static void hmap_free(hmap* h) { free(h->keys); free(h->vals); }

typedef struct {
  const float* D;
  int64_t n;
  float t;
  uint32_t p;
  const binom_t* b;
  const nbrs_t* g;
} coh_ctx;

/* all cofacets of the d-simplex s with diameter <= t, scaled by lam, appended
 * (Section 3.4: coboundary columns are generated on the fly) */
static int push_coboundary(const coh_ctx* x, int64_t sidx, float sdiam, int32_t d, uint32_t lam,
                           vec* out) {
  int64_t a[64], ca[64];
  vertices_of(x->b, sidx, d, x->n, a);
  /* candidate vertices: neighbours of the vertex of s with the fewest of them */
  int32_t best = 0;
  for (int32_t l = 1; l <= d; l++)
    if (x->g->off[a[l] + 1] - x->g->off[a[l]] < x->g->off[a[best] + 1] - x->g->off[a[best]]) best = l;
  for (int64_t q = x->g->off[a[best]]; q < x->g->off[a[best] + 1]; q++) {
    int64_t u = x->g->adj[q];
    float m = sdiam;
    int ok = 1, below = 0;
    for (int32_t l = 0; l <= d; l++) {
      if (a[l] == u) { ok = 0; break; }
      float v = dget(x->D, x->n, u, a[l]);
      if (v > x->t) { ok = 0; break; }
      if (v > m) m = v;
      if (a[l] < u) below++;
    }
    if (!ok) continue;
    int32_t k = 0;
    for (int32_t l = 0; l <= d; l++) {
      if (l == below) ca[k++] = u;
      ca[k++] = a[l];
    }
    if (below == d + 1) ca[k++] = u;
    /* u sits at position `below` of the cofacet: sign (-1)^below */
    uint32_t sign = (below % 2 == 0) ? 1u : x->p - 1;
    cent e = {m, index_of(x->b, ca, d + 1), (uint32_t)(((uint64_t)sign * lam) % x->p)};
    if (vec_push(out, &e)) return -3;
  }
  return 0;
}

/* Working coboundary column as a lazy binary heap (Section 4, "Pivot
 * extraction"): entries with the same row may appear several times and are
 * summed only when they reach the top.  The oldest row is on top. */
static int heap_push(vec* h, cent e) {
  if (vec_push(h, &e)) return -3;
  cent* a = (cent*)h->p;
  int64_t i = h->n - 1;
  while (i > 0) {
    int64_t up = (i - 1) / 2;
    if (!older(a[i].diam, a[i].idx, a[up].diam, a[up].idx)) break;
    cent t = a[i];
    a[i] = a[up];
    a[up] = t;
    i = up;
  }
  return 0;
}
static cent heap_pop(vec* h) {
  cent* a = (cent*)h->p;
  cent top = a[0];
  a[0] = a[--h->n];
  int64_t i = 0;
  for (;;) {
    int64_t l = 2 * i + 1, r = l + 1, m = i;
    if (l < h->n && older(a[l].diam, a[l].idx, a[m].diam, a[m].idx)) m = l;
    if (r < h->n && older(a[r].diam, a[r].idx, a[m].diam, a[m].idx)) m = r;
    if (m == i) break;
    cent t = a[i];
    a[i] = a[m];
    a[m] = t;
    i = m;
  }
  return top;
}
/* pivot of the column held in the heap: pop equal rows, summing their
 * coefficients, until a nonzero sum appears; it is pushed back and returned
 * (coefficient 0 means the column is zero) */
static cent heap_pivot(vec* h, uint32_t p) {
  while (h->n > 0) {
    cent e = heap_pop(h);
    uint64_t s = e.c;
    while (h->n > 0 && ((cent*)h->p)[0].idx == e.idx) s += heap_pop(h).c;
    e.c = (uint32_t)(s % p);
    if (e.c) {
      heap_push(h, e); /* cannot grow: an entry was just popped */
      return e;
    }
  }
  cent z = {0.0f, -1, 0};
  return z;
}

/* a stored column of V: (simplex index, diameter, coefficient) */
typedef struct {
  int64_t idx;
  float diam;
  uint32_t c;
} vent;

static int vadd(vec* V, const vent* w, int64_t wl, uint32_t lam, uint32_t p) {
  /* V <- V + lam * w, V sorted by idx */
  vec out = VEC(vent);
  int64_t i = 0, k = 0;
  while (i < V->n || k < wl) {
    vent e;
    if (k >= wl || (i < V->n && AT(*V, vent, i).idx < w[k].idx)) e = AT(*V, vent, i++);
    else {
      uint32_t add = (uint32_t)(((uint64_t)w[k].c * lam) % p);
      if (i < V->n && AT(*V, vent, i).idx == w[k].idx) {
        e = AT(*V, vent, i++);
        e.c = (uint32_t)(((uint64_t)e.c + add) % p);
      } else {
        e = w[k];
        e.c = add;
      }
      k++;
      if (!e.c) continue;
    }
    if (vec_push(&out, &e)) { vec_free(&out); return -3; }
  }
  vec_free(V);
  *V = out;
  return 0;
}

/* The representative cocycle of the bar just added: the column V_j of the
 * reduction, R_j = delta V_j (Sections 3.1 and 3.4), as (simplex index,
 * coefficient) in increasing index order.  For an essential class R_j = 0, so
 * V_j is a cocycle; for a pair (sigma_j, tau) delta V_j vanishes on every
 * (d+1)-simplex older than tau and not on tau. */
static int record_cocycle(oracle_result* res, const vec* V) {
  cospan* sp = (cospan*)res->cospans.p + (res->cospans.n - 1);
  sp->off = res->copool.n;
  sp->len = V->n;
  for (int64_t q = 0; q < V->n; q++) {
    const vent* v = &AT(*V, vent, q);
    oracle_cocycle_entry e = {v->idx, v->c};
    if (vec_push(&res->copool, &e)) return -3;
  }
  return 0;
}

static int oracle_coh(const float* D, int64_t n, int32_t dim_max, float t, uint32_t p,
                      oracle_result* res) {
  binom_t b;
  if (binom_init(&b, n, dim_max + 2)) return -3;
  if (C(&b, n, dim_max + 2) == INT64_MAX) { binom_free(&b); return -2; }
  nbrs_t g;
  if (nbrs_init(&g, D, n, t)) { binom_free(&b); return -3; }
  coh_ctx x = {D, n, t, p, &b, &g};
  int rc = 0;

  /* ---- dimension 0: Kruskal over edges in filtration order, union-find ---- */
  vec verts = VEC(simp), edges = VEC(simp);
  rc = vertex_list(n, &verts);
  if (!rc) rc = next_simplices(&b, D, n, t, &g, &verts, 1, &edges);
  vec cleared = VEC(simp); /* pivots of the previous dimension, sorted by idx */
  if (!rc) {
    simp* e = (simp*)edges.p;
    int64_t E = edges.n;
    simp* order = (simp*)malloc(sizeof(simp) * (size_t)(E ? E : 1));
    int64_t* parent = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
    int64_t* top = (int64_t*)malloc(sizeof(int64_t) * (size_t)n); /* oldest vertex = max index */
    if (!order || !parent || !top) rc = -3;
    if (!rc) {
      memcpy(order, e, sizeof(simp) * (size_t)E);
      qsort(order, (size_t)E, sizeof(simp), edge_filtration_cmp);
      for (int64_t v = 0; v < n; v++) { parent[v] = v; top[v] = v; }
      res->stats[0].simplices = n;
      res->stats[0].columns = n;
      for (int64_t i = 0; !rc && i < E; i++) {
        int64_t a[2];
        vertices_of(&b, order[i].idx, 1, n, a);
        int64_t ru = a[0], rv = a[1];
        while (parent[ru] != ru) ru = parent[ru] = parent[parent[ru]];
        while (parent[rv] != rv) rv = parent[rv] = parent[parent[rv]];
        if (ru == rv) continue;
        /* elder rule: the component whose oldest vertex is younger dies */
        int64_t die = top[ru] < top[rv] ? top[ru] : top[rv];
        int64_t live = top[ru] < top[rv] ? top[rv] : top[ru];
        parent[ru] = rv;
        top[rv] = live;
        res->stats[0].pairs++;
        if (order[i].diam == 0.0f) res->stats[0].zero_pairs++;
        if (order[i].diam != 0.0f || res->keep_zero) rc = add_bar(res, 0, 0.0f, order[i].diam, die, order[i].idx);
        if (!rc) rc = vec_push(&cleared, &order[i]);
      }
      for (int64_t v = 0; !rc && v < n; v++)
        if (parent[v] == v) {
          res->stats[0].essential++;
          rc = add_bar(res, 0, 0.0f, INFINITY, top[v], -1);
        }
    }
    free(order);
    free(parent);
    free(top);
  }
  if (!rc) qsort(cleared.p, (size_t)cleared.n, sizeof(simp), simp_idx_cmp);

  /* ---- dimensions 1..dim_max: Algorithm 2 on coboundary matrices ---- */
  vec simplices = edges; /* all d-simplices <= t */
  edges.p = NULL;
  vec_free(&verts);
  for (int32_t d = 1; !rc && d <= dim_max; d++) {
    if (d > 1) {
      vec nx = VEC(simp);
      rc = next_simplices(&b, D, n, t, &g, &simplices, d, &nx);
      vec_free(&simplices);
      simplices = nx;
      if (rc) break;
    }
    res->stats[d].simplices = simplices.n;
    /* columns: d-simplices that are not pivots of dimension d-1 (clearing) */
    vec cols = VEC(simp);
    for (int64_t s = 0; !rc && s < simplices.n; s++) {
      simp key = AT(simplices, simp, s);
      if (cleared.n && bsearch(&key, cleared.p, (size_t)cleared.n, sizeof(simp), simp_idx_cmp)) continue;
      rc = vec_push(&cols, &key);
    }
    if (rc) { vec_free(&cols); break; }
    qsort(cols.p, (size_t)cols.n, sizeof(simp), col_cmp);
    res->stats[d].columns = cols.n;

    hmap piv; /* pivot simplex index -> column ordinal */
    rc = hmap_init(&piv, cols.n + 16);
    uint32_t* pivc = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(cols.n + 1));
    int64_t* voff = (int64_t*)malloc(sizeof(int64_t) * (size_t)(cols.n + 1));
    int64_t* vlen = (int64_t*)malloc(sizeof(int64_t) * (size_t)(cols.n + 1));
    vec vpool = VEC(vent);
    vec next_cleared = VEC(simp);
    if (!pivc || !voff || !vlen) rc = -3;

    vec work = VEC(cent), tmp = VEC(cent), heap = VEC(cent), V = VEC(vent);
    for (int64_t j = 0; !rc && j < cols.n; j++) {
      simp sj = AT(cols, simp, j);
      work.n = 0;
      rc = push_coboundary(&x, sj.idx, sj.diam, d, 1, &work);
      if (rc) break;
      /* pivot = oldest entry of the unreduced coboundary */
      int64_t pi = -1;
      for (int64_t q = 0; q < work.n; q++)
        if (pi < 0 || older(AT(work, cent, q).diam, AT(work, cent, q).idx,
                            AT(work, cent, pi).diam, AT(work, cent, pi).idx))
          pi = q;
      V.n = 0;
      vent self = {sj.idx, sj.diam, 1};
      rc = vec_push(&V, &self);
      cent pv = {0.0f, -1, 0};
      if (pi >= 0) pv = AT(work, cent, pi);
      if (!rc && pi >= 0 && hmap_get(&piv, pv.idx) >= 0) {
        /* the pivot is taken by an earlier column: reduce (Algorithm 1 loop),
         * with the working coboundary R_j kept as a lazy heap */
        heap.n = 0;
        for (int64_t q = 0; !rc && q < work.n; q++) rc = heap_push(&heap, AT(work, cent, q));
        pv = heap_pivot(&heap, p);
        while (!rc && pv.c) {
          int64_t k = hmap_get(&piv, pv.idx);
          if (k < 0) break;
          uint32_t lam = (uint32_t)(((uint64_t)pv.c * modinv(pivc[k], p)) % p);
          uint32_t neg = (p - lam) % p;
          res->stats[d].additions++;
          /* R_j <- R_j - lam * D V_k, recomputing D V_k (implicit reduction) */
          tmp.n = 0;
          simp sk = AT(cols, simp, k);
          vent selfk = {sk.idx, sk.diam, 1};
          const vent* vk = vlen[k] > 0 ? &AT(vpool, vent, voff[k]) : &selfk;
          int64_t vkl = vlen[k] > 0 ? vlen[k] : 1;
          for (int64_t q = 0; !rc && q < vkl; q++)
            rc = push_coboundary(&x, vk[q].idx, vk[q].diam, d,
                                 (uint32_t)(((uint64_t)vk[q].c * neg) % p), &tmp);
          if (rc) break;
          for (int64_t q = 0; !rc && q < tmp.n; q++)
            if (AT(tmp, cent, q).c) rc = heap_push(&heap, AT(tmp, cent, q));
          /* V_j <- V_j - lam * V_k */
          rc = vadd(&V, vk, vkl, neg, p);
          if (!rc) pv = heap_pivot(&heap, p);
        }
        pi = pv.c ? 0 : -1;
      }
      if (rc) break;
      if (pi < 0) {
        res->stats[d].essential++;
        rc = add_bar(res, d, sj.diam, INFINITY, sj.idx, -1);
        if (!rc) rc = record_cocycle(res, &V);
      } else {
        rc = hmap_put(&piv, pv.idx, j);
        pivc[j] = pv.c;
        res->stats[d].pairs++;
        if (pv.diam == sj.diam) res->stats[d].zero_pairs++;
        if (!rc && (pv.diam != sj.diam || res->keep_zero)) {
          rc = add_bar(res, d, sj.diam, pv.diam, sj.idx, pv.idx);
          if (!rc) rc = record_cocycle(res, &V);
        }
        simp cl = {pv.idx, pv.diam};
        if (!rc) rc = vec_push(&next_cleared, &cl);
        /* store V_j for this death column (only if it is not just e_j) */
        vlen[j] = 0;
        if (!rc && V.n > 1) {
          voff[j] = vpool.n;
          vlen[j] = V.n;
          for (int64_t q = 0; !rc && q < V.n; q++) rc = vec_push(&vpool, &AT(V, vent, q));
        }
      }
    }
    vec_free(&work);
    vec_free(&tmp);
    vec_free(&heap);
    vec_free(&V);
    vec_free(&vpool);
    free(pivc);
    free(voff);
    free(vlen);
    hmap_free(&piv);
    vec_free(&cols);
    vec_free(&cleared);
    cleared = next_cleared;
    if (!rc) qsort(cleared.p, (size_t)cleared.n, sizeof(simp), simp_idx_cmp);
  }
  vec_free(&simplices);
  vec_free(&cleared);
  vec_free(&edges);
  nbrs_free(&g);
  binom_free(&b);
  return rc;
}

int oracle_barcodes(const float* D, int64_t n, int32_t dim_max, float threshold, uint32_t p,
                    int32_t method, oracle_result** out) {
  if (!out) return -1;
  *out = NULL;
  float t;
  if (check_input(D, n, threshold, &t)) return -1;
  if (dim_max < 0 || dim_max > 60 || !is_prime(p) || p >= 65536) return -1;
  int32_t keep_zero = (method & ORACLE_KEEP_ZERO) != 0;
  method &= ~ORACLE_KEEP_ZERO;
  if (method != ORACLE_DEF && method != ORACLE_COH) return -1;
  oracle_result* r = (oracle_result*)calloc(1, sizeof(oracle_result));
  if (!r) return -3;
  r->bars.elem = sizeof(oracle_bar);
  r->cospans.elem = sizeof(cospan);
  r->copool.elem = sizeof(oracle_cocycle_entry);
  r->t = t;
  r->dim_max = dim_max;
  r->keep_zero = keep_zero;
  int rc = method == ORACLE_DEF ? oracle_def(D, n, dim_max, t, p, r) : oracle_coh(D, n, dim_max, t, p, r);
  if (rc) {
    oracle_result_free(r);
    return rc;
  }
  *out = r;
  return 0;
}
