/*
 * Seeded synthetic graph generators for the node2vec walk workloads.
 *
 * This module is an input recipe only: it builds canonical CSR graphs (int64
 * row_ptr, strictly increasing int32 col per row, optional uint32 weights) and
 * holds none of the walk arithmetic.  Both the CUDA sampler's tests and the
 * CPU oracle's tests read their graphs from here.
 *
 * Randomness: SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom
 * number generators", OOPSLA 2014), written from that published definition.
 * It is deliberately a different generator from the Philox4x32-10 stream
 * that the walks draw from, so no walk arithmetic lives here.
 *
 * Graph models (Section 4.1 of the paper):
 *  - Erdos-Renyi G(n, m): m distinct unordered pairs {u, v}, u != v, drawn
 *    uniformly with rejection.
 *  - R-MAT(a, b, c, d) on 2^K vertices: each edge picks one of the four
 *    quadrants of the adjacency matrix with probabilities a, b, c, d, then
 *    recurses into it until a single cell is left (most significant bit
 *    first).  No noise and no vertex permutation, since the paper describes
 *    none.  Edges are symmetrised, self-loops dropped and duplicates merged.
 *  - Symmetric edge weights w(u,v) = lo + H(seed, min(u,v), max(u,v)) mod
 *    (hi - lo + 1), so w(u,v) == w(v,u) by construction.
 *
 * The canonical CSR is independent of the thread count: every edge's random
 * bits come from a counter-based stream keyed by its index, and every row is
 * sorted and deduplicated at the end.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define GOLDEN 0x9e3779b97f4a7c15ULL

static inline uint64_t sm64_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

static inline uint64_t sm64_next(uint64_t* s) {
  *s += GOLDEN;
  return sm64_mix(*s);
}

/* uniform integer in [0, n) from one 64-bit draw (multiply-high). */
static inline uint64_t below(uint64_t r, uint64_t n) {
  return (uint64_t)(((unsigned __int128)r * n) >> 64);
}

/* ------------------------------------------------------------------------ */
/* A tiny dynamic parallel-for over [0, n) in chunks of `grain`.             */

typedef void (*range_fn)(int64_t lo, int64_t hi, void* ctx);

typedef struct {
  int64_t n, grain;
  int64_t next;
  range_fn fn;
  void* ctx;
} pfor_t;

static void* pfor_worker(void* arg) {
  pfor_t* p = (pfor_t*)arg;
  for (;;) {
    int64_t lo = __atomic_fetch_add(&p->next, p->grain, __ATOMIC_RELAXED);
    if (lo >= p->n) break;
    int64_t hi = lo + p->grain < p->n ? lo + p->grain : p->n;
    p->fn(lo, hi, p->ctx);
  }
  return NULL;
}

static void parallel_for(int64_t n, int64_t grain, int nthreads, range_fn fn, void* ctx) {
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 256) nthreads = 256;
  pfor_t p = {n, grain > 0 ? grain : 1, 0, fn, ctx};
  pthread_t th[256];
  int started = 0;
  for (int i = 1; i < nthreads; ++i)
    if (pthread_create(&th[started], NULL, pfor_worker, &p) == 0) ++started;
  pfor_worker(&p);
  for (int i = 0; i < started; ++i) pthread_join(th[i], NULL);
}

/* ------------------------------------------------------------------------ */
/* Row sort + dedupe, shared by both generators.                             */

static int cmp_i32(const void* a, const void* b) {
  int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
  return (x > y) - (x < y);
}

static int64_t sort_unique(int32_t* a, int64_t n) {
  if (n <= 1) return n;
  if (n <= 24) {
    for (int64_t i = 1; i < n; ++i) {
      int32_t x = a[i];
      int64_t j = i - 1;
      while (j >= 0 && a[j] > x) { a[j + 1] = a[j]; --j; }
      a[j + 1] = x;
    }
  } else {
    qsort(a, (size_t)n, sizeof(int32_t), cmp_i32);
  }
  int64_t m = 1;
  for (int64_t i = 1; i < n; ++i)
    if (a[i] != a[m - 1]) a[m++] = a[i];
  return m;
}

typedef struct {
  const int64_t* row_ptr;
  int32_t* col;
  int64_t* udeg;
} rows_ctx;

static void rows_sort_fn(int64_t lo, int64_t hi, void* vctx) {
  rows_ctx* c = (rows_ctx*)vctx;
  for (int64_t u = lo; u < hi; ++u) {
    int64_t b = c->row_ptr[u], e = c->row_ptr[u + 1];
    c->udeg[u] = sort_unique(c->col + b, e - b);
  }
}

/* Sort and dedupe every row of a pre-CSR (row_ptr over raw counts), then
 * compact in place so that row_ptr becomes the canonical CSR offsets.
 * Returns the final nnz. */
static int64_t finish_csr(int64_t n, int64_t* row_ptr, int32_t* col, int nthreads) {
  int64_t* udeg = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  if (!udeg) return -2;
  rows_ctx rc = {row_ptr, col, udeg};
  parallel_for(n, 4096, nthreads, rows_sort_fn, &rc);
  int64_t out = 0;
  for (int64_t u = 0; u < n; ++u) {
    int64_t b = row_ptr[u];
    if (b != out && udeg[u] > 0) memmove(col + out, col + b, sizeof(int32_t) * (size_t)udeg[u]);
    row_ptr[u] = out;
    out += udeg[u];
  }
  row_ptr[n] = out;
  free(udeg);
  return out;
}

/* ------------------------------------------------------------------------ */
/* Erdos-Renyi G(n, m).                                                      */

/* Writes a symmetric CSR with exactly 2m adjacency entries.  row_ptr has
 * n+1 slots, col has 2m slots.  Returns 2m, or a negative value when m is
 * larger than the number of distinct pairs or memory runs out. */
int64_t n2v_gen_er(int64_t n, int64_t m, uint64_t seed, int64_t* row_ptr, int32_t* col) {
  if (n < 2 || m < 0 || (double)m > 0.5 * (double)n * (double)(n - 1)) return -1;
  if (n > INT32_MAX) return -1;
  uint64_t cap = 16;
  while (cap < (uint64_t)(4 * m + 16)) cap <<= 1;
  uint64_t* set = (uint64_t*)calloc(cap, sizeof(uint64_t));
  int32_t* eu = (int32_t*)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
  int32_t* ev = (int32_t*)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
  if (!set || !eu || !ev) { free(set); free(eu); free(ev); return -2; }
  uint64_t s = seed;
  int64_t have = 0;
  while (have < m) {
    int64_t a = (int64_t)below(sm64_next(&s), (uint64_t)n);
    int64_t b = (int64_t)below(sm64_next(&s), (uint64_t)n);
    if (a == b) continue;
    int64_t lo = a < b ? a : b, hi = a < b ? b : a;
    uint64_t key = (uint64_t)lo * (uint64_t)n + (uint64_t)hi + 1; /* never 0 */
    uint64_t h = sm64_mix(key) & (cap - 1);
    int dup = 0;
    while (set[h]) {
      if (set[h] == key) { dup = 1; break; }
      h = (h + 1) & (cap - 1);
    }
    if (dup) continue;
    set[h] = key;
    eu[have] = (int32_t)lo;
    ev[have] = (int32_t)hi;
    ++have;
  }
  free(set);
  memset(row_ptr, 0, sizeof(int64_t) * (size_t)(n + 1));
  for (int64_t i = 0; i < m; ++i) { row_ptr[eu[i] + 1]++; row_ptr[ev[i] + 1]++; }
  for (int64_t u = 0; u < n; ++u) row_ptr[u + 1] += row_ptr[u];
  int64_t* cur = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  if (!cur) { free(eu); free(ev); return -2; }
  memcpy(cur, row_ptr, sizeof(int64_t) * (size_t)n);
  for (int64_t i = 0; i < m; ++i) {
    col[cur[eu[i]]++] = ev[i];
    col[cur[ev[i]]++] = eu[i];
  }
  free(cur); free(eu); free(ev);
  return finish_csr(n, row_ptr, col, 1);
}

/* ------------------------------------------------------------------------ */
/* R-MAT.                                                                    */

typedef struct {
  int scale;
  uint64_t seed;
  uint64_t ta, tab, tabc; /* cumulative quadrant thresholds on a 32-bit draw */
  int64_t* row_ptr;       /* counts, then offsets */
  int64_t* cur;           /* fill cursors */
  int32_t* col;
} rmat_ctx;

static inline void rmat_edge(const rmat_ctx* c, uint64_t i, uint32_t* pu, uint32_t* pv) {
  uint64_t st = sm64_mix(c->seed ^ sm64_mix(i + 0x632be59bd9b4e019ULL));
  uint32_t u = 0, v = 0;
  uint64_t bits = 0;
  int avail = 0;
  for (int lev = c->scale - 1; lev >= 0; --lev) {
    if (!avail) { bits = sm64_next(&st); avail = 2; }
    uint64_t r = bits & 0xffffffffULL;
    bits >>= 32;
    --avail;
    uint32_t ubit, vbit;
    if (r < c->ta) { ubit = 0; vbit = 0; }
    else if (r < c->tab) { ubit = 0; vbit = 1; }
    else if (r < c->tabc) { ubit = 1; vbit = 0; }
    else { ubit = 1; vbit = 1; }
    u |= ubit << lev;
    v |= vbit << lev;
  }
  *pu = u;
  *pv = v;
}

static void rmat_count_fn(int64_t lo, int64_t hi, void* vctx) {
  rmat_ctx* c = (rmat_ctx*)vctx;
  for (int64_t i = lo; i < hi; ++i) {
    uint32_t u, v;
    rmat_edge(c, (uint64_t)i, &u, &v);
    if (u == v) continue;
    __atomic_fetch_add(&c->row_ptr[u + 1], 1, __ATOMIC_RELAXED);
    __atomic_fetch_add(&c->row_ptr[v + 1], 1, __ATOMIC_RELAXED);
  }
}

static void rmat_fill_fn(int64_t lo, int64_t hi, void* vctx) {
  rmat_ctx* c = (rmat_ctx*)vctx;
  for (int64_t i = lo; i < hi; ++i) {
    uint32_t u, v;
    rmat_edge(c, (uint64_t)i, &u, &v);
    if (u == v) continue;
    int64_t pu = __atomic_fetch_add(&c->cur[u], 1, __ATOMIC_RELAXED);
    int64_t pv = __atomic_fetch_add(&c->cur[v], 1, __ATOMIC_RELAXED);
    c->col[pu] = (int32_t)v;
    c->col[pv] = (int32_t)u;
  }
}

/* R-MAT with 2^scale vertices and edge_factor * 2^scale edge draws.
 * row_ptr has 2^scale + 1 slots; col must hold col_cap >= 2 * edge draws
 * entries (the pre-dedupe size).  Returns the final nnz, or negative on a
 * bad argument (-1) or allocation failure (-2). */
int64_t n2v_gen_rmat(int scale, int64_t edge_factor, double a, double b, double c, uint64_t seed,
                     int nthreads, int64_t* row_ptr, int32_t* col, int64_t col_cap) {
  if (scale < 1 || scale > 30 || edge_factor < 0) return -1;
  if (a < 0 || b < 0 || c < 0 || a + b + c > 1.0) return -1;
  int64_t n = (int64_t)1 << scale;
  int64_t m = edge_factor * n;
  if (col_cap < 2 * m) return -1;
  rmat_ctx ctx;
  ctx.scale = scale;
  ctx.seed = seed;
  ctx.ta = (uint64_t)(a * 4294967296.0);
  ctx.tab = (uint64_t)((a + b) * 4294967296.0);
  ctx.tabc = (uint64_t)((a + b + c) * 4294967296.0);
  ctx.row_ptr = row_ptr;
  ctx.col = col;
  memset(row_ptr, 0, sizeof(int64_t) * (size_t)(n + 1));
  parallel_for(m, 1 << 16, nthreads, rmat_count_fn, &ctx);
  for (int64_t u = 0; u < n; ++u) row_ptr[u + 1] += row_ptr[u];
  ctx.cur = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  if (!ctx.cur) return -2;
  memcpy(ctx.cur, row_ptr, sizeof(int64_t) * (size_t)n);
  parallel_for(m, 1 << 16, nthreads, rmat_fill_fn, &ctx);
  free(ctx.cur);
  return finish_csr(n, row_ptr, col, nthreads);
}

/* ------------------------------------------------------------------------ */
/* Symmetric weights.                                                        */

typedef struct {
  const int64_t* row_ptr;
  const int32_t* col;
  uint64_t key;
  uint32_t lo, span;
  uint32_t* w;
} wctx;

static void weights_fn(int64_t lo, int64_t hi, void* vctx) {
  wctx* c = (wctx*)vctx;
  for (int64_t u = lo; u < hi; ++u) {
    for (int64_t e = c->row_ptr[u]; e < c->row_ptr[u + 1]; ++e) {
      uint64_t x = (uint64_t)c->col[e];
      uint64_t mn = (uint64_t)u < x ? (uint64_t)u : x;
      uint64_t mx = (uint64_t)u < x ? x : (uint64_t)u;
      uint64_t h = sm64_mix(c->key ^ sm64_mix((mn << 32) | mx));
      c->w[e] = c->lo + (uint32_t)(h % c->span);
    }
  }
}

/* w[e] for every adjacency entry, uniform in [lo, hi] and symmetric. */
int n2v_gen_weights(int64_t n, const int64_t* row_ptr, const int32_t* col, uint64_t seed, uint32_t lo,
                    uint32_t hi, int nthreads, uint32_t* w) {
  if (hi < lo) return -1;
  wctx c = {row_ptr, col, sm64_mix(seed + GOLDEN), lo, hi - lo + 1, w};
  parallel_for(n, 4096, nthreads, weights_fn, &c);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Vectors of uniform integers for start sets and job parameters.            */

/* out[i] = uniform in [0, n) from stream (seed, stream), i in [0, count). */
void n2v_gen_uniform(uint64_t seed, uint64_t stream, uint64_t n, int64_t count, int64_t* out) {
  uint64_t s = sm64_mix(seed ^ sm64_mix(stream + 0x2545f4914f6cdd1dULL));
  for (int64_t i = 0; i < count; ++i) out[i] = (int64_t)below(sm64_next(&s), n);
}

/* out[i] = raw 64-bit draws of stream (seed, stream). */
void n2v_gen_raw64(uint64_t seed, uint64_t stream, int64_t count, uint64_t* out) {
  uint64_t s = sm64_mix(seed ^ sm64_mix(stream + 0x2545f4914f6cdd1dULL));
  for (int64_t i = 0; i < count; ++i) out[i] = sm64_next(&s);
}
