/*
 * Seeded synthetic graph generators and the symmetrising CSR builder.
 *
 * This module only synthesises inputs. It holds no connected-components
 * arithmetic and is shared by the CUDA path's tests/benchmarks and by the CPU
 * oracle's tests, which both receive the same arrays from it.
 *
 * Random numbers: a counter-based generator. Draw number `ctr` of stream `key`
 * is the splitmix64 output function (Steele, Lea and Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014; constants of Vigna's public
 * splitmix64) applied to key + (ctr + 1) * golden-gamma. Every edge/vertex
 * draws from its own counter, so the output does not depend on the thread
 * count.
 *
 * Graph families (they stand in for the road, social and Kronecker graphs the
 * paper evaluates in its Table I):
 *   - Erdos-Renyi: E edges, both endpoints uniform over [0, V); self-loops and
 *     duplicates are kept.
 *   - 2D grid: side x side lattice, row-major IDs, every lattice edge kept
 *     independently with probability p.
 *   - R-MAT (Chakrabarti, Zhan and Faloutsos, SDM 2004): recursive quadrant
 *     choice with probabilities (a, b, c, 1-a-b-c), no noise, followed by a
 *     keyed pseudo-random permutation of vertex IDs (4-round Feistel network
 *     with cycle walking, Luby-Rackoff).
 * Symmetrisation emits both (u,v) and (v,u) for every drawn edge, including
 * self-loops, so the CSR holds exactly 2E arcs; each row is sorted ascending so
 * the output is deterministic.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

#define GOLDEN_GAMMA 0x9E3779B97F4A7C15ULL

static inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* Draw `ctr` of the stream identified by `key`. */
static inline uint64_t draw(uint64_t key, uint64_t ctr) {
  return mix64(key + (ctr + 1) * GOLDEN_GAMMA);
}

/* Independent stream keys per (seed, purpose). */
static inline uint64_t stream_key(uint64_t seed, uint64_t purpose) {
  return mix64(mix64(seed ^ 0x5DEECE66DULL) + purpose * GOLDEN_GAMMA);
}

/* Uniform integer in [0, n) by 64x64->128 multiply-high (Lemire). */
static inline uint64_t bounded(uint64_t h, uint64_t n) {
  return (uint64_t)(((unsigned __int128)h * n) >> 64);
}

enum { PURPOSE_ER = 1, PURPOSE_GRID = 2, PURPOSE_RMAT = 3, PURPOSE_PERM = 4 };

/* ------------------------------------------------------------------------- */
/* A minimal parallel-for over [0, n) split into contiguous chunks.          */

typedef void (*range_fn)(void* ctx, int64_t lo, int64_t hi);

typedef struct {
  range_fn fn;
  void* ctx;
  int64_t lo, hi;
} range_job;

static void* range_thread(void* arg) {
  range_job* j = (range_job*)arg;
  j->fn(j->ctx, j->lo, j->hi);
  return NULL;
}

static void parallel_for(int64_t n, int nthreads, range_fn fn, void* ctx) {
  if (n <= 0) return;
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 256) nthreads = 256;
  if ((int64_t)nthreads > n) nthreads = (int)n;
  if (nthreads == 1 || n < 65536) {
    fn(ctx, 0, n);
    return;
  }
  pthread_t th[256];
  range_job jobs[256];
  int joined[256];
  for (int t = 0; t < nthreads; ++t) {
    jobs[t].fn = fn;
    jobs[t].ctx = ctx;
    jobs[t].lo = n * t / nthreads;
    jobs[t].hi = n * (t + 1) / nthreads;
    joined[t] = pthread_create(&th[t], NULL, range_thread, &jobs[t]) == 0;
    if (!joined[t]) range_thread(&jobs[t]); /* could not start a thread: run the chunk here */
  }
  for (int t = 0; t < nthreads; ++t)
    if (joined[t]) pthread_join(th[t], NULL);
}

/* ------------------------------------------------------------------------- */
/* Erdos-Renyi edge list.                                                     */

typedef struct {
  uint64_t key, V;
  int32_t *src, *dst;
} er_ctx;

static void er_range(void* p, int64_t lo, int64_t hi) {
  er_ctx* c = (er_ctx*)p;
  for (int64_t i = lo; i < hi; ++i) {
    c->src[i] = (int32_t)bounded(draw(c->key, 2 * (uint64_t)i), c->V);
    c->dst[i] = (int32_t)bounded(draw(c->key, 2 * (uint64_t)i + 1), c->V);
  }
}

int gen_er_coo(int64_t V, int64_t E, uint64_t seed, int32_t* src, int32_t* dst, int nthreads) {
  if (V < 0 || E < 0 || V > INT32_MAX) return -1;
  if (E > 0 && V == 0) return -1;
  er_ctx c = {stream_key(seed, PURPOSE_ER), (uint64_t)V, src, dst};
  parallel_for(E, nthreads, er_range, &c);
  return 0;
}

/* ------------------------------------------------------------------------- */
/* Pseudo-random permutation of [0, n): balanced Feistel network over the     */
/* smallest even bit width covering n-1, cycle-walking back into [0, n).      */

typedef struct {
  uint64_t key;
  uint32_t n;
  int half;
} perm_ctx;

static void perm_init(perm_ctx* p, uint64_t seed, uint32_t n) {
  p->key = stream_key(seed, PURPOSE_PERM);
  p->n = n;
  int bits = 0;
  while (bits < 32 && ((uint64_t)1 << bits) < (uint64_t)n) ++bits;
  if (bits & 1) ++bits;
  if (bits < 2) bits = 2;
  p->half = bits / 2;
}

static inline uint32_t perm_apply(const perm_ctx* p, uint32_t x) {
  if (p->n <= 1) return x;
  const uint32_t mask = (1u << p->half) - 1u;
  do {
    uint32_t L = x >> p->half, R = x & mask;
    for (uint32_t r = 0; r < 4; ++r) {
      uint32_t f = (uint32_t)draw(p->key, ((uint64_t)r << 32) | R) & mask;
      uint32_t t = L ^ f;
      L = R;
      R = t;
    }
    x = (L << p->half) | R;
  } while (x >= p->n);
  return x;
}

/* Exposed for tests: writes perm(i) for i in [0, n). */
int gen_permutation(uint32_t n, uint64_t seed, int32_t* out) {
  perm_ctx p;
  perm_init(&p, seed, n);
  for (uint32_t i = 0; i < n; ++i) out[i] = (int32_t)perm_apply(&p, i);
  return 0;
}

/* ------------------------------------------------------------------------- */
/* R-MAT edge list.                                                           */

typedef struct {
  uint64_t key;
  int scale;
  uint32_t ta, tab, tabc; /* cumulative quadrant thresholds in 2^-32 units */
  int permute;
  perm_ctx perm;
  int32_t *src, *dst;
} rmat_ctx;

static void rmat_range(void* p, int64_t lo, int64_t hi) {
  rmat_ctx* c = (rmat_ctx*)p;
  const uint64_t words = (uint64_t)(c->scale + 1) / 2; /* two 32-bit draws per word */
  for (int64_t i = lo; i < hi; ++i) {
    uint32_t u = 0, v = 0;
    uint64_t h = 0;
    for (int k = 0; k < c->scale; ++k) {
      if ((k & 1) == 0) h = draw(c->key, (uint64_t)i * words + (uint64_t)(k >> 1));
      uint32_t r = (k & 1) ? (uint32_t)h : (uint32_t)(h >> 32);
      uint32_t ub, vb;
      if (r < c->ta) { ub = 0; vb = 0; }
      else if (r < c->tab) { ub = 0; vb = 1; }
      else if (r < c->tabc) { ub = 1; vb = 0; }
      else { ub = 1; vb = 1; }
      u = (u << 1) | ub;
      v = (v << 1) | vb;
    }
    if (c->permute) {
      u = perm_apply(&c->perm, u);
      v = perm_apply(&c->perm, v);
    }
    c->src[i] = (int32_t)u;
    c->dst[i] = (int32_t)v;
  }
}

static uint32_t prob_to_u32(double q) {
  if (q <= 0.0) return 0;
  if (q >= 1.0) return UINT32_MAX;
  return (uint32_t)(q * 4294967296.0);
}

int gen_rmat_coo(int scale, int64_t E, double a, double b, double c, uint64_t seed, int permute,
                 int32_t* src, int32_t* dst, int nthreads) {
  if (scale < 0 || scale > 30 || E < 0) return -1;
  if (a < 0 || b < 0 || c < 0 || a + b + c > 1.0) return -1;
  rmat_ctx ctx;
  ctx.key = stream_key(seed, PURPOSE_RMAT);
  ctx.scale = scale;
  ctx.ta = prob_to_u32(a);
  ctx.tab = prob_to_u32(a + b);
  ctx.tabc = prob_to_u32(a + b + c);
  ctx.permute = permute;
  perm_init(&ctx.perm, seed, (uint32_t)1u << scale);
  ctx.src = src;
  ctx.dst = dst;
  parallel_for(E, nthreads, rmat_range, &ctx);
  return 0;
}

/* ------------------------------------------------------------------------- */
/* 2D grid, built directly as a sorted CSR.                                   */
/* Lattice edge IDs: horizontal (r,c)-(r,c+1) -> r*(n-1)+c;                   */
/*                   vertical   (r,c)-(r+1,c) -> n*(n-1) + r*n + c.           */

typedef struct {
  uint64_t key;
  int64_t n;
  uint64_t thresh; /* keep if draw >> 11 < thresh (53-bit fixed point) */
  int64_t* row_ptr;
  int32_t* col;
} grid_ctx;

static inline int grid_keep(const grid_ctx* g, uint64_t edge_id) {
  return (draw(g->key, edge_id) >> 11) < g->thresh;
}

static inline int grid_neighbors(const grid_ctx* g, int64_t v, int32_t out[4]) {
  const int64_t n = g->n, r = v / n, c = v % n;
  const uint64_t hbase = 0, vbase = (uint64_t)(n * (n - 1));
  int k = 0;
  if (r > 0 && grid_keep(g, vbase + (uint64_t)((r - 1) * n + c))) out[k++] = (int32_t)(v - n);
  if (c > 0 && grid_keep(g, hbase + (uint64_t)(r * (n - 1) + c - 1))) out[k++] = (int32_t)(v - 1);
  if (c < n - 1 && grid_keep(g, hbase + (uint64_t)(r * (n - 1) + c))) out[k++] = (int32_t)(v + 1);
  if (r < n - 1 && grid_keep(g, vbase + (uint64_t)(r * n + c))) out[k++] = (int32_t)(v + n);
  return k;
}

static void grid_count_range(void* p, int64_t lo, int64_t hi) {
  grid_ctx* g = (grid_ctx*)p;
  int32_t nb[4];
  for (int64_t v = lo; v < hi; ++v) g->row_ptr[v + 1] = grid_neighbors(g, v, nb);
}

static void grid_fill_range(void* p, int64_t lo, int64_t hi) {
  grid_ctx* g = (grid_ctx*)p;
  int32_t nb[4];
  for (int64_t v = lo; v < hi; ++v) {
    int k = grid_neighbors(g, v, nb);
    int64_t o = g->row_ptr[v];
    for (int j = 0; j < k; ++j) g->col[o + j] = nb[j];
  }
}

static void grid_init(grid_ctx* g, int64_t side, double p, uint64_t seed) {
  g->key = stream_key(seed, PURPOSE_GRID);
  g->n = side;
  if (p >= 1.0) g->thresh = (uint64_t)1 << 53;
  else if (p <= 0.0) g->thresh = 0;
  else g->thresh = (uint64_t)(p * 9007199254740992.0);
}

/* Fills row_ptr[0..side*side] (int64); returns nnz (or -1 on bad args). */
int64_t gen_grid_row_ptr(int64_t side, double p, uint64_t seed, int64_t* row_ptr, int nthreads) {
  if (side < 0 || side * side > INT32_MAX) return -1;
  grid_ctx g;
  grid_init(&g, side, p, seed);
  g.row_ptr = row_ptr;
  g.col = NULL;
  const int64_t V = side * side;
  row_ptr[0] = 0;
  parallel_for(V, nthreads, grid_count_range, &g);
  for (int64_t v = 0; v < V; ++v) row_ptr[v + 1] += row_ptr[v];
  return row_ptr[V];
}

int gen_grid_col(int64_t side, double p, uint64_t seed, const int64_t* row_ptr, int32_t* col, int nthreads) {
  if (side < 0 || side * side > INT32_MAX) return -1;
  grid_ctx g;
  grid_init(&g, side, p, seed);
  g.row_ptr = (int64_t*)row_ptr;
  g.col = col;
  parallel_for(side * side, nthreads, grid_fill_range, &g);
  return 0;
}

/* ------------------------------------------------------------------------- */
/* Symmetrising COO -> CSR: arcs (u,v) and (v,u) per edge, rows sorted.       */

typedef struct {
  int64_t V, E;
  const int32_t *src, *dst;
  int64_t* cnt;   /* degree counters / scatter cursors */
  int32_t* col;
  const int64_t* row_ptr;
  int bad;
} csr_ctx;

static void csr_count_range(void* p, int64_t lo, int64_t hi) {
  csr_ctx* c = (csr_ctx*)p;
  for (int64_t i = lo; i < hi; ++i) {
    int32_t u = c->src[i], v = c->dst[i];
    if (u < 0 || v < 0 || u >= c->V || v >= c->V) {
      __atomic_store_n(&c->bad, 1, __ATOMIC_RELAXED);
      continue;
    }
    __atomic_fetch_add(&c->cnt[u], 1, __ATOMIC_RELAXED);
    __atomic_fetch_add(&c->cnt[v], 1, __ATOMIC_RELAXED);
  }
}

static void csr_scatter_range(void* p, int64_t lo, int64_t hi) {
  csr_ctx* c = (csr_ctx*)p;
  for (int64_t i = lo; i < hi; ++i) {
    int32_t u = c->src[i], v = c->dst[i];
    int64_t pu = __atomic_fetch_add(&c->cnt[u], 1, __ATOMIC_RELAXED);
    c->col[pu] = v;
    int64_t pv = __atomic_fetch_add(&c->cnt[v], 1, __ATOMIC_RELAXED);
    c->col[pv] = u;
  }
}

static int cmp_i32(const void* a, const void* b) {
  int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
  return (x > y) - (x < y);
}

static void insertion_sort_i32(int32_t* a, int64_t n) {
  for (int64_t i = 1; i < n; ++i) {
    int32_t x = a[i];
    int64_t j = i - 1;
    while (j >= 0 && a[j] > x) { a[j + 1] = a[j]; --j; }
    a[j + 1] = x;
  }
}

static void csr_sort_range(void* p, int64_t lo, int64_t hi) {
  csr_ctx* c = (csr_ctx*)p;
  for (int64_t v = lo; v < hi; ++v) {
    int64_t b = c->row_ptr[v], e = c->row_ptr[v + 1];
    if (e - b <= 32) insertion_sort_i32(c->col + b, e - b);
    else qsort(c->col + b, (size_t)(e - b), sizeof(int32_t), cmp_i32);
  }
}

/* Pass 1: row_ptr[0..V] (int64) of the symmetrised CSR. Returns nnz, or -1 if */
/* an endpoint is outside [0, V).                                              */
int64_t gen_sym_csr_row_ptr(int64_t V, int64_t E, const int32_t* src, const int32_t* dst,
                            int64_t* row_ptr, int nthreads) {
  if (V < 0 || E < 0) return -1;
  memset(row_ptr, 0, sizeof(int64_t) * (size_t)(V + 1));
  csr_ctx c;
  memset(&c, 0, sizeof(c));
  c.V = V; c.E = E; c.src = src; c.dst = dst; c.cnt = row_ptr + 1;
  parallel_for(E, nthreads, csr_count_range, &c);
  if (c.bad) return -1;
  for (int64_t v = 0; v < V; ++v) row_ptr[v + 1] += row_ptr[v];
  return row_ptr[V];
}

/* Pass 2: col[0..nnz) given row_ptr from pass 1. `scratch` holds V int64. */
int gen_sym_csr_col(int64_t V, int64_t E, const int32_t* src, const int32_t* dst, const int64_t* row_ptr,
                    int32_t* col, int64_t* scratch, int nthreads) {
  if (V < 0 || E < 0) return -1;
  memcpy(scratch, row_ptr, sizeof(int64_t) * (size_t)V);
  csr_ctx c;
  memset(&c, 0, sizeof(c));
  c.V = V; c.E = E; c.src = src; c.dst = dst; c.cnt = scratch; c.col = col; c.row_ptr = row_ptr;
  parallel_for(E, nthreads, csr_scatter_range, &c);
  parallel_for(V, nthreads, csr_sort_range, &c);
  return 0;
}
