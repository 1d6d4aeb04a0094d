/*
 * Connected-components ORACLE. Test infrastructure, not part of the product.
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg may load
 * or run it; the library never calls it and has no CPU fallback.
 *
 * What it computes is the plain definition of Section II of the paper: two
 * vertices of the undirected graph G = (V, E) share a component iff an edge path
 * joins them, and each vertex receives the index of one representative vertex of
 * its component. The representative is fixed here as the minimum vertex ID of
 * the component:
 *
 *     label[v] = min { w in V : w is reachable from v }.
 *
 * Two independent sequential computations of that definition are provided, and
 * the tests require them to agree:
 *
 *   1. Traversal labelling (the sequential approach named in Section II): scan v
 *      in ascending order; an unlabelled v starts a breadth-first search that
 *      labels every vertex it reaches with v. Since the scan is ascending, v is
 *      the smallest vertex of the component it reaches.
 *
 *   2. Disjoint-set union-find (Galler-Fischer, with path halving per Tarjan and
 *      van Leeuwen 1984). A union links the larger of the two roots below the
 *      smaller one, so every root is the minimum of its set, and the final
 *      label is find(v).
 *
 * Arcs are read as undirected edges: each arc (u, v) joins u and v, whichever
 * direction it was stored in. Self-loops and duplicate edges are allowed.
 * Row offsets are int64 (the Python binding widens int32 offsets).
 *
 * Every function returns the number of components, or -1 if the input is
 * malformed (an endpoint outside [0, V), or offsets that are not a monotone
 * partition of [0, nnz)).
 *
 * No pins are missing: the tests check both functions by brute force on every
 * graph with up to 5 vertices, against closed forms (paths, edgeless graphs,
 * disjoint cliques, stars, full grids), against SciPy's connected_components,
 * and by invariants; textual mutants of this file must fail them.
 */
#include <stdint.h>
#include <stdlib.h>

static int csr_ok(int64_t V, const int64_t* row_ptr, const int32_t* col) {
  if (V < 0) return 0;
  if (row_ptr[0] != 0) return 0;
  for (int64_t v = 0; v < V; ++v)
    if (row_ptr[v + 1] < row_ptr[v]) return 0;
  const int64_t nnz = row_ptr[V];
  for (int64_t a = 0; a < nnz; ++a)
    if (col[a] < 0 || col[a] >= V) return 0;
  return 1;
}

/* ---------------------------------------------------------------- union-find */

/* Root of x's set; every vertex on the path is re-pointed at its grandparent. */
static int32_t uf_find(int32_t* parent, int32_t x) {
  while (parent[x] != x) {
    parent[x] = parent[parent[x]];
    x = parent[x];
  }
  return x;
}

/* Joins the sets of a and b; the larger root is placed below the smaller. */
static void uf_union(int32_t* parent, int32_t a, int32_t b) {
  int32_t ra = uf_find(parent, a);
  int32_t rb = uf_find(parent, b);
  if (ra == rb) return;
  if (ra < rb) parent[rb] = ra;
  else parent[ra] = rb;
}

static int64_t uf_finish(int64_t V, int32_t* label) {
  int64_t comps = 0;
  for (int64_t v = 0; v < V; ++v) {
    label[v] = uf_find(label, (int32_t)v);
    if (label[v] == v) ++comps;
  }
  return comps;
}

int64_t oracle_uf_csr(int64_t V, const int64_t* row_ptr, const int32_t* col, int32_t* label) {
  if (!csr_ok(V, row_ptr, col)) return -1;
  for (int64_t v = 0; v < V; ++v) label[v] = (int32_t)v;
  for (int64_t u = 0; u < V; ++u)
    for (int64_t a = row_ptr[u]; a < row_ptr[u + 1]; ++a)
      uf_union(label, (int32_t)u, col[a]);
  return uf_finish(V, label);
}

int64_t oracle_uf_coo(int64_t V, int64_t E, const int32_t* src, const int32_t* dst, int32_t* label) {
  if (V < 0 || E < 0) return -1;
  for (int64_t i = 0; i < E; ++i)
    if (src[i] < 0 || src[i] >= V || dst[i] < 0 || dst[i] >= V) return -1;
  for (int64_t v = 0; v < V; ++v) label[v] = (int32_t)v;
  for (int64_t i = 0; i < E; ++i) uf_union(label, src[i], dst[i]);
  return uf_finish(V, label);
}

/* ----------------------------------------------------- breadth-first search */

/* Undirected adjacency of an arc list: every arc (u, v) is listed at u and at v. */
typedef struct {
  int64_t* start; /* V + 1 */
  int32_t* nbr;   /* 2 * n_arcs */
} adjacency;

static int adj_build(adjacency* g, int64_t V, int64_t n_arcs, const int32_t* tail, const int64_t* row_ptr,
                     const int32_t* head) {
  /* tail[i] (or the CSR row of arc i when tail is NULL) and head[i] are the two endpoints of arc i. */
  g->start = (int64_t*)calloc((size_t)V + 1, sizeof(int64_t));
  g->nbr = (int32_t*)malloc(sizeof(int32_t) * (size_t)(2 * n_arcs + 1));
  if (!g->start || !g->nbr) return 0;
  int64_t u = 0;
  for (int64_t i = 0; i < n_arcs; ++i) {
    if (tail) u = tail[i];
    else while (row_ptr[u + 1] <= i) ++u;
    g->start[u + 1]++;
    g->start[head[i] + 1]++;
  }
  for (int64_t v = 0; v < V; ++v) g->start[v + 1] += g->start[v];
  int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)(V + 1));
  if (!fill) return 0;
  for (int64_t v = 0; v <= V; ++v) fill[v] = g->start[v];
  u = 0;
  for (int64_t i = 0; i < n_arcs; ++i) {
    if (tail) u = tail[i];
    else while (row_ptr[u + 1] <= i) ++u;
    g->nbr[fill[u]++] = head[i];
    g->nbr[fill[head[i]]++] = (int32_t)u;
  }
  free(fill);
  return 1;
}

static void adj_free(adjacency* g) {
  free(g->start);
  free(g->nbr);
}

static int64_t bfs_label(int64_t V, const adjacency* g, int32_t* label) {
  int32_t* queue = (int32_t*)malloc(sizeof(int32_t) * (size_t)(V + 1));
  if (!queue) return -1;
  for (int64_t v = 0; v < V; ++v) label[v] = -1;
  int64_t comps = 0;
  for (int64_t s = 0; s < V; ++s) {
    if (label[s] != -1) continue;
    ++comps;
    int64_t head = 0, tail = 0;
    label[s] = (int32_t)s;
    queue[tail++] = (int32_t)s;
    while (head < tail) {
      int32_t x = queue[head++];
      for (int64_t k = g->start[x]; k < g->start[x + 1]; ++k) {
        int32_t y = g->nbr[k];
        if (label[y] == -1) {
          label[y] = (int32_t)s;
          queue[tail++] = y;
        }
      }
    }
  }
  free(queue);
  return comps;
}

int64_t oracle_bfs_csr(int64_t V, const int64_t* row_ptr, const int32_t* col, int32_t* label) {
  if (!csr_ok(V, row_ptr, col)) return -1;
  adjacency g;
  if (!adj_build(&g, V, row_ptr[V], NULL, row_ptr, col)) { adj_free(&g); return -1; }
  int64_t c = bfs_label(V, &g, label);
  adj_free(&g);
  return c;
}

int64_t oracle_bfs_coo(int64_t V, int64_t E, const int32_t* src, const int32_t* dst, int32_t* label) {
  if (V < 0 || E < 0) return -1;
  for (int64_t i = 0; i < E; ++i)
    if (src[i] < 0 || src[i] >= V || dst[i] < 0 || dst[i] >= V) return -1;
  adjacency g;
  if (!adj_build(&g, V, E, src, NULL, dst)) { adj_free(&g); return -1; }
  int64_t c = bfs_label(V, &g, label);
  adj_free(&g);
  return c;
}

/* Label of one vertex by a search from it: the minimum vertex reached. Used to  */
/* check single sampled outputs of very large graphs. The CSR must be symmetric  */
/* (the reverse of every arc is present), since only out-arcs are followed.      */
/* `seen` and `queue` are caller-provided int32[V] work arrays; `seen` must be   */
/* all -1 on entry and is reset to -1 on return. Returns the label, or -1 on     */
/* malformed input.                                                              */
int64_t oracle_label_of(int64_t V, const int64_t* row_ptr, const int32_t* col, int64_t v, int32_t* seen,
                        int32_t* queue) {
  if (v < 0 || v >= V) return -1;
  int64_t head = 0, tail = 0, best = v;
  seen[v] = 1;
  queue[tail++] = (int32_t)v;
  while (head < tail) {
    int32_t x = queue[head++];
    if (x < best) best = x;
    for (int64_t a = row_ptr[x]; a < row_ptr[x + 1]; ++a) {
      int32_t y = col[a];
      if (y < 0 || y >= V) { best = -1; goto done; }
      if (seen[y] == -1) {
        seen[y] = 1;
        queue[tail++] = y;
      }
    }
  }
done:
  for (int64_t i = 0; i < tail; ++i) seen[queue[i]] = -1;
  return best;
}
