// Batched connected components: thousands of graphs of uneven size in one persistent launch.
//
// The batch is the disjoint union of its graphs over a graph-offset table: graph g owns the
// vertex range [v_off[g], v_off[g+1]) of the concatenated label array and the arc range
// [a_off[g], a_off[g+1]) of the concatenated col_idx; its row offsets (graph-local, V_g + 1 of
// them) start at row_ptr_cat + v_off[g] + g. Each graph is cut into windows of W vertices; a
// window is the unit of work of phase A.
//
//  - A graph of one window (V_g <= W) is labelled completely inside one CTA: every arc is hooked
//    on the shared-memory parent array and the compressed labels (graph-local minimum IDs) are
//    written once. No global atomics and no second pass.
//  - A larger graph is labelled on the concatenated array with global IDs (v_off[g] + local):
//    a window whose sampled arcs mostly stay inside it runs phase A of the two-phase hook (local
//    hooks, stars written, other arcs to the worklist); a window without that locality only
//    writes pi(x) = x and is hooked arc by arc in phase B. Phase B hooks the worklist and those
//    windows on pi in s' = 2|E'|/|V| segments, each followed by a Multi-Jump over the vertices of
//    the multi-window graphs; a last pass turns their global IDs into graph-local ones.
//
// Every write to pi is a CAS on a root towards a smaller vertex of the same graph (IDs of
// different graphs never meet: an arc only joins vertices of its own graph), so the argument of
// the single-graph kernels gives, per graph, the graph-local minimum vertex ID of each component.
#include "cc_internal.h"

namespace cc {

namespace {

constexpr int kMaxBlockB = 1024;
// Windows hooked arc by arc are cut into chunks, which warps take from a counter: a fixed split
// leaves the grid waiting on the slowest piece of a skewed graph when a batch has few such
// windows. A chunk is 2048 arcs, or less when the batch has fewer than four such chunks per warp
// (down to 128 arcs), so that small batches still spread over every warp.
constexpr int kPlainChunkArcs = 2048;
constexpr int kMinPlainChunkArcs = 128;

struct Batch {
  int n_graphs;
  const GraphDesc* desc;   // descriptor mode (nullptr: offset tables v_off / a_off)
  const long long* v_off;
  const long long* a_off;
  const int* rp_cat;
  const int* col_cat;
  int* labels;
  int* graph_status;       // nullable: per-graph error code
  long long* unit_start;   // [n_graphs + 1] first window of each graph (filled by the kernel)
  int* plain_units;        // windows hooked arc by arc in phase B
  int plain_cap;
  long long* plain_chunk_start;  // [plain_cap + 2] first chunk of each such window, then the chunk
                                 // size (filled by the kernel)
  int* graph_hint;               // [n_graphs] giant-star root of each graph (filled by the kernel)
  int total_v;             // label arena size (batch-global IDs are below it)
  int grid_a;              // CTAs of the first launch, whose count decided which graphs one CTA labels
  long long row_elems;     // descriptor mode: row-offset arena size
  long long arc_elems;     // descriptor mode: arc arena size
};

__device__ __forceinline__ long long units_of(long long vg, int W) { return vg <= 0 ? 0 : (vg + W - 1) / W; }

// Vertices of graph g; a descriptor that does not fit its arenas is reported (per graph and
// in the status word) and its graph gets no windows, so nothing reads or writes through it.
__device__ __forceinline__ long long graph_vertices(const Batch& b, int g, const Ctl& c) {
  if (!b.desc) return b.v_off[g + 1] - b.v_off[g];
  const GraphDesc d = b.desc[g];
  const bool ok = d.n_vertices >= 0 && d.n_arcs >= 0 && d.n_arcs <= 0x7fffffffLL && d.label_off >= 0 &&
                  d.label_off + d.n_vertices <= (long long)b.total_v && d.row_off >= 0 &&
                  d.row_off + d.n_vertices + 1 <= b.row_elems && d.arc_off >= 0 && d.arc_off + d.n_arcs <= b.arc_elems;
  if (!ok) {
    raise_input_error(c, kSiteValidate, (long long)g);
    if (b.graph_status) b.graph_status[g] = kErrOutOfRange;
    return 0;
  }
  return d.n_vertices;
}

// Block-wide inclusive scan of one value per thread (blockDim.x a multiple of 32).
__device__ __forceinline__ long long block_scan(long long x, long long* warp_sums, long long* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const long long y = __shfl_up_sync(kFull, x, d);
    if (lane >= d) x += y;
  }
  if (lane == 31) warp_sums[warp] = x;
  __syncthreads();
  if (warp == 0) {
    long long w = lane < nwarps ? warp_sums[lane] : 0;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const long long y = __shfl_up_sync(kFull, w, d);
      if (lane >= d) w += y;
    }
    if (lane < nwarps) warp_sums[lane] = w;
    if (lane == nwarps - 1) *total = w;
  }
  __syncthreads();
  const long long r = x + (warp > 0 ? warp_sums[warp - 1] : 0);
  __syncthreads();
  return r;
}

// How many CTAs share one window when there are too few windows to keep the grid busy.
__device__ __forceinline__ unsigned long long split_factor(unsigned long long items, unsigned grid) {
  if (items == 0) return 1;
  unsigned long long f = (2ull * grid + items - 1) / items;
  return f < 1 ? 1 : (f > 64 ? 64 : f);
}

// Graph owning window u: largest g with unit_start[g] <= u (graphs without vertices own none).
__device__ __forceinline__ int graph_of_unit(const long long* unit_start, int n, long long u) {
  int lo = 0, hi = n;  // unit_start[lo] <= u < unit_start[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (unit_start[mid] <= u) lo = mid;
    else hi = mid;
  }
  return lo;
}

struct UnitInfo {
  int g, w0, nrows, vbase, vg;
  bool single;
  long long nnz;
  const int* rp;
  const int* col;
};

__device__ __forceinline__ UnitInfo unit_info(const Batch& b, long long u, int W) {
  UnitInfo ui;
  ui.g = graph_of_unit(b.unit_start, b.n_graphs, u);
  long long vo, ro, ao;
  if (b.desc) {
    const GraphDesc d = b.desc[ui.g];
    vo = d.label_off;
    ro = d.row_off;
    ao = d.arc_off;
    ui.vg = d.n_vertices;
    ui.nnz = d.n_arcs;
  } else {
    vo = b.v_off[ui.g];
    ro = vo + ui.g;
    ao = b.a_off[ui.g];
    ui.vg = (int)(b.v_off[ui.g + 1] - vo);
    ui.nnz = b.a_off[ui.g + 1] - ao;
  }
  ui.vbase = (int)vo;
  const long long k = u - b.unit_start[ui.g];
  ui.single = (b.unit_start[ui.g + 1] - b.unit_start[ui.g]) == 1;
  ui.w0 = (int)(k * W);
  ui.nrows = (ui.vg - ui.w0) < W ? (ui.vg - ui.w0) : W;
  ui.rp = b.rp_cat + ro;
  ui.col = b.col_cat + ao;
  return ui;
}

// Graphs of one window are labelled by one CTA in shared memory, unless the batch has fewer
// windows than CTAs and the graph has more than kOneCtaArcs arcs: the other CTAs would then idle
// while one walks all its arcs, so such a graph is hooked arc by arc on pi in phase B instead
// (with batch-global IDs, like a window without locality).
constexpr long long kOneCtaArcs = 8192;
__device__ __forceinline__ bool one_cta(const UnitInfo& ui, long long n_units, int ctas) {
  return ui.single && (n_units >= (long long)ctas || ui.nnz <= kOneCtaArcs);
}

// Locality test of a multi-window graph by warp 0: the middle arc of 32 rows spread over the whole
// graph (the same rows whichever window asks, so every window of a graph decides alike: a graph
// whose windows disagreed would be neither filtered nor fully hooked in shared memory); true when
// the fraction f of sampled arcs that stay in their row's window is at least halfway from what
// random endpoints would give (W / V_g) to 1: f >= (1 + W / V_g) / 2. For large graphs that is one
// half; a graph of two windows needs three quarters, since random arcs already stay in a window
// half the time there.
__device__ __forceinline__ bool graph_is_local(const UnitInfo& ui, int W) {
  const int lane = threadIdx.x & 31;
  const int r = (int)(((long long)lane * ui.vg) / 32);
  bool sampled = false, local = false;
  const int a0 = ui.rp[r], a1 = ui.rp[r + 1];
  if (a0 >= 0 && a0 < a1 && (long long)a1 <= ui.nnz) {
    const int v = ui.col[a0 + (a1 - a0) / 2];
    if ((unsigned)v < (unsigned)ui.vg && v != r) {
      sampled = true;
      local = v / W == r / W;
    }
  }
  const int ns = __popc(__ballot_sync(kFull, sampled));
  const int nl = __popc(__ballot_sync(kFull, local));
  const long long w = (long long)W < (long long)ui.vg ? (long long)W : (long long)ui.vg;
  return 2ll * nl * ui.vg >= (long long)ns * ((long long)ui.vg + w);
}

// ----- the sampled-and-filtered hook of the windows without locality (symmetric batches) -----
// Slice 1 hooks the first kSampleArcs arcs of every row of those windows; a Multi-Jump over their
// vertices follows; then one warp per graph takes the most frequent root of 32 vertices spread
// over the graph as its giant-star hint (or -1); slice 2 reads only the rows whose vertex's parent
// is not the hint and hooks their remaining arcs in both directions. The single-graph argument
// holds per graph (arcs never leave their graph, and one hint serves all of a graph's rows): the
// reverse of a skipped arc is in a row that is read, unless both ends already share the star.
// Only graphs all of whose windows are hooked this way are filtered (see kMixedGraph).

// graph_hint value of a graph with a window hooked in phase A (never a vertex ID).
constexpr int kMixedGraph = -2;

// Rows [i0, i1) of window ui: the first kSampleArcs arcs of each. A thread takes kHeadRows rows
// (i, i + blockDim.x, ...) per step and hooks their arcs together, so the loads and root walks
// of several rows are in flight at once: with one CTA per SM (the window's shared memory) a
// thread has many rows to go through, and one row at a time left the phase bound on the
// latency of each row's chain of dependent loads.
constexpr int kHeadRows = 2;
__device__ __forceinline__ void batched_row_heads(const Batch& b, const UnitInfo& ui, int i0, int i1, const Ctl& c) {
  constexpr int K = kHeadRows * kSampleArcs;
  for (int i = i0 + threadIdx.x; i < i1; i += kHeadRows * blockDim.x) {
    int uu[K], vv[K];
    bool live[K];
#pragma unroll
    for (int r = 0; r < kHeadRows; ++r) {
      const int ir = i + r * (int)blockDim.x;
      const int u = ui.w0 + ir;
      int a0 = 0, a1 = 0;
      if (ir < i1) {
        a0 = ui.rp[u];
        a1 = ui.rp[u + 1];
        if (!(a0 >= 0 && a0 <= a1 && (long long)a1 <= ui.nnz)) {
          raise_input_error(c, kSiteHookArc, (long long)ui.g);
          if (b.graph_status) b.graph_status[ui.g] = kErrOutOfRange;
          a1 = a0;
        }
      }
#pragma unroll
      for (int j = 0; j < kSampleArcs; ++j) {
        const int k = r * kSampleArcs + j;
        const bool has = (long long)a0 + j < (long long)a1;
        const int v = has ? ld_stream(ui.col + a0 + j) : 0;
        const bool in_range = (unsigned)v < (unsigned)ui.vg;
        if (has && !in_range) {
          raise_input_error(c, kSiteHookArc, (long long)ui.g);
          if (b.graph_status) b.graph_status[ui.g] = kErrOutOfRange;
        }
        live[k] = has && in_range && v != u;
        uu[k] = ui.vbase + u;
        vv[k] = ui.vbase + v;
      }
    }
    atomic_hook_k<K>(b.labels, uu, vv, live, b.total_v, c);
  }
}

// Multi-Jump (Fig. 3, bottom) of the vertices base + [i0, i1) of one window: a thread takes
// kJumpVerts vertices (i, i + blockDim.x, ...) per step, whose parents and grandparents are
// loaded together before each walk goes on alone, writing every step.
constexpr int kJumpVerts = 4;
__device__ __forceinline__ void batched_jump(int* labels, int base, int i0, int i1, int total_v, const Ctl& c) {
  for (int i = i0 + threadIdx.x; i < i1; i += kJumpVerts * blockDim.x) {
    int x[kJumpVerts], p[kJumpVerts], g[kJumpVerts];
#pragma unroll
    for (int j = 0; j < kJumpVerts; ++j) {
      const int ij = i + j * (int)blockDim.x;
      x[j] = base + ij;
      p[j] = ij < i1 ? ld_pi(labels + x[j]) : x[j];
    }
#pragma unroll
    for (int j = 0; j < kJumpVerts; ++j) g[j] = p[j] != x[j] ? ld_pi(labels + p[j]) : p[j];
#pragma unroll
    for (int j = 0; j < kJumpVerts; ++j)
      if (g[j] != p[j]) jump_from(labels, x[j], p[j], g[j], total_v, c);
  }
}

// Rows [i0, i1) of window ui whose vertex's parent is not `hint`: their arcs from position
// kSampleArcs on, both directions; one row per lane, rows of more than 32 such arcs by the warp.
__device__ __forceinline__ void batched_rows_outside(const Batch& b, const UnitInfo& ui, int i0, int i1, int hint,
                                                     const Ctl& c) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  for (int base = i0 + warp * 32; base < i1; base += nwarps * 32) {  // warp-uniform
    const int i = base + lane;
    const int u = ui.w0 + i;
    int a0 = 0, a1 = 0;
    if (i < i1 && ld_pi(b.labels + ui.vbase + u) != hint) {
      a0 = ui.rp[u];
      a1 = ui.rp[u + 1];
      if (!(a0 >= 0 && a0 <= a1 && (long long)a1 <= ui.nnz)) a1 = a0;  // reported by slice 1
      a0 = a1 - a0 > kSampleArcs ? a0 + kSampleArcs : a1;
    }
    const bool heavy = a1 - a0 > 32;
    if (!heavy) {
      for (int a = a0; a < a1; ++a) {
        const int v = ld_stream(ui.col + a);
        if ((unsigned)v >= (unsigned)ui.vg) {
          raise_input_error(c, kSiteHookArc, (long long)ui.g);
          if (b.graph_status) b.graph_status[ui.g] = kErrOutOfRange;
          continue;
        }
        if (v != u) atomic_hook(b.labels, ui.vbase + u, ui.vbase + v, b.total_v, c);
      }
    }
    unsigned hv = __ballot_sync(kFull, heavy);
    while (hv) {
      const int h = __ffs(hv) - 1;
      hv &= hv - 1;
      const int hu = __shfl_sync(kFull, u, h);
      const int h0 = __shfl_sync(kFull, a0, h), h1 = __shfl_sync(kFull, a1, h);
      for (long long bb = h0; bb < h1; bb += 32) {
        const long long a = bb + lane;
        const bool has = a < h1;
        const int v = has ? ld_stream(ui.col + a) : 0;
        const bool in_range = (unsigned)v < (unsigned)ui.vg;
        if (has && !in_range) {
          raise_input_error(c, kSiteHookArc, (long long)ui.g);
          if (b.graph_status) b.graph_status[ui.g] = kErrOutOfRange;
        }
        const int uu[1] = {ui.vbase + hu}, vv[1] = {ui.vbase + v};
        const bool live[1] = {has && in_range && v != hu};
        atomic_hook_k<1>(b.labels, uu, vv, live, b.total_v, c);
      }
    }
  }
}

// First launch (one CTA per SM: the window's parent array in shared memory): the unit table, then
// phase A over every window.
template <bool SYM>
__device__ __forceinline__ void batched_front(const Batch& b, int* smem, const Ctl& c) {
  __shared__ long long s_warp_sums[32];
  __shared__ long long s_total;
  __shared__ unsigned long long s_unit;
  __shared__ int s_ovf, s_bad, s_plain;
  if (launch_blocked(c)) return;
  unsigned epoch = 0;
  const int W = c.tile_w;

  // Windows per graph -> unit_start (block 0).
  if (blockIdx.x == 0) {
    long long carry = 0;
    if (threadIdx.x == 0) b.unit_start[0] = 0;
    for (int base = 0; base < b.n_graphs; base += blockDim.x) {
      const int g = base + threadIdx.x;
      const long long n = g < b.n_graphs ? units_of(graph_vertices(b, g, c), W) : 0;
      const long long incl = block_scan(n, s_warp_sums, &s_total);
      if (g < b.n_graphs) {
        b.unit_start[g + 1] = carry + incl;
        b.graph_hint[g] = 0;  // set to kMixedGraph by phase A below
      }
      carry += s_total;
    }
  }
  if (!grid_sync(c, epoch)) return;
  const long long n_units = *reinterpret_cast<volatile long long*>(b.unit_start + b.n_graphs);

  // Phase A over all windows of all graphs.
  int* lp = smem;
  WarpSink sink;
  warp_scratch_init(sink, reinterpret_cast<unsigned char*>(smem + W));
  for (;;) {
    if (threadIdx.x == 0) {
      s_unit = atomicAdd(&c.st->counters[0], 1ull);
      s_ovf = 0;
      s_bad = 0;
    }
    __syncthreads();
    const unsigned long long k = s_unit;
    if (k >= (unsigned long long)n_units) break;
    const UnitInfo ui = unit_info(b, (long long)k, W);
    for (int i = threadIdx.x; i < ui.nrows; i += blockDim.x) lp[i] = i;
    if (threadIdx.x < 32) {  // warp 0 decides how the window is hooked
      // With fewer windows than CTAs, phase A would leave most of the GPU idle while a few
      // CTAs walk whole windows: every window (but those of graphs small enough for one CTA)
      // is then hooked arc by arc in phase B, spread over all warps.
      bool local = true;
      if (!ui.single)
        local = (c.window_mode == kWindowsPlain || n_units < (long long)gridDim.x) ? false : graph_is_local(ui, W);
      else if (!one_cta(ui, n_units, (int)gridDim.x))
        local = false;
      if (ui.nnz > 0x7fffffffLL) {  // graph too large for int32 row offsets: reported, not hooked
        local = true;
        if (threadIdx.x == 0) {
          raise_input_error(c, kSiteHookArc, (long long)ui.g);
          s_bad = 1;
        }
      }
      if (threadIdx.x == 0) s_plain = !local;
    }
    __syncthreads();
    if (s_plain) {
      for (int i = threadIdx.x; i < ui.nrows; i += blockDim.x) b.labels[ui.vbase + ui.w0 + i] = ui.vbase + ui.w0 + i;
      if (threadIdx.x == 0) {
        const unsigned long long j = atomicAdd(&c.st->counters[3], 1ull);
        if (j < (unsigned long long)b.plain_cap) b.plain_units[j] = (int)k;
        else raise_error(c.st, kErrInternal, kSiteHookGuard, (long long)k);  // capacity is the window count
      }
    } else {
      // A graph with a window hooked in phase A is not filtered: phase A drops the arcs with
      // v < u of a symmetric CSR, leaving them to the reverse arcs, which the filter may skip.
      if (threadIdx.x == 0 && !one_cta(ui, n_units, (int)gridDim.x)) b.graph_hint[ui.g] = kMixedGraph;
      if (ui.nnz <= 0x7fffffffLL)
        phase_a_window<int, SYM, int>(ui.rp, ui.col, ui.vg, (int)ui.nnz, ui.w0, ui.nrows, ui.vbase, lp, sink, &s_ovf,
                                 &s_bad, c);
      else
        __syncthreads();
      volatile int* vlp = lp;
      if (one_cta(ui, n_units, (int)gridDim.x)) {
        for (int i = threadIdx.x; i < ui.nrows; i += blockDim.x) b.labels[ui.vbase + i] = lfind(vlp, i);
      } else {
        const int base = ui.vbase + ui.w0;
        for (int i = threadIdx.x; i < ui.nrows; i += blockDim.x) b.labels[base + i] = base + lfind(vlp, i);
      }
      if (threadIdx.x == 0 && s_ovf) {  // worklist full: hook this window arc by arc in phase B
        const unsigned long long j = atomicAdd(&c.st->counters[3], 1ull);
        if (j < (unsigned long long)b.plain_cap) b.plain_units[j] = (int)k;
      }
    }
    if (threadIdx.x == 0 && s_bad && b.graph_status) b.graph_status[ui.g] = kErrOutOfRange;
    __syncthreads();
  }
}

// Second launch (no shared-memory window, so two 1024-thread CTAs per SM: twice the threads of the
// first launch for phases bound by chains of dependent loads): the sampled-and-filtered hook of the
// windows without locality, phase B, the Multi-Jumps and the relabelling. The first launch's
// decisions reach it through global memory (unit table, worklist and window counters, labels).
template <bool SYM>
__device__ __forceinline__ void batched_back(const Batch& b, const Ctl& c) {
  __shared__ long long s_warp_sums[32];
  __shared__ long long s_total;
  __shared__ int s_warp_bad[kMaxBlockB / 32];
  if (launch_blocked(c)) return;
  unsigned epoch = 0;
  const int W = c.tile_w;
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nt = (long long)gridDim.x * blockDim.x;
  const long long n_units = *reinterpret_cast<const volatile long long*>(b.unit_start + b.n_graphs);

  const unsigned long long cur = *reinterpret_cast<volatile unsigned long long*>(&c.st->counters[2]);
  const unsigned long long n_pairs = cur < c.wl_cap ? cur : c.wl_cap;
  unsigned long long n_plain = *reinterpret_cast<volatile unsigned long long*>(&c.st->counters[3]);
  n_plain = n_plain < (unsigned long long)b.plain_cap ? n_plain : (unsigned long long)b.plain_cap;
  long long s2 = c.segments_b > 0 ? c.segments_b : (long long)((2.0 * (double)n_pairs) / (double)b.total_v + 0.5);
  s2 = s2 < 1 ? 1 : (s2 > 4096 ? 4096 : s2);
  if (n_pairs == 0 && n_plain == 0) s2 = 0;  // every tree is already a star: only the relabelling is left
  if (tid == 0) {
    c.st->report[0] = n_pairs;
    c.st->report[1] = (unsigned long long)s2;
  }
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const unsigned long long pparts = split_factor(n_plain, gridDim.x);
  if (SYM && n_plain > 0) {
    // Sampled-and-filtered hook of the windows without locality: slice 1, then a Multi-Jump
    // over their vertices, then the per-graph hints (slice 2 runs with the worklist below).
    for (unsigned long long item = blockIdx.x; item < n_plain * pparts; item += gridDim.x) {
      const UnitInfo ui = unit_info(b, b.plain_units[item / pparts], W);
      const long long part = (long long)(item % pparts);
      batched_row_heads(b, ui, split_point<int>(ui.nrows, (long long)pparts, part),
                        split_point<int>(ui.nrows, (long long)pparts, part + 1), c);
    }
    if (!grid_sync(c, epoch)) return;
    for (unsigned long long item = blockIdx.x; item < n_plain * pparts; item += gridDim.x) {
      const UnitInfo ui = unit_info(b, b.plain_units[item / pparts], W);
      const long long part = (long long)(item % pparts);
      batched_jump(b.labels, ui.vbase + ui.w0, split_point<int>(ui.nrows, (long long)pparts, part),
                   split_point<int>(ui.nrows, (long long)pparts, part + 1), b.total_v, c);
    }
    if (!grid_sync(c, epoch)) return;
    for (long long gw = tid >> 5; gw < b.n_graphs; gw += nt >> 5) {  // one warp per graph
      const int gi = (int)gw;
      const long long u0 = b.unit_start[gi], u1 = b.unit_start[gi + 1];
      int hint = -1;
      const int mark = b.graph_hint[gi];
      if (mark == kMixedGraph) {
        hint = kMixedGraph;  // matches no vertex: every row is read
      } else if (u1 > u0) {
        const UnitInfo ui = unit_info(b, u0, W);
        if (!one_cta(ui, n_units, b.grid_a)) {
          const int x = ui.vbase + (int)(((long long)lane * ui.vg) / 32);
          const int val = ld_pi(b.labels + x);
          const unsigned grp = __match_any_sync(kFull, val);
          const int best = __reduce_max_sync(kFull, (unsigned)((__popc(grp) << 5) | lane));
          const int val_best = __shfl_sync(kFull, val, best & 31);
          if ((best >> 5) >= 4) hint = val_best;  // at least an eighth of the 32 samples
        }
      }
      if (lane == 0) b.graph_hint[gi] = hint;
    }
    if (!grid_sync(c, epoch)) return;
  }
  // Chunk table of the windows hooked arc by arc (block 0; batches without CC_FLAG_SYMMETRIC):
  // window j owns chunks [chunk_start[j], chunk_start[j + 1]) of chunk_start[n_plain + 1] arcs
  // each; a window whose row offsets are inconsistent gets one chunk, which reports it.
  if (!SYM && n_plain > 0) {
    if (blockIdx.x == 0) {
      long long arcs = 0;
      for (unsigned long long j = threadIdx.x; j < n_plain; j += blockDim.x) {
        const UnitInfo ui = unit_info(b, b.plain_units[j], W);
        const int a0 = ui.rp[ui.w0], a1 = ui.rp[ui.w0 + ui.nrows];
        if (a0 >= 0 && a0 <= a1 && (long long)a1 <= ui.nnz) arcs += a1 - a0;
      }
      block_scan(arcs, s_warp_sums, &s_total);
      const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
      long long chunk = s_total / (4 * warps);
      chunk = chunk < kMinPlainChunkArcs ? kMinPlainChunkArcs : (chunk > kPlainChunkArcs ? kPlainChunkArcs : chunk);
      chunk = (chunk + 31) & ~31ll;
      long long carry = 0;
      if (threadIdx.x == 0) {
        b.plain_chunk_start[0] = 0;
        b.plain_chunk_start[n_plain + 1] = chunk;
      }
      for (unsigned long long base = 0; base < n_plain; base += blockDim.x) {
        const unsigned long long j = base + threadIdx.x;
        long long n = 0;
        if (j < n_plain) {
          const UnitInfo ui = unit_info(b, b.plain_units[j], W);
          const int a0 = ui.rp[ui.w0], a1 = ui.rp[ui.w0 + ui.nrows];
          n = (a0 >= 0 && a0 <= a1 && (long long)a1 <= ui.nnz) ? ((long long)(a1 - a0) + chunk - 1) / chunk : 1;
        }
        const long long incl = block_scan(n, s_warp_sums, &s_total);
        if (j < n_plain) b.plain_chunk_start[j + 1] = carry + incl;
        carry += s_total;
      }
    }
    if (!grid_sync(c, epoch)) return;
  }
  for (long long seg = 0; seg < s2; ++seg) {
    const unsigned long long p0 = split_point<unsigned long long>(n_pairs, s2, seg);
    const unsigned long long p1 = split_point<unsigned long long>(n_pairs, s2, seg + 1);
    hook_worklist(b.labels, c.wl, p0, p1, tid, nt, b.total_v, c);
    if (SYM && seg == 0 && n_plain > 0) {  // slice 2 of the windows without locality
      for (unsigned long long item = blockIdx.x; item < n_plain * pparts; item += gridDim.x) {
        const UnitInfo ui = unit_info(b, b.plain_units[item / pparts], W);
        const long long part = (long long)(item % pparts);
        batched_rows_outside(b, ui, split_point<int>(ui.nrows, (long long)pparts, part),
                             split_point<int>(ui.nrows, (long long)pparts, part + 1), b.graph_hint[ui.g], c);
      }
    }
    if (!SYM && seg == 0 && n_plain > 0) {  // windows without locality: every arc on pi, in chunks from a counter
      const long long n_chunks = *reinterpret_cast<volatile long long*>(b.plain_chunk_start + n_plain);
      const long long chunk = *reinterpret_cast<volatile long long*>(b.plain_chunk_start + n_plain + 1);
      if (lane == 0) s_warp_bad[warp] = 0;
      __syncwarp();
      for (;;) {
        long long t = 0;
        if (lane == 0) t = (long long)atomicAdd(&c.st->counters[1], 1ull);
        t = __shfl_sync(kFull, t, 0);
        if (t >= n_chunks) break;
        const int j = graph_of_unit(b.plain_chunk_start, (int)n_plain, t);
        const UnitInfo ui = unit_info(b, b.plain_units[j], W);
        const int a0 = ui.rp[ui.w0], a1 = ui.rp[ui.w0 + ui.nrows];
        if (a0 >= 0 && a0 <= a1 && (long long)a1 <= ui.nnz) {
          const long long k = t - b.plain_chunk_start[j];
          const int t0 = (int)((long long)a0 + k * chunk);
          const int t1 = (long long)t0 + chunk < (long long)a1 ? (int)((long long)t0 + chunk) : a1;
          if (t0 < t1)
            hook_csr_range<int, SYM, kHookK>(ui.rp, ui.col, b.labels, ui.vg, t0, t1, c, ui.w0, ui.vbase,
                                             s_warp_bad + warp);
        } else if (lane == 0) {
          raise_input_error(c, kSiteHookArc, (long long)ui.g);
          s_warp_bad[warp] = 1;
        }
        __syncwarp();
        if (lane == 0 && s_warp_bad[warp]) {
          if (b.graph_status) b.graph_status[ui.g] = kErrOutOfRange;
          s_warp_bad[warp] = 0;
        }
        __syncwarp();
      }
    }
    if (!grid_sync(c, epoch)) return;
    // Multi-Jump over the vertices of multi-window graphs (global IDs), windows split over CTAs.
    const unsigned long long vparts = split_factor((unsigned long long)n_units, gridDim.x);
    for (unsigned long long item = blockIdx.x; item < (unsigned long long)n_units * vparts; item += gridDim.x) {
      const UnitInfo ui = unit_info(b, (long long)(item / vparts), W);
      if (one_cta(ui, n_units, b.grid_a)) continue;
      const long long part = (long long)(item % vparts);
      batched_jump(b.labels, ui.vbase + ui.w0, split_point<int>(ui.nrows, (long long)vparts, part),
                   split_point<int>(ui.nrows, (long long)vparts, part + 1), b.total_v, c);
    }
    if (!grid_sync(c, epoch)) return;
  }
  // Global IDs of multi-window graphs -> graph-local labels.
  const unsigned long long cparts = split_factor((unsigned long long)n_units, gridDim.x);
  for (unsigned long long item = blockIdx.x; item < (unsigned long long)n_units * cparts; item += gridDim.x) {
    const UnitInfo ui = unit_info(b, (long long)(item / cparts), W);
    if (one_cta(ui, n_units, b.grid_a)) continue;
    const long long part = (long long)(item % cparts);
    const int base = ui.vbase + ui.w0;
    const int i0 = split_point<int>(ui.nrows, (long long)cparts, part);
    const int i1 = split_point<int>(ui.nrows, (long long)cparts, part + 1);
    // four labels per thread and step, all loaded before any is stored
    for (int i = i0 + threadIdx.x; i < i1; i += 4 * blockDim.x) {
      int l[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) l[j] = i + j * (int)blockDim.x < i1 ? b.labels[base + i + j * (int)blockDim.x] : 0;
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (i + j * (int)blockDim.x < i1) b.labels[base + i + j * (int)blockDim.x] = l[j] - ui.vbase;
    }
  }
}

// Phase timestamps (CC_FLAG_PHASE_TIMES): slot 0 the start, slot 1 the first launch's barrier, slot 2 the
// end of phase A (the first launch's last block), then the second launch's barriers from slot 3.
constexpr int kBatchedPhaseAEndSlot = 2;

template <bool SYM>
__global__ void __launch_bounds__(kMaxBlockB, 1) k_batched(Batch b, Ctl c) {
  extern __shared__ int dyn_smem[];
  if (c.phase_ns && blockIdx.x == 0 && threadIdx.x == 0) c.phase_ns[0] = now_ns();
  batched_front<SYM>(b, dyn_smem, c);
  if (c.phase_ns && threadIdx.x == 0) atomicMax(c.phase_ns + kBatchedPhaseAEndSlot, now_ns());
}

template <bool SYM>
__global__ void __launch_bounds__(kMaxBlockB, 2) k_batched_b(Batch b, Ctl c) {
  batched_back<SYM>(b, c);
  if (c.phase_ns && threadIdx.x == 0) atomicMax(c.phase_ns + (c.phase_cap - 1), now_ns());
}

template <typename K>
cudaError_t launch_cooperative(K k, LaunchShape s, size_t smem, cudaStream_t stream, const Batch& b, const Ctl& c) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)s.grid);
  cfg.blockDim = dim3((unsigned)s.block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k, b, c);
}

template <typename F>
auto with_batched(bool sym, F&& f) {
  return sym ? f(k_batched<true>) : f(k_batched<false>);
}

template <typename F>
auto with_batched_b(bool sym, F&& f) {
  return sym ? f(k_batched_b<true>) : f(k_batched_b<false>);
}

}  // namespace

int batched_blocks_per_sm(bool sym, int block, int W) {
  const size_t smem = tiled_smem_bytes(W, block);
  return with_batched(sym, [&](auto k) {
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, block, smem) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    return n;
  });
}

cudaError_t launch_batched(const BatchProblem& p, const Ctl& c, LaunchShape s, cudaStream_t stream) {
  Batch b;
  b.n_graphs = p.n_graphs;
  b.desc = p.desc;
  b.v_off = p.v_off;
  b.a_off = p.a_off;
  b.rp_cat = p.rp_cat;
  b.col_cat = p.col_cat;
  b.labels = p.labels;
  b.graph_status = p.graph_status;
  b.unit_start = p.unit_start;
  b.plain_units = p.plain_units;
  b.plain_cap = p.plain_cap;
  b.plain_chunk_start = p.plain_chunk_start;
  b.graph_hint = p.graph_hint;
  b.total_v = (int)p.total_v;
  b.grid_a = s.grid;
  b.row_elems = p.row_elems;
  b.arc_elems = p.arc_elems;
  const size_t smem = tiled_smem_bytes(c.tile_w, s.block);
  cudaError_t e = with_batched(p.sym, [&](auto k) {
    if (smem > 48 * 1024) {
      cudaError_t e1 = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e1 != cudaSuccess) return e1;
    }
    return launch_cooperative(k, s, smem, stream, b, c);
  });
  if (e != cudaSuccess) return e;
  // The second launch counts its grid barriers from zero again; its other status fields (work
  // counters, worklist cursor) carry the first launch's results.
  e = cudaMemsetAsync(&c.st->bar, 0, sizeof(c.st->bar), stream);
  if (e != cudaSuccess) return e;
  // Two CTAs per SM where the first launch fits one (the same SMs, scaled by the occupancy ratio).
  const int per_sm_a = std::max(1, batched_blocks_per_sm(p.sym, s.block, c.tile_w));
  const int per_sm_b = with_batched_b(p.sym, [&](auto k) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, s.block, 0) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    return n;
  });
  if (per_sm_b <= 0) return cudaErrorInvalidConfiguration;
  const LaunchShape sb{std::max(1, (int)((long long)s.grid * per_sm_b / per_sm_a)), s.block};
  Ctl cb = c;
  cb.phase_off = kBatchedPhaseAEndSlot;
  cb.skip_arrival_block = -1;  // the test hook stops an arrival at the call's first barrier only
  return with_batched_b(p.sym, [&](auto k) { return launch_cooperative(k, sb, 0, stream, b, cb); });
}

}  // namespace cc
