/*
 * cc.h - C ABI of the GB300 (sm_103a) connected-components library (libcc.so).
 *
 * The library labels every vertex of an undirected graph G(V, E) with the index
 * of a representative vertex of its connected component (Section II of Sutton,
 * Ben-Nun, Barak, Pai, Pingali, "Adaptive Work-Efficient Connected Components
 * on the GPU", arXiv:1612.01178). The representative is the MINIMUM vertex ID of
 * the component: it falls out of the high-to-low hooking rule (Section II, Fig. 2
 * and Section III-A, Fig. 3), which only ever points a tree root at a smaller
 * vertex, so the root of every tree is its minimum vertex.
 *
 * Method (Section III, Fig. 4, "Adaptive Hook-Compress"):
 *   pi(v) <- v for all v;
 *   split the arcs into s = 2|E|/|V| segments (the average degree; Section III-B);
 *   for each segment: Atomic-Hook every arc of the segment (Fig. 3, top: CAS a
 *   root H = max to L = min, climbing until the CAS succeeds or both endpoints
 *   share a tree), then Multi-Jump every vertex (Fig. 3, bottom: pointer-jump
 *   until pi(v) is a root, writing every step).
 * The whole loop runs on the device; no host round-trip decides convergence.
 *
 * Conventions shared by every entry point:
 *   - Graph and label pointers are DEVICE pointers owned by the caller (except
 *     cc_labels_csr_host, which takes host pointers). The library keeps no
 *     reference to them after the call returns and never frees them.
 *   - labels is int32[n_vertices], written in place: it is the parent array pi
 *     of the method and holds the final labels when the work completes. No
 *     other per-vertex memory is allocated. labels must not overlap the graph
 *     arrays (checked on the host: CC_ERR_INVALID_ARG).
 *   - Every arc/edge is read as an undirected edge. Self-loops and duplicate
 *     edges are allowed. n_vertices = 0 and zero arcs are legal.
 *   - Calls are asynchronous and ordered on the context's stream unless
 *     CC_FLAG_SYNC is set. Argument errors are returned at once. Errors found
 *     on the device are sticky in the context's device status block and are
 *     returned by cc_sync (or by the call itself with CC_FLAG_SYNC), which also
 *     clears them. They come in two kinds:
 *       - malformed input (CC_ERR_OUT_OF_RANGE: an endpoint outside [0, V),
 *         offsets inconsistent with n_arcs): the bad arc or row is skipped and
 *         reported, the call runs to its end (in a batch, every other graph is
 *         labelled normally) and later calls are not affected; the labels of
 *         the graph concerned are unspecified;
 *       - fatal (CC_ERR_TIMEOUT, CC_ERR_INTERNAL): while one is pending, later
 *         device work of the same context exits early.
 *     Device code never traps.
 *   - A context is used by one host thread at a time.
 */
#ifndef CC_H_
#define CC_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cc_ctx cc_ctx;

typedef enum cc_status {
  CC_OK = 0,
  CC_ERR_INVALID_ARG = 1,  /* bad argument detected on the host (sizes, null pointers, types) */
  CC_ERR_OUT_OF_RANGE = 2, /* device, malformed input: an endpoint outside [0, V) or bad offsets */
  CC_ERR_OOM = 3,          /* a context-owned allocation failed */
  CC_ERR_CUDA = 4,         /* a CUDA runtime call failed; see cc_last_error_message */
  CC_ERR_TIMEOUT = 5,      /* device: a grid-wide wait exceeded cc_options.timeout_ns */
  CC_ERR_INTERNAL = 6      /* device: an iteration guard fired (impossible on valid input) */
} cc_status;

/* Row-offset element type of a CSR graph. */
typedef enum cc_index_type { CC_INDEX_I32 = 4, CC_INDEX_I64 = 8 } cc_index_type;

/* Flags (cc_options.flags, or'ed). */
enum {
  /* Every arc (u,v) has its reverse (v,u) (a symmetrised CSR): arcs with u >= v
     are skipped, halving the hooks without changing any label. */
  CC_FLAG_SYMMETRIC = 1,
  /* Check offsets (row_ptr[0] = 0, non-decreasing, row_ptr[V] = n_arcs) and
     endpoints on the device before hooking; if a check fails the call reports
     CC_ERR_OUT_OF_RANGE and does not hook at all. Endpoints are always
     range-checked while hooking; this adds the offset checks. */
  CC_FLAG_VALIDATE = 2,
  /* Block until the device work of the call is done and return its status. */
  CC_FLAG_SYNC = 4,
  /* Record a device timestamp at every grid barrier of a persistent launch
     (read with cc_last_phase_times). Costs one store per barrier. */
  CC_FLAG_PHASE_TIMES = 8
};

/* How the segment loop of Fig. 4 is driven on the device. */
typedef enum cc_mode {
  CC_MODE_AUTO = 0,        /* CC_MODE_PERSISTENT, except that a symmetric CSR (CC_FLAG_SYMMETRIC) with
                              tile_vertices = 0 and no ID locality runs CC_MODE_FILTERED when its
                              degrees are skewed (from 2^17 vertices: at least a quarter of the
                              sampled rows below a quarter of the mean degree, as in power-law
                              graphs) or its mean degree n_arcs / V is at least auto_dense_degree
                              (8; any size); cc_last_run_info reports the mode that ran */
  CC_MODE_PERSISTENT = 1,  /* one cooperative launch; phases separated by grid barriers */
  CC_MODE_MULTI_LAUNCH = 2, /* host-driven (Section III): one init, then a Hook and a Multi-Jump launch per segment */
  /* The baselines the paper measures against (Section IV, Fig. 5), CSR only: the host loop of
     Fig. 1 with the non-atomic Hook and the single Jump of Fig. 2, reading a device change flag
     after every Hook round and every Jump (one CPU-GPU round trip each) ... */
  CC_MODE_SOMAN = 3,
  /* ... and the same loop with each Compress done by one Multi-Jump launch. */
  CC_MODE_SOMAN_MULTIJUMP = 4,
  /* Sampled-and-filtered hook, CSR with CC_FLAG_SYMMETRIC only (else CC_ERR_INVALID_ARG): one
     cooperative launch running Fig. 4 with two arc subsets picked for the edge filter. The first
     2 arcs of every row are hooked, a Multi-Jump makes every tree a star, the root of the largest
     star is estimated from 256 sampled vertices, and then only the rows of vertices outside that
     star are read, their remaining arcs hooked in both directions (the reverse of a skipped arc
     is in a row that is read, unless both ends already share the star); a final Multi-Jump. On a
     graph with a giant component most arcs are never read. Without a star holding an eighth of
     the sample, the second subset is every arc, hooked as in CC_MODE_PERSISTENT. `segments`,
     `tile_vertices` do not apply. Arcs that are never read are not range-checked: an endpoint
     outside [0, V) in a skipped row goes unreported (CC_FLAG_VALIDATE checks every arc first). */
  CC_MODE_FILTERED = 5,
  /* Small graphs, CSR only: one launch of one thread-block cluster (8 CTAs, or 16 where the GPU
     allows it) holding pi in the CTAs' distributed shared memory, so root walks and hooks are
     shared-memory accesses and the phases are separated by the cluster barrier. With
     CC_FLAG_SYMMETRIC it runs the sampled-and-filtered hook, else every arc in one segment.
     At most 16 x 32768 vertices (8 x 32768 where clusters of 16 are not available), else
     CC_ERR_INVALID_ARG. CC_MODE_AUTO picks it only up to cluster_max_vertices vertices (off by
     default; an autotuner knob). */
  CC_MODE_CLUSTER = 6
} cc_mode;

typedef struct cc_options {
  int32_t mode;        /* cc_mode */
  int32_t segments;    /* s of Fig. 4. -1 = the paper's s = max(1, round(2|E| / |V|)) (Section III-B;
                          2|E| = n_arcs). 0 = this library's default from the same sweep on GB300:
                          s = 4 when 2|E|/|V| < 3, else s = 1 (the two-phase hook splits its
                          worklist E' into max(1, round(2|E'|/|V|)) segments). > 0 = exactly s. */
  int32_t block;       /* threads per block (a multiple of 32, at most 1024); 0 = 256 for the
                          plain hook and 1024 for the two-phase hook. A block that cannot be
                          co-resident is halved until it can. */
  int32_t grid_blocks; /* blocks per launch; 0 = all co-resident blocks (occupancy x SMs) */
  int32_t flags;       /* CC_FLAG_* */
  int32_t chunk_arcs;  /* global Atomic-Hook work split: -1 = one fixed slice of the segment per
                          warp; > 0 (a multiple of 32) = warps take chunks of this many arcs from a
                          shared counter; 0 = automatic (chunks of 2048 arcs when a segment holds
                          at least 2048 arcs per warp of the launch, else fixed slices) */
  int32_t tile_vertices; /* window of the two-phase hierarchical Atomic-Hook (CSR, persistent mode):
                          a power of two, 256 .. 32768. Phase A hooks every arc whose two ends lie
                          in the same window of this many consecutive IDs in shared memory and
                          writes those stars to pi; the other arcs form a worklist E' that phase B
                          hooks on pi in s' = 2|E'|/|V| segments (or `segments` if set), each
                          followed by a Multi-Jump. -1 = off: every arc is hooked on pi, one
                          segment after the other (Section III). 0 = automatic: graphs of at least 2^17 vertices whose
                          sampled arcs mostly stay inside 16384-vertex windows use the two-phase
                          hook, with a window balanced over the co-resident CTAs (a multiple of
                          256, at most 18432); the sample is a small kernel plus a
                          synchronisation on the first call for a given (row_ptr, col_idx, V,
                          n_arcs), reused afterwards. */
  int32_t sm_limit;    /* > 0: the launches of this context fill at most this many SMs' worth of
                          co-resident blocks (a share of the GPU, so that the launches of several
                          contexts on different streams run side by side); 0 = all SMs */
  int64_t timeout_ns;  /* limit of every device-side wait; 0 = 2 s */
  int64_t stream_arcs; /* cc_labels_csr_host only: > 0 = leave the arcs in host memory and stream
                          them in segments of this many arcs (see cc_labels_csr_host); -1 = never
                          stream (copy the whole graph, then run the automatic hook); 0 = stream
                          only when the graph does not fit in free device memory */
  /* Knobs of the automatic choices, for an autotuner (0 = the default in brackets): */
  int32_t hook_k;      /* arcs per lane per step of the plain CSR hook: 1, 2 or 4 [1] */
  int32_t auto_min_vertices;    /* below this many vertices CC_MODE_AUTO keeps the plain hook [2^17] */
  int32_t auto_local_permille;  /* sampled arcs inside one window, per mille, for the two-phase hook [500] */
  int32_t auto_lowdeg_permille; /* sampled rows below a quarter of the mean degree, per mille, for the
                                   sampled-and-filtered hook [250] */
  int32_t cluster_max_vertices; /* CC_MODE_AUTO runs the cluster kernel up to this many vertices (and
                                   2^23 arcs per 2^18 vertices) [0 = never] */
  int32_t auto_dense_degree;    /* mean degree n_arcs / V from which a symmetric CSR without ID
                                   locality takes the sampled-and-filtered hook even with unskewed
                                   degrees, at any size; -1 = only skewed graphs [8] */
} cc_options;

/* Fills *opt with the defaults (all zero fields resolved as documented above). */
void cc_default_options(cc_options* opt);

/* Creates a context on `device`. `stream` is a cudaStream_t to issue work on
   (NULL = the legacy default stream). `opt` may be NULL (defaults). Allocates a
   small device status block and a pinned host mirror of it. The context holds the
   state that Section III keeps on the device so that the segment loop of Fig. 4 runs
   without host round trips: the grid-barrier counter, the work counters and the
   error words of the status block. Returns CC_ERR_INVALID_ARG for bad options,
   CC_ERR_CUDA or CC_ERR_OOM when the device or the allocation fails. */
cc_status cc_create(cc_ctx** out, int device, void* stream, const cc_options* opt);

/* Replaces the stream / options of a context. */
cc_status cc_set_stream(cc_ctx* ctx, void* stream);
cc_status cc_set_options(cc_ctx* ctx, const cc_options* opt);

/* Per-call input status without a synchronisation (the paper has one graph per call and no
   failure reporting; this serves a caller that keeps several calls in flight on one context,
   such as a serving loop). With device_status a device int32 pointer, every following
   labelling call of the context first sets *device_status = 0 on the context's stream, and
   its kernels set it to CC_ERR_OUT_OF_RANGE if they find malformed input; read it after the
   call's work (stream order). NULL turns the output off. The pointer is the caller's and must
   stay valid while calls use it; the sticky status of the context is kept as well. */
cc_status cc_set_launch_status(cc_ctx* ctx, int32_t* device_status);

/* Connected components of a CSR graph (Fig. 4 over the arcs of the CSR).
 *   n_vertices  V >= 0.
 *   n_arcs      number of stored arcs (= row_ptr[V]); for a symmetrised CSR, 2|E|.
 *   row_ptr     device, int32 or int64 (row_ptr_type) [V + 1]; arcs of row u are
 *               col_idx[row_ptr[u] .. row_ptr[u+1]).
 *   col_idx     device int32 [n_arcs], values in [0, V).
 *   labels      device int32 [V], caller-owned output (also the work array pi).
 * The s segments are s contiguous, equal-length ranges of the arc array
 * (Fig. 4: "s distinct subsets of E"). */
cc_status cc_labels_csr(cc_ctx* ctx, int64_t n_vertices, int64_t n_arcs, const void* row_ptr,
                        cc_index_type row_ptr_type, const int32_t* col_idx, int32_t* labels);

/* Connected components of a CSR graph with 64-bit vertex IDs, for graphs of more than 2^31 - 1
 * vertices (Section III-B: the method's working set is the |V|-sized parent array, so the vertex
 * count is bounded by device memory, 8 bytes per vertex here, not by 32-bit IDs).
 *   row_ptr     device int64 [V + 1];  col_idx  device int64 [n_arcs], values in [0, V);
 *   labels      device int64 [V], caller-owned output (also the work array pi).
 * Runs Fig. 4 with one segment as three launches (init, Atomic-Hook of every arc, Multi-Jump).
 * CC_FLAG_SYMMETRIC and CC_FLAG_SYNC apply as for cc_labels_csr; the other options do not.
 * Labels are the minimum vertex ID of each component, as for cc_labels_csr. */
cc_status cc_labels_csr64(cc_ctx* ctx, int64_t n_vertices, int64_t n_arcs, const int64_t* row_ptr,
                          const int64_t* col_idx, int64_t* labels);

/* Connected components of an edge list (COO): edge i joins src[i] and dst[i]. The
 * graph of Section II given by its edge set E, labelled with Fig. 4 over E: each
 * edge is Atomic-Hooked once (Fig. 3, top), each of the s edge segments followed by
 * a Multi-Jump (Fig. 3, bottom).
 *   src, dst    device int32 [n_edges], values in [0, V); each edge is undirected
 *               and is hooked once.
 *   labels      device int32 [V], caller-owned output (min-ID labels).
 * Segments: cc_options.segments; 0 = 4 when 2 n_edges / V < 3, else 1 (the GB300
 * measurement of Fig. 6); -1 = the paper's max(1, round(2 n_edges / V)) (Section
 * III-B counts |E| edges, two arcs each). An endpoint outside [0, V) is skipped and
 * reported as CC_ERR_OUT_OF_RANGE; the inputs are not modified. */
cc_status cc_labels_coo(cc_ctx* ctx, int64_t n_vertices, int64_t n_edges, const int32_t* src,
                        const int32_t* dst, int32_t* labels);

/* Connected components of a batch of independent graphs in one persistent launch
 * (the paper has one graph per call; batching is this library's addition). Graph g has
 * V_g = v_off[g+1] - v_off[g] vertices and n_g = a_off[g+1] - a_off[g] arcs:
 *   v_off, a_off     device int64 [n_graphs + 1], non-decreasing, v_off[0] = a_off[0] = 0,
 *                    v_off[n_graphs] = total_vertices, a_off[n_graphs] = total_arcs.
 *   row_ptr_cat      device int32; graph g's row offsets (graph-local arc indices, V_g + 1
 *                    of them) start at row_ptr_cat + v_off[g] + g (total_vertices + n_graphs
 *                    entries in all).
 *   col_idx_cat      device int32 [total_arcs]; graph g's arcs at a_off[g] .. a_off[g+1],
 *                    graph-local vertex IDs in [0, V_g).
 *   labels_cat       device int32 [total_vertices], output: graph g's labels at v_off[g],
 *                    graph-local minimum vertex IDs.
 *   graph_status     device int32 [n_graphs] or NULL: set to CC_OK, or to
 *                    CC_ERR_OUT_OF_RANGE for a graph with an endpoint outside [0, V_g) or
 *                    inconsistent offsets. Such a graph's labels are unspecified; every other
 *                    graph of the batch is labelled normally (the context's status reports
 *                    CC_ERR_OUT_OF_RANGE as well).
 * total_vertices must be below 2^31 (labels are computed with batch-global IDs); each graph
 * must have fewer than 2^31 arcs. Graphs of at most tile_vertices vertices (default 32768)
 * are labelled inside one CTA's shared memory; larger graphs go through the two-phase hook
 * with a locality sample per window (tile_vertices = -1: their windows are hooked arc by arc).
 * CC_FLAG_SYMMETRIC, CC_FLAG_SYNC and CC_FLAG_PHASE_TIMES apply as for cc_labels_csr. */
cc_status cc_labels_batched(cc_ctx* ctx, int32_t n_graphs, int64_t total_vertices, int64_t total_arcs,
                            const int64_t* v_off, const int64_t* a_off, const int32_t* row_ptr_cat,
                            const int32_t* col_idx_cat, int32_t* labels_cat, int32_t* graph_status);

/* One graph of a descriptor-mode batch: element offsets of its labels (label_off, V
   entries), row offsets (row_off, V + 1 graph-local offsets) and arcs (arc_off, n_arcs
   graph-local IDs) inside three device arenas. */
typedef struct cc_graph_desc {
  int64_t label_off;
  int64_t row_off;
  int64_t arc_off;
  int64_t n_arcs;
  int32_t n_vertices;
  int32_t reserved; /* 0 */
} cc_graph_desc;

/* cc_labels_batched for graphs placed anywhere in three device arenas (a serving loop keeps
 * requests wherever its allocator put them). descs is a device array [n_graphs]; label ranges
 * [label_off, label_off + n_vertices) must not overlap. A descriptor that does not fit its arena
 * sizes is reported in graph_status (and the status word) and its graph is skipped.
 * label_arena_elems must be below 2^31. Results are graph-local minimum IDs at label_off. */
cc_status cc_labels_batched_desc(cc_ctx* ctx, int32_t n_graphs, const cc_graph_desc* descs,
                                 const int32_t* row_arena, int64_t row_arena_elems, const int32_t* arc_arena,
                                 int64_t arc_arena_elems, int32_t* label_arena, int64_t label_arena_elems,
                                 int32_t* graph_status);

/* cc_labels_csr with HOST buffers: copies row_ptr and col_idx from host memory
   (pinned memory gives full copy bandwidth) into context-owned device buffers,
   runs the method, copies the labels back into the host array `labels`, and
   returns after the copy completes (always synchronous). The device buffers
   grow to the largest graph seen and are freed by cc_destroy.
   Graphs larger than device memory (Section III-B: the segments bound the
   working set to the |V|-sized parent array): when cc_options.stream_arcs > 0,
   or (stream_arcs = 0) when row_ptr + col_idx + labels do not fit in free
   device memory, the arcs stay in host memory. row_ptr and the labels (pi) are copied to / kept on the
   device, and Fig. 4 runs with s = ceil(n_arcs / seg) contiguous segments of
   seg arcs (stream_arcs, or two buffers sized from the free memory): segment i
   is copied in on a copy stream while segment i - 1 is Atomic-Hooked (plain
   hook), and a Multi-Jump follows every segment. The device then holds only
   row_ptr, labels and two segment buffers. CC_FLAG_VALIDATE does not apply
   (endpoints are range-checked while hooking); cc_last_run_info reports
   streamed_segments. Returns CC_ERR_OOM if row_ptr and labels themselves do not
   fit. */
cc_status cc_labels_csr_host(cc_ctx* ctx, int64_t n_vertices, int64_t n_arcs, const void* row_ptr,
                             cc_index_type row_ptr_type, const int32_t* col_idx, int32_t* labels);

/* Waits for all work issued on the context's stream, then returns the first
   device error recorded since the last cc_sync (CC_OK if none) and clears it. */
cc_status cc_sync(cc_ctx* ctx);

/* What the last labelling call ran with (filled on the host at issue time). */
typedef struct cc_run_info {
  int32_t mode;        /* cc_mode actually used */
  int32_t segments;    /* s actually used */
  int32_t grid_blocks; /* blocks per launch */
  int32_t block;       /* threads per block */
  int32_t launches;    /* kernel launches issued by the call */
  int32_t tile_vertices; /* window of the hierarchical hook (0 = plain hook) */
  int64_t worklist_capacity; /* pairs the worklist could hold (hierarchical hook) */
  int32_t host_round_trips;  /* device-to-host flag reads that decided convergence (Soman modes) */
  int32_t hook_rounds;       /* Hook rounds of the host loop (Soman modes) */
  int32_t streamed_segments; /* cc_labels_csr_host: arc segments streamed from host memory (0 = none) */
  int32_t reserved;
} cc_run_info;

/* Worklist of the last hierarchical-hook launch: waits for the context's stream, then
   stores the number of arcs phase A left for phase B (*pairs) and the segments phase B
   used (*segments); both 0 if every arc was joined inside its window. */
cc_status cc_last_worklist(cc_ctx* ctx, int64_t* pairs, int32_t* segments);
cc_status cc_last_run_info(const cc_ctx* ctx, cc_run_info* info);

/* Phase timestamps of the last persistent launch made with CC_FLAG_PHASE_TIMES:
   waits for the context's stream, then writes ns[0] = 0 (kernel start),
   ns[k] = time block 0 left grid barrier k (k = 1 .. n-2) and ns[n-1] = the
   end of the last block, all in ns relative to the start; *n = entries written
   (at most cap, at most 64). Barrier 1 ends init; barriers 2i and 2i+1 end the
   Atomic-Hook and the Multi-Jump of segment i. */
cc_status cc_last_phase_times(cc_ctx* ctx, int64_t* ns, int32_t cap, int32_t* n);

/* Text of the last CUDA error seen by the context ("" if none). */
const char* cc_last_error_message(const cc_ctx* ctx);

/* Static description of a status code. */
const char* cc_status_string(cc_status status);

/* Releases the context and everything it allocated (the device state of
   cc_create, worklist and staging buffers). NULL is ignored. Waits for the
   context's stream first. */
void cc_destroy(cc_ctx* ctx);

/* Allocation-free variant of cc_labels_csr (the paper has no counterpart: this
   entry point exists for callers that cannot allocate device memory, such as code
   running inside a device memory allocator or pool, plug-ins whose host owns all
   device memory, or real-time paths that must not allocate).
   It needs no context and calls no cudaMalloc/cudaFree or allocating routine. The
   only scratch the persistent kernel needs beyond the caller's arrays (its 96-byte
   status block: grid-barrier counter, work counters and error word) lives in a
   static 256-byte device array inside libcc.so, held on every GPU that loads the
   library until the process exits; its size does not grow with the graph. It runs
   the plain Atomic-Hook in one cooperative launch with cc_labels_csr's default
   segment plan and work split (the two-phase and filtered hooks of cc_labels_csr
   need a worklist or a sampling buffer, which this entry point does not have). The graph limits are those of
   cc_labels_csr: n_vertices <= 2^31 - 1, and n_arcs <= 2^31 - 1 with int32
   offsets; anything larger, or any other flag than CC_FLAG_SYMMETRIC, returns
   CC_ERR_INVALID_ARG.
     row_ptr, col_idx, labels: device pointers as for cc_labels_csr, on the
       current device; stream: cudaStream_t (NULL = legacy default stream).
   The call issues on `stream`, waits for it, and returns the device status of
   this call (CC_OK, CC_ERR_OUT_OF_RANGE, CC_ERR_TIMEOUT, ...). Because it waits,
   it cannot be issued on a stream that is being captured: such a call returns
   CC_ERR_INVALID_ARG without touching the stream. The first call on a device
   looks up the scratch array's device address (cudaGetSymbolAddress, once per
   device), which must not happen during a stream capture on that device. All calls share the scratch array, which keeps the last call's
   contents; each call clears it before launching. Calls whose GPU work could
   overlap (unordered streams, or concurrent host threads) race on it and must
   not be issued. */
cc_status cc_labels_csr_noalloc(int64_t n_vertices, int64_t n_arcs, const void* row_ptr,
                                cc_index_type row_ptr_type, const int32_t* col_idx, int32_t* labels,
                                void* stream, int32_t flags);

/* Test hook: with block >= 0, that block of the next persistent launch does not
   arrive at its first grid barrier, so every other block's wait runs out after
   timeout_ns and the call reports CC_ERR_TIMEOUT; the context stays usable.
   The hook disarms itself after one launch. Returns CC_ERR_INVALID_ARG for a
   NULL context. */
cc_status cc_debug_skip_barrier_arrival(cc_ctx* ctx, int32_t block);

#ifdef __cplusplus
}
#endif

#endif /* CC_H_ */
