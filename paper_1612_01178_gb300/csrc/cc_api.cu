// C ABI of libcc.so (declared in include/cc.h): contexts, argument checks, launch-shape
// choice, device status handling and the host-buffer entry point.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>

#include "cc.h"
#include "cc_internal.h"

struct cc_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  cc_options opt{};
  int num_sms = 0;
  cc::DevStatus* d_status = nullptr;  // device status block
  cc::DevStatus* h_status = nullptr;  // pinned host mirror
  cc_run_info last{};
  int skip_arrival_block = -1;
  char last_error[256] = {0};
  int32_t* status_out = nullptr;          // cc_set_launch_status: per-call input status (device)
  unsigned long long* d_phase = nullptr;  // CC_FLAG_PHASE_TIMES timestamps (kPhaseSlots)
  bool phase_valid = false;
  // worklist of the two-phase hierarchical hook
  int2* d_wl = nullptr;
  size_t d_wl_pairs = 0;
  int* d_ovf = nullptr;
  size_t d_ovf_n = 0;
  long long* d_unit_start = nullptr;  // batched: first window of each graph
  size_t d_unit_start_n = 0;
  long long* d_chunk_start = nullptr;  // batched: chunk table of the windows hooked arc by arc
  size_t d_chunk_start_n = 0;
  int* d_hint = nullptr;  // batched: giant-star root per graph
  size_t d_hint_n = 0;
  // automatic hook choice: locality sample buffer and the last decision
  unsigned long long* d_sample = nullptr;
  unsigned long long* h_sample = nullptr;
  const void* auto_rp = nullptr;
  const void* auto_col = nullptr;
  long long auto_V = -1, auto_m = -1;
  int auto_w = 0;
  bool auto_skewed = false;  // the sampled degrees are skewed (most rows far below the mean)
  // staging buffers of cc_labels_csr_host
  void* d_rp = nullptr;
  size_t d_rp_bytes = 0;
  int32_t* d_col = nullptr;
  size_t d_col_bytes = 0;
  int32_t* d_labels = nullptr;
  size_t d_labels_bytes = 0;
  // streamed arcs of cc_labels_csr_host (graphs whose arcs stay in host memory)
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t seg_copied[2] = {nullptr, nullptr};
  cudaEvent_t seg_used[2] = {nullptr, nullptr};
  int32_t* d_seg[2] = {nullptr, nullptr};
  size_t d_seg_arcs = 0;
};

namespace cc {

// s of Section III-B: 2|E|/|V| = arcs per vertex, rounded, at least 1.
static int paper_segments(long long arcs, long long V) {
  if (V <= 0 || arcs <= 0) return 1;
  const double s = std::floor((double)arcs / (double)V + 0.5);
  return (int)std::max(1.0, std::min(s, 1.0e6));
}

// Segment count when the caller leaves it to the library (segments = 0). The segmentation
// sweep of Fig. 6 repeated on GB300 (ER graphs of average degree 2..128, both drivers) puts the
// fastest s at 1..4 for every degree, far below the paper's 2|E|/|V| (at degree 86 that choice
// is 1.65x slower than s = 1): with root walks that halve paths as they go, intermediate
// compresses rarely pay for their full O(V) pass. Only very sparse graphs gained from a few
// segments (degree 2: s = 4, 1.1x to 2.5x over s = 1). segments = -1 selects the paper's s.
int default_segments(long long arcs, long long V, int requested) {
  if (requested > 0) return requested;
  if (requested < 0) return paper_segments(arcs, V);
  if (V <= 0 || arcs <= 0) return 1;
  return (double)arcs / (double)V < 3.0 ? 4 : 1;
}

// Automatic work split of the plain hook: warps take chunks of kAutoChunkArcs arcs from a counter
// when a segment holds at least that many arcs per warp of the launch (a fixed slice per warp
// leaves the grid waiting on the slowest slice of a skewed graph); smaller segments use fixed
// slices (-1).
int auto_chunk_arcs(long long arcs_per_segment, long long warps) {
  constexpr int kAutoChunkArcs = 2048;
  return arcs_per_segment >= (long long)kAutoChunkArcs * warps ? kAutoChunkArcs : -1;
}

}  // namespace cc

namespace {

constexpr long long kDefaultTimeoutNs = 2000000000LL;
constexpr int kDefaultChunkArcs = 0;  // automatic
// Default window of the two-phase hook: single graphs use 16384 vertices (64 KB of 32-bit local
// parents, two 1024-thread CTAs per SM); the batched kernel keeps whole graphs of up to 32768
// vertices in one CTA.
constexpr int kDefaultTileVertices = 16384;
constexpr int kBatchedTileVertices = 32768;
// Widest automatic window of a single graph: 18432 x 4 bytes of local parents plus the per-warp
// scratch of 32 warps still lets two 1024-thread CTAs share an SM's 228 KB.
constexpr int kMaxAutoWindow = 18432;
constexpr int kMinAutoWindow = 2048;
constexpr int kMaxTileVertices = 32768;
constexpr int kPlainBlock = 256;   // default block of the plain hook
constexpr int kTiledBlock = 1024;  // default block of the two-phase hook
constexpr int kPhaseABlock = 1024; // default block of its phase-A launch
constexpr int kSampleThreads = 16384;
constexpr double kLocalFractionForTiles = 0.5;     // cc_options.auto_local_permille = 0
// Automatic choice of the sampled-and-filtered hook (CC_FLAG_SYMMETRIC, no locality): at least
// this fraction of sampled rows has a degree below a quarter of the mean, as in power-law graphs
// whose arcs sit mostly in the long rows of a giant component (on R-MAT the filter skips most
// arcs) ...
constexpr double kLowDegreeFractionForFilter = 0.25;  // cc_options.auto_lowdeg_permille = 0
constexpr long long kAutoMinVertices = 1 << 17;      // cc_options.auto_min_vertices = 0
// ... and, at any size, for a symmetric CSR without ID locality whose mean degree n_arcs / V is at
// least this (cc_options.auto_dense_degree = 0): with the grid barrier's relaxed polling the filter
// measured faster than the plain hook on ER graphs of mean degree 16 to 40 (ER 100k / 1M 0.090 vs
// 0.138 ms, ER 16M / 128M 0.65 vs 1.81 ms), slower on sparse ones (ER 20k / 30k 0.065 vs 0.051 ms).
constexpr int kDenseDegreeForFilter = 8;
// Block of the sampled-and-filtered hook: 1024-thread CTAs, two per SM, so that each of its grid
// barriers counts 304 arrivals instead of 1216 (an empty barrier measured 1.7 vs 5.0 us); R-MAT 26
// 1.72 -> 1.70 ms, ER 100k / 1M 0.105 -> 0.090 ms.
constexpr int kFilterBlock = 1024;
constexpr int kPhaseSlots = 64;
// Automatic choice of the cluster kernel (CC_MODE_AUTO, CSR) up to cc_options.cluster_max_vertices
// vertices (0 = never: on GB300 the grid-wide kernels measured faster on most small graphs, the
// cluster kernel on some power-law ones, so the choice is left to the autotuner) and
// kClusterAutoMaxArcs arcs per 2^18 vertices.
constexpr long long kClusterAutoMaxArcs = 1 << 23;

// Makes `device` current for the scope of a call and restores the caller's device after.
struct DeviceGuard {
  int prev = -1;
  bool ok = false;
  explicit DeviceGuard(int device) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    ok = (prev == device) || cudaSetDevice(device) == cudaSuccess;
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

cc_status cuda_fail(cc_ctx* ctx, cudaError_t e, const char* where) {
  if (ctx) std::snprintf(ctx->last_error, sizeof(ctx->last_error), "%s: %s", where, cudaGetErrorString(e));
  cudaGetLastError();  // clear a non-sticky error so the context stays usable
  return CC_ERR_CUDA;
}

void resolve_options(cc_options* o) {
  if (o->timeout_ns <= 0) o->timeout_ns = kDefaultTimeoutNs;
}

// SMs a context's launches may fill: cc_options.sm_limit (a share of the GPU, so that launches of
// several contexts run side by side), or all of them.
int usable_sms(const cc_ctx* ctx) {
  const int lim = ctx->opt.sm_limit;
  return lim > 0 && lim < ctx->num_sms ? lim : ctx->num_sms;
}

// Window of the two-phase hook for `want` vertices: a power of two, at least 256, no wider
// than needed to cover V.
int window_for(long long V, int want) {
  int w = 256;
  while (w < want && w < V) w <<= 1;
  return w;
}

// Automatic window (tile_vertices = 0, two-phase hook chosen): phase A hands windows to the
// co-resident CTAs from a counter, so its time is set by the number of rounds of windows per
// CTA. The window is the smallest multiple of 256 that covers V in whole rounds of all CTAs,
// with no more rounds than kMaxAutoWindow needs (a window count just above a multiple of the
// CTA count would leave most CTAs idle in the last round).
int balanced_window(const cc_ctx* ctx, cc::Problem p, int block) {
  p.tile_w = kMaxAutoWindow;
  const long long ctas = (long long)std::max(1, cc::phase_a_blocks_per_sm(p, block)) * usable_sms(ctx);
  const long long rounds = std::max<long long>(1, (p.V + ctas * kMaxAutoWindow - 1) / (ctas * kMaxAutoWindow));
  long long w = (p.V + rounds * ctas - 1) / (rounds * ctas);
  w = (w + 255) / 256 * 256;
  return (int)std::min<long long>(kMaxAutoWindow, std::max<long long>(kMinAutoWindow, w));
}

// Automatic hook choice (tile_vertices = 0): the two-phase hook pays off when most arcs join
// vertices of the same window, i.e. when the vertex numbering has locality (meshes, road
// networks in their natural order); otherwise the plain hook is used, or, for a symmetric CSR
// whose sampled degrees are skewed (*skewed_out) or whose mean degree is high (the caller's
// test, which needs no sample), the sampled-and-filtered hook. A small
// sampling kernel measures both on the first call for a given graph (row_ptr, col_idx, V,
// n_arcs); the answers are kept and reused while those stay the same. Only the speed depends
// on them.
cc_status auto_window(cc_ctx* ctx, const cc::Problem& p, int* w_out, bool* skewed_out) {
  *w_out = 0;
  *skewed_out = false;
  const cc_options& o = ctx->opt;
  if (p.V < (o.auto_min_vertices > 0 ? (long long)o.auto_min_vertices : kAutoMinVertices)) return CC_OK;  // no sample
  const int w = window_for(p.V, kDefaultTileVertices);
  if (ctx->auto_rp == p.rp && ctx->auto_col == p.col && ctx->auto_V == p.V && ctx->auto_m == p.m) {
    *w_out = ctx->auto_w;
    *skewed_out = ctx->auto_skewed;
    return CC_OK;
  }
  if (!ctx->d_sample) {
    if (cudaMalloc(&ctx->d_sample, 4 * sizeof(unsigned long long)) != cudaSuccess ||
        cudaMallocHost(&ctx->h_sample, 4 * sizeof(unsigned long long)) != cudaSuccess) {
      cudaGetLastError();
      return CC_ERR_OOM;
    }
  }
  cudaError_t e = cudaMemsetAsync(ctx->d_sample, 0, 4 * sizeof(unsigned long long), ctx->stream);
  if (e == cudaSuccess) e = cc::launch_sample_locality(p, w, ctx->d_sample, kSampleThreads, ctx->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(ctx->h_sample, ctx->d_sample, 4 * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                        ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "locality sample");
  const double total = (double)ctx->h_sample[1];
  const double frac = total > 0 ? (double)ctx->h_sample[0] / total : 0.0;
  ctx->auto_rp = p.rp;
  ctx->auto_col = p.col;
  ctx->auto_V = p.V;
  ctx->auto_m = p.m;
  const double local_min = o.auto_local_permille > 0 ? o.auto_local_permille / 1000.0 : kLocalFractionForTiles;
  const double lowdeg_min = o.auto_lowdeg_permille > 0 ? o.auto_lowdeg_permille / 1000.0 : kLowDegreeFractionForFilter;
  ctx->auto_w = frac >= local_min ? w : 0;
  const double rows = (double)ctx->h_sample[3];
  ctx->auto_skewed = rows > 0 && (double)ctx->h_sample[2] / rows >= lowdeg_min;
  *w_out = ctx->auto_w;
  *skewed_out = ctx->auto_skewed;
  return CC_OK;
}

bool options_ok(const cc_options* o) {
  if (o->mode < CC_MODE_AUTO || o->mode > CC_MODE_CLUSTER) return false;
  if (o->segments < -1 || o->grid_blocks < 0) return false;
  if (o->chunk_arcs < -1 || (o->chunk_arcs > 0 && o->chunk_arcs % 32 != 0)) return false;
  if (o->tile_vertices != 0 && o->tile_vertices != -1 &&
      (o->tile_vertices < 256 || o->tile_vertices > kMaxTileVertices ||
       (o->tile_vertices & (o->tile_vertices - 1)) != 0))
    return false;
  if (o->sm_limit < 0 || o->stream_arcs < -1 || o->auto_dense_degree < -1) return false;
  if (o->hook_k != 0 && o->hook_k != 1 && o->hook_k != 2 && o->hook_k != 4) return false;
  if (o->auto_min_vertices < 0 || o->auto_local_permille < 0 || o->auto_local_permille > 1000 ||
      o->auto_lowdeg_permille < 0 || o->auto_lowdeg_permille > 1000 || o->cluster_max_vertices < 0)
    return false;
  if (o->block != 0 && (o->block < 32 || o->block > 1024 || o->block % 32 != 0)) return false;
  if (o->flags & ~(CC_FLAG_SYMMETRIC | CC_FLAG_VALIDATE | CC_FLAG_SYNC | CC_FLAG_PHASE_TIMES)) return false;
  return true;
}

cc_status read_and_clear_status(cc_ctx* ctx) {
  cudaError_t e = cudaMemcpyAsync(ctx->h_status, ctx->d_status, sizeof(cc::DevStatus), cudaMemcpyDeviceToHost,
                                  ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cc_sync");
  const cc::DevStatus& h = *ctx->h_status;
  const int err = h.error != 0 ? h.error : h.input_error;
  if (err != 0) {
    if (h.error != 0)
      std::snprintf(ctx->last_error, sizeof(ctx->last_error), "device error %d at site %d (info %lld)", err,
                    h.error_where, h.error_info);
    else
      std::snprintf(ctx->last_error, sizeof(ctx->last_error), "malformed input (error %d) at site %d (info %lld)",
                    err, h.input_where, h.input_info);
    e = cudaMemsetAsync(ctx->d_status, 0, sizeof(cc::DevStatus), ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cc_sync clear");
    return (cc_status)err;
  }
  return CC_OK;
}

// A call with nothing to label: the caller's status output (if any) still reads 0 afterwards.
cc_status finish_empty_call(cc_ctx* ctx) {
  if (ctx->status_out) {
    cudaError_t e = cudaMemsetAsync(ctx->status_out, 0, sizeof(int32_t), ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "status reset");
  }
  return (ctx->opt.flags & CC_FLAG_SYNC) ? read_and_clear_status(ctx) : CC_OK;
}

// Grows a context-owned device buffer to at least `n` elements of T.
template <typename T>
cudaError_t grow_buffer(T** buf, size_t* have, size_t n) {
  if (n <= *have) return cudaSuccess;
  if (*buf) cudaFree(*buf);
  *buf = nullptr;
  *have = 0;
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(buf), n * sizeof(T));
  if (e != cudaSuccess) {
    *buf = nullptr;
    cudaGetLastError();
    return e;
  }
  *have = n;
  return cudaSuccess;
}

// Reads DevStatus::changed after zeroing it and running `launch` (one CPU-GPU round trip).
template <typename F>
cc_status flag_round(cc_ctx* ctx, F&& launch, bool* changed, cc_run_info* info) {
  cudaError_t e = cudaMemsetAsync(&ctx->d_status->changed, 0, sizeof(unsigned int), ctx->stream);
  if (e == cudaSuccess) e = launch();
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(ctx->h_status, ctx->d_status, sizeof(cc::DevStatus), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "host loop");
  info->launches += 1;
  info->host_round_trips += 1;
  if (ctx->h_status->error != 0) return read_and_clear_status(ctx);
  *changed = ctx->h_status->changed != 0;
  return CC_OK;
}

// The host-driven loop of the Hook-Compress baseline (Section II): repeat { Hook all arcs;
// Compress } until a Hook round changes nothing, each decision read back from the device
// change flag. Compress is a single Jump repeated until it changes nothing, or one Multi-Jump.
cc_status run_host_loop(cc_ctx* ctx, const cc::Problem& p, const cc::Ctl& c, cc::LaunchShape s, bool multijump,
                        cc_run_info* info) {
  cudaError_t e = cc::launch_init_only(p, c, s, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "init launch");
  info->launches += 1;
  const long long guard = 2LL * p.V + 64;
  for (long long round = 0;; ++round) {
    if (round > guard) {
      std::snprintf(ctx->last_error, sizeof(ctx->last_error), "host loop did not converge");
      return CC_ERR_INTERNAL;
    }
    bool hooked = false;
    cc_status st = flag_round(ctx, [&] { return cc::launch_hook_nonatomic(p, c, s, ctx->stream); }, &hooked, info);
    if (st != CC_OK) return st;
    info->hook_rounds += 1;
    if (!hooked) break;
    if (multijump) {
      e = cc::launch_jump_multi(p, c, s, ctx->stream);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "multi-jump launch");
      info->launches += 1;
    } else {
      for (long long j = 0;; ++j) {
        if (j > guard) {
          std::snprintf(ctx->last_error, sizeof(ctx->last_error), "jump loop did not converge");
          return CC_ERR_INTERNAL;
        }
        bool jumped = false;
        st = flag_round(ctx, [&] { return cc::launch_jump_single(p, c, s, ctx->stream); }, &jumped, info);
        if (st != CC_OK) return st;
        if (!jumped) break;
      }
    }
  }
  return CC_OK;
}

// Runs one single-graph problem on the context's stream.
cc_status run_problem(cc_ctx* ctx, cc::Problem& p) {
  const cc_options& o = ctx->opt;
  int block = o.block > 0 ? o.block : kPlainBlock;
  p.segments = cc::default_segments(p.m, p.V, o.segments);
  if (p.m == 0) p.segments = 1;

  cc::Ctl c;
  c.st = ctx->d_status;
  c.timeout_ns = o.timeout_ns;
  c.skip_arrival_block = -1;
  c.chunk_arcs = o.chunk_arcs;
  c.hook_k = o.hook_k > 0 ? o.hook_k : 1;

  // Work-proportional grid, capped by what is co-resident (the persistent kernel needs it).
  const long long work = std::max<long long>(p.V, p.m / 4);
  long long want = (work + block - 1) / block;
  want = std::max<long long>(want, 1);

  cc_run_info info{};
  info.segments = p.segments;
  int mode = o.mode == CC_MODE_AUTO ? CC_MODE_PERSISTENT : o.mode;
  info.mode = mode;
  p.filtered = false;
  if (mode == CC_MODE_FILTERED) {
    if (p.kind != cc::kKindCsr || !p.sym) {
      std::snprintf(ctx->last_error, sizeof(ctx->last_error),
                    "CC_MODE_FILTERED needs CSR input with CC_FLAG_SYMMETRIC");
      return CC_ERR_INVALID_ARG;
    }
    p.filtered = true;
    p.segments = 2;  // the two arc subsets
    info.segments = 2;
    mode = CC_MODE_PERSISTENT;  // one cooperative launch, shaped like the persistent one
  }

  info.block = block;
  const long long cluster_max_v = o.cluster_max_vertices;
  const bool want_cluster =
      p.kind == cc::kKindCsr && p.m > 0 &&
      (o.mode == CC_MODE_CLUSTER || (o.mode == CC_MODE_AUTO && o.tile_vertices == 0 && p.V <= cluster_max_v &&
                                     p.m <= kClusterAutoMaxArcs * std::max<long long>(1, cluster_max_v >> 18)));
  const int cluster = want_cluster ? cc::cluster_size_for(p) : 0;
  if (o.mode == CC_MODE_CLUSTER && cluster == 0) {
    std::snprintf(ctx->last_error, sizeof(ctx->last_error), "graph does not fit one thread-block cluster");
    return CC_ERR_INVALID_ARG;
  }
  // Per-call status: the per-launch fields of the status block (validation's abort flag
  // included) and the caller's status output start at zero.
  {
    cudaError_t e0 = cudaMemsetAsync(ctx->d_status, 0, cc::kPerLaunchStatusBytes, ctx->stream);
    if (e0 == cudaSuccess && ctx->status_out) e0 = cudaMemsetAsync(ctx->status_out, 0, sizeof(int32_t), ctx->stream);
    if (e0 != cudaSuccess) return cuda_fail(ctx, e0, "status reset");
    c.status_out = ctx->status_out;
  }
  if (o.flags & CC_FLAG_VALIDATE) {
    cc::LaunchShape vs{(int)std::min<long long>(want, (long long)usable_sms(ctx) * 8), block};
    cudaError_t e = cc::launch_validate(p, c, vs, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "validate launch");
    info.launches += 1;
  }

  if (cluster > 0) {
    cudaError_t e = cudaSuccess;
    if (o.flags & CC_FLAG_PHASE_TIMES) {
      if (!ctx->d_phase && cudaMalloc(&ctx->d_phase, kPhaseSlots * sizeof(unsigned long long)) != cudaSuccess) {
        ctx->d_phase = nullptr;
        cudaGetLastError();
        return CC_ERR_OOM;
      }
      e = cudaMemsetAsync(ctx->d_phase, 0, kPhaseSlots * sizeof(unsigned long long), ctx->stream);
      c.phase_ns = ctx->d_phase;
      c.phase_cap = kPhaseSlots;
      ctx->phase_valid = true;
    } else {
      ctx->phase_valid = false;
    }
    if (e == cudaSuccess) e = cc::launch_cluster(p, c, cluster, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cluster launch");
    info.mode = CC_MODE_CLUSTER;
    info.segments = p.sym ? 2 : 1;
    info.grid_blocks = cluster;
    info.block = 1024;
    info.launches += 1;
    ctx->last = info;
    if (o.flags & CC_FLAG_SYNC) return read_and_clear_status(ctx);
    return CC_OK;
  }

  // Two-phase hierarchical hook (CSR, persistent mode): windows of W vertices.
  p.tile_w = 0;
  int w = 0;
  if (p.kind == cc::kKindCsr && mode == CC_MODE_PERSISTENT && p.m > 0 && !p.filtered) {
    if (o.tile_vertices > 0) {
      w = window_for(p.V, o.tile_vertices);
    } else if (o.tile_vertices == 0) {
      bool skewed = false;
      const int dense_deg = o.auto_dense_degree == 0 ? kDenseDegreeForFilter : o.auto_dense_degree;
      const bool dense = dense_deg > 0 && p.m >= (long long)dense_deg * p.V;
      const cc_status st = auto_window(ctx, p, &w, &skewed);
      if (st != CC_OK) return st;
      if (w > 0) {
        w = balanced_window(ctx, p, o.block > 0 ? o.block : kPhaseABlock);
      } else if (p.sym && o.mode == CC_MODE_AUTO && (skewed || dense)) {
        // no locality, skewed degrees or a high mean degree: the sampled-and-filtered hook (one
        // cooperative launch)
        p.filtered = true;
        p.segments = 2;
        info.segments = 2;
        info.mode = CC_MODE_FILTERED;
      }
    }
  }
  if (w > 0) {
    if (o.block <= 0) block = kTiledBlock;
    p.tile_w = w;
    // Worklist capacity: one pair per vertex (at least 2^20, at most one per arc). Windows
    // whose appends overflow it are re-hooked arc by arc in phase B instead.
    const size_t cap = (size_t)std::min<long long>(p.m, std::max<long long>(p.V, 1 << 20));
    const size_t n_units = (size_t)((p.V + w - 1) / w);
    if (grow_buffer(&ctx->d_wl, &ctx->d_wl_pairs, cap) != cudaSuccess ||
        grow_buffer(&ctx->d_ovf, &ctx->d_ovf_n, n_units) != cudaSuccess) {
      std::snprintf(ctx->last_error, sizeof(ctx->last_error), "worklist allocation failed");
      return CC_ERR_OOM;
    }
    c.tile_w = w;
    c.wl = ctx->d_wl;
    c.wl_cap = ctx->d_wl_pairs;
    c.ovf_units = ctx->d_ovf;
    c.ovf_cap = (int)std::min<size_t>(ctx->d_ovf_n, INT32_MAX);
    c.segments_b = o.segments > 0 ? o.segments : 0;
  }

  if (p.filtered && o.block <= 0) block = kFilterBlock;
  if (mode == CC_MODE_PERSISTENT) {
    // The requested block size must be co-resident at least once per SM; halve it until it is
    // (a kernel variant may need more registers or shared memory than the request allows).
    int per_sm = cc::persistent_blocks_per_sm(p, block);
    while (per_sm <= 0 && block > 32) {
      block /= 2;
      per_sm = cc::persistent_blocks_per_sm(p, block);
    }
    info.block = block;
    if (per_sm <= 0) return cuda_fail(ctx, cudaErrorInvalidConfiguration, "persistent occupancy");
    want = std::max<long long>(1, (work + block - 1) / block);
    const long long cap = (long long)per_sm * usable_sms(ctx);
    long long grid = o.grid_blocks > 0 ? std::min<long long>(o.grid_blocks, cap) : std::min(want, cap);
    cc::LaunchShape s{(int)grid, block};
    if (o.chunk_arcs == 0) {
      const long long warps = grid * (block / 32);
      c.chunk_arcs = cc::auto_chunk_arcs(p.m / std::max(1, p.segments), warps);
    }
    c.skip_arrival_block = ctx->skip_arrival_block;
    ctx->skip_arrival_block = -1;
    cudaError_t e = cudaSuccess;
    if (o.flags & CC_FLAG_PHASE_TIMES) {
      if (!ctx->d_phase && cudaMalloc(&ctx->d_phase, kPhaseSlots * sizeof(unsigned long long)) != cudaSuccess) {
        ctx->d_phase = nullptr;
        cudaGetLastError();
        return CC_ERR_OOM;
      }
      e = cudaMemsetAsync(ctx->d_phase, 0, kPhaseSlots * sizeof(unsigned long long), ctx->stream);
      c.phase_ns = ctx->d_phase;
      c.phase_cap = kPhaseSlots;
      ctx->phase_valid = true;
    } else {
      ctx->phase_valid = false;
    }
    if (e == cudaSuccess && p.tile_w > 0) {
      // Phase A: one CTA per window at most, as many as are co-resident.
      int block_a = o.block > 0 ? o.block : kPhaseABlock;
      int per_sm_a = cc::phase_a_blocks_per_sm(p, block_a);
      while (per_sm_a <= 0 && block_a > 32) {
        block_a /= 2;
        per_sm_a = cc::phase_a_blocks_per_sm(p, block_a);
      }
      if (per_sm_a <= 0) return cuda_fail(ctx, cudaErrorInvalidConfiguration, "phase A occupancy");
      const long long n_units = (p.V + p.tile_w - 1) / p.tile_w;
      const long long grid_a = std::min<long long>(n_units, (long long)per_sm_a * usable_sms(ctx));
      e = cc::launch_two_phase(p, c, cc::LaunchShape{(int)grid_a, block_a}, s, ctx->stream);
      info.launches += 2;
    } else if (e == cudaSuccess) {
      e = cc::launch_persistent(p, c, s, ctx->stream);
      info.launches += 1;
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "persistent launch");
    info.grid_blocks = s.grid;
  } else if (mode == CC_MODE_SOMAN || mode == CC_MODE_SOMAN_MULTIJUMP) {
    if (p.kind != cc::kKindCsr) return CC_ERR_INVALID_ARG;
    const int per_sm = std::max(1, cc::stage_blocks_per_sm(p, block));
    const long long cap = (long long)per_sm * usable_sms(ctx);
    long long grid = o.grid_blocks > 0 ? o.grid_blocks : std::min(want, cap);
    cc::LaunchShape s{(int)grid, block};
    const cc_status st = run_host_loop(ctx, p, c, s, mode == CC_MODE_SOMAN_MULTIJUMP, &info);
    if (st != CC_OK) return st;
    info.grid_blocks = s.grid;
  } else {
    const int per_sm = std::max(1, cc::stage_blocks_per_sm(p, block));
    const long long cap = (long long)per_sm * usable_sms(ctx);
    long long grid = o.grid_blocks > 0 ? o.grid_blocks : std::min(want, cap);
    cc::LaunchShape s{(int)grid, block};
    int n = 0;
    cudaError_t e = cc::launch_multi(p, c, s, ctx->stream, &n);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "multi launch");
    info.grid_blocks = s.grid;
    info.launches += n;
  }
  info.tile_vertices = p.tile_w;
  info.worklist_capacity = p.tile_w > 0 ? (int64_t)ctx->d_wl_pairs : 0;
  ctx->last = info;
  if (o.flags & CC_FLAG_SYNC) return read_and_clear_status(ctx);
  return CC_OK;
}

}  // namespace

extern "C" {

void cc_default_options(cc_options* opt) {
  if (!opt) return;
  std::memset(opt, 0, sizeof(*opt));
  opt->mode = CC_MODE_AUTO;
  opt->block = 0;
  opt->chunk_arcs = kDefaultChunkArcs;
  opt->tile_vertices = 0;
  opt->timeout_ns = kDefaultTimeoutNs;
}

cc_status cc_create(cc_ctx** out, int device, void* stream, const cc_options* opt) {
  if (!out) return CC_ERR_INVALID_ARG;
  *out = nullptr;
  cc_options o;
  cc_default_options(&o);
  if (opt) {
    if (!options_ok(opt)) return CC_ERR_INVALID_ARG;
    o = *opt;
  }
  resolve_options(&o);
  int n_dev = 0;
  if (cudaGetDeviceCount(&n_dev) != cudaSuccess || device < 0 || device >= n_dev) {
    cudaGetLastError();
    return device < 0 ? CC_ERR_INVALID_ARG : CC_ERR_CUDA;
  }
  DeviceGuard g(device);
  if (!g.ok) return CC_ERR_CUDA;
  cc_ctx* ctx = new (std::nothrow) cc_ctx();
  if (!ctx) return CC_ERR_OOM;
  ctx->device = device;
  ctx->stream = static_cast<cudaStream_t>(stream);
  ctx->opt = o;
  if (cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
    delete ctx;
    cudaGetLastError();
    return CC_ERR_CUDA;
  }
  if (cudaMalloc(&ctx->d_status, sizeof(cc::DevStatus)) != cudaSuccess ||
      cudaMallocHost(&ctx->h_status, sizeof(cc::DevStatus)) != cudaSuccess) {
    cudaGetLastError();
    if (ctx->d_status) cudaFree(ctx->d_status);
    delete ctx;
    return CC_ERR_OOM;
  }
  std::memset(ctx->h_status, 0, sizeof(cc::DevStatus));
  cudaError_t e = cudaMemsetAsync(ctx->d_status, 0, sizeof(cc::DevStatus), ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    cudaFree(ctx->d_status);
    cudaFreeHost(ctx->h_status);
    delete ctx;
    return CC_ERR_CUDA;
  }
  *out = ctx;
  return CC_OK;
}

cc_status cc_set_stream(cc_ctx* ctx, void* stream) {
  if (!ctx) return CC_ERR_INVALID_ARG;
  ctx->stream = static_cast<cudaStream_t>(stream);
  return CC_OK;
}

cc_status cc_set_launch_status(cc_ctx* ctx, int32_t* device_status) {
  if (!ctx) return CC_ERR_INVALID_ARG;
  ctx->status_out = device_status;
  return CC_OK;
}

cc_status cc_set_options(cc_ctx* ctx, const cc_options* opt) {
  if (!ctx || !opt || !options_ok(opt)) return CC_ERR_INVALID_ARG;
  ctx->opt = *opt;
  resolve_options(&ctx->opt);
  return CC_OK;
}

static bool overlaps(const void* a, size_t a_bytes, const void* b, size_t b_bytes) {
  if (!a || !b || a_bytes == 0 || b_bytes == 0) return false;
  const uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
  return x < y + b_bytes && y < x + a_bytes;
}

cc_status cc_labels_csr(cc_ctx* ctx, int64_t n_vertices, int64_t n_arcs, const void* row_ptr,
                        cc_index_type row_ptr_type, const int32_t* col_idx, int32_t* labels) {
  if (!ctx) return CC_ERR_INVALID_ARG;
  if (n_vertices < 0 || n_vertices > INT32_MAX || n_arcs < 0) return CC_ERR_INVALID_ARG;
  if (row_ptr_type != CC_INDEX_I32 && row_ptr_type != CC_INDEX_I64) return CC_ERR_INVALID_ARG;
  if (row_ptr_type == CC_INDEX_I32 && n_arcs > INT32_MAX) return CC_ERR_INVALID_ARG;
  if (!row_ptr) return CC_ERR_INVALID_ARG;
  if (n_vertices > 0 && !labels) return CC_ERR_INVALID_ARG;
  if (n_arcs > 0 && (!col_idx || n_vertices == 0)) return CC_ERR_INVALID_ARG;
  const size_t lab_bytes = (size_t)n_vertices * 4;
  if (overlaps(labels, lab_bytes, row_ptr, (size_t)(n_vertices + 1) * (size_t)row_ptr_type) ||
      overlaps(labels, lab_bytes, col_idx, (size_t)n_arcs * 4))
    return CC_ERR_INVALID_ARG;
  DeviceGuard g(ctx->device);
  if (!g.ok) return CC_ERR_CUDA;
  ctx->last = cc_run_info{};
  if (n_vertices == 0) return finish_empty_call(ctx);
  cc::Problem p{};
  p.kind = cc::kKindCsr;
  p.rp = row_ptr;
  p.rp64 = row_ptr_type == CC_INDEX_I64;
  p.col = col_idx;
  p.pi = labels;
  p.V = (int)n_vertices;
  p.m = n_arcs;
  p.sym = (ctx->opt.flags & CC_FLAG_SYMMETRIC) != 0;
  return run_problem(ctx, p);
}

cc_status cc_labels_csr64(cc_ctx* ctx, int64_t n_vertices, int64_t n_arcs, const int64_t* row_ptr,
                          const int64_t* col_idx, int64_t* labels) {
  if (!ctx) return CC_ERR_INVALID_ARG;
  if (n_vertices < 0 || n_vertices > (INT64_MAX >> 4) || n_arcs < 0 || n_arcs > (INT64_MAX >> 4)) return CC_ERR_INVALID_ARG;
  if (!row_ptr || (n_vertices > 0 && !labels) || (n_arcs > 0 && (!col_idx || n_vertices == 0))) return CC_ERR_INVALID_ARG;
  const size_t lab_bytes = (size_t)n_vertices * 8;
  if (overlaps(labels, lab_bytes, row_ptr, (size_t)(n_vertices + 1) * 8) ||
      overlaps(labels, lab_bytes, col_idx, (size_t)n_arcs * 8))
    return CC_ERR_INVALID_ARG;
  DeviceGuard g(ctx->device);
  if (!g.ok) return CC_ERR_CUDA;
  ctx->last = cc_run_info{};
  if (n_vertices == 0) return finish_empty_call(ctx);
  const cc_options& o = ctx->opt;
  cc::Ctl c;
  c.st = ctx->d_status;
  c.timeout_ns = o.timeout_ns;
  c.status_out = ctx->status_out;
  cudaError_t e = cudaMemsetAsync(ctx->d_status, 0, cc::kPerLaunchStatusBytes, ctx->stream);
  if (e == cudaSuccess && ctx->status_out) e = cudaMemsetAsync(ctx->status_out, 0, sizeof(int32_t), ctx->stream);
  const bool sym = (o.flags & CC_FLAG_SYMMETRIC) != 0;
  const int per_sm = std::max(1, cc::wide_blocks_per_sm(sym));
  const long long want = std::max<long long>(1, (std::max(n_vertices, n_arcs / 4) + 255) / 256);
  const int grid = (int)std::min<long long>(want, (long long)per_sm * usable_sms(ctx));
  if (e == cudaSuccess)
    e = cc::launch_wide(reinterpret_cast<const long long*>(row_ptr), reinterpret_cast<const long long*>(col_idx),
                        reinterpret_cast<long long*>(labels), n_vertices, n_arcs, sym, c, grid, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "64-bit labelling");
  cc_run_info info{};
  info.mode = CC_MODE_MULTI_LAUNCH;
  info.segments = 1;
  info.grid_blocks = grid;
  info.block = 256;
  info.launches = 3;
  ctx->last = info;
  if (o.flags & CC_FLAG_SYNC) return read_and_clear_status(ctx);
  return CC_OK;
}

cc_status cc_labels_coo(cc_ctx* ctx, int64_t n_vertices, int64_t n_edges, const int32_t* src, const int32_t* dst,
                        int32_t* labels) {
  if (!ctx) return CC_ERR_INVALID_ARG;
  if (n_vertices < 0 || n_vertices > INT32_MAX || n_edges < 0) return CC_ERR_INVALID_ARG;
  if (n_vertices > 0 && !labels) return CC_ERR_INVALID_ARG;
  if (n_edges > 0 && (!src || !dst || n_vertices == 0)) return CC_ERR_INVALID_ARG;
  if (overlaps(labels, (size_t)n_vertices * 4, src, (size_t)n_edges * 4) ||
      overlaps(labels, (size_t)n_vertices * 4, dst, (size_t)n_edges * 4))
    return CC_ERR_INVALID_ARG;
  DeviceGuard g(ctx->device);
  if (!g.ok) return CC_ERR_CUDA;
  ctx->last = cc_run_info{};
  if (n_vertices == 0) return finish_empty_call(ctx);
  cc::Problem p{};
  p.kind = cc::kKindCoo;
  p.src = src;
  p.dst = dst;
  p.pi = labels;
  p.V = (int)n_vertices;
  p.m = n_edges;
  p.sym = false;
  cc_options saved = ctx->opt;
  // Section III-B counts |E| edges: a COO edge stands for two arcs.
  ctx->opt.segments = cc::default_segments(2 * n_edges, n_vertices, ctx->opt.segments);
  cc_status st = run_problem(ctx, p);
  ctx->opt = saved;
  return st;
}

// Launches one batch (offset-table or descriptor mode) on the context's stream.
static cc_status run_batch(cc_ctx* ctx, cc::BatchProblem& p, long long total_arcs) {
  const cc_options& o = ctx->opt;
  const int n_graphs = p.n_graphs;
  const long long total_vertices = p.total_v;
  const int W = o.tile_vertices > 0 ? window_for(INT32_MAX, o.tile_vertices) : kBatchedTileVertices;
  int block = o.block > 0 ? o.block : kTiledBlock;
  const bool sym = (o.flags & CC_FLAG_SYMMETRIC) != 0;
  int per_sm = cc::batched_blocks_per_sm(sym, block, W);
  while (per_sm <= 0 && block > 32) {
    block /= 2;
    per_sm = cc::batched_blocks_per_sm(sym, block, W);
  }
  if (per_sm <= 0) return cuda_fail(ctx, cudaErrorInvalidConfiguration, "batched occupancy");
  long long grid = (long long)per_sm * usable_sms(ctx);
  if (o.grid_blocks > 0) grid = std::min<long long>(grid, o.grid_blocks);

  // Scratch: window table, worklist (one pair per vertex, at least 2^20, at most one per arc),
  // and the list of windows hooked arc by arc (at most one entry per window).
  const size_t n_windows = (size_t)(total_vertices / W) + (size_t)n_graphs + 1;
  const size_t cap = (size_t)std::max<long long>(1, std::min<long long>(std::max<long long>(total_arcs, 1),
                                                                        std::max<long long>(total_vertices, 1 << 20)));
  if (grow_buffer(&ctx->d_unit_start, &ctx->d_unit_start_n, (size_t)n_graphs + 1) != cudaSuccess ||
      grow_buffer(&ctx->d_wl, &ctx->d_wl_pairs, cap) != cudaSuccess ||
      grow_buffer(&ctx->d_ovf, &ctx->d_ovf_n, n_windows) != cudaSuccess ||
      grow_buffer(&ctx->d_chunk_start, &ctx->d_chunk_start_n, n_windows + 2) != cudaSuccess ||
      grow_buffer(&ctx->d_hint, &ctx->d_hint_n, (size_t)n_graphs + 1) != cudaSuccess) {
    std::snprintf(ctx->last_error, sizeof(ctx->last_error), "batched scratch allocation failed");
    return CC_ERR_OOM;
  }
  cc::Ctl c;
  c.st = ctx->d_status;
  c.timeout_ns = o.timeout_ns;
  c.tile_w = W;
  c.wl = ctx->d_wl;
  c.wl_cap = ctx->d_wl_pairs;
  c.segments_b = o.segments > 0 ? o.segments : 0;
  c.window_mode = o.tile_vertices == -1 ? cc::kWindowsPlain : cc::kWindowsSampled;
  c.skip_arrival_block = ctx->skip_arrival_block;
  ctx->skip_arrival_block = -1;
  p.unit_start = ctx->d_unit_start;
  p.plain_units = ctx->d_ovf;
  p.plain_cap = (int)std::min<size_t>(std::min(ctx->d_ovf_n, ctx->d_chunk_start_n - 2), INT32_MAX);
  p.plain_chunk_start = ctx->d_chunk_start;
  p.graph_hint = ctx->d_hint;
  p.sym = sym;

  cudaError_t e = cudaMemsetAsync(ctx->d_status, 0, cc::kPerLaunchStatusBytes, ctx->stream);
  if (e == cudaSuccess && ctx->status_out) e = cudaMemsetAsync(ctx->status_out, 0, sizeof(int32_t), ctx->stream);
  c.status_out = ctx->status_out;
  if (e == cudaSuccess && p.graph_status)
    e = cudaMemsetAsync(p.graph_status, 0, sizeof(int32_t) * n_graphs, ctx->stream);
  if (e == cudaSuccess && (o.flags & CC_FLAG_PHASE_TIMES)) {
    if (!ctx->d_phase && cudaMalloc(&ctx->d_phase, kPhaseSlots * sizeof(unsigned long long)) != cudaSuccess) {
      ctx->d_phase = nullptr;
      cudaGetLastError();
      return CC_ERR_OOM;
    }
    e = cudaMemsetAsync(ctx->d_phase, 0, kPhaseSlots * sizeof(unsigned long long), ctx->stream);
    c.phase_ns = ctx->d_phase;
    c.phase_cap = kPhaseSlots;
    ctx->phase_valid = true;
  } else {
    ctx->phase_valid = false;
  }
  if (e == cudaSuccess) e = cc::launch_batched(p, c, cc::LaunchShape{(int)grid, block}, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "batched launch");
  cc_run_info info{};
  info.mode = CC_MODE_PERSISTENT;
  info.segments = o.segments;
  info.grid_blocks = (int)grid;
  info.block = block;
  info.launches = 2;  // phase A with the window in shared memory, then the rest (cc_batched.cu)
  info.tile_vertices = W;
  info.worklist_capacity = (int64_t)ctx->d_wl_pairs;
  ctx->last = info;
  if (o.flags & CC_FLAG_SYNC) return read_and_clear_status(ctx);
  return CC_OK;
}

cc_status cc_labels_batched(cc_ctx* ctx, int32_t n_graphs, int64_t total_vertices, int64_t total_arcs,
                            const int64_t* v_off, const int64_t* a_off, const int32_t* row_ptr_cat,
                            const int32_t* col_idx_cat, int32_t* labels_cat, int32_t* graph_status) {
  if (!ctx) return CC_ERR_INVALID_ARG;
  if (n_graphs < 0 || total_vertices < 0 || total_vertices >= INT32_MAX || total_arcs < 0) return CC_ERR_INVALID_ARG;
  if (n_graphs > 0 && (!v_off || !a_off || !row_ptr_cat)) return CC_ERR_INVALID_ARG;
  if (total_vertices > 0 && !labels_cat) return CC_ERR_INVALID_ARG;
  if (total_arcs > 0 && (!col_idx_cat || total_vertices == 0)) return CC_ERR_INVALID_ARG;
  if (overlaps(labels_cat, (size_t)total_vertices * 4, col_idx_cat, (size_t)total_arcs * 4) ||
      overlaps(labels_cat, (size_t)total_vertices * 4, row_ptr_cat, (size_t)(total_vertices + n_graphs) * 4))
    return CC_ERR_INVALID_ARG;
  DeviceGuard g(ctx->device);
  if (!g.ok) return CC_ERR_CUDA;
  ctx->last = cc_run_info{};
  if (n_graphs == 0) return finish_empty_call(ctx);
  cc::BatchProblem p{};
  p.n_graphs = n_graphs;
  p.v_off = reinterpret_cast<const long long*>(v_off);
  p.a_off = reinterpret_cast<const long long*>(a_off);
  p.rp_cat = row_ptr_cat;
  p.col_cat = col_idx_cat;
  p.labels = labels_cat;
  p.graph_status = graph_status;
  p.total_v = total_vertices;
  return run_batch(ctx, p, total_arcs);
}

cc_status cc_labels_batched_desc(cc_ctx* ctx, int32_t n_graphs, const cc_graph_desc* descs,
                                 const int32_t* row_arena, int64_t row_arena_elems, const int32_t* arc_arena,
                                 int64_t arc_arena_elems, int32_t* label_arena, int64_t label_arena_elems,
                                 int32_t* graph_status) {
  if (!ctx) return CC_ERR_INVALID_ARG;
  if (n_graphs < 0 || label_arena_elems < 0 || label_arena_elems >= INT32_MAX || row_arena_elems < 0 ||
      arc_arena_elems < 0)
    return CC_ERR_INVALID_ARG;
  if (n_graphs > 0 && (!descs || !row_arena || !label_arena)) return CC_ERR_INVALID_ARG;
  if (overlaps(label_arena, (size_t)label_arena_elems * 4, arc_arena, (size_t)arc_arena_elems * 4) ||
      overlaps(label_arena, (size_t)label_arena_elems * 4, row_arena, (size_t)row_arena_elems * 4))
    return CC_ERR_INVALID_ARG;
  DeviceGuard g(ctx->device);
  if (!g.ok) return CC_ERR_CUDA;
  ctx->last = cc_run_info{};
  if (n_graphs == 0) return finish_empty_call(ctx);
  static_assert(sizeof(cc_graph_desc) == sizeof(cc::GraphDesc), "descriptor layouts must agree");
  cc::BatchProblem p{};
  p.n_graphs = n_graphs;
  p.desc = reinterpret_cast<const cc::GraphDesc*>(descs);
  p.rp_cat = row_arena;
  p.col_cat = arc_arena;
  p.labels = label_arena;
  p.graph_status = graph_status;
  p.total_v = label_arena_elems;
  p.row_elems = row_arena_elems;
  p.arc_elems = arc_arena_elems;
  return run_batch(ctx, p, std::max<long long>(arc_arena_elems, 1));
}

static cc_status grow(cc_ctx* ctx, void** buf, size_t* have, size_t need) {
  if (need <= *have) return CC_OK;
  if (*buf) cudaFree(*buf);
  *buf = nullptr;
  *have = 0;
  if (cudaMalloc(buf, need) != cudaSuccess) {
    cudaGetLastError();
    *buf = nullptr;
    std::snprintf(ctx->last_error, sizeof(ctx->last_error), "staging allocation of %zu bytes failed", need);
    return CC_ERR_OOM;
  }
  *have = need;
  return CC_OK;
}

// Arcs per streamed segment for cc_labels_csr_host (0 = copy the whole graph, then label it; -1 =
// not even row_ptr and labels fit). cc_options.stream_arcs > 0 is taken as given and -1 never
// streams. Automatically (0): only a graph that does not fit in free device memory next to a
// margin streams, through two buffers sized from the memory left after row_ptr and labels.
// (Streaming a graph that fits, to hide the labelling under the copy, measured on GB300: R-MAT 26
// 46.7 -> 45.3 ms per call in the median, but the host link's occasional stalls of 50-180 ms hit
// the streamed calls more often, 71.8 against 53.9 ms in the mean of 20 calls; the 4096^2 grid
// 2.2 -> 2.7 ms, the Multi-Jumps after every segment outweighing the copy.)
static long long stream_segment_arcs(cc_ctx* ctx, size_t rp_bytes, size_t col_bytes, size_t lab_bytes) {
  if (ctx->opt.stream_arcs > 0) return ctx->opt.stream_arcs;
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  const size_t avail = free_b + ctx->d_rp_bytes + ctx->d_col_bytes + ctx->d_labels_bytes +
                       2 * ctx->d_seg_arcs * sizeof(int32_t);  // buffers this call may reuse
  const size_t margin = (size_t)1 << 30;
  if (rp_bytes + col_bytes + lab_bytes + margin <= avail) return 0;
  if (ctx->opt.stream_arcs < 0) return -1;
  const size_t min_seg_bytes = (size_t)1 << 22;
  if (rp_bytes + lab_bytes + margin + 2 * min_seg_bytes > avail) return -1;
  const size_t seg_bytes = std::min<size_t>((avail - rp_bytes - lab_bytes - margin) / 2, (size_t)1 << 30);
  return (long long)(seg_bytes / sizeof(int32_t));
}

// Fig. 4 with the arcs left in host memory: row_ptr and labels (pi) live on the device, and the
// s = ceil(n_arcs / seg) segments of the arc array are copied in one after the other on a copy
// stream, into two device buffers used in turn. Segment i is Atomic-Hooked (plain hook) as soon
// as it has landed, while segment i + 1 is copied; a Multi-Jump follows every segment. The
// device holds 4 (V + 1) or 8 (V + 1) + 4 V + 8 seg bytes, whatever n_arcs is.
static cc_status run_streamed(cc_ctx* ctx, int64_t n_vertices, int64_t n_arcs, const void* row_ptr,
                              cc_index_type row_ptr_type, const int32_t* col_idx, int32_t* labels, long long seg) {
  const cc_options& o = ctx->opt;
  const size_t rp_bytes = (size_t)(n_vertices + 1) * (size_t)row_ptr_type;
  const size_t lab_bytes = (size_t)n_vertices * sizeof(int32_t);
  // the resident arc buffer of the non-streamed path is not needed here
  if (ctx->d_col) {
    cudaFree(ctx->d_col);
    ctx->d_col = nullptr;
    ctx->d_col_bytes = 0;
  }
  cc_status st = grow(ctx, &ctx->d_rp, &ctx->d_rp_bytes, std::max<size_t>(rp_bytes, 16));
  if (st == CC_OK) st = grow(ctx, (void**)&ctx->d_labels, &ctx->d_labels_bytes, std::max<size_t>(lab_bytes, 16));
  if (st != CC_OK) return st;
  if (ctx->d_seg_arcs < (size_t)seg) {
    for (int b = 0; b < 2; ++b) {
      if (ctx->d_seg[b]) cudaFree(ctx->d_seg[b]);
      ctx->d_seg[b] = nullptr;
    }
    ctx->d_seg_arcs = 0;
    for (int b = 0; b < 2; ++b) {
      if (cudaMalloc(&ctx->d_seg[b], (size_t)seg * sizeof(int32_t)) != cudaSuccess) {
        cudaGetLastError();
        std::snprintf(ctx->last_error, sizeof(ctx->last_error), "segment buffer of %lld arcs failed", seg);
        return CC_ERR_OOM;
      }
    }
    ctx->d_seg_arcs = (size_t)seg;
  }
  if (!ctx->copy_stream) {
    if (cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      ctx->copy_stream = nullptr;
      return cuda_fail(ctx, cudaErrorUnknown, "copy stream");
    }
    for (int b = 0; b < 2; ++b) {
      if (cudaEventCreateWithFlags(&ctx->seg_copied[b], cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&ctx->seg_used[b], cudaEventDisableTiming) != cudaSuccess)
        return cuda_fail(ctx, cudaGetLastError(), "segment events");
    }
  }
  cudaStream_t s = ctx->stream;
  cc::Problem p{};
  p.kind = cc::kKindCsr;
  p.rp = ctx->d_rp;
  p.rp64 = row_ptr_type == CC_INDEX_I64;
  p.col = nullptr;  // not resident
  p.pi = ctx->d_labels;
  p.V = (int)n_vertices;
  p.m = n_arcs;
  p.sym = (o.flags & CC_FLAG_SYMMETRIC) != 0;
  const long long n_seg = (n_arcs + seg - 1) / seg;
  p.segments = (int)std::min<long long>(n_seg, INT32_MAX);
  cc::Ctl c;
  c.st = ctx->d_status;
  c.timeout_ns = o.timeout_ns;
  c.status_out = ctx->status_out;
  const int block = o.block > 0 ? o.block : kPlainBlock;
  const int per_sm = std::max(1, cc::stage_blocks_per_sm(p, block));
  const long long work = std::max<long long>(p.V, std::min<long long>(n_arcs, seg) / 4);
  const long long grid = std::max<long long>(1, std::min<long long>((work + block - 1) / block,
                                                                    (long long)per_sm * usable_sms(ctx)));
  const cc::LaunchShape shape{(int)grid, block};
  cudaError_t e = cudaMemsetAsync(ctx->d_status, 0, cc::kPerLaunchStatusBytes, s);
  if (e == cudaSuccess && ctx->status_out) e = cudaMemsetAsync(ctx->status_out, 0, sizeof(int32_t), s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ctx->d_rp, row_ptr, rp_bytes, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cc::launch_init_only(p, c, shape, s);
  cc_run_info info{};
  info.mode = CC_MODE_MULTI_LAUNCH;
  info.segments = p.segments;
  info.grid_blocks = (int)grid;
  info.block = block;
  info.launches = 1;
  info.streamed_segments = p.segments;
  for (long long i = 0; i < n_seg && e == cudaSuccess; ++i) {
    const int b = (int)(i & 1);
    const long long a0 = i * seg, a1 = std::min<long long>(n_arcs, a0 + seg);
    if (i >= 2) e = cudaStreamWaitEvent(ctx->copy_stream, ctx->seg_used[b], 0);  // buffer free again
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(ctx->d_seg[b], col_idx + a0, (size_t)(a1 - a0) * sizeof(int32_t), cudaMemcpyHostToDevice,
                          ctx->copy_stream);
    if (e == cudaSuccess) e = cudaEventRecord(ctx->seg_copied[b], ctx->copy_stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ctx->seg_copied[b], 0);
    c.chunk_arcs = o.chunk_arcs != 0 ? o.chunk_arcs : cc::auto_chunk_arcs(a1 - a0, grid * (block / 32));
    if (e == cudaSuccess) e = cc::launch_hook_segment(p, ctx->d_seg[b], a0, a1, c, shape, s);
    if (e == cudaSuccess) e = cudaEventRecord(ctx->seg_used[b], s);
    if (e == cudaSuccess) e = cc::launch_jump_multi(p, c, shape, s);  // Multi-Jump after every segment
    info.launches += 2;
  }
  if (e == cudaSuccess && lab_bytes) e = cudaMemcpyAsync(labels, ctx->d_labels, lab_bytes, cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "streamed labelling");
  ctx->last = info;
  return read_and_clear_status(ctx);
}

cc_status cc_labels_csr_host(cc_ctx* ctx, int64_t n_vertices, int64_t n_arcs, const void* row_ptr,
                             cc_index_type row_ptr_type, const int32_t* col_idx, int32_t* labels) {
  if (!ctx) return CC_ERR_INVALID_ARG;
  if (n_vertices < 0 || n_vertices > INT32_MAX || n_arcs < 0 || !row_ptr) return CC_ERR_INVALID_ARG;
  if (row_ptr_type != CC_INDEX_I32 && row_ptr_type != CC_INDEX_I64) return CC_ERR_INVALID_ARG;
  if (n_vertices > 0 && !labels) return CC_ERR_INVALID_ARG;
  if (n_arcs > 0 && !col_idx) return CC_ERR_INVALID_ARG;
  DeviceGuard g(ctx->device);
  if (!g.ok) return CC_ERR_CUDA;
  const size_t rp_bytes = (size_t)(n_vertices + 1) * (size_t)row_ptr_type;
  const size_t col_bytes = (size_t)n_arcs * sizeof(int32_t);
  const size_t lab_bytes = (size_t)n_vertices * sizeof(int32_t);
  if (n_vertices > 0 && n_arcs > 0) {
    const long long seg = stream_segment_arcs(ctx, rp_bytes, col_bytes, lab_bytes);
    if (seg < 0) {
      std::snprintf(ctx->last_error, sizeof(ctx->last_error), "the graph does not fit on the device");
      return CC_ERR_OOM;
    }
    if (seg > 0 && seg < n_arcs) {
      ctx->last = cc_run_info{};
      return run_streamed(ctx, n_vertices, n_arcs, row_ptr, row_ptr_type, col_idx, labels, seg);
    }
  }
  cc_status st = grow(ctx, &ctx->d_rp, &ctx->d_rp_bytes, std::max<size_t>(rp_bytes, 16));
  if (st == CC_OK) st = grow(ctx, (void**)&ctx->d_col, &ctx->d_col_bytes, std::max<size_t>(col_bytes, 16));
  if (st == CC_OK) st = grow(ctx, (void**)&ctx->d_labels, &ctx->d_labels_bytes, std::max<size_t>(lab_bytes, 16));
  if (st != CC_OK) return st;
  cudaError_t e = cudaMemcpyAsync(ctx->d_rp, row_ptr, rp_bytes, cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess && col_bytes)
    e = cudaMemcpyAsync(ctx->d_col, col_idx, col_bytes, cudaMemcpyHostToDevice, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "host-to-device copy");
  const int saved_flags = ctx->opt.flags;
  ctx->opt.flags &= ~CC_FLAG_SYNC;
  st = cc_labels_csr(ctx, n_vertices, n_arcs, ctx->d_rp, row_ptr_type, ctx->d_col, ctx->d_labels);
  ctx->opt.flags = saved_flags;
  if (st != CC_OK) return st;
  if (lab_bytes) {
    e = cudaMemcpyAsync(labels, ctx->d_labels, lab_bytes, cudaMemcpyDeviceToHost, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "device-to-host copy");
  }
  return read_and_clear_status(ctx);
}

cc_status cc_sync(cc_ctx* ctx) {
  if (!ctx) return CC_ERR_INVALID_ARG;
  DeviceGuard g(ctx->device);
  if (!g.ok) return CC_ERR_CUDA;
  return read_and_clear_status(ctx);
}

cc_status cc_last_run_info(const cc_ctx* ctx, cc_run_info* info) {
  if (!ctx || !info) return CC_ERR_INVALID_ARG;
  *info = ctx->last;
  return CC_OK;
}

cc_status cc_last_phase_times(cc_ctx* ctx, int64_t* ns, int32_t cap, int32_t* n) {
  if (!ctx || !ns || !n || cap <= 0) return CC_ERR_INVALID_ARG;
  *n = 0;
  if (!ctx->d_phase || !ctx->phase_valid) return CC_OK;
  DeviceGuard g(ctx->device);
  if (!g.ok) return CC_ERR_CUDA;
  unsigned long long host[kPhaseSlots];
  cudaError_t e = cudaMemcpyAsync(host, ctx->d_phase, sizeof(host), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cc_last_phase_times");
  // slot 0 = start, slots 1.. = barriers passed (until the first unused slot), last slot = end
  int used = 1;
  while (used < kPhaseSlots - 1 && host[used] != 0) ++used;
  const int m = std::min(used + 1, (int)cap);
  for (int i = 0; i < m; ++i) {
    const unsigned long long t = (i == used) ? host[kPhaseSlots - 1] : host[i];
    ns[i] = t >= host[0] ? (int64_t)(t - host[0]) : 0;
  }
  *n = m;
  return CC_OK;
}

cc_status cc_last_worklist(cc_ctx* ctx, int64_t* pairs, int32_t* segments) {
  if (!ctx || !pairs || !segments) return CC_ERR_INVALID_ARG;
  DeviceGuard g(ctx->device);
  if (!g.ok) return CC_ERR_CUDA;
  cc::DevStatus host;
  cudaError_t e = cudaMemcpyAsync(&host, ctx->d_status, sizeof(host), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cc_last_worklist");
  *pairs = (int64_t)host.report[0];
  *segments = (int32_t)host.report[1];
  return CC_OK;
}

const char* cc_last_error_message(const cc_ctx* ctx) { return ctx ? ctx->last_error : ""; }

const char* cc_status_string(cc_status s) {
  switch (s) {
    case CC_OK: return "CC_OK";
    case CC_ERR_INVALID_ARG: return "CC_ERR_INVALID_ARG: invalid argument";
    case CC_ERR_OUT_OF_RANGE: return "CC_ERR_OUT_OF_RANGE: endpoint outside [0, V) or malformed offsets";
    case CC_ERR_OOM: return "CC_ERR_OOM: allocation failed";
    case CC_ERR_CUDA: return "CC_ERR_CUDA: CUDA runtime error";
    case CC_ERR_TIMEOUT: return "CC_ERR_TIMEOUT: a device-side wait exceeded its limit";
    case CC_ERR_INTERNAL: return "CC_ERR_INTERNAL: device iteration guard fired";
  }
  return "unknown cc_status";
}

void cc_destroy(cc_ctx* ctx) {
  if (!ctx) return;
  {
    DeviceGuard g(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    if (ctx->d_rp) cudaFree(ctx->d_rp);
    if (ctx->d_col) cudaFree(ctx->d_col);
    if (ctx->d_labels) cudaFree(ctx->d_labels);
    for (int b = 0; b < 2; ++b) {
      if (ctx->d_seg[b]) cudaFree(ctx->d_seg[b]);
      if (ctx->seg_copied[b]) cudaEventDestroy(ctx->seg_copied[b]);
      if (ctx->seg_used[b]) cudaEventDestroy(ctx->seg_used[b]);
    }
    if (ctx->copy_stream) {
      cudaStreamSynchronize(ctx->copy_stream);
      cudaStreamDestroy(ctx->copy_stream);
    }
    if (ctx->d_phase) cudaFree(ctx->d_phase);
    if (ctx->d_wl) cudaFree(ctx->d_wl);
    if (ctx->d_ovf) cudaFree(ctx->d_ovf);
    if (ctx->d_unit_start) cudaFree(ctx->d_unit_start);
    if (ctx->d_chunk_start) cudaFree(ctx->d_chunk_start);
    if (ctx->d_hint) cudaFree(ctx->d_hint);
    if (ctx->d_sample) cudaFree(ctx->d_sample);
    if (ctx->h_sample) cudaFreeHost(ctx->h_sample);
    if (ctx->d_status) cudaFree(ctx->d_status);
    if (ctx->h_status) cudaFreeHost(ctx->h_status);
    cudaGetLastError();
  }
  delete ctx;
}

cc_status cc_debug_skip_barrier_arrival(cc_ctx* ctx, int32_t block) {
  if (!ctx) return CC_ERR_INVALID_ARG;
  ctx->skip_arrival_block = block;
  return CC_OK;
}

}  // extern "C"
