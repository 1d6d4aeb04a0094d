// Single-graph kernels: the persistent driver of Fig. 4 (one cooperative launch, grid
// barriers between Hook and Multi-Jump phases), the two launches of the hierarchical hook, and
// the per-phase kernels of a host-driven loop (one launch per Hook and per Multi-Jump), for CSR (int32 / int64 offsets, plain or
// symmetrised) and COO inputs.
#include "cc_internal.h"

namespace cc {

namespace {

constexpr int kMaxBlock = 1024;

__device__ __forceinline__ long long global_tid() {
  return (long long)blockIdx.x * blockDim.x + threadIdx.x;
}
__device__ __forceinline__ long long global_threads() { return (long long)gridDim.x * blockDim.x; }

__device__ __forceinline__ void phase_start(const Ctl& c) {
  if (c.phase_ns && blockIdx.x == 0 && threadIdx.x == 0) c.phase_ns[0] = now_ns();
}
__device__ __forceinline__ void phase_end(const Ctl& c) {
  if (c.phase_ns && threadIdx.x == 0) atomicMax(c.phase_ns + (c.phase_cap - 1), now_ns());
}

__device__ __forceinline__ unsigned long long ld_volatile_u64(const unsigned long long* p) {
  return *reinterpret_cast<const volatile unsigned long long*>(p);
}

// Adaptive Hook-Compress (Fig. 4) over the arcs of a CSR graph, in one launch: init pi; for i
// in 1..s: Atomic-Hook(E_i); barrier; Multi-Jump(V); barrier. Hook phase i takes its work from
// counter i % 2; thread 0 zeroes the other counter during the phase, and the barriers in
// between publish the reset before its next use.
template <typename OffT, bool SYM>
__device__ __forceinline__ void csr_persistent_body(const OffT* __restrict__ rp, const int* __restrict__ col,
                                                    int* pi, int V, OffT nnz, int s, const Ctl& c) {
  if (launch_blocked(c)) return;  // a pending fatal error or a failed validation stops device work
  unsigned epoch = 0;
  const long long tid = global_tid(), nt = global_threads();
  init_pi(pi, V, tid, nt);
  if (!grid_sync(c, epoch)) return;
  for (int i = 0; i < s; ++i) {
    if (tid == 0) c.st->counters[(i + 1) % kWorkCounters] = 0ull;
    const OffT a0 = split_point<OffT>(nnz, s, i);
    const OffT a1 = split_point<OffT>(nnz, s, i + 1);
    hook_csr_arcs<OffT, SYM>(rp, col, pi, V, a0, a1, tid, nt, &c.st->counters[i % kWorkCounters], c);
    if (!grid_sync(c, epoch)) return;
    multi_jump(pi, V, tid, nt, c);
    if (i + 1 < s && !grid_sync(c, epoch)) return;
  }
}

template <typename OffT, bool SYM>
__global__ void __launch_bounds__(kMaxBlock, 2) k_csr_persistent(const OffT* __restrict__ rp,
                                                                 const int* __restrict__ col, int* pi, int V,
                                                                 OffT nnz, int s, Ctl c) {
  phase_start(c);
  csr_persistent_body<OffT, SYM>(rp, col, pi, V, nnz, s, c);
  phase_end(c);
}

// Sampled-and-filtered hook (CSR, CC_FLAG_SYMMETRIC), one cooperative launch: init pi; hook the
// first kSampleArcs arcs of every row; Multi-Jump; estimate the largest star's root (block 0,
// published in counters[3]); hook the remaining arcs of the rows outside that star (or, without
// a large star, every arc with the plain hook); Multi-Jump.
template <typename OffT>
__global__ void __launch_bounds__(kMaxBlock, 2) k_csr_filtered(const OffT* __restrict__ rp,
                                                               const int* __restrict__ col, int* pi, int V, OffT nnz,
                                                               Ctl c) {
  phase_start(c);
  if (!launch_blocked(c)) {
    unsigned epoch = 0;
    const long long tid = global_tid(), nt = global_threads();
    init_pi(pi, V, tid, nt);
    bool go = grid_sync(c, epoch);
    if (go) {
      hook_row_heads<OffT>(rp, col, pi, V, nnz, tid, nt, c);
      go = grid_sync(c, epoch);
    }
    if (go) {
      multi_jump(pi, V, tid, nt, c);
      go = grid_sync(c, epoch);
    }
    if (go) {
      if (blockIdx.x == 0) {
        const int g = giant_root(pi, V);
        if (threadIdx.x == 0) c.st->counters[3] = (unsigned long long)(unsigned)g;
      }
      go = grid_sync(c, epoch);
    }
    if (go) {
      const int g = (int)(unsigned)ld_volatile_u64(&c.st->counters[3]);
      if (g >= 0) hook_rows_outside<OffT>(rp, col, pi, V, nnz, g, tid, nt, c);
      else hook_csr_arcs<OffT, true>(rp, col, pi, V, (OffT)0, nnz, tid, nt, &c.st->counters[0], c);
      go = grid_sync(c, epoch);
    }
    if (go) multi_jump(pi, V, tid, nt, c);
  }
  phase_end(c);
}

// Two-phase hierarchical hook, first launch: phase A (window-local hooks in shared memory, pi
// written, worklist E' built). Windows are taken from a work counter, so the grid needs no
// co-residency; at the default window two 1024-thread CTAs share an SM.
template <typename OffT, bool SYM>
__global__ void __launch_bounds__(kMaxBlock, 2) k_phase_a(const OffT* __restrict__ rp, const int* __restrict__ col,
                                                          int* pi, int V, OffT nnz, Ctl c) {
  extern __shared__ __align__(16) unsigned char dyn_smem_a[];
  phase_start(c);
  if (!launch_blocked(c)) tiled_phase_a<OffT, SYM, int>(rp, col, pi, V, nnz, dyn_smem_a, c);
  if (c.phase_ns && threadIdx.x == 0) atomicMax(c.phase_ns + 1, now_ns());
}

// Second launch (cooperative): Fig. 4 over E', s' = 2|E'|/|V| segments, each Atomic-Hook on pi
// followed by Multi-Jump(V). The windows whose worklist appends overflowed are hooked arc by
// arc in the first segment.
template <typename OffT, bool SYM>
__global__ void __launch_bounds__(kMaxBlock, 1) k_phase_b(const OffT* __restrict__ rp, const int* __restrict__ col,
                                                          int* pi, int V, OffT nnz, Ctl c) {
  if (!launch_blocked(c)) {
    unsigned epoch = 0;
    const long long tid = global_tid(), nt = global_threads();
    const unsigned long long cur = ld_volatile_u64(&c.st->counters[2]);
    const unsigned long long n_pairs = cur < c.wl_cap ? cur : c.wl_cap;
    unsigned long long n_ovf = ld_volatile_u64(&c.st->counters[3]);
    n_ovf = n_ovf < (unsigned long long)c.ovf_cap ? n_ovf : (unsigned long long)c.ovf_cap;
    if (n_pairs != 0 || n_ovf != 0) {  // else every tree is already a star rooted at its minimum
      long long s2 = c.segments_b;
      if (s2 <= 0) s2 = (long long)((2.0 * (double)n_pairs) / (double)V + 0.5);
      s2 = s2 < 1 ? 1 : (s2 > 4096 ? 4096 : s2);
      if (tid == 0) {
        c.st->report[0] = n_pairs;
        c.st->report[1] = (unsigned long long)s2;
      }
      for (long long i = 0; i < s2; ++i) {
        tiled_phase_b<OffT, SYM>(rp, col, pi, V, nnz, split_point<unsigned long long>(n_pairs, s2, i),
                                 split_point<unsigned long long>(n_pairs, s2, i + 1), i == 0, n_ovf, tid, nt, c);
        if (!grid_sync(c, epoch)) break;
        multi_jump(pi, V, tid, nt, c);
        if (i + 1 < s2 && !grid_sync(c, epoch)) break;
      }
    }
  }
  phase_end(c);
}

__device__ __forceinline__ void coo_persistent_body(const int* __restrict__ src, const int* __restrict__ dst,
                                                    int* pi, int V, long long E, int s, const Ctl& c) {
  if (launch_blocked(c)) return;
  unsigned epoch = 0;
  const long long tid = global_tid(), nt = global_threads();
  init_pi(pi, V, tid, nt);
  if (!grid_sync(c, epoch)) return;
  for (int i = 0; i < s; ++i) {
    hook_coo_edges(src, dst, pi, V, split_point<long long>(E, s, i), split_point<long long>(E, s, i + 1), tid, nt,
                   c);
    if (!grid_sync(c, epoch)) return;
    multi_jump(pi, V, tid, nt, c);
    if (i + 1 < s && !grid_sync(c, epoch)) return;
  }
}

__global__ void __launch_bounds__(kMaxBlock, 1) k_coo_persistent(const int* __restrict__ src,
                                                              const int* __restrict__ dst, int* pi, int V,
                                                              long long E, int s, Ctl c) {
  phase_start(c);
  coo_persistent_body(src, dst, pi, V, E, s, c);
  phase_end(c);
}

// ----- per-phase kernels (the host loop of Fig. 4) -----
// Work counter 0 is zeroed by the kernel before each hook kernel (init or jump); the
// launches are stream-ordered, so no hook kernel overlaps a reset.

__global__ void __launch_bounds__(kMaxBlock) k_init(int* pi, int V, Ctl c) {
  if (global_tid() == 0) c.st->counters[0] = 0ull;
  if (launch_blocked(c)) return;
  init_pi(pi, V, global_tid(), global_threads());
}

template <typename OffT, bool SYM>
__global__ void __launch_bounds__(kMaxBlock) k_hook_csr(const OffT* __restrict__ rp, const int* __restrict__ col,
                                                        int* pi, int V, OffT a0, OffT a1, Ctl c) {
  if (launch_blocked(c)) return;
  hook_csr_arcs<OffT, SYM>(rp, col, pi, V, a0, a1, global_tid(), global_threads(), &c.st->counters[0], c);
}

__global__ void __launch_bounds__(kMaxBlock) k_hook_coo(const int* __restrict__ src, const int* __restrict__ dst,
                                                        int* pi, int V, long long e0, long long e1, Ctl c) {
  if (launch_blocked(c)) return;
  hook_coo_edges(src, dst, pi, V, e0, e1, global_tid(), global_threads(), c);
}

template <typename OffT, bool SYM>
__global__ void __launch_bounds__(kMaxBlock) k_hook_csr_nonatomic(const OffT* __restrict__ rp,
                                                                  const int* __restrict__ col, int* pi, int V, OffT nnz,
                                                                  Ctl c) {
  if (launch_blocked(c)) return;
  hook_csr_arcs<OffT, SYM, kHookNonAtomic>(rp, col, pi, V, (OffT)0, nnz, global_tid(), global_threads(), nullptr, c);
}

__global__ void __launch_bounds__(kMaxBlock) k_jump_single(int* pi, int V, Ctl c) {
  if (launch_blocked(c)) return;
  single_jump(pi, V, global_tid(), global_threads(), c);
}

__global__ void __launch_bounds__(kMaxBlock) k_jump(int* pi, int V, Ctl c) {
  if (global_tid() == 0) c.st->counters[0] = 0ull;
  if (launch_blocked(c)) return;
  multi_jump(pi, V, global_tid(), global_threads(), c);
}

// ----- locality sample (automatic choice of the hook variant) -----
// Thread t looks at the middle arc of row t * V / T and counts it as local when both ends lie
// in the same window of W vertices. out[0] += local arcs, out[1] += sampled arcs.
template <typename OffT>
__global__ void __launch_bounds__(256) k_sample_locality(const OffT* __restrict__ rp, const int* __restrict__ col,
                                                         int V, OffT nnz, int W, unsigned long long* out) {
  const long long t = global_tid(), T = global_threads();
  const int u = (int)((t * (long long)V) / T);
  bool sampled = false, local = false, row = false, low = false;
  if (u < V) {
    const OffT a0 = rp[u], a1 = rp[u + 1];
    if (a0 >= 0 && a0 <= a1 && a1 <= nnz) {
      row = true;
      low = 4.0 * (double)(a1 - a0) * (double)V < (double)nnz;  // degree below a quarter of the mean
    }
    if (a0 >= 0 && a0 < a1 && a1 <= nnz) {
      const int v = col[a0 + (a1 - a0) / 2];
      if ((unsigned)v < (unsigned)V && v != u) {
        sampled = true;
        local = (u / W) == (v / W);
      }
    }
  }
  const unsigned ns = __popc(__ballot_sync(kFull, sampled));
  const unsigned nl = __popc(__ballot_sync(kFull, local));
  const unsigned nr = __popc(__ballot_sync(kFull, row));
  const unsigned nlow = __popc(__ballot_sync(kFull, low));
  if ((threadIdx.x & 31) == 0 && ns) {
    atomicAdd(out, (unsigned long long)nl);
    atomicAdd(out + 1, (unsigned long long)ns);
  }
  if ((threadIdx.x & 31) == 0 && nr) {
    atomicAdd(out + 2, (unsigned long long)nlow);
    atomicAdd(out + 3, (unsigned long long)nr);
  }
}

// ----- validation (CC_FLAG_VALIDATE) -----
// A failed check is reported as an input error and stops the rest of the call (DevStatus::abort),
// so the hooks never follow offsets found bad.
__device__ __forceinline__ void fail_validation(const Ctl& c, long long info) {
  raise_input_error(c, kSiteValidate, info);
  c.st->abort = 1u;
}

template <typename OffT>
__global__ void __launch_bounds__(kMaxBlock) k_validate_csr(const OffT* __restrict__ rp, const int* __restrict__ col,
                                                            int V, OffT nnz, Ctl c) {
  const long long tid = global_tid(), nt = global_threads();
  if (tid == 0 && (rp[0] != 0 || rp[V] != nnz)) fail_validation(c, -1);
  for (long long v = tid; v < V; v += nt)
    if (rp[v + 1] < rp[v]) fail_validation(c, v);
  for (long long a = tid; a < (long long)nnz; a += nt)
    if ((unsigned)col[a] >= (unsigned)V) fail_validation(c, a);
}

__global__ void __launch_bounds__(kMaxBlock) k_validate_coo(const int* __restrict__ src, const int* __restrict__ dst,
                                                            int V, long long E, Ctl c) {
  for (long long i = global_tid(); i < E; i += global_threads())
    if ((unsigned)src[i] >= (unsigned)V || (unsigned)dst[i] >= (unsigned)V)
      fail_validation(c, i);
}

// ----- host helpers -----

template <typename F>
int blocks_per_sm(F kernel, int block, size_t smem) {
  if (smem > 48 * 1024 &&
      cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, block, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

template <typename... Args>
cudaError_t launch_kernel(void (*kernel)(Args...), LaunchShape s, size_t smem, bool coop, cudaStream_t stream,
                          Args... args) {
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)s.grid);
  cfg.blockDim = dim3((unsigned)s.block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = coop ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// Calls f(kernel) with the cooperative CSR kernel of p: the plain persistent driver, or phase B
// of the hierarchical hook.
template <typename OffT, typename F>
auto with_csr_persistent(const Problem& p, F&& f) {
  const bool tiled = p.tile_w > 0;
  if (p.sym) return tiled ? f(k_phase_b<OffT, true>) : f(k_csr_persistent<OffT, true>);
  return tiled ? f(k_phase_b<OffT, false>) : f(k_csr_persistent<OffT, false>);
}

template <typename OffT, typename F>
auto with_phase_a(const Problem& p, F&& f) {
  return p.sym ? f(k_phase_a<OffT, true>) : f(k_phase_a<OffT, false>);
}

template <typename OffT, typename F>
auto with_phase_b(const Problem& p, F&& f) {
  return p.sym ? f(k_phase_b<OffT, true>) : f(k_phase_b<OffT, false>);
}

template <typename OffT, typename F>
auto with_csr_hook(const Problem& p, F&& f) {
  return p.sym ? f(k_hook_csr<OffT, true>) : f(k_hook_csr<OffT, false>);
}

}  // namespace

size_t phase_a_smem_bytes(const Problem& p, int block) {
  return tiled_smem_bytes(p.tile_w, block, (int)sizeof(int));
}

int persistent_blocks_per_sm(const Problem& p, int block) {
  if (p.kind == kKindCoo) return blocks_per_sm(k_coo_persistent, block, 0);
  if (p.filtered)
    return p.rp64 ? blocks_per_sm(k_csr_filtered<long long>, block, 0) : blocks_per_sm(k_csr_filtered<int>, block, 0);
  auto occ = [&](auto k) { return blocks_per_sm(k, block, 0); };
  return p.rp64 ? with_csr_persistent<long long>(p, occ) : with_csr_persistent<int>(p, occ);
}

int phase_a_blocks_per_sm(const Problem& p, int block) {
  const size_t smem = phase_a_smem_bytes(p, block);
  auto occ = [&](auto k) { return blocks_per_sm(k, block, smem); };
  return p.rp64 ? with_phase_a<long long>(p, occ) : with_phase_a<int>(p, occ);
}

int stage_blocks_per_sm(const Problem& p, int block) {
  if (p.kind == kKindCoo) return blocks_per_sm(k_hook_coo, block, 0);
  auto occ = [&](auto k) { return blocks_per_sm(k, block, 0); };
  return p.rp64 ? with_csr_hook<long long>(p, occ) : with_csr_hook<int>(p, occ);
}

cudaError_t launch_persistent(const Problem& p, const Ctl& c, LaunchShape s, cudaStream_t stream) {
  if (p.kind == kKindCoo)
    return launch_kernel(k_coo_persistent, s, 0, true, stream, p.src, p.dst, p.pi, p.V, p.m, p.segments, c);
  if (p.filtered) {
    if (p.rp64)
      return launch_kernel(k_csr_filtered<long long>, s, 0, true, stream, static_cast<const long long*>(p.rp), p.col,
                           p.pi, p.V, (long long)p.m, c);
    return launch_kernel(k_csr_filtered<int>, s, 0, true, stream, static_cast<const int*>(p.rp), p.col, p.pi, p.V,
                         (int)p.m, c);
  }
  if (p.rp64) {
    const long long* rp = static_cast<const long long*>(p.rp);
    return p.sym ? launch_kernel(k_csr_persistent<long long, true>, s, 0, true, stream, rp, p.col, p.pi, p.V,
                                 (long long)p.m, p.segments, c)
                 : launch_kernel(k_csr_persistent<long long, false>, s, 0, true, stream, rp, p.col, p.pi, p.V,
                                 (long long)p.m, p.segments, c);
  }
  const int* rp = static_cast<const int*>(p.rp);
  return p.sym ? launch_kernel(k_csr_persistent<int, true>, s, 0, true, stream, rp, p.col, p.pi, p.V, (int)p.m,
                               p.segments, c)
               : launch_kernel(k_csr_persistent<int, false>, s, 0, true, stream, rp, p.col, p.pi, p.V, (int)p.m,
                               p.segments, c);
}

cudaError_t launch_two_phase(const Problem& p, const Ctl& c, LaunchShape sa, LaunchShape sb, cudaStream_t stream) {
  const size_t smem = phase_a_smem_bytes(p, sa.block);
  Ctl cb = c;
  cb.phase_off = 1;  // slot 1 holds the end of phase A
  if (p.rp64) {
    const long long* rp = static_cast<const long long*>(p.rp);
    cudaError_t e = with_phase_a<long long>(p, [&](auto k) {
      return launch_kernel(k, sa, smem, false, stream, rp, p.col, p.pi, p.V, (long long)p.m, c);
    });
    if (e != cudaSuccess) return e;
    return with_phase_b<long long>(p, [&](auto k) {
      return launch_kernel(k, sb, 0, true, stream, rp, p.col, p.pi, p.V, (long long)p.m, cb);
    });
  }
  const int* rp = static_cast<const int*>(p.rp);
  cudaError_t e = with_phase_a<int>(p, [&](auto k) {
    return launch_kernel(k, sa, smem, false, stream, rp, p.col, p.pi, p.V, (int)p.m, c);
  });
  if (e != cudaSuccess) return e;
  return with_phase_b<int>(p, [&](auto k) {
    return launch_kernel(k, sb, 0, true, stream, rp, p.col, p.pi, p.V, (int)p.m, cb);
  });
}

cudaError_t launch_multi(const Problem& p, const Ctl& c, LaunchShape s, cudaStream_t stream, int* launches) {
  int n = 0;
  cudaError_t e = launch_kernel(k_init, s, 0, false, stream, p.pi, p.V, c);
  if (e != cudaSuccess) return e;
  ++n;
  const size_t smem = 0;  // the per-phase kernels use the plain hook
  for (int i = 0; i < p.segments; ++i) {
    if (p.kind == kKindCoo) {
      e = launch_kernel(k_hook_coo, s, 0, false, stream, p.src, p.dst, p.pi, p.V,
                        split_point<long long>(p.m, p.segments, i), split_point<long long>(p.m, p.segments, i + 1), c);
    } else if (p.rp64) {
      const long long* rp = static_cast<const long long*>(p.rp);
      const long long a0 = split_point<long long>(p.m, p.segments, i);
      const long long a1 = split_point<long long>(p.m, p.segments, i + 1);
      e = with_csr_hook<long long>(p, [&](auto k) { return launch_kernel(k, s, smem, false, stream, rp, p.col, p.pi, p.V, a0, a1, c); });
    } else {
      const int* rp = static_cast<const int*>(p.rp);
      const int a0 = split_point<int>((int)p.m, p.segments, i), a1 = split_point<int>((int)p.m, p.segments, i + 1);
      e = with_csr_hook<int>(p, [&](auto k) { return launch_kernel(k, s, smem, false, stream, rp, p.col, p.pi, p.V, a0, a1, c); });
    }
    if (e != cudaSuccess) return e;
    e = launch_kernel(k_jump, s, 0, false, stream, p.pi, p.V, c);
    if (e != cudaSuccess) return e;
    n += 2;
  }
  *launches = n;
  return cudaSuccess;
}

cudaError_t launch_sample_locality(const Problem& p, int W, unsigned long long* out, int threads, cudaStream_t stream) {
  const LaunchShape s{(threads + 255) / 256, 256};
  if (p.rp64)
    return launch_kernel(k_sample_locality<long long>, s, 0, false, stream, static_cast<const long long*>(p.rp), p.col,
                         p.V, (long long)p.m, W, out);
  return launch_kernel(k_sample_locality<int>, s, 0, false, stream, static_cast<const int*>(p.rp), p.col, p.V, (int)p.m,
                       W, out);
}

cudaError_t launch_hook_segment(const Problem& p, const int* col_seg, long long a0, long long a1, const Ctl& c,
                                LaunchShape s, cudaStream_t stream) {
  // col_seg holds the arcs [a0, a1); the kernel indexes arcs by their position in the whole arc
  // array, so it gets the address col_seg would have if the whole array were resident (only
  // positions in [a0, a1) are ever read through it).
  const int* col = reinterpret_cast<const int*>(reinterpret_cast<uintptr_t>(col_seg) - (uintptr_t)a0 * sizeof(int));
  if (p.rp64) {
    const long long* rp = static_cast<const long long*>(p.rp);
    return with_csr_hook<long long>(p, [&](auto k) {
      return launch_kernel(k, s, 0, false, stream, rp, col, p.pi, p.V, a0, a1, c);
    });
  }
  const int* rp = static_cast<const int*>(p.rp);
  return with_csr_hook<int>(p, [&](auto k) {
    return launch_kernel(k, s, 0, false, stream, rp, col, p.pi, p.V, (int)a0, (int)a1, c);
  });
}

cudaError_t launch_init_only(const Problem& p, const Ctl& c, LaunchShape s, cudaStream_t stream) {
  return launch_kernel(k_init, s, 0, false, stream, p.pi, p.V, c);
}

cudaError_t launch_hook_nonatomic(const Problem& p, const Ctl& c, LaunchShape s, cudaStream_t stream) {
  if (p.rp64) {
    const long long* rp = static_cast<const long long*>(p.rp);
    return p.sym ? launch_kernel(k_hook_csr_nonatomic<long long, true>, s, 0, false, stream, rp, p.col, p.pi, p.V,
                                 (long long)p.m, c)
                 : launch_kernel(k_hook_csr_nonatomic<long long, false>, s, 0, false, stream, rp, p.col, p.pi, p.V,
                                 (long long)p.m, c);
  }
  const int* rp = static_cast<const int*>(p.rp);
  return p.sym ? launch_kernel(k_hook_csr_nonatomic<int, true>, s, 0, false, stream, rp, p.col, p.pi, p.V, (int)p.m, c)
               : launch_kernel(k_hook_csr_nonatomic<int, false>, s, 0, false, stream, rp, p.col, p.pi, p.V, (int)p.m, c);
}

cudaError_t launch_jump_single(const Problem& p, const Ctl& c, LaunchShape s, cudaStream_t stream) {
  return launch_kernel(k_jump_single, s, 0, false, stream, p.pi, p.V, c);
}

cudaError_t launch_jump_multi(const Problem& p, const Ctl& c, LaunchShape s, cudaStream_t stream) {
  return launch_kernel(k_jump, s, 0, false, stream, p.pi, p.V, c);
}

cudaError_t launch_validate(const Problem& p, const Ctl& c, LaunchShape s, cudaStream_t stream) {
  if (p.kind == kKindCoo)
    return launch_kernel(k_validate_coo, s, 0, false, stream, p.src, p.dst, p.V, p.m, c);
  if (p.rp64)
    return launch_kernel(k_validate_csr<long long>, s, 0, false, stream, static_cast<const long long*>(p.rp), p.col,
                         p.V, (long long)p.m, c);
  return launch_kernel(k_validate_csr<int>, s, 0, false, stream, static_cast<const int*>(p.rp), p.col, p.V, (int)p.m,
                       c);
}

}  // namespace cc
