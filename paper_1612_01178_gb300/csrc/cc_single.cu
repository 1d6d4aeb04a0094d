// Single-graph kernels: the persistent driver of Fig. 4 (one cooperative launch, grid
// barriers between Hook and Multi-Jump phases) and the per-phase kernels of the printed
// host loop, for CSR (int32 / int64 offsets, plain or symmetrised) and COO inputs.
#include "cc_internal.h"

namespace cc {

namespace {

__device__ __forceinline__ long long global_tid() {
  return (long long)blockIdx.x * blockDim.x + threadIdx.x;
}
__device__ __forceinline__ long long global_threads() { return (long long)gridDim.x * blockDim.x; }

// Adaptive Hook-Compress (Fig. 4) over the arcs of a CSR graph, in one launch:
//   init pi; for i in 1..s: Atomic-Hook(E_i); barrier; Multi-Jump(V); barrier.
template <typename OffT, bool SYM>
__global__ void __launch_bounds__(256) k_csr_persistent(const OffT* __restrict__ rp, const int* __restrict__ col,
                                                        int* pi, int V, OffT nnz, int s, Ctl c) {
  if (ld_relaxed(&c.st->error) != 0) return;  // a pending error stops all device work
  unsigned epoch = 0;
  const long long tid = global_tid(), nt = global_threads();
  init_pi(pi, V, tid, nt);
  if (!grid_sync(c, epoch)) return;
  for (int i = 0; i < s; ++i) {
    const OffT a0 = split_point<OffT>(nnz, s, i);
    const OffT a1 = split_point<OffT>(nnz, s, i + 1);
    hook_csr_arcs<OffT, SYM>(rp, col, pi, V, a0, a1, tid, nt, c);
    if (!grid_sync(c, epoch)) return;
    multi_jump(pi, V, tid, nt, c);
    if (i + 1 < s && !grid_sync(c, epoch)) return;
  }
}

__global__ void __launch_bounds__(256) k_coo_persistent(const int* __restrict__ src, const int* __restrict__ dst,
                                                        int* pi, int V, long long E, int s, Ctl c) {
  if (ld_relaxed(&c.st->error) != 0) return;
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

// ----- per-phase kernels (the host loop of Fig. 4) -----

__global__ void __launch_bounds__(256) k_init(int* pi, int V, Ctl c) {
  if (ld_relaxed(&c.st->error) != 0) return;
  init_pi(pi, V, global_tid(), global_threads());
}

template <typename OffT, bool SYM>
__global__ void __launch_bounds__(256) k_hook_csr(const OffT* __restrict__ rp, const int* __restrict__ col, int* pi,
                                                  int V, OffT a0, OffT a1, Ctl c) {
  if (ld_relaxed(&c.st->error) != 0) return;
  hook_csr_arcs<OffT, SYM>(rp, col, pi, V, a0, a1, global_tid(), global_threads(), c);
}

__global__ void __launch_bounds__(256) k_hook_coo(const int* __restrict__ src, const int* __restrict__ dst, int* pi,
                                                  int V, long long e0, long long e1, Ctl c) {
  if (ld_relaxed(&c.st->error) != 0) return;
  hook_coo_edges(src, dst, pi, V, e0, e1, global_tid(), global_threads(), c);
}

__global__ void __launch_bounds__(256) k_jump(int* pi, int V, Ctl c) {
  if (ld_relaxed(&c.st->error) != 0) return;
  multi_jump(pi, V, global_tid(), global_threads(), c);
}

// ----- validation (CC_FLAG_VALIDATE) -----

template <typename OffT>
__global__ void __launch_bounds__(256) k_validate_csr(const OffT* __restrict__ rp, const int* __restrict__ col, int V,
                                                      OffT nnz, Ctl c) {
  const long long tid = global_tid(), nt = global_threads();
  if (tid == 0 && (rp[0] != 0 || rp[V] != nnz)) raise_error(c.st, kErrOutOfRange, kSiteValidate, -1);
  for (long long v = tid; v < V; v += nt)
    if (rp[v + 1] < rp[v]) raise_error(c.st, kErrOutOfRange, kSiteValidate, v);
  for (long long a = tid; a < (long long)nnz; a += nt)
    if ((unsigned)col[a] >= (unsigned)V) raise_error(c.st, kErrOutOfRange, kSiteValidate, a);
}

__global__ void __launch_bounds__(256) k_validate_coo(const int* __restrict__ src, const int* __restrict__ dst, int V,
                                                      long long E, Ctl c) {
  for (long long i = global_tid(); i < E; i += global_threads())
    if ((unsigned)src[i] >= (unsigned)V || (unsigned)dst[i] >= (unsigned)V)
      raise_error(c.st, kErrOutOfRange, kSiteValidate, i);
}

template <typename F>
int blocks_per_sm(F kernel, int block) {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, block, 0) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

template <typename... Args>
cudaError_t launch_coop(void (*kernel)(Args...), LaunchShape s, cudaStream_t stream, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)s.grid);
  cfg.blockDim = dim3((unsigned)s.block);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

}  // namespace

int persistent_blocks_per_sm(const Problem& p, int block) {
  if (p.kind == kKindCoo) return blocks_per_sm(k_coo_persistent, block);
  if (p.rp64)
    return p.sym ? blocks_per_sm(k_csr_persistent<long long, true>, block)
                 : blocks_per_sm(k_csr_persistent<long long, false>, block);
  return p.sym ? blocks_per_sm(k_csr_persistent<int, true>, block)
               : blocks_per_sm(k_csr_persistent<int, false>, block);
}

int stage_blocks_per_sm(const Problem& p, int block) {
  if (p.kind == kKindCoo) return blocks_per_sm(k_hook_coo, block);
  if (p.rp64)
    return p.sym ? blocks_per_sm(k_hook_csr<long long, true>, block) : blocks_per_sm(k_hook_csr<long long, false>, block);
  return p.sym ? blocks_per_sm(k_hook_csr<int, true>, block) : blocks_per_sm(k_hook_csr<int, false>, block);
}

cudaError_t launch_persistent(const Problem& p, const Ctl& c, LaunchShape s, cudaStream_t stream) {
  if (p.kind == kKindCoo)
    return launch_coop(k_coo_persistent, s, stream, p.src, p.dst, p.pi, p.V, p.m, p.segments, c);
  if (p.rp64) {
    const long long* rp = static_cast<const long long*>(p.rp);
    if (p.sym)
      return launch_coop(k_csr_persistent<long long, true>, s, stream, rp, p.col, p.pi, p.V, p.m, p.segments, c);
    return launch_coop(k_csr_persistent<long long, false>, s, stream, rp, p.col, p.pi, p.V, p.m, p.segments, c);
  }
  const int* rp = static_cast<const int*>(p.rp);
  const int nnz = (int)p.m;
  if (p.sym) return launch_coop(k_csr_persistent<int, true>, s, stream, rp, p.col, p.pi, p.V, nnz, p.segments, c);
  return launch_coop(k_csr_persistent<int, false>, s, stream, rp, p.col, p.pi, p.V, nnz, p.segments, c);
}

cudaError_t launch_multi(const Problem& p, const Ctl& c, LaunchShape s, cudaStream_t stream, int* launches) {
  int n = 0;
  k_init<<<s.grid, s.block, 0, stream>>>(p.pi, p.V, c);
  ++n;
  for (int i = 0; i < p.segments; ++i) {
    if (p.kind == kKindCoo) {
      k_hook_coo<<<s.grid, s.block, 0, stream>>>(p.src, p.dst, p.pi, p.V, split_point<long long>(p.m, p.segments, i),
                                                 split_point<long long>(p.m, p.segments, i + 1), c);
    } else if (p.rp64) {
      const long long* rp = static_cast<const long long*>(p.rp);
      const long long a0 = split_point<long long>(p.m, p.segments, i), a1 = split_point<long long>(p.m, p.segments, i + 1);
      if (p.sym) k_hook_csr<long long, true><<<s.grid, s.block, 0, stream>>>(rp, p.col, p.pi, p.V, a0, a1, c);
      else k_hook_csr<long long, false><<<s.grid, s.block, 0, stream>>>(rp, p.col, p.pi, p.V, a0, a1, c);
    } else {
      const int* rp = static_cast<const int*>(p.rp);
      const int a0 = split_point<int>((int)p.m, p.segments, i), a1 = split_point<int>((int)p.m, p.segments, i + 1);
      if (p.sym) k_hook_csr<int, true><<<s.grid, s.block, 0, stream>>>(rp, p.col, p.pi, p.V, a0, a1, c);
      else k_hook_csr<int, false><<<s.grid, s.block, 0, stream>>>(rp, p.col, p.pi, p.V, a0, a1, c);
    }
    k_jump<<<s.grid, s.block, 0, stream>>>(p.pi, p.V, c);
    n += 2;
  }
  *launches = n;
  return cudaGetLastError();
}

cudaError_t launch_validate(const Problem& p, const Ctl& c, LaunchShape s, cudaStream_t stream) {
  if (p.kind == kKindCoo) {
    k_validate_coo<<<s.grid, s.block, 0, stream>>>(p.src, p.dst, p.V, p.m, c);
  } else if (p.rp64) {
    k_validate_csr<long long><<<s.grid, s.block, 0, stream>>>(static_cast<const long long*>(p.rp), p.col, p.V, p.m, c);
  } else {
    k_validate_csr<int><<<s.grid, s.block, 0, stream>>>(static_cast<const int*>(p.rp), p.col, p.V, (int)p.m, c);
  }
  return cudaGetLastError();
}

}  // namespace cc
