// Small graphs in one thread-block cluster: the parent array pi lives in the distributed shared
// memory of the cluster's CTAs instead of global memory, so every step of a root walk and every
// CAS of the Atomic-Hook (Fig. 3) is a shared-memory access (local, or a neighbour SM's through
// DSMEM) rather than an L2 round trip, and the phases are separated by the cluster's hardware
// barrier instead of a grid barrier. The method is the one of the single-graph kernels:
//   symmetric CSR: the sampled-and-filtered hook (first 2 arcs of every row; Multi-Jump; the
//     largest star's root from a sample; the remaining arcs of the rows outside that star, both
//     directions; Multi-Jump);
//   otherwise: every arc hooked (one segment of Fig. 4), then Multi-Jump.
// CTA r of C owns the vertices [r P, r P + P) (P a power of two): their parents sit in its shared
// memory, and it reads their rows. Only the rows' arcs come from global memory; the labels are
// written once at the end.
#include <cooperative_groups.h>

#include "cc_internal.h"

namespace cg = cooperative_groups;

namespace cc {

namespace {

constexpr int kClusterBlock = 1024;

// Distributed parent array: vertex x is entry x & mask of CTA x >> shift.
struct DsmPi {
  unsigned base;  // shared-window address of this CTA's part
  int shift;
  int mask;
  __device__ __forceinline__ unsigned addr(int x) const {
    const unsigned a = base + 4u * (unsigned)(x & mask);
    unsigned r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"((unsigned)(x >> shift)));
    return r;
  }
  __device__ __forceinline__ int ld(int x) const {
    int v;
    asm volatile("ld.relaxed.cluster.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(addr(x)) : "memory");
    return v;
  }
  __device__ __forceinline__ void st(int x, int v) const {
    asm volatile("st.relaxed.cluster.shared::cluster.u32 [%0], %1;" ::"r"(addr(x)), "r"(v) : "memory");
  }
  __device__ __forceinline__ int cas(int x, int cmp, int val) const {
    int old;
    asm volatile("atom.relaxed.cluster.shared::cluster.cas.b32 %0, [%1], %2, %3;"
                 : "=r"(old)
                 : "r"(addr(x)), "r"(cmp), "r"(val)
                 : "memory");
    return old;
  }
};

// Root of x with path halving (the invariant pi(x) <= x of the global kernels holds here too).
__device__ __forceinline__ int dsm_find(const DsmPi& d, int x) {
  int px = d.ld(x);
  while (px != x) {
    const int gx = d.ld(px);
    if (gx == px) return px;
    d.st(x, gx);
    x = gx;
    px = d.ld(x);
  }
  return x;
}

// Atomic-Hook of (u, v) (Fig. 3, top): CAS the higher root to the lower one until it succeeds or
// the roots agree; the larger root strictly decreases on every retry, so V bounds the loop.
__device__ __forceinline__ void dsm_hook(const DsmPi& d, int u, int v, int V, const Ctl& c) {
  int ru = dsm_find(d, u), rv = dsm_find(d, v);
  int guard = 0;
  while (ru != rv) {
    const int H = ru > rv ? ru : rv;
    const int L = ru > rv ? rv : ru;
    const int old = d.cas(H, H, L);
    if (old == H || old == L) return;
    ru = dsm_find(d, old);
    rv = dsm_find(d, L);
    if (++guard > V) {
      raise_error(c.st, kErrInternal, kSiteHookGuard, (long long)H);
      return;
    }
  }
}

// Multi-Jump of this CTA's vertices [v0, v1) (Fig. 3, bottom): roots do not change during it, and
// every step writes the parent reached (a vertex whose grandparent is a root ends in one step).
__device__ __forceinline__ void dsm_jump(const DsmPi& d, int* part, int v0, int v1, int V, const Ctl& c) {
  for (int x = v0 + (int)threadIdx.x; x < v1; x += blockDim.x) {
    int p = part[x - v0];
    if (p == x) continue;
    int g = d.ld(p);
    int guard = 0;
    while (g != p) {
      part[x - v0] = g;
      p = g;
      g = d.ld(p);
      if (++guard > V) {
        raise_error(c.st, kErrInternal, kSiteJumpGuard, (long long)x);
        break;
      }
    }
  }
}

// Arcs from position `skip` on of the rows [v0, v1) whose parent is not `giant` (every row when
// giant < 0), one row per lane; rows with more than 32 such arcs are walked by the whole warp.
template <typename OffT>
__device__ __forceinline__ void dsm_hook_rows(const DsmPi& d, const int* part, const OffT* __restrict__ rp,
                                              const int* __restrict__ col, int V, OffT nnz, int v0, int v1, int skip,
                                              int giant, const Ctl& c) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  for (int base = v0 + warp * 32; base < v1; base += nwarps * 32) {  // warp-uniform
    const int u = base + lane;
    long long a0 = 0, a1 = 0;
    if (u < v1 && (giant < 0 || part[u - v0] != giant)) {
      a0 = (long long)ld_ro(rp + u);
      a1 = (long long)ld_ro(rp + u + 1);
      if (!(a0 >= 0 && a0 <= a1 && a1 <= (long long)nnz)) {
        raise_input_error(c, kSiteHookArc, (long long)u);
        a1 = a0;
      }
      a0 = a0 + skip < a1 ? a0 + skip : a1;
    }
    const bool heavy = a1 - a0 > 32;
    if (!heavy) {
      for (long long a = a0; a < a1; ++a) {
        const int v = ld_stream(col + a);
        if ((unsigned)v >= (unsigned)V) {
          raise_input_error(c, kSiteHookArc, a);
          continue;
        }
        if (v != u) dsm_hook(d, u, v, V, c);
      }
    }
    unsigned hv = __ballot_sync(kFull, heavy);
    while (hv) {
      const int h = __ffs(hv) - 1;
      hv &= hv - 1;
      const int hu = __shfl_sync(kFull, u, h);
      const long long h0 = __shfl_sync(kFull, a0, h), h1 = __shfl_sync(kFull, a1, h);
      for (long long bb = h0; bb < h1; bb += 32) {
        const long long a = bb + lane;
        if (a < h1) {
          const int v = ld_stream(col + a);
          if ((unsigned)v >= (unsigned)V) raise_input_error(c, kSiteHookArc, a);
          else if (v != hu) dsm_hook(d, hu, v, V, c);
        }
      }
    }
  }
}

// The first kSampleArcs arcs of the rows [v0, v1), one row per thread.
template <typename OffT>
__device__ __forceinline__ void dsm_hook_heads(const DsmPi& d, const OffT* __restrict__ rp,
                                               const int* __restrict__ col, int V, OffT nnz, int v0, int v1,
                                               const Ctl& c) {
  for (int u = v0 + (int)threadIdx.x; u < v1; u += blockDim.x) {
    OffT a0 = ld_ro(rp + u), a1 = ld_ro(rp + u + 1);
    if (!(a0 >= 0 && a0 <= a1 && a1 <= nnz)) {
      raise_input_error(c, kSiteHookArc, (long long)u);
      a1 = a0;
    }
    int v[kSampleArcs];
#pragma unroll
    for (int j = 0; j < kSampleArcs; ++j) v[j] = (long long)a0 + j < (long long)a1 ? ld_stream(col + a0 + j) : u;
#pragma unroll
    for (int j = 0; j < kSampleArcs; ++j) {
      if ((unsigned)v[j] >= (unsigned)V) raise_input_error(c, kSiteHookArc, (long long)a0 + j);
      else if (v[j] != u) dsm_hook(d, u, v[j], V, c);
    }
  }
}

template <typename OffT, bool SYM>
__global__ void __launch_bounds__(kClusterBlock, 1) k_csr_cluster(const OffT* __restrict__ rp,
                                                                  const int* __restrict__ col, int* labels, int V,
                                                                  OffT nnz, int shift, Ctl c) {
  extern __shared__ __align__(16) int part[];
  __shared__ int s_giant;
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  const int P = 1 << shift;
  const DsmPi d{(unsigned)__cvta_generic_to_shared(part), shift, P - 1};
  const int v0 = rank * P < V ? rank * P : V;
  const int v1 = v0 + P < V ? v0 + P : V;
  // Every CTA passes the same cluster barriers whatever happens; a pending error only skips work.
  const bool go = !launch_blocked(c);
  if (c.phase_ns && rank == 0 && threadIdx.x == 0) c.phase_ns[0] = now_ns();
  for (int i = threadIdx.x; i < P; i += blockDim.x) part[i] = rank * P + i;
  cl.sync();
  int giant = -1;
  if (SYM) {
    if (go) dsm_hook_heads<OffT>(d, rp, col, V, nnz, v0, v1, c);
    cl.sync();
    if (go) dsm_jump(d, part, v0, v1, V, c);
    cl.sync();
    if (rank == 0) {  // the most frequent root of 256 vertices spread over [0, V)
      __shared__ int s_samples[kGiantSamples];
      __shared__ unsigned long long s_best;
      if (threadIdx.x == 0) s_best = 0ull;
      if (threadIdx.x < kGiantSamples) {
        const long long x = ((long long)threadIdx.x * V) / kGiantSamples;
        s_samples[threadIdx.x] = go ? d.ld((int)(x < V ? x : V - 1)) : -1;
      }
      __syncthreads();
      if (threadIdx.x < kGiantSamples) {
        const int mine = s_samples[threadIdx.x];
        unsigned cnt = 0;
        for (int j = 0; j < kGiantSamples; ++j) cnt += s_samples[j] == mine ? 1u : 0u;
        atomicMax(&s_best, ((unsigned long long)cnt << 32) | (unsigned)mine);
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        const unsigned long long best = s_best;
        const int g = 8ull * (best >> 32) >= (unsigned long long)kGiantSamples ? (int)(best & 0xffffffffull) : -1;
        for (int r = 0; r < (int)cl.num_blocks(); ++r) *cl.map_shared_rank(&s_giant, r) = g;
      }
    }
    cl.sync();
    giant = s_giant;
    if (go) dsm_hook_rows<OffT>(d, part, rp, col, V, nnz, v0, v1, kSampleArcs, giant, c);
  } else {
    if (go) dsm_hook_rows<OffT>(d, part, rp, col, V, nnz, v0, v1, 0, -1, c);
  }
  cl.sync();
  if (go) dsm_jump(d, part, v0, v1, V, c);
  cl.sync();  // all parts final; no CTA exits while another may still read its shared memory
  if (go)
    for (int x = v0 + (int)threadIdx.x; x < v1; x += blockDim.x) labels[x] = part[x - v0];
  if (c.phase_ns && threadIdx.x == 0) atomicMax(c.phase_ns + (c.phase_cap - 1), now_ns());
}

template <typename OffT, typename F>
auto with_cluster_kernel(bool sym, F&& f) {
  return sym ? f(k_csr_cluster<OffT, true>) : f(k_csr_cluster<OffT, false>);
}

// Smallest shift with C << shift >= V.
int part_shift(long long V, int C) {
  int s = 0;
  while (((long long)C << s) < V) ++s;
  return s < 2 ? 2 : s;
}

template <typename OffT>
cudaError_t cluster_launch(const Problem& p, const Ctl& c, int C, cudaStream_t stream, bool check_only, bool* fits) {
  const int shift = part_shift(p.V, C);
  const size_t smem = ((size_t)1 << shift) * sizeof(int);
  *fits = false;
  return with_cluster_kernel<OffT>(p.sym, [&](auto k) -> cudaError_t {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess && C > 8) e = cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return check_only ? cudaSuccess : e;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)C);
    cfg.blockDim = dim3((unsigned)kClusterBlock);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    e = cudaOccupancyMaxActiveClusters(&n, k, &cfg);
    if (e != cudaSuccess || n < 1) {
      cudaGetLastError();
      return check_only ? cudaSuccess : (e != cudaSuccess ? e : cudaErrorInvalidConfiguration);
    }
    *fits = true;
    if (check_only) return cudaSuccess;
    return cudaLaunchKernelEx(&cfg, k, static_cast<const OffT*>(p.rp), p.col, p.pi, p.V, (OffT)p.m, shift, c);
  });
}

}  // namespace

int cluster_size_for(const Problem& p) {
  if (p.kind != kKindCsr || p.V <= 0) return 0;
  for (int C : {8, 16}) {
    if (((long long)C << kClusterMaxShift) < p.V) continue;
    bool fits = false;
    Ctl c;
    const cudaError_t e = p.rp64 ? cluster_launch<long long>(p, c, C, nullptr, true, &fits)
                                 : cluster_launch<int>(p, c, C, nullptr, true, &fits);
    if (e == cudaSuccess && fits) return C;
  }
  return 0;
}

cudaError_t launch_cluster(const Problem& p, const Ctl& c, int C, cudaStream_t stream) {
  bool fits = false;
  return p.rp64 ? cluster_launch<long long>(p, c, C, stream, false, &fits)
                : cluster_launch<int>(p, c, C, stream, false, &fits);
}

}  // namespace cc
