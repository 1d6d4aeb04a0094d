// Graphs with more than 2^31 - 1 vertices: the adaptive Hook-Compress method of Fig. 4 with one
// segment, every vertex ID, row offset and parent 64 bits wide. Three stream-ordered launches:
//   init pi(v) = v;
//   Atomic-Hook (Fig. 3, top) of every arc, warps taking 32 rows at a time (one row per lane, rows
//   of more than 32 arcs by the whole warp), 64-bit CAS on roots;
//   Multi-Jump (Fig. 3, bottom) of every vertex.
// The invariant pi(x) <= x and the high-to-low rule are those of the 32-bit kernels, so every
// label is the minimum vertex ID of its component.
#include "cc_internal.h"

namespace cc {

namespace {

constexpr int kWideBlock = 256;

__device__ __forceinline__ long long ld_pi64(const long long* p) {
  long long v;
  asm volatile("ld.global.s64 %0, [%1];" : "=l"(v) : "l"(p));
  return v;
}

__device__ __forceinline__ void st_pi64(long long* p, long long v) {
  asm volatile("st.global.s64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ long long find_root64(long long* pi, long long x) {
  long long px = ld_pi64(pi + x);
  while (px != x) {
    const long long gx = ld_pi64(pi + px);
    if (gx == px) return px;
    st_pi64(pi + x, gx);
    x = gx;
    px = ld_pi64(pi + x);
  }
  return x;
}

__device__ __forceinline__ void atomic_hook64(long long* pi, long long u, long long v, long long V, const Ctl& c) {
  long long ru = find_root64(pi, u), rv = find_root64(pi, v);
  long long guard = 0;
  while (ru != rv) {
    const long long H = ru > rv ? ru : rv;
    const long long L = ru > rv ? rv : ru;
    const long long old = (long long)atomicCAS(reinterpret_cast<unsigned long long*>(pi + H),
                                               (unsigned long long)H, (unsigned long long)L);
    if (old == H || old == L) return;
    ru = find_root64(pi, old);
    rv = find_root64(pi, L);
    if (++guard > V) {
      raise_error(c.st, kErrInternal, kSiteHookGuard, H);
      return;
    }
  }
}

__global__ void __launch_bounds__(kWideBlock) k_init64(long long* pi, long long V, Ctl c) {
  if (launch_blocked(c)) return;
  const long long T = (long long)gridDim.x * blockDim.x;
  for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += T) pi[v] = v;
}

template <bool SYM>
__global__ void __launch_bounds__(kWideBlock) k_hook64(const long long* __restrict__ rp,
                                                       const long long* __restrict__ col, long long* pi, long long V,
                                                       long long nnz, Ctl c) {
  if (launch_blocked(c)) return;
  const int lane = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  long long bad_at = -1;
  for (long long base = warp * 32; base < V; base += nwarps * 32) {  // warp-uniform
    const long long u = base + lane;
    long long a0 = 0, a1 = 0;
    if (u < V) {
      a0 = __ldg(rp + u);
      a1 = __ldg(rp + u + 1);
      if (!(a0 >= 0 && a0 <= a1 && a1 <= nnz)) {
        bad_at = u;
        a1 = a0;
      }
    }
    const bool heavy = a1 - a0 > 32;
    if (!heavy) {
      for (long long a = a0; a < a1; ++a) {
        const long long v = __ldcs(col + a);
        if ((unsigned long long)v >= (unsigned long long)V) {
          bad_at = a;
          continue;
        }
        if (SYM ? v > u : v != u) atomic_hook64(pi, u, v, V, c);
      }
    }
    unsigned hv = __ballot_sync(kFull, heavy);
    while (hv) {
      const int h = __ffs(hv) - 1;
      hv &= hv - 1;
      const long long hu = __shfl_sync(kFull, u, h);
      const long long h0 = __shfl_sync(kFull, a0, h), h1 = __shfl_sync(kFull, a1, h);
      for (long long a = h0 + lane; a < h1; a += 32) {
        const long long v = __ldcs(col + a);
        if ((unsigned long long)v >= (unsigned long long)V) bad_at = a;
        else if (SYM ? v > hu : v != hu) atomic_hook64(pi, hu, v, V, c);
      }
    }
  }
  if (bad_at >= 0) raise_input_error(c, kSiteHookArc, bad_at);
}

__global__ void __launch_bounds__(kWideBlock) k_jump64(long long* pi, long long V, Ctl c) {
  if (launch_blocked(c)) return;
  const long long T = (long long)gridDim.x * blockDim.x;
  for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += T) {
    long long p = ld_pi64(pi + v);
    if (p == v) continue;
    long long g = ld_pi64(pi + p);
    long long guard = 0;
    while (g != p) {
      st_pi64(pi + v, g);
      p = g;
      g = ld_pi64(pi + p);
      if (++guard > V) {
        raise_error(c.st, kErrInternal, kSiteJumpGuard, v);
        break;
      }
    }
  }
}

}  // namespace

int wide_blocks_per_sm(bool sym) {
  int n = 0;
  const cudaError_t e = sym ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_hook64<true>, kWideBlock, 0)
                            : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_hook64<false>, kWideBlock, 0);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

cudaError_t launch_wide(const long long* rp, const long long* col, long long* pi, long long V, long long nnz, bool sym,
                        const Ctl& c, int grid, cudaStream_t stream) {
  k_init64<<<grid, kWideBlock, 0, stream>>>(pi, V, c);
  if (sym) k_hook64<true><<<grid, kWideBlock, 0, stream>>>(rp, col, pi, V, nnz, c);
  else k_hook64<false><<<grid, kWideBlock, 0, stream>>>(rp, col, pi, V, nnz, c);
  k_jump64<<<grid, kWideBlock, 0, stream>>>(pi, V, c);
  return cudaGetLastError();
}

}  // namespace cc
