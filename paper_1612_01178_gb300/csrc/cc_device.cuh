// Device building blocks of the adaptive Hook-Compress method (arXiv:1612.01178):
// the parent array pi, root finding, Atomic-Hook (Fig. 3, top), Multi-Jump
// (Fig. 3, bottom), the CSR arc-segment walker and the bounded grid barrier that
// replaces the host loop of Fig. 4 inside one persistent launch.
//
// Invariant used throughout (it is what makes every race below benign):
//   pi(x) <= x for every x at every moment.
// Init writes pi(x) = x. A hook writes L < H into pi(H), and only while pi(H) = H.
// A jump or a path-halving step writes pi(pi(x)) <= pi(x). So every value ever
// stored at x is an ancestor of x, ancestors stay ancestors (trees only merge),
// and a root is the minimum vertex of its tree. A stale read therefore yields an
// older ancestor, never a wrong tree; a CAS on a root is the only decision point.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace cc {

constexpr unsigned kFull = 0xffffffffu;

// Device status block owned by the context. `bar` is zeroed before each
// persistent launch; `error` is sticky until the host reads and clears it.
struct DevStatus {
  unsigned int bar;
  unsigned int pad0;
  int error;
  int error_where;
  long long error_info;
  unsigned long long counters[4];
};

// Where an error was raised (DevStatus::error_where).
enum ErrorSite : int {
  kSiteBarrier = 1,
  kSiteHookArc = 2,
  kSiteHookGuard = 3,
  kSiteJumpGuard = 4,
  kSiteValidate = 5,
  kSiteFindGuard = 6,
};

// Status codes mirrored from cc.h (device code does not include the C header).
enum DevError : int { kErrOutOfRange = 2, kErrTimeout = 5, kErrInternal = 6 };

struct Ctl {
  DevStatus* st;
  long long timeout_ns;
  int skip_arrival_block;  // test hook (-1 = off)
};

// ---------------------------------------------------------------------------------------------
// Memory access flavours.
//
// pi is read with plain (weak) loads so that the tree walks of nearby vertices hit in L1;
// inline asm keeps the compiler from caching a value across iterations of a racy loop.
// Within one phase a weak load may return an older ancestor (see the invariant above), which
// never changes a decision: a hook decides with a CAS, and a jump only stops at a vertex
// whose pi it read as itself, i.e. a root. The grid barrier between phases releases and
// acquires at GPU scope, so a phase never reads pi values from before the previous phase.

__device__ __forceinline__ int ld_pi(const int* p) {
  int v;
  asm volatile("ld.global.s32 %0, [%1];" : "=r"(v) : "l"(p));
  return v;
}

__device__ __forceinline__ void st_pi(int* p, int v) {
  asm volatile("st.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ int ld_relaxed(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void red_release_add(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Streaming read of the arc array: each element is read once (evict-first).
__device__ __forceinline__ int ld_stream(const int* p) { return __ldcs(p); }

template <typename T>
__device__ __forceinline__ T ld_ro(const T* p) {
  return __ldg(p);
}

__device__ __forceinline__ void raise_error(DevStatus* st, int code, int where, long long info) {
  if (atomicCAS(&st->error, 0, code) == 0) {
    st->error_where = where;
    st->error_info = info;
  }
}

// ---------------------------------------------------------------------------------------------
// Grid barrier with a time limit. Every block calls it the same number of times; `epoch`
// counts the calls. Returns false (in every thread of the block) when the launch must stop:
// an error is pending, or the wait ran out (which raises CC_ERR_TIMEOUT).

__device__ __forceinline__ bool grid_sync(const Ctl& c, unsigned& epoch) {
  __shared__ int s_go;
  __syncthreads();
  if (threadIdx.x == 0) {
    ++epoch;
    const unsigned target = epoch * gridDim.x;
    const bool skip = (epoch == 1) && ((int)blockIdx.x == c.skip_arrival_block);
    __threadfence();
    if (!skip) red_release_add(&c.st->bar, 1u);
    int go = 1;
    const unsigned long long t0 = now_ns();
    for (unsigned spin = 0;; ++spin) {
      if (ld_acquire(&c.st->bar) >= target) break;
      if (ld_relaxed(&c.st->error) != 0) {
        go = 0;
        break;
      }
      if ((spin & 31u) == 31u && (long long)(now_ns() - t0) > c.timeout_ns) {
        raise_error(c.st, kErrTimeout, kSiteBarrier, (long long)epoch);
        go = 0;
        break;
      }
    }
    if (go && ld_relaxed(&c.st->error) != 0) go = 0;
    __threadfence();
    s_go = go;
  }
  __syncthreads();
  return s_go != 0;
}

// ---------------------------------------------------------------------------------------------
// Root of x's tree. Path halving: each visited vertex whose grandparent differs from its
// parent is re-pointed at the grandparent, so later walks are shorter. x strictly decreases
// along the walk (pi(y) < y for non-roots), so it ends within V steps.

__device__ __forceinline__ int find_root(int* pi, int x) {
  int px = ld_pi(pi + x);
  while (px != x) {
    const int gx = ld_pi(pi + px);
    if (gx == px) return px;
    st_pi(pi + x, gx);
    x = gx;
    px = ld_pi(pi + x);
  }
  return x;
}

// Atomic-Hook of one edge (u, v) (Fig. 3, top; Section III-A). Both endpoints are walked to
// their roots; while they differ, the higher root H is CASed from H (still a root) to the
// lower one L. A failed CAS means another thread hooked H first; the walk resumes from the
// value the CAS returned. The larger of the two roots strictly decreases on every retry, so
// the loop ends within V retries; the guard only trips on corrupted memory.
__device__ __forceinline__ void atomic_hook(int* pi, int u, int v, int V, const Ctl& c) {
  int ru = find_root(pi, u);
  int rv = find_root(pi, v);
  int guard = 0;
  while (ru != rv) {
    const int H = ru > rv ? ru : rv;
    const int L = ru > rv ? rv : ru;
    const int old = atomicCAS(pi + H, H, L);
    if (old == H) return;
    ru = find_root(pi, old);
    rv = find_root(pi, L);
    if (++guard > V) {
      raise_error(c.st, kErrInternal, kSiteHookGuard, (long long)H);
      return;
    }
  }
}

// pi(v) <- v over [0, V), grid-strided.
__device__ __forceinline__ void init_pi(int* pi, int V, long long tid, long long nthreads) {
  for (long long v = tid; v < V; v += nthreads) pi[v] = (int)v;
}

// Multi-Jump (Fig. 3, bottom; Section III-A): every vertex jumps pi(v) <- pi(pi(v)) until
// pi(v) is a root, writing the intermediate value each step (optimisation (i)). Thread t
// takes vertices t, t + T, ... so lower IDs, the tops of the trees, are served first
// (optimisation (ii)). No hook runs concurrently, so roots are fixed during the phase.
__device__ __forceinline__ void multi_jump(int* pi, int V, long long tid, long long nthreads, const Ctl& c) {
  for (long long vv = tid; vv < V; vv += nthreads) {
    const int v = (int)vv;
    int p = ld_pi(pi + v);
    if (p == v) continue;
    int g = ld_pi(pi + p);
    int guard = 0;
    while (g != p) {
      st_pi(pi + v, g);
      p = g;
      g = ld_pi(pi + p);
      if (++guard > V) {
        raise_error(c.st, kErrInternal, kSiteJumpGuard, (long long)v);
        break;
      }
    }
  }
}

// ---------------------------------------------------------------------------------------------
// Segments and partitions: part i of n equal parts of [0, len).
template <typename T>
__host__ __device__ __forceinline__ T split_point(T len, long long parts, long long i) {
  const T base = len / (T)parts;
  const T rem = len % (T)parts;
  return (T)i * base + ((T)i < rem ? (T)i : rem);
}

// Largest r in [lo, hi) with rp[r] <= a, given rp[lo] <= a (warp-cooperative, 32-ary search).
// Every lane returns the same value. Memory-safe for any rp contents: probes stay in [lo, hi).
template <typename OffT>
__device__ __forceinline__ int warp_row_search(const OffT* rp, int lo, int hi, OffT a) {
  const int lane = threadIdx.x & 31;
  while (hi - lo > 32) {
    const long long step = ((long long)(hi - lo) + 31) >> 5;
    const long long probe = (long long)lo + lane * step;
    const bool le = probe < hi && ld_ro(rp + probe) <= a;
    const unsigned m = __ballot_sync(kFull, le) | 1u;
    const int k = 31 - __clz(m);
    lo = (int)((long long)lo + k * step);
    const long long nh = (long long)lo + step;
    hi = nh < hi ? (int)nh : hi;
  }
  const int probe = lo + lane;
  const bool le = probe < hi && ld_ro(rp + probe) <= a;
  const unsigned m = __ballot_sync(kFull, le) | 1u;
  return lo + (31 - __clz(m));
}

// Number of lanes l whose row end e_l (non-decreasing in l) is <= a (0..32).
template <typename OffT>
__device__ __forceinline__ int window_count(OffT e, OffT a) {
  int pos = 0;
#pragma unroll
  for (int step = 16; step > 0; step >>= 1) {
    const OffT probe = __shfl_sync(kFull, e, pos + step - 1);
    if (probe <= a) pos += step;
  }
  const OffT last = __shfl_sync(kFull, e, 31);
  if (pos == 31 && last <= a) pos = 32;
  return pos;
}

// Atomic-Hook over the arcs [a0, a1) of a CSR graph (one segment E_i of Fig. 4). Each warp
// takes one contiguous slice of the segment and walks it 32 arcs at a time (coalesced
// col_idx reads). The source row of every arc comes from a window of 32 row offsets held
// one per lane: lane l holds the end of row r + l, and an arc's row is r + (number of window
// ends <= arc). A warp searches row_ptr only at the start of its slice and when a batch runs
// past its window (rows with few or no arcs).
// SYM: the CSR holds both directions of every edge, so arcs with u > v are skipped.
template <typename OffT, bool SYM>
__device__ __forceinline__ void hook_csr_arcs(const OffT* __restrict__ rp, const int* __restrict__ col, int* pi,
                                              int V, OffT a0, OffT a1, long long tid, long long nthreads,
                                              const Ctl& c) {
  const int lane = threadIdx.x & 31;
  const long long warp = tid >> 5;
  const long long nwarps = nthreads >> 5;
  const OffT len = a1 - a0;
  const OffT t0 = a0 + split_point<OffT>(len, nwarps, warp);
  const OffT t1 = a0 + split_point<OffT>(len, nwarps, warp + 1);
  if (t0 >= t1) return;  // warp-uniform
  int r = warp_row_search<OffT>(rp, 0, V, t0);
  for (OffT b = t0; b < t1; b += 32) {
    const OffT a = b + lane;
    const bool valid = a < t1;
    const OffT aq = valid ? a : b;
    const int v = valid ? ld_stream(col + a) : 0;
    const long long wi = (long long)r + 1 + lane;
    OffT e = ld_ro(rp + (wi < V ? wi : V));
    int cnt = window_count<OffT>(e, aq);
    int u = cnt < 32 ? r + cnt : -1;
    unsigned pend = __ballot_sync(kFull, valid && u < 0);
    while (pend) {
      if ((long long)r + 32 >= V) {
        // Only reachable when row_ptr[V] != n_arcs: the remaining arcs have no row.
        if (valid && u < 0) u = V;
        break;
      }
      const int first = __ffs(pend) - 1;
      const OffT amin = __shfl_sync(kFull, aq, first);
      r = warp_row_search<OffT>(rp, r + 32, V, amin);
      const long long wj = (long long)r + 1 + lane;
      e = ld_ro(rp + (wj < V ? wj : V));
      cnt = window_count<OffT>(e, aq);
      if (valid && u < 0 && cnt < 32) u = r + cnt;
      pend = __ballot_sync(kFull, valid && u < 0);
    }
    const long long last_valid = (long long)(t1 - b) - 1;
    r = __shfl_sync(kFull, u, last_valid < 31 ? (int)last_valid : 31);
    r = r < V ? r : V;
    if (!valid) continue;
    if ((unsigned)v >= (unsigned)V || (unsigned)u >= (unsigned)V) {
      raise_error(c.st, kErrOutOfRange, kSiteHookArc, (long long)a);
      continue;
    }
    if (SYM ? (u >= v) : (u == v)) continue;
    atomic_hook(pi, u, v, V, c);
  }
}

// Atomic-Hook over edges [e0, e1) of an edge list.
__device__ __forceinline__ void hook_coo_edges(const int* __restrict__ src, const int* __restrict__ dst, int* pi,
                                               int V, long long e0, long long e1, long long tid,
                                               long long nthreads, const Ctl& c) {
  for (long long i = e0 + tid; i < e1; i += nthreads) {
    const int u = ld_stream(src + i);
    const int v = ld_stream(dst + i);
    if ((unsigned)u >= (unsigned)V || (unsigned)v >= (unsigned)V) {
      raise_error(c.st, kErrOutOfRange, kSiteHookArc, i);
      continue;
    }
    if (u != v) atomic_hook(pi, u, v, V, c);
  }
}

}  // namespace cc
