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

// Device status block owned by the context. The per-launch fields are zeroed before each
// labelling call; the sticky fields stay set until the host reads and clears them.
struct DevStatus {
  // per-launch fields (zeroed before every call)
  unsigned int bar;
  unsigned int changed;  // change flag of the host-driven modes (Fig. 1)
  unsigned long long counters[4];  // [0],[1] work counters; [2] worklist cursor; [3] overflowed units
  unsigned long long report[2];    // [0] worklist pairs, [1] worklist segments (hierarchical hook)
  unsigned int abort;    // validation failed: the launches of this call stop before hooking
  unsigned int pad;
  // sticky fields (cleared when the host reads them)
  int error;             // fatal (a wait ran out, a guard fired): later launches of the context exit early
  int error_where;
  long long error_info;
  int input_error;       // malformed input found (CC_ERR_OUT_OF_RANGE): reported, later launches run normally
  int input_where;
  long long input_info;
};
constexpr size_t kPerLaunchStatusBytes = 64;  // bar, changed, counters, report, abort, pad

// Where an error was raised (DevStatus::error_where).
enum ErrorSite : int {
  kSiteBarrier = 1,
  kSiteHookArc = 2,
  kSiteHookGuard = 3,
  kSiteJumpGuard = 4,
  kSiteValidate = 5,
  kSiteFindGuard = 6,
  kSiteWindowRow = 7,  // phase A: info = graph-local vertex whose row holds an endpoint outside [0, V)
};

// Status codes mirrored from cc.h (device code does not include the C header).
enum DevError : int { kErrOutOfRange = 2, kErrTimeout = 5, kErrInternal = 6 };

// Launch-wide control block passed by value to every kernel.
struct Ctl {
  DevStatus* st = nullptr;
  long long timeout_ns = 2000000000LL;
  int skip_arrival_block = -1;            // test hook (-1 = off)
  int chunk_arcs = -1;                    // dynamic Atomic-Hook chunk (<= 0: one static slice per warp)
  int tile_w = 0;                         // hierarchical hook window (vertices; 0 = plain hook)
  int2* wl = nullptr;                     // worklist of arcs left for the global hook
  unsigned long long wl_cap = 0;
  int* ovf_units = nullptr;               // windows whose worklist appends overflowed
  int ovf_cap = 0;
  int segments_b = 0;                     // segments of the global phase (0 = 2|E'|/|V|)
  int hook_k = 1;                         // arcs per lane per step of the plain CSR hook: 1, 2 or 4
  int window_mode = 0;                    // batched: kWindowsSampled or kWindowsPlain
  int* status_out = nullptr;              // optional per-call input status (CC_ERR_OUT_OF_RANGE or left 0)
  unsigned long long* phase_ns = nullptr; // optional per-barrier timestamps (block 0)
  int phase_cap = 0;
  int phase_off = 0;                      // slot of the first barrier's timestamp, minus one
};

// How the batched kernel hooks windows of multi-window graphs.
enum WindowMode : int { kWindowsSampled = 0, kWindowsPlain = 1 };

// DevStatus::counters[0..1] are the work counters of the dynamically scheduled phases.
constexpr int kWorkCounters = 2;

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

// A fatal device error: the launch stops at its next grid barrier and later launches of the
// context exit at once until the host has read the error.
__device__ __forceinline__ void raise_error(DevStatus* st, int code, int where, long long info) {
  if (atomicCAS(&st->error, 0, code) == 0) {
    st->error_where = where;
    st->error_info = info;
  }
}

// Malformed input (an arc endpoint outside [0, V), offsets inconsistent with n_arcs): the bad
// arc or row is skipped and reported; the launch and later launches carry on, so in a batch
// every other graph is still labelled. Also written to the call's status output, if any.
__device__ __forceinline__ void raise_input_error(const Ctl& c, int where, long long info) {
  if (atomicCAS(&c.st->input_error, 0, (int)kErrOutOfRange) == 0) {
    c.st->input_where = where;
    c.st->input_info = info;
  }
  if (c.status_out) *c.status_out = (int)kErrOutOfRange;
}

// True when this launch must not run: a fatal error is pending or the call's validation failed.
__device__ __forceinline__ bool launch_blocked(const Ctl& c) {
  return ld_relaxed(&c.st->error) != 0 || ld_relaxed(reinterpret_cast<const int*>(&c.st->abort)) != 0;
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
    // The wait polls with relaxed loads and sleeps briefly between polls; the fence after the
    // loop makes it an acquire. An acquire load inside the loop measured slower: blocks that
    // reach the barrier early slowed the blocks still hooking on the same SMs (ER 262k / 4M:
    // first hook slice 168 -> 64 us).
    for (unsigned spin = 0;; ++spin) {
      if ((unsigned)ld_relaxed(reinterpret_cast<const int*>(&c.st->bar)) >= target) break;
      __nanosleep(64);
      if (launch_blocked(c)) {
        go = 0;
        break;
      }
      if ((spin & 31u) == 31u && (long long)(now_ns() - t0) > c.timeout_ns) {
        raise_error(c.st, kErrTimeout, kSiteBarrier, (long long)epoch);
        go = 0;
        break;
      }
    }
    if (go && launch_blocked(c)) go = 0;
    __threadfence();
    if (c.phase_ns && blockIdx.x == 0 && (int)epoch + c.phase_off < c.phase_cap - 1)
      c.phase_ns[epoch + c.phase_off] = now_ns();
    s_go = go;
  }
  __syncthreads();
  return s_go != 0;
}

// ---------------------------------------------------------------------------------------------
// Root of x's tree, walked two levels per step without writing: the first levels of a hook's
// walks already halve the path (root_from2), and the stores of a second halving pass measured
// slower (they contend with the hooks on the few hot vertices near the roots). x strictly
// decreases along the walk (pi(y) < y for non-roots), so it ends within V steps.

__device__ __forceinline__ int find_root(int* pi, int x) {
  int px = ld_pi(pi + x);
  while (px != x) {
    const int gx = ld_pi(pi + px);
    if (gx == px) return px;
    x = gx;
    px = ld_pi(pi + x);
  }
  return x;
}

// Atomic-Hook of one edge (u, v) (Fig. 3, top; Section III-A). Both endpoints are walked to
// their roots; while they differ, the higher root H is CASed from H (still a root) to the
// lower one L. A failed CAS means another thread hooked H first; the walk resumes from the
// value the CAS returned, unless that value is L itself (H already hangs under L: done, which
// spares the two walks when many threads hook the same pair of roots). The larger of the two roots strictly decreases on every retry, so
// the loop ends within V retries; the guard only trips on corrupted memory.
__device__ __forceinline__ void atomic_hook(int* pi, int u, int v, int V, const Ctl& c) {
  int ru = find_root(pi, u);
  int rv = find_root(pi, v);
  int guard = 0;
  while (ru != rv) {
    const int H = ru > rv ? ru : rv;
    const int L = ru > rv ? rv : ru;
    const int old = atomicCAS(pi + H, H, L);
    if (old == H || old == L) return;
    ru = find_root(pi, old);
    rv = find_root(pi, L);
    if (++guard > V) {
      raise_error(c.st, kErrInternal, kSiteHookGuard, (long long)H);
      return;
    }
  }
}

// Root of x, given px = pi(x) != x (the walk of find_root, resumed).
__device__ __forceinline__ int root_from(int* pi, int x, int px) {
  for (;;) {
    const int gx = ld_pi(pi + px);
    if (gx == px) return px;
    st_pi(pi + x, gx);
    x = gx;
    px = ld_pi(pi + x);
    if (px == x) return x;
  }
}

// Root of a from its parent pa and grandparent ga (already loaded), halving one step if
// the walk must go on.
__device__ __forceinline__ int root_from2(int* pi, int a, int pa, int ga) {
  if (pa == a) return a;
  if (ga == pa) return pa;
  st_pi(pi + a, ga);
  const int pg = ld_pi(pi + ga);
  return pg == ga ? ga : root_from(pi, ga, pg);
}

// Atomic-Hook of K independent edges per thread. The first two levels of all 2K root walks
// are loaded together and all first CASes are issued together, so a thread keeps up to 2K
// loads or K atomics in flight instead of one dependent chain; deeper walks and failed CASes
// then finish one edge at a time exactly as in atomic_hook.
// DEDUP (the whole warp must call, converged): lanes whose edge j has the same pair of parents
// (pi(u), pi(v)), or later the same pair of roots (H, L), leave it to the lowest such lane, whose
// hook joins exactly those two trees (u and v lie in them); this keeps thousands of root walks
// and CASes off the same few roots when many edges join the same two components.
template <int K, bool DEDUP = false>
__device__ __forceinline__ void atomic_hook_k(int* pi, const int (&u)[K], const int (&v)[K], const bool (&live_in)[K],
                                              int V, const Ctl& c) {
  int pu[K], pv[K];
  bool live[K];
#pragma unroll
  for (int j = 0; j < K; ++j) {
    live[j] = live_in[j];
    pu[j] = live[j] ? ld_pi(pi + u[j]) : 0;
    pv[j] = live[j] ? ld_pi(pi + v[j]) : 0;
  }
  if (DEDUP) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int j = 0; j < K; ++j) {
      const unsigned long long key =
          live[j] ? (((unsigned long long)(unsigned)pu[j] << 32) | (unsigned)pv[j]) : ~0ull;
      const unsigned grp = __match_any_sync(kFull, key);
      live[j] = live[j] && lane == __ffs(grp) - 1;
    }
  }
  int gu[K], gv[K];
#pragma unroll
  for (int j = 0; j < K; ++j) {
    gu[j] = (live[j] && pu[j] != u[j]) ? ld_pi(pi + pu[j]) : pu[j];
    gv[j] = (live[j] && pv[j] != v[j]) ? ld_pi(pi + pv[j]) : pv[j];
  }
  int H[K], L[K], old[K];
#pragma unroll
  for (int j = 0; j < K; ++j) {
    H[j] = -1;
    if (!live[j]) continue;
    const int ru = root_from2(pi, u[j], pu[j], gu[j]);
    const int rv = root_from2(pi, v[j], pv[j], gv[j]);
    if (ru == rv) continue;
    H[j] = ru > rv ? ru : rv;
    L[j] = ru > rv ? rv : ru;
  }
  if (DEDUP) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int j = 0; j < K; ++j) {
      const unsigned long long key =
          H[j] >= 0 ? (((unsigned long long)(unsigned)H[j] << 32) | (unsigned)L[j]) : ~0ull;
      const unsigned grp = __match_any_sync(kFull, key);
      if (H[j] >= 0 && lane != __ffs(grp) - 1) H[j] = -1;
    }
  }
#pragma unroll
  for (int j = 0; j < K; ++j)
    if (H[j] >= 0) old[j] = atomicCAS(pi + H[j], H[j], L[j]);
#pragma unroll
  for (int j = 0; j < K; ++j)
    if (H[j] >= 0 && old[j] != H[j] && old[j] != L[j]) atomic_hook(pi, old[j], L[j], V, c);
}

// pi(v) <- v over [0, V), grid-strided; 16-byte stores when pi is 16-byte aligned.
__device__ __forceinline__ void init_pi(int* pi, int V, long long tid, long long nthreads) {
  if ((reinterpret_cast<uintptr_t>(pi) & 15) == 0) {
    const long long n4 = V >> 2;
    int4* p4 = reinterpret_cast<int4*>(pi);
    for (long long q = tid; q < n4; q += nthreads) {
      const int v = (int)(q << 2);
      p4[q] = make_int4(v, v + 1, v + 2, v + 3);
    }
    for (long long v = (n4 << 2) + tid; v < V; v += nthreads) pi[v] = (int)v;
  } else {
    for (long long v = tid; v < V; v += nthreads) pi[v] = (int)v;
  }
}

// Multi-Jump (Fig. 3, bottom; Section III-A): every vertex jumps pi(v) <- pi(pi(v)) until
// pi(v) is a root, writing the intermediate value each step (optimisation (i)). Thread t
// takes vertices t, t + T, ... so lower IDs, the tops of the trees, are served first
// (optimisation (ii)). No hook runs concurrently, so roots are fixed during the phase.
__device__ __forceinline__ void jump_from(int* pi, int v, int p, int g, int V, const Ctl& c) {
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

__device__ __forceinline__ int4 ld_pi4(const int* p) {
  int4 v;
  asm volatile("ld.global.v4.s32 {%0, %1, %2, %3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(p));
  return v;
}

__device__ __forceinline__ void st_pi4(int* p, int4 v) {
  asm volatile("st.global.v4.s32 [%0], {%1, %2, %3, %4};" ::"l"(p), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w) : "memory");
}

// Jump of four consecutive vertices v..v+3 whose parents p were loaded: the grandparents g and
// great-grandparents h of all four are loaded together. A vertex whose grandparent is a root
// (h == g) ends at g; the four results go out in one 16-byte store when any moved. Deeper walks
// continue one step at a time, writing every step.
struct Jump4 {
  int4 p, g, h;
};

__device__ __forceinline__ int jump_gather(int* pi, int v, int p) { return p != v ? ld_pi(pi + p) : p; }

__device__ __forceinline__ void jump4_load(int* pi, int v, Jump4& s) {
  s.p = ld_pi4(pi + v);
}
__device__ __forceinline__ void jump4_level2(int* pi, int v, Jump4& s) {
  s.g = make_int4(jump_gather(pi, v, s.p.x), jump_gather(pi, v + 1, s.p.y), jump_gather(pi, v + 2, s.p.z),
                  jump_gather(pi, v + 3, s.p.w));
}
__device__ __forceinline__ void jump4_level3(int* pi, Jump4& s) {
  s.h = make_int4(jump_gather(pi, s.p.x, s.g.x), jump_gather(pi, s.p.y, s.g.y), jump_gather(pi, s.p.z, s.g.z),
                  jump_gather(pi, s.p.w, s.g.w));
}
__device__ __forceinline__ void jump4_finish(int* pi, int v, const Jump4& s, int V, const Ctl& c) {
  if (s.g.x != s.p.x || s.g.y != s.p.y || s.g.z != s.p.z || s.g.w != s.p.w) {
    st_pi4(pi + v, s.g);
    if (s.h.x != s.g.x) jump_from(pi, v, s.g.x, s.h.x, V, c);
    if (s.h.y != s.g.y) jump_from(pi, v + 1, s.g.y, s.h.y, V, c);
    if (s.h.z != s.g.z) jump_from(pi, v + 2, s.g.z, s.h.z, V, c);
    if (s.h.w != s.g.w) jump_from(pi, v + 3, s.g.w, s.h.w, V, c);
  }
}

__device__ __forceinline__ void multi_jump(int* pi, int V, long long tid, long long nthreads, const Ctl& c) {
  long long first_scalar = 0;
  if ((reinterpret_cast<uintptr_t>(pi) & 15) == 0) {
    // Two groups of four consecutive vertices per thread and step (groups q and q + T): their
    // 16-byte parent loads, then the grandparent and great-grandparent gathers of all eight are
    // issued level by level, so each thread keeps eight walks in flight.
    const long long n4 = V >> 2;
    for (long long q = tid; q < n4; q += 2 * nthreads) {
      const long long q2 = q + nthreads;
      const bool two = q2 < n4;
      const int v = (int)(q << 2), v2 = two ? (int)(q2 << 2) : v;
      Jump4 a, b;
      jump4_load(pi, v, a);
      if (two) jump4_load(pi, v2, b);
      else b.p = make_int4(v, v + 1, v + 2, v + 3);
      jump4_level2(pi, v, a);
      jump4_level2(pi, v2, b);
      jump4_level3(pi, a);
      jump4_level3(pi, b);
      jump4_finish(pi, v, a, V, c);
      if (two) jump4_finish(pi, v2, b, V, c);
    }
    first_scalar = n4 << 2;
  }
  for (long long vv = first_scalar + tid; vv < V; vv += nthreads) {
    const int v = (int)vv;
    const int p = ld_pi(pi + v);
    if (p == v) continue;
    jump_from(pi, v, p, ld_pi(pi + p), V, c);
  }
}

// One Jump of Fig. 2 over every vertex: pi(v) <- pi(pi(v)); sets `changed` if any value moved.
__device__ __forceinline__ void single_jump(int* pi, int V, long long tid, long long nthreads, const Ctl& c) {
  bool ch = false;
  for (long long vv = tid; vv < V; vv += nthreads) {
    const int v = (int)vv;
    const int p = ld_pi(pi + v);
    const int g = ld_pi(pi + p);
    if (g != p) {
      st_pi(pi + v, g);
      ch = true;
    }
  }
  if (__ballot_sync(kFull, ch) && (threadIdx.x & 31) == 0) c.st->changed = 1u;
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

// Root of x in a CTA-local parent array (shared memory), with path halving. The local array obeys the same invariant as pi (lp(x) <= x), so the walk ends
// within W steps.
template <typename LT>
__device__ __forceinline__ int lfind(volatile LT* lp, int x) {
  int px = lp[x];
  while (px != x) {
    const int gx = lp[px];
    if (gx == px) return px;
    lp[x] = (LT)gx;
    x = gx;
    px = lp[x];
  }
  return x;
}

__device__ __forceinline__ int cas_local(int* p, int cmp, int val) { return atomicCAS(p, cmp, val); }

// Atomic-Hook of local indices (a, b) on the shared-memory parent array: both roots are found,
// and the higher is CAS-linked to the lower until the CAS succeeds or the roots agree.
template <typename LT>
__device__ __forceinline__ void local_hook(LT* lp, int a, int b) {
  volatile LT* vlp = lp;
  int ra = lfind(vlp, a), rb = lfind(vlp, b);
  while (ra != rb) {
    const int H = ra > rb ? ra : rb;
    const int L = ra > rb ? rb : ra;
    const int old = cas_local(lp + H, H, L);
    if (old == H || old == L) return;
    ra = lfind(vlp, old);
    rb = lfind(vlp, L);
  }
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

// Row of the arc aq of this lane, from a window of 32 row ends held one per lane: lane l
// holds the end of row r + l, so the row is r + (number of window ends <= aq). When a lane's
// arc lies past the window (rows with few or no arcs), the warp searches row_ptr from r + 32.
// Returns V if no row exists (only when row_ptr[V] != n_arcs). Afterwards r is the row of the
// arc of lane `last` (the batch's last valid lane), the start of the next window. (rc, ec)
// caches the end ec of row rc: while the batch's last arc lies before the end of row r, every
// arc of the batch is in row r (arcs only increase), and the row needs no load and no search.
template <typename OffT>
__device__ __forceinline__ int resolve_row(const OffT* __restrict__ rp, int V, int& r, OffT aq, bool valid,
                                           int last, int& rc, OffT& ec) {
  const int lane = threadIdx.x & 31;
  const OffT alast = __shfl_sync(kFull, aq, last);
  if (rc == r && alast < ec) return r;  // warp-uniform
  const long long wi = (long long)r + 1 + lane;
  OffT e = ld_ro(rp + (wi < V ? wi : V));
  rc = r;
  ec = __shfl_sync(kFull, e, 0);
  if (alast < ec) return r;
  int cnt = window_count<OffT>(e, aq);
  int u = cnt < 32 ? r + cnt : -1;
  unsigned pend = __ballot_sync(kFull, valid && u < 0);
  while (pend) {
    if ((long long)r + 32 >= V) {
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
  const int nr = __shfl_sync(kFull, u, last);
  r = nr < V ? nr : V;
  return u;
}

// Per-warp staging buffer in shared memory for the worklist of the two-phase hook: arcs are
// appended by ballot (no atomics) and flushed to the global worklist with one atomic per flush.
constexpr int kSinkPairs = 112;
// Local hooks that the fast path of phase A could not finish wait in a per-warp queue of
// kDeferCap packed pairs (two 16-bit local indices) and are finished 32 at a time.
constexpr int kDeferCap = 64;
constexpr int kWarpScratchBytes = kSinkPairs * (int)sizeof(int2) + kDeferCap * (int)sizeof(unsigned);

// Flags a lane gathers during phase A (reported at the end of the window): bit 0 = a worklist
// append did not fit; bit 1 = an arc endpoint was outside [0, V), with (local row + 1) << 2 of
// the last such row above them.
constexpr int kSinkOverflow = 1;
constexpr int kSinkBadArc = 2;

struct WarpSink {
  int2* buf;   // kSinkPairs entries in shared memory, private to the warp, then kDeferCap
               // deferred local hooks
  int count;   // warp-uniform
  int dcount;  // warp-uniform, < 32 between calls
  int flags;   // kSinkOverflow | kSinkBadArc | bad row, per lane
  __device__ __forceinline__ unsigned* dq() const { return reinterpret_cast<unsigned*>(buf + kSinkPairs); }
};

// Points s at the calling warp's part of the per-warp scratch that starts at `base`.
__device__ __forceinline__ void warp_scratch_init(WarpSink& s, unsigned char* base) {
  s.buf = reinterpret_cast<int2*>(base + (threadIdx.x >> 5) * kWarpScratchBytes);
  s.count = 0;
  s.dcount = 0;
  s.flags = 0;
}

__device__ __forceinline__ void sink_flush(WarpSink& s, const Ctl& c) {
  if (s.count == 0) return;
  const int lane = threadIdx.x & 31;
  __syncwarp();
  unsigned long long base = 0;
  if (lane == 0) base = atomicAdd(&c.st->counters[2], (unsigned long long)s.count);
  base = __shfl_sync(kFull, base, 0);
  for (int i = lane; i < s.count; i += 32) {
    const unsigned long long pos = base + (unsigned long long)i;
    if (pos < c.wl_cap) c.wl[pos] = s.buf[i];
    else s.flags |= kSinkOverflow;
  }
  __syncwarp();
  s.count = 0;
}

// The local hook of (a, b) when it needs no root walk: done if a and b have the same parent or
// the same grandparent; else, if a parent is a root (its own parent) whose ID is above the other
// endpoint's grandparent, or both parents are roots, a CAS links that root to the other
// grandparent (or the larger root to the smaller): an ancestor of the other endpoint, so the
// invariant lp(x) <= x holds and the two trees are joined. Returns false when the hook is left for
// local_hook.
template <typename LT>
__device__ __forceinline__ bool local_hook_try(LT* lp, int a, int b) {
  volatile LT* vl = lp;
  const int pa = vl[a], pb = vl[b];
  if (pa == pb) return true;
  const int ga = vl[pa], gb = vl[pb];
  if (ga == gb) return true;
  const bool ra = pa == ga, rb = pb == gb;  // pa / pb is a root
  int H, L;
  if (ra && rb) {
    H = pa > pb ? pa : pb;
    L = pa > pb ? pb : pa;
  } else if (rb && pb > ga) {
    H = pb;
    L = ga;
  } else if (ra && pa > gb) {
    H = pa;
    L = gb;
  } else {
    return false;
  }
  return cas_local(lp + H, H, L) == H;
}

// Queues the hooks that local_hook_try left (lanes with `take`) and finishes 32 of them, one per
// lane, whenever 32 are waiting, so the root walks run with every lane busy.
template <typename LT>
__device__ __forceinline__ void defer_push(WarpSink& s, bool take, int a, int b, LT* lp) {
  const unsigned m = __ballot_sync(kFull, take);
  if (!m) return;
  const int lane = threadIdx.x & 31;
  if (take) s.dq()[s.dcount + __popc(m & ((1u << lane) - 1u))] = (unsigned)a | ((unsigned)b << 16);
  s.dcount += __popc(m);
  if (s.dcount >= 32) {
    __syncwarp();
    const unsigned e = s.dq()[s.dcount - 32 + lane];
    __syncwarp();
    s.dcount -= 32;
    local_hook(lp, (int)(e & 0xffffu), (int)(e >> 16));
  }
}

// Finishes the hooks still queued (fewer than 32).
template <typename LT>
__device__ __forceinline__ void defer_drain(WarpSink& s, LT* lp) {
  if (s.dcount == 0) return;
  const int lane = threadIdx.x & 31;
  __syncwarp();
  if (lane < s.dcount) {
    const unsigned e = s.dq()[lane];
    local_hook(lp, (int)(e & 0xffffu), (int)(e >> 16));
  }
  __syncwarp();
  s.dcount = 0;
}

__device__ __forceinline__ void sink_push(WarpSink& s, bool take, int u, int v, const Ctl& c) {
  const unsigned m = __ballot_sync(kFull, take);
  if (!m) return;
  const int n = __popc(m);
  if (s.count + n > kSinkPairs) sink_flush(s, c);
  const int lane = threadIdx.x & 31;
  if (take) s.buf[s.count + __popc(m & ((1u << lane) - 1u))] = make_int2(u, v);
  s.count += n;
}

// Atomic-Hook over the arcs [t0, t1) of a CSR graph by one warp, 32 x K arcs per step: lane l
// takes arcs b + l + 32 j, j < K (each j a coalesced read of col_idx), and the next step's
// arcs are loaded before the current ones are hooked, so the arc stream stays in flight.
// SYM: the CSR holds both directions of every edge, so arcs with u > v are skipped. Every arc
// is Atomic-Hooked on pi, K at a time (or with the plain-store hook of Fig. 2). lo_row is a row
// with rp[lo_row] <= t0; vbase is added to both endpoints (a graph of a batch) and `bad`
// records an endpoint outside [0, V).
// How hook_csr_range joins an arc's trees.
enum HookKind : int {
  kHookAtomic = 0,    // Atomic-Hook (Fig. 3, top)
  kHookNonAtomic = 1  // Hook of Fig. 2: pi(max(pi(u), pi(v))) <- min(...), plain store, sets `changed`
};

template <typename OffT, bool SYM, int K, int HOOK = kHookAtomic>
__device__ __forceinline__ void hook_csr_range(const OffT* __restrict__ rp, const int* __restrict__ col, int* pi,
                                               int V, OffT t0, OffT t1, const Ctl& c, int lo_row, int vbase = 0,
                                               volatile int* bad = nullptr) {
  const int lane = threadIdx.x & 31;
  int r = warp_row_search<OffT>(rp, lo_row, V, t0);
  int rc = -1;  // row whose end ec is cached by resolve_row
  OffT ec = 0;
  long long bad_at = -1;  // an arc with an endpoint outside [0, V), reported after the loop
  int vn[K];
#pragma unroll
  for (int j = 0; j < K; ++j) {
    const OffT a = t0 + 32 * j + lane;
    vn[j] = a < t1 ? ld_stream(col + a) : 0;
  }
  for (OffT b = t0; b < t1; b += 32 * K) {
    int v[K];
#pragma unroll
    for (int j = 0; j < K; ++j) v[j] = vn[j];
    const OffT nb = b + 32 * K;
    if (nb < t1) {
#pragma unroll
      for (int j = 0; j < K; ++j) {
        const OffT a = nb + 32 * j + lane;
        vn[j] = a < t1 ? ld_stream(col + a) : 0;
      }
    }
    int u[K];
    bool live[K];
#pragma unroll
    for (int j = 0; j < K; ++j) {
      const OffT bj = b + 32 * j;
      u[j] = -1;
      live[j] = false;
      if (bj < t1) {  // warp-uniform
        const OffT a = bj + lane;
        const bool valid = a < t1;
        const long long rem = (long long)(t1 - bj) - 1;
        u[j] = resolve_row<OffT>(rp, V, r, valid ? a : bj, valid, rem < 31 ? (int)rem : 31, rc, ec);
        if (valid) {
          const bool in_range = (unsigned)v[j] < (unsigned)V && (unsigned)u[j] < (unsigned)V;
          bad_at = in_range ? bad_at : (long long)a;
          live[j] = in_range && !(SYM ? (u[j] >= v[j]) : (u[j] == v[j]));
        }
      }
    }
    if (HOOK == kHookNonAtomic) {
      // Fig. 2: every tree is a star when a Hook round starts (the Compress before it ran to the
      // end), so pi(u) and pi(v) are roots; the larger is pointed at the smaller with a plain store.
      // Concurrent stores to one root may overwrite each other; the round then reports a change
      // and the host repeats it (Fig. 1), which is why this hook needs no atomics.
      bool ch = false;
#pragma unroll
      for (int j = 0; j < K; ++j) {
        if (!live[j]) continue;
        const int pu = ld_pi(pi + u[j]), pv = ld_pi(pi + v[j]);
        if (pu != pv) {
          st_pi(pi + (pu > pv ? pu : pv), pu > pv ? pv : pu);
          ch = true;
        }
      }
      if (__ballot_sync(kFull, ch) && lane == 0) c.st->changed = 1u;
    } else {
      if (vbase != 0) {  // graph of a batch: hook global IDs
#pragma unroll
        for (int j = 0; j < K; ++j) {
          u[j] += vbase;
          v[j] += vbase;
        }
      }
      atomic_hook_k<K>(pi, u, v, live, vbase + V, c);
    }
  }
  if (bad_at >= 0) {
    raise_input_error(c, kSiteHookArc, bad_at);
    if (bad) *bad = 1;
  }
}

constexpr int kHookK = 1;   // default arcs per lane per step of the plain hook (Ctl::hook_k)
constexpr int kPairK = 4;   // worklist pairs per thread per step of phase B

// hook_csr_range with c.hook_k arcs per lane per step (an autotuned choice: more arcs in flight per
// lane against fewer lanes' worth of registers).
template <typename OffT, bool SYM, int HOOK>
__device__ __forceinline__ void hook_csr_range_k(const OffT* __restrict__ rp, const int* __restrict__ col, int* pi,
                                                 int V, OffT t0, OffT t1, const Ctl& c) {
  if (HOOK == kHookAtomic && c.hook_k == 2) hook_csr_range<OffT, SYM, 2, HOOK>(rp, col, pi, V, t0, t1, c, 0);
  else if (HOOK == kHookAtomic && c.hook_k == 4) hook_csr_range<OffT, SYM, 4, HOOK>(rp, col, pi, V, t0, t1, c, 0);
  else hook_csr_range<OffT, SYM, kHookK, HOOK>(rp, col, pi, V, t0, t1, c, 0);
}

// Atomic-Hook over the arcs [a0, a1) of a CSR graph (one segment E_i of Fig. 4). With
// c.chunk_arcs > 0, warps take chunks of that many arcs from the work counter `ctr` (zeroed
// before the phase) until the segment is exhausted; otherwise each warp takes one fixed
// contiguous slice.
template <typename OffT, bool SYM, int HOOK = kHookAtomic>
__device__ __forceinline__ void hook_csr_arcs(const OffT* __restrict__ rp, const int* __restrict__ col, int* pi,
                                              int V, OffT a0, OffT a1, long long tid, long long nthreads,
                                              unsigned long long* ctr, const Ctl& c) {
  const OffT len = a1 - a0;
  if (len <= 0) return;
  if (c.chunk_arcs <= 0 || ctr == nullptr) {
    const long long warp = tid >> 5, nwarps = nthreads >> 5;
    const OffT t0 = a0 + split_point<OffT>(len, nwarps, warp);
    const OffT t1 = a0 + split_point<OffT>(len, nwarps, warp + 1);
    if (t0 < t1) hook_csr_range_k<OffT, SYM, HOOK>(rp, col, pi, V, t0, t1, c);
    return;
  }
  const OffT C = (OffT)c.chunk_arcs;
  const unsigned long long n_chunks = (unsigned long long)((len + C - 1) / C);
  const int lane = threadIdx.x & 31;
  for (;;) {
    unsigned long long t = 0;
    if (lane == 0) t = atomicAdd(ctr, 1ull);
    t = __shfl_sync(kFull, t, 0);
    if (t >= n_chunks) break;
    const OffT t0 = a0 + (OffT)t * C;
    const OffT t1 = (len - (OffT)t * C) > C ? t0 + C : a1;
    hook_csr_range_k<OffT, SYM, HOOK>(rp, col, pi, V, t0, t1, c);
  }
}

// ---------------------------------------------------------------------------------------------
// Sampled-and-filtered hook (CSR with CC_FLAG_SYMMETRIC): Fig. 4 with two arc subsets chosen for
// the edge filter. Slice 1 hooks the first kSampleArcs arcs of every row, a Multi-Jump makes every
// tree a star, and the largest star is found from a sample of roots. Slice 2 then reads only the
// rows of vertices outside that star and hooks their remaining arcs in both directions: an arc
// (u, v) whose row u lies in the star is not read, because u is already joined to the star and
// the reverse arc (v, u) is read from v's row unless v is in the star too (then u and v already
// share a tree). Without a star of at least kGiantSamples / 8 sampled roots, slice 2 is the plain
// hook of every arc.

constexpr int kSampleArcs = 2;
constexpr int kGiantSamples = 256;

// Slice 1: the first kSampleArcs arcs of rows tid, tid + T, ..., hooked together.
template <typename OffT>
__device__ __forceinline__ void hook_row_heads(const OffT* __restrict__ rp, const int* __restrict__ col, int* pi,
                                               int V, OffT nnz, long long tid, long long nthreads, const Ctl& c) {
  long long bad_at = -1;  // a row with bad offsets or an arc outside [0, V), reported after the loop
  for (long long x = tid; x < V; x += nthreads) {
    const int u = (int)x;
    OffT a0 = ld_ro(rp + u), a1 = ld_ro(rp + u + 1);
    const bool span_ok = a0 >= 0 && a0 <= a1 && a1 <= nnz;
    bad_at = span_ok ? bad_at : (long long)u;
    a1 = span_ok ? a1 : a0;
    int uu[kSampleArcs], v[kSampleArcs];
    bool live[kSampleArcs];
#pragma unroll
    for (int j = 0; j < kSampleArcs; ++j) {
      const bool has = (long long)a0 + j < (long long)a1;
      v[j] = has ? ld_stream(col + a0 + j) : 0;
      const bool in_range = (unsigned)v[j] < (unsigned)V;
      bad_at = (has && !in_range) ? (long long)a0 + j : bad_at;
      live[j] = has && in_range && v[j] != u;
      uu[j] = u;
    }
    atomic_hook_k<kSampleArcs>(pi, uu, v, live, V, c);
  }
  if (bad_at >= 0) raise_input_error(c, kSiteHookArc, bad_at);
}

// The most frequent root among n = min(kGiantSamples, blockDim.x) vertices spread over [0, V),
// if it holds at least one eighth of them, else -1. Called by one whole block after a Multi-Jump
// (pi(x) is then x's root). Only the speed depends on the answer: slice 2 is correct for any
// value, since a row is skipped only when its vertex's parent is that value.
__device__ __forceinline__ int giant_root(const int* pi, int V) {
  __shared__ int s_samples[kGiantSamples];
  __shared__ unsigned long long s_best;
  const int t = threadIdx.x;
  const int n = blockDim.x < kGiantSamples ? (int)blockDim.x : kGiantSamples;
  if (t == 0) s_best = 0ull;
  if (t < n) {
    const long long x = ((long long)t * (long long)V) / n + ((t * 40503) % 977) % (V / n + 1);
    s_samples[t] = ld_pi(pi + (x < V ? x : V - 1));
  }
  __syncthreads();
  if (t < n) {
    const int mine = s_samples[t];
    unsigned cnt = 0;
    for (int j = 0; j < n; ++j) cnt += s_samples[j] == mine ? 1u : 0u;
    atomicMax(&s_best, ((unsigned long long)cnt << 32) | (unsigned)mine);
  }
  __syncthreads();
  const unsigned long long best = s_best;
  return 8ull * (best >> 32) >= (unsigned long long)n ? (int)(best & 0xffffffffull) : -1;
}

// Slice 2: the arcs from position kSampleArcs on of every row whose vertex is not in the tree of
// `giant`, both directions, one row per lane; rows of more than 32 such arcs are walked by the
// whole warp, 32 arcs at a time.
template <typename OffT>
__device__ __forceinline__ void hook_rows_outside(const OffT* __restrict__ rp, const int* __restrict__ col, int* pi,
                                                  int V, OffT nnz, int giant, long long tid, long long nthreads,
                                                  const Ctl& c) {
  const int lane = threadIdx.x & 31;
  const long long warp = tid >> 5, nwarps = nthreads >> 5;
  long long bad_at = -1;  // an arc outside [0, V), reported after the loop
  for (long long base = warp * 32; base < V; base += nwarps * 32) {  // warp-uniform
    const long long x = base + lane;
    const int u = (int)x;
    long long a0 = 0, a1 = 0;
    if (x < V && ld_pi(pi + u) != giant) {
      a0 = (long long)ld_ro(rp + u);
      a1 = (long long)ld_ro(rp + u + 1);
      if (!(a0 >= 0 && a0 <= a1 && a1 <= (long long)nnz)) a1 = a0;  // reported by slice 1
      a0 = a0 + kSampleArcs < a1 ? a0 + kSampleArcs : a1;
    }
    const bool heavy = a1 - a0 > 32;
    if (!heavy) {
      for (long long a = a0; a < a1; ++a) {
        const int v = ld_stream(col + a);
        const bool in_range = (unsigned)v < (unsigned)V;
        bad_at = in_range ? bad_at : a;
        if (in_range && v != u) atomic_hook(pi, u, v, V, c);
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
        const bool has = a < h1;
        const int v = has ? ld_stream(col + a) : 0;
        const bool in_range = (unsigned)v < (unsigned)V;
        bad_at = (has && !in_range) ? a : bad_at;
        const int uu[1] = {hu}, vv[1] = {v};
        const bool live[1] = {has && in_range && v != hu};
        atomic_hook_k<1>(pi, uu, vv, live, V, c);
      }
    }
  }
  if (bad_at >= 0) raise_input_error(c, kSiteHookArc, bad_at);
}

// Bytes of dynamic shared memory of phase A for a block of `block` threads: the window's parent
// array (W entries of lt_bytes each) followed by the per-warp scratch (worklist sink and queue
// of deferred local hooks).
__host__ __device__ __forceinline__ size_t tiled_smem_bytes(int W, int block, int lt_bytes = (int)sizeof(int)) {
  const size_t lp = ((size_t)W * (size_t)lt_bytes + 15) & ~(size_t)15;
  return lp + (size_t)(block / 32) * kWarpScratchBytes;
}

// Rows with more arcs than this are walked by a whole warp in phase A.
constexpr int kHeavyRow = 32;
// Rows of more than kHeavyRow arcs that a window can hand to the whole CTA (more are walked by
// the warp that found them).
constexpr int kHeavyCap = 128;

// Rows of a window handed to the whole CTA: row i has arcs [a0, a1); blocks of 32 arcs are
// numbered across the rows (prefix[h] = first block of row h).
struct HeavyRows {
  int n;
  int row[kHeavyCap];
  long long a0[kHeavyCap];
  long long a1[kHeavyCap];
  int prefix[kHeavyCap + 1];
};
// Arcs of a row loaded together in phase A.
constexpr int kGroup = 4;

// Arc span [x0, x1) of window row i (0, 0 past the end of the warp's rows).
template <typename OffT>
__device__ __forceinline__ void load_row_span(const OffT* __restrict__ rp, int w0, int i, int end, OffT& x0,
                                              OffT& x1) {
  if (i < end) {
    x0 = ld_ro(rp + w0 + i);
    x1 = ld_ro(rp + w0 + i + 1);
  } else {
    x0 = 0;
    x1 = 0;
  }
}

// Offsets inconsistent with n_arcs are reported and replaced by an empty span, so no read
// of col_idx leaves [0, n_arcs).
template <typename OffT>
__device__ __forceinline__ void check_span(OffT& x0, OffT& x1, OffT nnz, int u, const Ctl& c) {
  if (!(x0 >= 0 && x0 <= x1 && x1 <= nnz)) {
    raise_input_error(c, kSiteHookArc, (long long)u);
    x0 = 0;
    x1 = 0;
  }
}

// Arcs x0 + kGroup*g + j (j < kGroup) of a row, 0 beyond its end.
template <typename OffT>
__device__ __forceinline__ void load_group(const int* __restrict__ col, OffT x0, OffT x1, int g, int (&v)[kGroup]) {
#pragma unroll
  for (int j = 0; j < kGroup; ++j) {
    const long long a = (long long)x0 + g * kGroup + j;  // no wrap for an int32 x1 near 2^31
    v[j] = a < (long long)x1 ? ld_stream(col + a) : 0;
  }
}

// Phase A work for one arc (u, v) of window [w0, w0 + nrows), u = w0 + i in the window. IDs
// are local to the graph (< V); worklist entries get vbase added (the graph's first vertex in a
// batch). An endpoint outside [0, V) is only flagged here (no branch on the hot path);
// phase_a_window reports it once per window. ia >= 0: the arc to u + 1 is hooked from local row
// ia instead of i (the first row of the run of u -> u + 1 arcs that reaches u).
template <bool SYM, typename LT>
__device__ __forceinline__ void phase_a_arc(bool has, int i, int u, int v, int V, int w0, int nrows, LT* lp,
                                            WarpSink& sink, int vbase, const Ctl& c, int ia = -1) {
  const bool in_range = has && (unsigned)v < (unsigned)V;
  sink.flags = (has && !in_range) ? ((sink.flags & kSinkOverflow) | kSinkBadArc | ((i + 1) << 2)) : sink.flags;
  const bool live = in_range && (SYM ? (v > u) : (v != u));
  const int b = v - w0;
  const bool local = live && (unsigned)b < (unsigned)nrows;
  const int a = (ia >= 0 && v == u + 1) ? ia : i;
  const bool left = local && !local_hook_try(lp, a, b);
  defer_push(sink, left, a, b, lp);
  sink_push(sink, live && !local, u + vbase, v + vbase, c);
}

// Phase A of one window [w0, w0 + nrows) of a graph with V vertices and nnz arcs (rows rp,
// arcs col, graph-local IDs), by the whole CTA: lp must hold lp[i] = i on entry (and a barrier
// must separate that from this call); on return (after a barrier) lp holds the window's local
// forest. Warps take 32-row chunks (one row per lane) in an interleaved order, so the CTA sweeps
// the window roughly in ID order and new vertices mostly join components that already have
// short paths to their roots. Row offsets are loaded one chunk ahead. Rows of more than
// kHeavyRow arcs are set aside (up to kHeavyCap per window) and walked after the light rows by
// all warps of the CTA together, 32 consecutive arcs per warp step, so one hub row does not
// hold its warp, and with it the window, for thousands of steps; past kHeavyCap the warp that
// found a heavy row walks it itself.
template <typename OffT, bool SYM, typename LT>
__device__ __forceinline__ void phase_a_window(const OffT* __restrict__ rp, const int* __restrict__ col, int V,
                                               OffT nnz, int w0, int nrows, int vbase, LT* lp, WarpSink& sink,
                                               volatile int* ovf, volatile int* bad, const Ctl& c) {
  __shared__ HeavyRows s_heavy;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int step = nwarps * 32;
  const int r_begin = warp * 32;
  const int r_end = nrows;
  if (threadIdx.x == 0) s_heavy.n = 0;
  __syncthreads();
  if (r_begin < r_end) {  // warp-uniform
    OffT a0, a1, na0, na1;
    load_row_span<OffT>(rp, w0, r_begin + lane, r_end, na0, na1);
    for (int base = r_begin; base < r_end; base += step) {
      a0 = na0;
      a1 = na1;
      check_span<OffT>(a0, a1, nnz, w0 + base + lane, c);
      int v[kGroup];
      load_group<OffT>(col, a0, a1, 0, v);
      load_row_span<OffT>(rp, w0, base + step + lane, r_end, na0, na1);
      const int i = base + lane;
      const int u = w0 + i;
      const long long deg = (long long)(a1 - a0);
      const bool heavy = deg > kHeavyRow;
      // Arcs u -> u + 1 inside the warp's 32 rows form runs of consecutive rows; the arc into row
      // u + 1 is hooked from the run's first row instead (the same tree joined through the run),
      // so a run becomes one star rather than a chain of parents.
      bool right = false;
#pragma unroll
      for (int j = 0; j < kGroup; ++j) right |= (!heavy && j < deg && v[j] == u + 1);
      right = right && lane < 31 && i + 1 < nrows;
      const unsigned rmask = __ballot_sync(kFull, right);
      const unsigned below = ~rmask & ((2u << lane) - 1u);
      const int run0 = below ? 32 - __clz(below) : 0;
      const int ia = right ? i - lane + run0 : -1;
#pragma unroll
      for (int j = 0; j < kGroup; ++j)
        phase_a_arc<SYM, LT>(!heavy && j < deg, i, u, v[j], V, w0, nrows, lp, sink, vbase, c, ia);
      const int maxdeg = __reduce_max_sync(kFull, heavy ? 0 : (int)deg);
      for (int g = 1; g * kGroup < maxdeg; ++g) {
        int w[kGroup];
        load_group<OffT>(col, a0, heavy ? a0 : a1, g, w);
#pragma unroll
        for (int j = 0; j < kGroup; ++j)
          phase_a_arc<SYM, LT>(!heavy && g * kGroup + j < deg, i, u, w[j], V, w0, nrows, lp, sink, vbase, c);
      }
      bool handed = false;
      if (heavy) {
        const int slot = atomicAdd(&s_heavy.n, 1);
        if (slot < kHeavyCap) {
          s_heavy.row[slot] = i;
          s_heavy.a0[slot] = (long long)a0;
          s_heavy.a1[slot] = (long long)a1;
          handed = true;
        }
      }
      unsigned hv = __ballot_sync(kFull, heavy && !handed);
      while (hv) {  // heavy rows the CTA list could not take: the warp walks each one 32 arcs at a time
        const int h = __ffs(hv) - 1;
        hv &= hv - 1;
        const int hi = __shfl_sync(kFull, i, h);
        // 64-bit positions: an int32 nnz near 2^31 must not wrap past the row's end
        const long long h0 = (long long)__shfl_sync(kFull, a0, h), h1 = (long long)__shfl_sync(kFull, a1, h);
        for (long long bb = h0; bb < h1; bb += 32) {
          const long long a = bb + lane;
          const bool has = a < h1;
          const int vv = has ? ld_stream(col + a) : 0;
          phase_a_arc<SYM, LT>(has, hi, w0 + hi, vv, V, w0, nrows, lp, sink, vbase, c);
        }
      }
    }
  }
  __syncthreads();
  const int nh = s_heavy.n < kHeavyCap ? s_heavy.n : kHeavyCap;
  if (nh > 0) {  // CTA-uniform: the handed-over heavy rows, 32-arc blocks spread over all warps
    if (warp == 0) {
      int carry = 0;
      for (int h0 = 0; h0 < nh; h0 += 32) {
        const int h = h0 + lane;
        int nb = h < nh ? (int)((s_heavy.a1[h] - s_heavy.a0[h] + 31) >> 5) : 0;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
          const int y = __shfl_up_sync(kFull, nb, d);
          if (lane >= d) nb += y;
        }
        if (h < nh) s_heavy.prefix[h + 1] = carry + nb;
        carry += __shfl_sync(kFull, nb, 31);
      }
      if (lane == 0) s_heavy.prefix[0] = 0;
    }
    __syncthreads();
    const int total = s_heavy.prefix[nh];
    for (int k = warp; k < total; k += nwarps) {
      int lo = 0, hi = nh;  // prefix[lo] <= k < prefix[hi]
      while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (s_heavy.prefix[mid] <= k) lo = mid;
        else hi = mid;
      }
      const int hr = s_heavy.row[lo];
      const long long a = s_heavy.a0[lo] + 32ll * (k - s_heavy.prefix[lo]) + lane;
      const bool has = a < s_heavy.a1[lo];
      const int vv = has ? ld_stream(col + a) : 0;
      phase_a_arc<SYM, LT>(has, hr, w0 + hr, vv, V, w0, nrows, lp, sink, vbase, c);
    }
  }
  defer_drain(sink, lp);
  sink_flush(sink, c);
  if (sink.flags & kSinkOverflow) *ovf = 1;
  if (sink.flags & kSinkBadArc) {
    raise_input_error(c, kSiteWindowRow, (long long)w0 + (sink.flags >> 2) - 1);
    *bad = 1;
  }
  sink.flags = 0;
  __syncthreads();
}

// lp[i] = i for the window's rows, four entries per 16-byte shared store (lp is 16-byte aligned).
template <typename LT>
__device__ __forceinline__ void local_init(LT* lp, int nrows) {
  if (sizeof(LT) == 4) {
    int4* lp4 = reinterpret_cast<int4*>(lp);
    for (int q = threadIdx.x; q < (nrows >> 2); q += blockDim.x) lp4[q] = make_int4(4 * q, 4 * q + 1, 4 * q + 2, 4 * q + 3);
    for (int i = (nrows & ~3) + threadIdx.x; i < nrows; i += blockDim.x) lp[i] = (LT)i;
  } else {
    for (int i = threadIdx.x; i < nrows; i += blockDim.x) lp[i] = (LT)i;
  }
}

// pi(w0 + i) = w0 + local root of i for the window's rows. Four consecutive rows per thread:
// their parents, grandparents and great-grandparents are read level by level, a root found at
// the second level ends the walk (deeper trees finish with lfind), and the four labels leave in
// one 16-byte store when pi + w0 is 16-byte aligned.
template <typename LT>
__device__ __forceinline__ void publish_window(int* pi, int w0, LT* lp, int nrows) {
  volatile LT* vlp = lp;
  int q_end = 0;
  if (sizeof(LT) == 4 && (reinterpret_cast<uintptr_t>(pi + w0) & 15) == 0) {
    q_end = nrows >> 2;
    for (int q = threadIdx.x; q < q_end; q += blockDim.x) {
      int r[4], g[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) r[k] = vlp[4 * q + k];
#pragma unroll
      for (int k = 0; k < 4; ++k) g[k] = vlp[r[k]];
#pragma unroll
      for (int k = 0; k < 4; ++k) r[k] = g[k] == r[k] ? r[k] : lfind(vlp, g[k]);
      *reinterpret_cast<int4*>(pi + w0 + 4 * q) = make_int4(w0 + r[0], w0 + r[1], w0 + r[2], w0 + r[3]);
    }
  }
  for (int i = 4 * q_end + threadIdx.x; i < nrows; i += blockDim.x) pi[w0 + i] = w0 + lfind(vlp, i);
}

// Two-phase hierarchical Atomic-Hook, phase A. The vertices are cut into windows of W
// consecutive IDs; a CTA takes windows from work counter 0. For window [w0, w0 + W) it keeps a
// local parent array lp in shared memory and streams the arcs of the window's rows once, one
// row per lane (rows of more than kHeavyRow arcs by the whole warp): an arc with both
// endpoints in the window is Atomic-Hooked on lp (the high-to-low CAS rule on local indices);
// any other arc goes to the worklist. The local trees are then compressed and written as the
// window's part of pi with plain stores: pi(x) = w0 + local root of x, the minimum vertex of
// x's local component. Every vertex belongs to exactly one window, so this also initialises
// pi, and no two CTAs write the same entry. If the worklist is full, the window is recorded as
// overflowed and phase B hooks all of its arcs again on pi. LT is the type of the local parent
// entries (a 32-bit shared-memory CAS must exist for it).
template <typename OffT, bool SYM, typename LT>
__device__ __forceinline__ void tiled_phase_a(const OffT* __restrict__ rp, const int* __restrict__ col, int* pi,
                                              int V, OffT nnz, unsigned char* smem, const Ctl& c) {
  __shared__ unsigned long long s_unit;
  __shared__ int s_ovf, s_bad;
  const int W = c.tile_w;
  LT* lp = reinterpret_cast<LT*>(smem);
  const long long n_units = ((long long)V + W - 1) / W;
  WarpSink sink;
  warp_scratch_init(sink, smem + (((size_t)W * sizeof(LT) + 15) & ~(size_t)15));
  for (;;) {
    if (threadIdx.x == 0) {
      s_unit = atomicAdd(&c.st->counters[0], 1ull);
      s_ovf = 0;
      s_bad = 0;
    }
    __syncthreads();
    const unsigned long long k = s_unit;
    if (k >= (unsigned long long)n_units) break;
    const int w0 = (int)(k * (unsigned long long)W);
    const int nrows = (V - w0) < W ? (V - w0) : W;
    local_init(lp, nrows);
    __syncthreads();
    phase_a_window<OffT, SYM, LT>(rp, col, V, nnz, w0, nrows, 0, lp, sink, &s_ovf, &s_bad, c);
    publish_window(pi, w0, lp, nrows);
    if (threadIdx.x == 0 && s_ovf) {
      const unsigned long long j = atomicAdd(&c.st->counters[3], 1ull);
      if (j < (unsigned long long)c.ovf_cap) c.ovf_units[j] = (int)k;
    }
    __syncthreads();
  }
}

// Atomic-Hook on pi of worklist pairs [p0, p1), K per thread and step (each j a coalesced read),
// with the pairs that reach the same two roots in a warp hooked once. The loop is warp-uniform
// (lanes past the end carry no pair), as the deduplication needs.
__device__ __forceinline__ void hook_worklist(int* pi, const int2* __restrict__ wl, unsigned long long p0,
                                              unsigned long long p1, long long tid, long long nthreads, int V,
                                              const Ctl& c) {
  constexpr int K = kPairK;
  const unsigned long long T = (unsigned long long)nthreads;
  const unsigned long long lane = (unsigned long long)(threadIdx.x & 31);
  for (unsigned long long base = p0 + (unsigned long long)tid; base - lane < p1; base += T * K) {
    int u[K], v[K];
    bool live[K];
#pragma unroll
    for (int j = 0; j < K; ++j) {
      const unsigned long long i = base + (unsigned long long)j * T;
      live[j] = i < p1;
      const int2 e = live[j] ? wl[i] : make_int2(0, 0);
      u[j] = e.x;
      v[j] = e.y;
    }
    atomic_hook_k<K, true>(pi, u, v, live, V, c);
  }
}

// Phase B, one segment: Atomic-Hook on pi of worklist pairs [p0, p1) and, when `overflowed` is
// set, of every arc of the windows listed as overflowed (one CTA per window).
template <typename OffT, bool SYM>
__device__ __forceinline__ void tiled_phase_b(const OffT* __restrict__ rp, const int* __restrict__ col, int* pi,
                                              int V, OffT nnz, unsigned long long p0, unsigned long long p1,
                                              bool overflowed, unsigned long long n_ovf, long long tid,
                                              long long nthreads, const Ctl& c) {
  hook_worklist(pi, c.wl, p0, p1, tid, nthreads, V, c);
  if (!overflowed) return;
  const int W = c.tile_w;
  const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  for (unsigned long long j = blockIdx.x; j < n_ovf; j += gridDim.x) {
    const int w0 = c.ovf_units[j] * W;
    const int nrows = (V - w0) < W ? (V - w0) : W;
    const OffT u0 = ld_ro(rp + w0), u1 = ld_ro(rp + w0 + nrows);
    if (!(u0 >= 0 && u0 <= u1 && u1 <= nnz)) continue;
    const OffT t0 = u0 + split_point<OffT>(u1 - u0, nwarps, warp);
    const OffT t1 = u0 + split_point<OffT>(u1 - u0, nwarps, warp + 1);
    if (t0 < t1) hook_csr_range<OffT, SYM, kHookK>(rp, col, pi, V, t0, t1, c, w0);
  }
}

// Atomic-Hook over edges [e0, e1) of an edge list, K edges per thread per step.
__device__ __forceinline__ void hook_coo_edges(const int* __restrict__ src, const int* __restrict__ dst, int* pi,
                                               int V, long long e0, long long e1, long long tid,
                                               long long nthreads, const Ctl& c) {
  constexpr int K = kHookK;
  long long bad_at = -1;  // an edge with an endpoint outside [0, V), reported after the loop
  for (long long base = e0 + tid; base < e1; base += nthreads * K) {
    int u[K], v[K];
    bool live[K];
#pragma unroll
    for (int j = 0; j < K; ++j) {
      const long long i = base + (long long)j * nthreads;
      const bool valid = i < e1;
      u[j] = valid ? ld_stream(src + i) : 0;
      v[j] = valid ? ld_stream(dst + i) : 0;
      const bool in_range = (unsigned)u[j] < (unsigned)V && (unsigned)v[j] < (unsigned)V;
      bad_at = (valid && !in_range) ? i : bad_at;
      live[j] = valid && in_range && u[j] != v[j];
    }
    atomic_hook_k<K>(pi, u, v, live, V, c);
  }
  if (bad_at >= 0) raise_input_error(c, kSiteHookArc, bad_at);
}

}  // namespace cc
