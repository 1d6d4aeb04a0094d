// Host-side declarations shared by the library's translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "cc_device.cuh"

namespace cc {

// One single-graph problem as the kernels see it.
struct Problem {
  int kind;            // kKindCsr or kKindCoo
  const void* rp;      // CSR row offsets (int32 or int64)
  bool rp64;
  const int* col;      // CSR col_idx
  const int* src;      // COO
  const int* dst;      // COO
  int* pi;             // labels / parent array
  int V;
  long long m;         // arcs (CSR) or edges (COO)
  int segments;
  bool sym;
  int tile_w;          // > 0: hierarchical hook with this window (CSR only)
  bool filtered;       // sampled-and-filtered hook (CSR with sym only)
};

enum : int { kKindCsr = 1, kKindCoo = 2 };

struct LaunchShape {
  int grid;
  int block;
};

// Blocks of the cooperative kernel of p (the plain persistent driver, or phase B of the
// hierarchical hook when p.tile_w > 0) that fit on one SM at `block` threads (0 if it cannot run).
int persistent_blocks_per_sm(const Problem& p, int block);
int stage_blocks_per_sm(const Problem& p, int block);
// Blocks of the phase-A kernel of the hierarchical hook per SM, with its window in shared memory.
int phase_a_blocks_per_sm(const Problem& p, int block);

// Segment plan of Fig. 4 (Section III-B): requested > 0 = exactly that many segments; -1 = the
// paper's s = max(1, round(arcs / V)); 0 = this library's default from the segmentation sweep on
// GB300 (s = 4 below an average degree of 3, else 1).
int default_segments(long long arcs, long long V, int requested);
// Automatic work split of the plain hook for a launch of `warps` warps: the chunk size (arcs)
// warps take from a counter, or -1 for one fixed slice of the segment per warp.
int auto_chunk_arcs(long long arcs_per_segment, long long warps);

// One cooperative launch running init + all segments (Hook, barrier, Multi-Jump, barrier).
cudaError_t launch_persistent(const Problem& p, const Ctl& c, LaunchShape s, cudaStream_t stream);

// Hierarchical hook (p.tile_w > 0): the phase-A launch (shape sa, windows from a work counter),
// then the cooperative phase-B launch (shape sb: worklist segments, each with a Multi-Jump).
cudaError_t launch_two_phase(const Problem& p, const Ctl& c, LaunchShape sa, LaunchShape sb, cudaStream_t stream);

// The adaptive method of Section III driven by the host: init, then per segment one Hook launch
// and one Multi-Jump launch.
// Returns the number of launches issued in *launches.
cudaError_t launch_multi(const Problem& p, const Ctl& c, LaunchShape s, cudaStream_t stream, int* launches);

// One graph of a descriptor-mode batch: its labels, row offsets and arcs sit at these element
// offsets of the label, row-offset and arc arenas (layout-compatible with cc_graph_desc).
struct GraphDesc {
  long long label_off;
  long long row_off;
  long long arc_off;
  long long n_arcs;
  int n_vertices;
  int reserved;
};

// A batch of graphs over a graph-offset table or descriptors (see cc_batched.cu).
struct BatchProblem {
  int n_graphs;
  const GraphDesc* desc;
  const long long* v_off;
  const long long* a_off;
  const int* rp_cat;
  const int* col_cat;
  int* labels;
  int* graph_status;
  long long* unit_start;
  int* plain_units;
  int plain_cap;
  long long* plain_chunk_start;  // [plain_cap + 2] chunk table of plain_units and chunk size (kernel-filled)
  int* graph_hint;               // [n_graphs] giant-star root per graph (kernel-filled, symmetric batches)
  long long total_v;    // label arena size
  long long row_elems;  // descriptor mode: arena sizes
  long long arc_elems;
  bool sym;
};
int batched_blocks_per_sm(bool sym, int block, int W);
cudaError_t launch_batched(const BatchProblem& p, const Ctl& c, LaunchShape s, cudaStream_t stream);

// Locality sample: out[0] += sampled arcs with both ends in one window of W vertices,
// out[1] += sampled arcs (out must be zeroed by the caller).
// out[2] += sampled rows whose degree is below a quarter of the mean, out[3] += sampled rows.
cudaError_t launch_sample_locality(const Problem& p, int W, unsigned long long* out, int threads, cudaStream_t stream);

// Kernels of the host-driven loop of Fig. 1 (Soman et al.'s Hook-Compress with the Hook and
// Jump of Fig. 2), kept for the ablation of Section IV: pi init; one non-atomic Hook round over
// all arcs; one single Jump over all vertices; one Multi-Jump over all vertices. The Hook and
// Jump rounds set DevStatus::changed.
cudaError_t launch_init_only(const Problem& p, const Ctl& c, LaunchShape s, cudaStream_t stream);
cudaError_t launch_hook_nonatomic(const Problem& p, const Ctl& c, LaunchShape s, cudaStream_t stream);
cudaError_t launch_jump_single(const Problem& p, const Ctl& c, LaunchShape s, cudaStream_t stream);
cudaError_t launch_jump_multi(const Problem& p, const Ctl& c, LaunchShape s, cudaStream_t stream);

// Atomic-Hook of the arcs [a0, a1) of a CSR graph whose arcs are not resident: col_seg is a
// device buffer holding exactly those arcs (one segment of Fig. 4 streamed in from the host).
// p.rp and p.pi are on the device. Work counter 0 must be zero (k_init / k_jump reset it).
cudaError_t launch_hook_segment(const Problem& p, const int* col_seg, long long a0, long long a1, const Ctl& c,
                                LaunchShape s, cudaStream_t stream);

// Small graphs in one thread-block cluster (cc_cluster.cu): pi in the distributed shared memory of
// C CTAs (8, or 16 where the GPU allows it), at most 2^kClusterMaxShift vertices per CTA.
constexpr int kClusterMaxShift = 15;
// Cluster size that can hold p in one cluster of co-resident CTAs, or 0.
int cluster_size_for(const Problem& p);
// One launch of C CTAs: writes the labels into p.pi.
cudaError_t launch_cluster(const Problem& p, const Ctl& c, int C, cudaStream_t stream);

// 64-bit vertex IDs (cc_wide.cu): init, Atomic-Hook of every arc, Multi-Jump; three launches of
// `grid` blocks on `stream`. wide_blocks_per_sm: co-resident blocks of the hook kernel per SM.
int wide_blocks_per_sm(bool sym);
cudaError_t launch_wide(const long long* rp, const long long* col, long long* pi, long long V, long long nnz, bool sym,
                        const Ctl& c, int grid, cudaStream_t stream);

// Device checks of CSR offsets and endpoints (CC_FLAG_VALIDATE).
cudaError_t launch_validate(const Problem& p, const Ctl& c, LaunchShape s, cudaStream_t stream);

}  // namespace cc
