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
};

enum : int { kKindCsr = 1, kKindCoo = 2 };

struct LaunchShape {
  int grid;
  int block;
};

// Blocks of the persistent kernel that fit on one SM at `block` threads (0 if it cannot run).
int persistent_blocks_per_sm(const Problem& p, int block);
int stage_blocks_per_sm(const Problem& p, int block);

// One cooperative launch running init + all segments (Hook, barrier, Multi-Jump, barrier).
cudaError_t launch_persistent(const Problem& p, const Ctl& c, LaunchShape s, cudaStream_t stream);

// Fig. 4 as printed: init, then per segment one Hook launch and one Multi-Jump launch.
// Returns the number of launches issued in *launches.
cudaError_t launch_multi(const Problem& p, const Ctl& c, LaunchShape s, cudaStream_t stream, int* launches);

// Device checks of CSR offsets and endpoints (CC_FLAG_VALIDATE).
cudaError_t launch_validate(const Problem& p, const Ctl& c, LaunchShape s, cudaStream_t stream);

}  // namespace cc
