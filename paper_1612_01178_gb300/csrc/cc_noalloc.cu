// cc_labels_csr_noalloc: the persistent CSR labelling without any allocation.
//
// Some callers cannot call cudaMalloc: code running inside a custom device allocator or
// memory pool (which must not re-enter the allocator), plug-ins of hosts that own all device
// memory and forbid others from allocating, and tight real-time paths that must not pay for
// (or fail in) an allocation. This entry point needs no context. Its only scratch memory, the
// status block (grid-barrier counter, work counters, error word) that the persistent kernel
// needs beyond the caller's input and output arrays, lives in the file-scope device array below.
//
// The array is allocated when the library is loaded and stays allocated on every GPU that
// loads the library until the process exits. Every call shares it and it keeps the last
// call's contents, so each call clears it on its stream before the launch; two calls whose
// work overlaps on the GPU (different streams, no ordering between them) race on it and
// must not be issued.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "cc.h"
#include "cc_internal.h"

namespace {

constexpr size_t kScratchBytes = 256;  // the stated maximum: one status block (sizeof(DevStatus) = 96 bytes used)
static_assert(sizeof(cc::DevStatus) <= kScratchBytes, "status block must fit the static scratch");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void* g_scratch_ptr[kMaxDevices] = {nullptr};
int g_num_sms[kMaxDevices] = {0};

// Once per device, with that device current: the device address of the static scratch.
cudaError_t scratch_for_device(int device, cc::DevStatus** out, int* num_sms) {
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) return e;
    g_num_sms[device] = sms;
    g_scratch_ptr[device] = p;
  }
  *out = static_cast<cc::DevStatus*>(g_scratch_ptr[device]);
  *num_sms = g_num_sms[device];
  return cudaSuccess;
}

}  // namespace

extern "C" cc_status cc_labels_csr_noalloc(int64_t n_vertices, int64_t n_arcs, const void* row_ptr,
                                           cc_index_type row_ptr_type, const int32_t* col_idx, int32_t* labels,
                                           void* stream, int32_t flags) {
  if (n_vertices < 0 || n_vertices > INT32_MAX || n_arcs < 0) return CC_ERR_INVALID_ARG;
  if (row_ptr_type != CC_INDEX_I32 && row_ptr_type != CC_INDEX_I64) return CC_ERR_INVALID_ARG;
  if (row_ptr_type == CC_INDEX_I32 && n_arcs > INT32_MAX) return CC_ERR_INVALID_ARG;
  if (flags & ~CC_FLAG_SYMMETRIC) return CC_ERR_INVALID_ARG;
  if (!row_ptr || (n_vertices > 0 && !labels) || (n_arcs > 0 && (!col_idx || n_vertices == 0)))
    return CC_ERR_INVALID_ARG;
  const size_t lab_bytes = (size_t)n_vertices * 4;
  const uintptr_t lab = (uintptr_t)labels, rp = (uintptr_t)row_ptr, col = (uintptr_t)col_idx;
  const size_t rp_bytes = (size_t)(n_vertices + 1) * (size_t)row_ptr_type, col_bytes = (size_t)n_arcs * 4;
  if (lab && rp && lab < rp + rp_bytes && rp < lab + lab_bytes) return CC_ERR_INVALID_ARG;
  if (lab && col && col_bytes && lab < col + col_bytes && col < lab + lab_bytes) return CC_ERR_INVALID_ARG;
  if (n_vertices == 0) return CC_OK;

  int device = -1;
  if (cudaGetDevice(&device) != cudaSuccess || device < 0 || device >= kMaxDevices) {
    cudaGetLastError();
    return CC_ERR_CUDA;
  }
  cc::DevStatus* scratch = nullptr;
  int num_sms = 0;
  if (scratch_for_device(device, &scratch, &num_sms) != cudaSuccess) {
    cudaGetLastError();
    return CC_ERR_CUDA;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // The call reads its status back and waits for the stream, which a capturing stream does not
  // allow: refuse before touching the stream, so the caller's capture stays valid.
  cudaStreamCaptureStatus cap_status = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap_status) != cudaSuccess) {
    cudaGetLastError();
    return CC_ERR_CUDA;
  }
  if (cap_status != cudaStreamCaptureStatusNone) return CC_ERR_INVALID_ARG;

  cc::Problem p{};
  p.kind = cc::kKindCsr;
  p.rp = row_ptr;
  p.rp64 = row_ptr_type == CC_INDEX_I64;
  p.col = col_idx;
  p.pi = labels;
  p.V = (int)n_vertices;
  p.m = n_arcs;
  p.sym = (flags & CC_FLAG_SYMMETRIC) != 0;
  // the same segment plan as cc_labels_csr with default options
  p.segments = n_arcs > 0 ? cc::default_segments(n_arcs, n_vertices, 0) : 1;

  const int block = 256;
  const int per_sm = cc::persistent_blocks_per_sm(p, block);
  if (per_sm <= 0) {
    cudaGetLastError();
    return CC_ERR_CUDA;
  }
  const long long work = n_vertices > n_arcs / 4 ? n_vertices : n_arcs / 4;
  long long grid = (work + block - 1) / block;
  const long long cap = (long long)per_sm * num_sms;
  if (grid > cap) grid = cap;
  if (grid < 1) grid = 1;

  cc::Ctl c;
  c.st = scratch;
  c.timeout_ns = 2000000000LL;
  c.skip_arrival_block = -1;
  c.chunk_arcs = cc::auto_chunk_arcs(n_arcs / p.segments, grid * (block / 32));

  // The scratch keeps the previous call's barrier count and error word: clear them first.
  cudaError_t e = cudaMemsetAsync(scratch, 0, sizeof(cc::DevStatus), s);
  if (e == cudaSuccess) e = cc::launch_persistent(p, c, cc::LaunchShape{(int)grid, block}, s);
  cc::DevStatus result;
  std::memset(&result, 0, sizeof(result));
  if (e == cudaSuccess) e = cudaMemcpyAsync(&result, scratch, sizeof(result), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return CC_ERR_CUDA;
  }
  return (cc_status)(result.error != 0 ? result.error : result.input_error);
}
