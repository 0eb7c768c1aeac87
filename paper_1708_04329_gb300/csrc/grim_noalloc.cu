// grim_filter_noalloc: grim_filter without a caller-supplied workspace and
// without any device allocation.
//
// Some callers cannot allocate device memory on the path that calls the
// filter: a host process whose memory manager owns the whole GPU (a library
// cudaMalloc would fail, or fragment that manager's pool), or a latency-bound
// serving loop that keeps cudaMalloc/cudaFree off its request path because
// those calls can synchronise the device.  For them the scratch the filter
// needs (tokens, per-read thresholds, unsorted records, sort buffers, the
// control block) lives in one fixed array in the library's own device
// memory, sized GRIM_NOALLOC_SCRATCH_BYTES.  Every GPU that loads the library
// holds that array until the process exits.
#include <mutex>

#include "grim_internal.cuh"

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[GRIM_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once
// per device and kept for the life of the process (one CUDA context per
// device is assumed: a cudaDeviceReset would leave the kept address stale).
// In host code the array's name is only a host-side handle, so the kernels
// must be given this address instead.
int scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return GRIM_E_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return GRIM_E_UNSUPPORTED;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return GRIM_E_CUDA;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return GRIM_OK;
}

}  // namespace

extern "C" int grim_filter_noalloc(const grim_index* idx, const char* reads,
                                   const uint64_t* offsets, const uint32_t* lens, uint32_t n_reads,
                                   const uint16_t* e, const int32_t* cand, const uint64_t* cand_off,
                                   uint64_t n_cand, uint32_t* out_read, uint32_t* out_bin,
                                   uint8_t* out_count, uint64_t cap, uint64_t* n_out,
                                   void* stream) {
  if (!idx || !n_out) return GRIM_E_ARG;
  *n_out = 0;
  // reject, before touching the device, any call whose scratch would not fit
  const uint64_t need = grim_filter_workspace_size(idx, n_reads, n_cand, cap);
  if (need > (uint64_t)GRIM_NOALLOC_SCRATCH_BYTES) return GRIM_E_WORKSPACE;
  void* scratch = nullptr;
  const int rc = scratch_address(&scratch);
  if (rc != GRIM_OK) return rc;
  // grim_filter clears the control block at the start of every call and
  // writes every other scratch byte before reading it, so the previous call's
  // contents never leak into this one.
  return grim_filter(idx, reads, offsets, lens, n_reads, e, cand, cand_off, n_cand, out_read,
                     out_bin, out_count, cap, n_out, scratch, GRIM_NOALLOC_SCRATCH_BYTES, stream);
}

extern "C" uint64_t grim_noalloc_scratch_bytes(void) { return GRIM_NOALLOC_SCRATCH_BYTES; }
