// Measurement helper, not part of the filter: the practical ceiling of the
// candidate-list path's memory access on this GPU.
//
// A candidate costs one random gather of a 128-byte (q = 5) or 512-byte
// (q = 6) bin vector (§GRIM-Filter, Fig. 5: the bin holding a candidate
// location is fetched and tested).  Random rows of that size cannot reach
// the copy bandwidth: DRAM spends a row activation on every 128 bytes.  This
// kernel does the gather alone -- row numbers come from a hash of the
// gather's index, so no id is loaded, and each lane folds its 16 bytes into
// one word -- with the candidate kernel's lane split (16 bytes a lane, U rows
// in flight per lane group).  Its rate is what any kernel on this access
// pattern can hope for.
//
//   int grim_probe_gather(const void* table, uint64_t rows, uint32_t row_bytes,
//                         uint64_t n, uint32_t unroll, uint32_t* sink,
//                         uint64_t sink_words, void* stream);
//
// table: device, rows x row_bytes bytes, 16-byte aligned, rows < 2^32.
// row_bytes: 128 or 512.  n: rows gathered.  unroll: 1, 2 or 4.  sink:
// device, written (one word a thread) so the loads are not dropped; it must
// hold the launch's threads, which grim_probe_gather_sink_words returns.  Returns 0, -1 for a
// bad argument, or -3 when the launch fails.  Asynchronous on `stream`.
#include <cstdint>
#include <cuda_runtime.h>

namespace {

constexpr int kThreads = 256;

// A row in [0, rows) from the gather's index: C. Wellons' "lowbias32" integer
// hash, then a multiply-shift range reduction (no division, which would make
// the probe bound by arithmetic instead of by memory).  rows < 2^32.
__device__ __forceinline__ uint32_t row_of(uint64_t i, uint32_t rows) {
  uint32_t x = (uint32_t)i ^ (uint32_t)(i >> 32) * 0x9e3779b9u;
  x ^= x >> 16;
  x *= 0x7feb352du;
  x ^= x >> 15;
  x *= 0x846ca68bu;
  x ^= x >> 16;
  return (uint32_t)(((uint64_t)x * rows) >> 32);
}

template <int U, int ROWB>
__global__ void __launch_bounds__(kThreads) k_probe_gather(const uint4* __restrict__ tab,
                                                           uint32_t rows, uint64_t n,
                                                           uint32_t* __restrict__ sink) {
  constexpr int G = ROWB / 16, CPW = 32 / G;
  const uint32_t lane = threadIdx.x & 31, sub = lane % G, slot = lane / G;
  const uint64_t warp = (blockIdx.x * (uint64_t)kThreads + threadIdx.x) >> 5;
  const uint64_t n_warps = ((uint64_t)gridDim.x * kThreads) >> 5;
  uint32_t acc = 0;
  for (uint64_t base = warp * CPW * U; base < n; base += n_warps * CPW * U) {
    uint4 v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const uint64_t i = base + u * CPW + slot;
      const uint64_t row = row_of(i, rows);
      v[u] = i < n ? __ldg(tab + row * G + sub) : make_uint4(0, 0, 0, 0);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) acc += (v[u].x ^ v[u].y) + (v[u].z ^ v[u].w);
  }
  sink[blockIdx.x * (uint64_t)kThreads + threadIdx.x] = acc;
}

template <int U, int ROWB>
int launch(const void* table, uint32_t rows, uint64_t n, uint32_t* sink, uint64_t sink_words,
           cudaStream_t st) {
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -3;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_probe_gather<U, ROWB>, kThreads, 0);
  if (per_sm < 1) per_sm = 1;
  const uint64_t grid = (uint64_t)sms * per_sm;
  if (sink_words < grid * kThreads) return -1;
  k_probe_gather<U, ROWB><<<(unsigned)grid, kThreads, 0, st>>>(
      static_cast<const uint4*>(table), rows, n, sink);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

}  // namespace

extern "C" uint64_t grim_probe_gather_sink_words(void) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return (uint64_t)sms * (2048 / kThreads) * kThreads;  // at most 2048 threads per SM
}

extern "C" int grim_probe_gather(const void* table, uint64_t rows, uint32_t row_bytes, uint64_t n,
                                 uint32_t unroll, uint32_t* sink, uint64_t sink_words,
                                 void* stream) {
  if (!table || !sink || rows == 0 || rows > 0xFFFFFFFFull ||
      (reinterpret_cast<uintptr_t>(table) & 15u))
    return -1;
  if (n == 0) return 0;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (row_bytes == 128) {
    if (unroll == 1) return launch<1, 128>(table, (uint32_t)rows, n, sink, sink_words, st);
    if (unroll == 2) return launch<2, 128>(table, (uint32_t)rows, n, sink, sink_words, st);
    if (unroll == 4) return launch<4, 128>(table, (uint32_t)rows, n, sink, sink_words, st);
  } else if (row_bytes == 512) {
    if (unroll == 1) return launch<1, 512>(table, (uint32_t)rows, n, sink, sink_words, st);
    if (unroll == 2) return launch<2, 512>(table, (uint32_t)rows, n, sink, sink_words, st);
    if (unroll == 4) return launch<4, 512>(table, (uint32_t)rows, n, sink, sink_words, st);
  }
  return -1;
}
