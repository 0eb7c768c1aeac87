// Stream compaction of the passing (read, bin, count) records
// (§Mapping GRIM-Filter: the filter's result per read is a vector over bins;
// here only the set entries are kept, read by read).
//
// The filter kernels append records in whatever order their warps finish, so
// the order is restored by a least-significant-digit radix sort on the record
// key -- (read << bin_bits | bin) in all-bins mode, the global candidate index
// in candidate mode; keys are unique, so the output order is unique too.
// Each 8-bit pass is a per-block digit histogram, one exclusive scan over
// all blocks' histograms, and a stable scatter (per-warp ranks from
// __match_any_sync, then warp order, then round order).  A last kernel splits
// the keys into the caller's read / bin / count arrays.
#include "grim_internal.cuh"

namespace grim {
namespace {

constexpr uint32_t kSortThreads = 256;
constexpr uint32_t kSortItems = 16;  // per thread per pass
constexpr uint32_t kSortTile = kSortThreads * kSortItems;

// Live record counts: *n_live (capped at n) when n_live is set, else n; a
// gate (ctl, path) makes the kernel a no-op unless the batch took that path.
__device__ __forceinline__ uint64_t live_n(const unsigned long long* n_live, uint64_t n) {
  if (!n_live) return n;
  const uint64_t v = *n_live;
  return v < n ? v : n;
}
__device__ __forceinline__ bool gate_off(const Ctl* c, uint32_t gate) {
  return c && gate && c->path != gate;
}

__global__ void __launch_bounds__(kSortThreads) k_rs_hist(const unsigned long long* __restrict__ keys,
                                                          uint64_t n, uint32_t shift,
                                                          uint32_t* __restrict__ hist, uint32_t nb,
                                                          const unsigned long long* n_live,
                                                          const Ctl* gc, uint32_t gate) {
  __shared__ uint32_t cnt[256];
  if (gate_off(gc, gate)) return;
  n = live_n(n_live, n);
  if ((uint64_t)blockIdx.x * kSortTile >= n) return;  // past the live records
  cnt[threadIdx.x] = 0;
  __syncthreads();
  const uint64_t base = (uint64_t)blockIdx.x * kSortTile;
  for (uint32_t i = 0; i < kSortItems; ++i) {
    const uint64_t idx = base + (uint64_t)i * kSortThreads + threadIdx.x;
    if (idx < n) atomicAdd(&cnt[(keys[idx] >> shift) & 0xFFu], 1u);
  }
  __syncthreads();
  hist[(uint64_t)threadIdx.x * nb + blockIdx.x] = cnt[threadIdx.x];
}

// Exclusive scan, with one block, of the digit-major histogram of the live
// blocks: entry (d, blk) at h[d * nb + blk] for blk < nb_live, scanned in
// the logical order i = d * nb_live + blk.  Warp w owns the logical range
// [w*S, (w+1)*S): it sums the range (32 consecutive entries per step, so the
// loads coalesce), the 32 warp totals are scanned, and each warp rescans its
// range with shuffles, carrying its running offset.
__device__ __forceinline__ uint64_t hist_at(uint32_t i, uint32_t nb_live, uint64_t nb) {
  return (uint64_t)(i / nb_live) * nb + (i % nb_live);
}

__global__ void __launch_bounds__(1024) k_rs_scan(uint32_t* __restrict__ h, uint64_t nb, uint64_t n,
                                                  const unsigned long long* n_live, const Ctl* gc,
                                                  uint32_t gate) {
  __shared__ uint32_t s_warp[32];
  if (gate_off(gc, gate)) return;
  n = live_n(n_live, n);
  const uint32_t nb_live = (uint32_t)((n + kSortTile - 1) / kSortTile);
  if (nb_live == 0) return;
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t m = 256u * nb_live;
  const uint32_t span = (m + 31) / 32;
  const uint32_t lo = min(warp * span, m), hi = min(lo + span, m);
  uint32_t total = 0;
  for (uint32_t i = lo + lane; i < hi; i += 32) total += h[hist_at(i, nb_live, nb)];
  total = __reduce_add_sync(0xFFFFFFFFu, total);
  if (lane == 0) s_warp[warp] = total;
  __syncthreads();
  if (warp == 0) {
    const uint32_t v = s_warp[lane];
    uint32_t incl = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, incl, d);
      if (lane >= (uint32_t)d) incl += t;
    }
    s_warp[lane] = incl - v;  // exclusive
  }
  __syncthreads();
  uint32_t carry = s_warp[warp];
  for (uint32_t c = lo; c < hi; c += 32) {
    const uint32_t i = c + lane;
    const bool in = i < hi;
    const uint64_t j = in ? hist_at(i, nb_live, nb) : 0;
    const uint32_t v = in ? h[j] : 0u;
    uint32_t incl = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, incl, d);
      if (lane >= (uint32_t)d) incl += t;
    }
    if (in) h[j] = carry + incl - v;
    carry += __shfl_sync(0xFFFFFFFFu, incl, 31);
  }
}

__global__ void __launch_bounds__(kSortThreads) k_rs_scatter(
    const unsigned long long* __restrict__ kin, const uint8_t* __restrict__ cin,
    unsigned long long* __restrict__ kout, uint8_t* __restrict__ cout, uint64_t n, uint32_t shift,
    const uint32_t* __restrict__ hist, uint32_t nb, const unsigned long long* n_live, const Ctl* gc,
    uint32_t gate) {
  constexpr uint32_t kW = kSortThreads / 32;
  __shared__ uint32_t s_base[256];
  __shared__ uint32_t s_wcnt[kW][256];
  if (gate_off(gc, gate)) return;
  n = live_n(n_live, n);
  if ((uint64_t)blockIdx.x * kSortTile >= n) return;  // past the live records
  const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  s_base[tid] = hist[(uint64_t)tid * nb + blockIdx.x];
  const uint64_t base = (uint64_t)blockIdx.x * kSortTile;
  for (uint32_t round = 0; round < kSortItems; ++round) {
    for (uint32_t i = tid; i < kW * 256; i += kSortThreads) (&s_wcnt[0][0])[i] = 0;
    __syncthreads();
    const uint64_t idx = base + (uint64_t)round * kSortThreads + tid;
    const bool valid = idx < n;
    unsigned long long key = valid ? kin[idx] : 0ull;
    const uint8_t c = valid ? cin[idx] : (uint8_t)0;
    const uint32_t d = (uint32_t)(key >> shift) & 0xFFu;
    // invalid lanes get a value no valid digit has, so they never match
    const uint32_t peers = __match_any_sync(0xFFFFFFFFu, valid ? d : 256u + lane);
    const uint32_t rank = __popc(peers & ((1u << lane) - 1u));
    if (valid && rank == 0) s_wcnt[warp][d] = __popc(peers);
    __syncthreads();
    if (valid) {
      uint32_t off = s_base[d] + rank;
      for (uint32_t w = 0; w < warp; ++w) off += s_wcnt[w][d];
      kout[off] = key;
      cout[off] = c;
    }
    __syncthreads();
    uint32_t add = 0;
    for (uint32_t w = 0; w < kW; ++w) add += s_wcnt[w][tid];
    s_base[tid] += add;
    __syncthreads();  // s_wcnt is cleared again at the top of the next round
  }
}

__global__ void k_emit(const unsigned long long* __restrict__ keys,
                       const uint8_t* __restrict__ counts, uint64_t n, bool cand_mode,
                       uint32_t bin_bits, const int32_t* __restrict__ cand,
                       const uint64_t* __restrict__ cand_off, uint32_t n_reads,
                       uint32_t* __restrict__ out_read, uint32_t* __restrict__ out_bin,
                       uint8_t* __restrict__ out_count, const unsigned long long* n_live,
                       const uint32_t* n_reads_live, const Ctl* gc, uint32_t gate) {
  const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (gate_off(gc, gate)) return;
  if (i >= live_n(n_live, n)) return;
  if (n_reads_live) n_reads = *n_reads_live;
  const unsigned long long key = keys[i];
  uint32_t r, b;
  if (cand_mode) {
    b = (uint32_t)cand[key];
    // largest r with cand_off[r] <= key
    uint32_t lo = 0, hi = n_reads - 1;
    while (lo < hi) {
      const uint32_t mid = lo + (hi - lo + 1) / 2;
      if (cand_off[mid] <= key) lo = mid;
      else hi = mid - 1;
    }
    r = lo;
  } else {
    r = (uint32_t)(key >> bin_bits);
    b = (uint32_t)(key & ((bin_bits >= 64) ? ~0ull : ((1ull << bin_bits) - 1ull)));
  }
  out_read[i] = r;
  out_bin[i] = b;
  out_count[i] = counts[i];
}

// Survivors of the coarse pass (keys read << cbits | super-bin, sorted) become
// candidate lists of the members of each surviving super-bin: candidates
// f*i .. f*i+f-1 are bins f*s .. f*s+f-1, and read r's list starts at f times
// the number of survivors of reads before r.
__global__ void k_expand(const unsigned long long* __restrict__ keys, uint64_t n_surv,
                         uint32_t cbits, uint32_t f, uint32_t n_reads, int32_t* __restrict__ cand,
                         uint64_t* __restrict__ cand_off, const Ctl* lc, uint32_t gate) {
  const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (lc) {
    if (gate_off(lc, gate)) return;
    n_surv = lc->n_surv;
    n_reads = lc->live_reads;
  }
  const unsigned long long mask = cbits >= 64 ? ~0ull : ((1ull << cbits) - 1ull);
  if (i < n_surv) {
    const uint32_t s = (uint32_t)(keys[i] & mask);
    for (uint32_t k = 0; k < f; ++k) cand[f * i + k] = (int32_t)(f * s + k);
  }
  if (i <= n_reads) {
    const unsigned long long target = (unsigned long long)i << cbits;
    uint64_t lo = 0, hi = n_surv;  // first survivor with key >= target
    while (lo < hi) {
      const uint64_t mid = (lo + hi) / 2;
      if (keys[mid] < target) lo = mid + 1;
      else hi = mid;
    }
    cand_off[i] = f * lo;
  }
}

}  // namespace

uint64_t sort_workspace_bytes(uint64_t cap) {
  const uint64_t nb = (cap + kSortTile - 1) / kSortTile;
  return 256ull * (nb ? nb : 1) * sizeof(uint32_t);
}

void expand_survivors(const unsigned long long* keys, uint64_t n_surv, uint32_t cbits, uint32_t f,
                      uint32_t n_reads, int32_t* cand, uint64_t* cand_off, cudaStream_t st,
                      const Ctl* live_ctl, uint32_t gate) {
  const uint64_t n = n_surv > (uint64_t)n_reads + 1 ? n_surv : (uint64_t)n_reads + 1;
  ProfScope ps("expand", st);
  k_expand<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(keys, n_surv, cbits, f, n_reads, cand,
                                                       cand_off, live_ctl, gate);
}

RecordsView sort_records(RecordsView a, RecordsView b, uint64_t n, uint32_t key_bits, void* hist,
                         cudaStream_t st, const unsigned long long* n_live, const Ctl* gate_ctl,
                         uint32_t gate) {
  if (n == 0) return a;
  const uint32_t nb = (uint32_t)((n + kSortTile - 1) / kSortTile);
  uint32_t* h = static_cast<uint32_t*>(hist);
  RecordsView src = a, dst = b;
  const uint32_t passes = (key_bits + 7) / 8;
  for (uint32_t p = 0; p < passes; ++p) {
    const uint32_t shift = 8 * p;
    {
      ProfScope ps("sort_hist", st);
      k_rs_hist<<<nb, kSortThreads, 0, st>>>(src.keys, n, shift, h, nb, n_live, gate_ctl, gate);
    }
    {
      ProfScope ps("sort_scan", st);
      k_rs_scan<<<1, 1024, 0, st>>>(h, nb, n, n_live, gate_ctl, gate);
    }
    {
      ProfScope ps("sort_scatter", st);
      k_rs_scatter<<<nb, kSortThreads, 0, st>>>(src.keys, src.counts, dst.keys, dst.counts, n,
                                                shift, h, nb, n_live, gate_ctl, gate);
    }
    RecordsView t = src;
    src = dst;
    dst = t;
  }
  return src;
}

void sort_and_emit(RecordsView a, RecordsView b, uint64_t n, uint32_t key_bits, void* hist,
                   bool candidate_mode, uint32_t bin_bits, const int32_t* cand,
                   const uint64_t* cand_off, uint32_t n_reads, uint32_t* out_read,
                   uint32_t* out_bin, uint8_t* out_count, cudaStream_t st,
                   const unsigned long long* n_live, const uint32_t* n_reads_live,
                   const Ctl* gate_ctl, uint32_t gate) {
  if (n == 0) return;
  const RecordsView src = sort_records(a, b, n, key_bits, hist, st, n_live, gate_ctl, gate);
  ProfScope ps("emit", st);
  k_emit<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(src.keys, src.counts, n, candidate_mode,
                                                      bin_bits, cand, cand_off, n_reads, out_read,
                                                      out_bin, out_count, n_live, n_reads_live,
                                                      gate_ctl, gate);
}

}  // namespace grim
