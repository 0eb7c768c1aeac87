// Read tokenising (§GRIM-Filter step 1: every token of the read is
// extracted) and the per-read threshold of Fig. 3, plus the validation of
// candidate-list offsets.
#include "grim_internal.cuh"

namespace grim {
namespace {

constexpr int kTokWarps = 8;
constexpr uint32_t kMaxStride = 256;  // token stride: <= 255 tokens rounded up to 16

// One warp per read.  The read's tokens (row indices of the table: the token
// value for a clean q-gram, rowInvalid for one holding a non-base -- it still
// counts among the L-q+1 tokens and can never be found -- and rowPad after
// the last token) are written to tokens[(r*copies + k)*ts ...].  With a
// presence table they are written rarest first -- q-grams with a non-base,
// which every bin misses, then ascending number of (super-)bins holding the
// token, ties by position, and the repeats of a value already seen after all
// distinct ones -- so that the all-bins kernels see misses as early as
// possible; a sum does not depend on the order.  meta[r] = ntok | D' << 8
// with D' = min(q*e, ntok): a bin passes iff at most D' of the read's tokens
// are missing from it, which is sum >= (L-q+1) - q*e.
//
// copies = 4 (the 256-bin tiles of q = 6): a tile row is 32 bytes, so the
// row's bank group in shared memory is row & 3, and 16 reads of a warp
// loading random rows collide in bank groups.  The order is then made
// class-cyclic -- position p holds a token of row class p & 3, each class
// rarest first, for as long as every class has tokens left; the rest follow
// rarest first -- and copy k rotates every 16-token block by k positions.  A
// group g of the all-bins kernel reads copy g & 3, so at each load the
// warp's 16 groups cover the four bank groups four times each.  Every block
// holds the same tokens in every copy, so the per-block early exit and every
// sum are unchanged.
__global__ void __launch_bounds__(kTokWarps * 32) k_tokenise(
    const char* __restrict__ reads, const uint64_t* __restrict__ offsets,
    const uint32_t* __restrict__ lens, const uint16_t* __restrict__ e, uint32_t n_reads, uint32_t q,
    uint32_t max_read_len, uint32_t r4, uint32_t ts, const uint32_t* __restrict__ presence,
    uint16_t* __restrict__ tokens, uint32_t* __restrict__ meta, Ctl* ctl, Live live,
    uint32_t max_e, uint64_t max_bases, uint32_t copies) {
  __shared__ unsigned long long s_key[kTokWarps][kMaxStride];
  __shared__ uint16_t s_row[kTokWarps][kMaxStride];
  __shared__ uint16_t s_seq[kTokWarps][kMaxStride];
  __shared__ uint8_t s_crank[kTokWarps][kMaxStride];
  __shared__ uint8_t s_code[kTokWarps][kMaxStride + 16];  // per base: code | 4 if not a base
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint64_t r = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
  if (r >= live_reads(ctl, live, n_reads)) return;  // whole warps: warp syncs stay uniform
  if (e[r] > max_e && lane == 0) atomicOr(&ctl->status, kStatusArg);
  const uint32_t L = lens[r];
  const uint64_t off = offsets[r];
  uint16_t* out = tokens + r * copies * ts;
  bool bad = false;
  if (L < q) {
    if (lane == 0) atomicOr(&ctl->status, kStatusShort);
    bad = true;
  } else if (L > max_read_len || L - q + 1 > kMaxTokens) {
    if (lane == 0) atomicOr(&ctl->status, kStatusLong);
    bad = true;
  } else if (off > max_bases || L > max_bases - off) {  // past the end of the reads buffer
    if (lane == 0) atomicOr(&ctl->status, kStatusArg);
    bad = true;
  }
  const uint32_t ntok = bad ? 0 : L - q + 1;
  // each base read once (coalesced) and coded into shared memory
  for (uint32_t i = lane; i < (bad ? 0u : L); i += 32) {
    const uint32_t u = (uint8_t)reads[off + i] & 0xDFu;  // fold lowercase letters
    const bool ok = (u == 0x41u) | (u == 0x43u) | (u == 0x47u) | (u == 0x54u);
    s_code[warp][i] = (uint8_t)((((u >> 1) ^ (u >> 2)) & 3u) | (ok ? 0u : 4u));  // A0 C1 G2 T3
  }
  __syncwarp();
  for (uint32_t j = lane; j < ntok; j += 32) {
    uint32_t v = 0, flags = 0;
    for (uint32_t i = 0; i < q; ++i) {
      const uint32_t c = s_code[warp][j + i];
      v = (v << 2) | (c & 3u);
      flags |= c;
    }
    const bool clean = (flags & 4u) == 0;
    const uint32_t row = clean ? v : rowInvalid(r4);
    if (!presence && copies == 1) {  // no order wanted (candidate lists): positions as they are
      out[j] = (uint16_t)row;
      continue;
    }
    s_row[warp][j] = (uint16_t)row;
    s_seq[warp][j] = (uint16_t)row;  // the order without a presence table
  }
  __syncwarp();
  for (uint32_t j = lane; j < ntok && (presence || copies > 1); j += 32) {
    // a clean token whose value already occurred earlier in the read misses
    // exactly the bins its first occurrence misses: it adds no new bins to
    // the dead set, so repeats go after every distinct token (1024-bin
    // tiles: 1.7% fewer bit tests at q = 5; at q = 6 repeats are rare and the
    // scan did not pay for itself)
    const uint32_t row = s_row[warp][j];
    bool repeat = false;
    if (copies == 1 && row != rowInvalid(r4))
      for (uint32_t i = 0; i < j && !repeat; ++i) repeat = s_row[warp][i] == row;
    const unsigned long long rare =
        !presence ? 0ull : row != rowInvalid(r4) ? (unsigned long long)presence[row] + 1 : 0ull;
    s_key[warp][j] = ((unsigned long long)repeat << 48) | (rare << 8) | j;
  }
  __syncwarp();
  if (presence && copies == 1) {
    // rank = number of smaller keys (keys are distinct: position breaks ties)
    for (uint32_t j = lane; j < ntok; j += 32) {
      const unsigned long long mine = s_key[warp][j];
      uint32_t rank = 0;
      for (uint32_t i = 0; i < ntok; ++i) rank += s_key[warp][i] < mine;
      out[rank] = s_row[warp][j];
    }
  } else if (copies > 1) {
    if (presence) {
      // rank of each token within its row class, and the size of each class
      uint32_t cnt = 0;  // 4 byte counters: tokens of class c counted by this lane
      for (uint32_t j = lane; j < ntok; j += 32) {
        const unsigned long long mine = s_key[warp][j];
        const uint32_t c = s_row[warp][j] & 3u;
        uint32_t rank = 0;
        for (uint32_t i = 0; i < ntok; ++i)
          rank += (s_row[warp][i] & 3u) == c && s_key[warp][i] < mine;
        s_crank[warp][j] = (uint8_t)rank;
        cnt += 1u << (8 * c);
      }
      cnt = __reduce_add_sync(0xFFFFFFFFu, cnt);
      const uint32_t m = min(min(cnt & 0xFFu, (cnt >> 8) & 0xFFu),
                             min((cnt >> 16) & 0xFFu, cnt >> 24));  // complete cycles
      __syncwarp();
      // the first 4m positions cycle through the classes; the tokens left over
      // follow, rarest first
      for (uint32_t j = lane; j < ntok; j += 32) {
        const uint32_t rc = s_crank[warp][j];
        uint32_t pos;
        if (rc < m) {
          pos = 4u * rc + (s_row[warp][j] & 3u);
        } else {
          const unsigned long long mine = s_key[warp][j];
          uint32_t rank = 0;
          for (uint32_t i = 0; i < ntok; ++i) rank += s_crank[warp][i] >= m && s_key[warp][i] < mine;
          pos = 4u * m + rank;
        }
        s_seq[warp][pos] = s_row[warp][j];
      }
    }
    __syncwarp();
    // copy k: every 16-token block rotated by k positions
    for (uint32_t k = 0; k < copies; ++k) {
      uint16_t* o = out + k * ts;
      for (uint32_t p = lane; p < ts; p += 32) {
        const uint32_t src = (p & ~15u) | ((p + k) & 15u);
        o[p] = src < ntok ? s_seq[warp][src] : (uint16_t)rowPad(r4);
      }
    }
  }
  if (copies == 1)
    for (uint32_t j = ntok + lane; j < ts; j += 32) out[j] = (uint16_t)rowPad(r4);
  if (lane == 0) {
    uint32_t d = q * (uint32_t)e[r];
    if (d > ntok) d = ntok;
    meta[r] = ntok | (d << 8);
    // most batches share one budget: skip the atomics once the max is reached
    if (d > *reinterpret_cast<volatile uint32_t*>(&ctl->max_d)) atomicMax(&ctl->max_d, d);
    if (255u - d > *reinterpret_cast<volatile uint32_t*>(&ctl->d_lo)) atomicMax(&ctl->d_lo, 255u - d);
    const uint32_t tight = 255u - (ntok - d);
    if (tight > *reinterpret_cast<volatile uint32_t*>(&ctl->max_tight))
      atomicMax(&ctl->max_tight, tight);
  }
}

// The spread of the reads' 16-token block counts (ctl->blk_max, blk_lo =
// 32 - the fewest): the all-bins kernel can let a warp's lane groups take
// their next reads together when every read spans as many blocks.  Reads
// shorter than q are left out (the tokeniser fails the batch for them).
__global__ void k_block_spread(const uint32_t* __restrict__ lens, uint32_t n_reads, uint32_t q,
                               Ctl* ctl) {
  uint32_t hi = 0, lo = 0;  // most blocks, 32 - fewest blocks
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n_reads;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t L = lens[i];
    if (L < q) continue;
    const uint32_t ntok = min(L - q + 1, kMaxTokens);
    const uint32_t nblk = (ntok + kBlockTokens - 1) / kBlockTokens;
    hi = max(hi, nblk);
    lo = max(lo, 32u - nblk);
  }
  hi = __reduce_max_sync(0xFFFFFFFFu, hi);
  lo = __reduce_max_sync(0xFFFFFFFFu, lo);
  if ((threadIdx.x & 31) == 0) {
    if (hi) atomicMax(&ctl->blk_max, hi);
    if (lo) atomicMax(&ctl->blk_lo, lo);
  }
}

__global__ void k_check_csr(const uint64_t* __restrict__ cand_off, uint32_t n_reads,
                            uint64_t n_cand, Ctl* ctl, Live live) {
  const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (live.on) {
    n_reads = ctl->live_reads;
    n_cand = ctl->live_cand;
  }
  if (i < n_reads && cand_off[i] > cand_off[i + 1]) atomicOr(&ctl->status, kStatusBadCsr);
  if (i == 0 && cand_off[n_reads] != n_cand) atomicOr(&ctl->status, kStatusBadCsr);
}

// Reverse complement, one warp per read: out[off + L-1-j] = comp(reads[off + j])
// with A<->T and C<->G in either case (case kept); other bytes unchanged.
__global__ void k_reverse_complement(const char* __restrict__ reads,
                                     const uint64_t* __restrict__ offsets,
                                     const uint32_t* __restrict__ lens, uint32_t n_reads,
                                     char* __restrict__ out) {
  const uint64_t r = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
  const uint32_t lane = threadIdx.x & 31;
  if (r >= n_reads) return;
  const uint64_t off = offsets[r];
  const uint32_t L = lens[r];
  for (uint32_t j = lane; j < L; j += 32) {
    const uint32_t c = (uint8_t)reads[off + j];
    const uint32_t u = c & 0xDFu, low = c & 0x20u;
    uint32_t d = c;
    if (u == 0x41u) d = 0x54u | low;       // A -> T
    else if (u == 0x54u) d = 0x41u | low;  // T -> A
    else if (u == 0x43u) d = 0x47u | low;  // C -> G
    else if (u == 0x47u) d = 0x43u | low;  // G -> C
    out[off + L - 1 - j] = (char)d;
  }
}

}  // namespace

void launch_reverse_complement(const char* reads, const uint64_t* offsets, const uint32_t* lens,
                               uint32_t n_reads, char* out, cudaStream_t st) {
  if (n_reads == 0) return;
  const uint32_t threads = 256;
  const uint64_t grid = ((uint64_t)n_reads * 32 + threads - 1) / threads;
  k_reverse_complement<<<(unsigned)grid, threads, 0, st>>>(reads, offsets, lens, n_reads, out);
}

void launch_tokenise(const char* reads, const uint64_t* offsets, const uint32_t* lens,
                     const uint16_t* e, const IndexView& ix, ReadsView rv, uint16_t* tokens,
                     uint32_t* meta, Ctl* ctl, cudaStream_t st, Live live, uint32_t max_e,
                     uint64_t max_bases) {
  const uint32_t copies = rv.copies;
  if (rv.n_reads == 0) return;
  const uint32_t threads = kTokWarps * 32;
  uint64_t grid = ((uint64_t)rv.n_reads * 32 + threads - 1) / threads;
  ProfScope ps("tokenise", st);
  k_tokenise<<<(unsigned)grid, threads, 0, st>>>(reads, offsets, lens, e, rv.n_reads, ix.q,
                                                 ix.max_read_len, ix.r4, rv.ts, ix.presence, tokens,
                                                 meta, ctl, live, max_e, max_bases, copies);
}

void launch_block_spread(const uint32_t* lens, uint32_t n_reads, uint32_t q, Ctl* ctl,
                         cudaStream_t st) {
  if (n_reads == 0) return;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const uint64_t need = ((uint64_t)n_reads + 255) / 256;
  const uint64_t cap = (uint64_t)(sms > 0 ? sms : 1) * 4;
  const uint32_t grid = (uint32_t)(need < cap ? need : cap);
  ProfScope ps("block_spread", st);
  k_block_spread<<<grid, 256, 0, st>>>(lens, n_reads, q, ctl);
}

void launch_check_candidates(const uint64_t* cand_off, uint32_t n_reads, uint64_t n_cand, Ctl* ctl,
                             cudaStream_t st, Live live) {
  const uint64_t n = (uint64_t)n_reads + 1;
  ProfScope ps("check_candidates", st);
  k_check_csr<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(cand_off, n_reads, n_cand, ctl, live);
}

}  // namespace grim
