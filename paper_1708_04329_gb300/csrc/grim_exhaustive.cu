// All-bins filter over the token-major table (§GRIM-Filter steps 2-3;
// §Mapping GRIM-Filter: a row of p bins' existence bits per token is fetched
// and p counters are incremented, then p comparators give a pass bit per bin).
//
// GB300 mapping
// -------------
// * A persistent CTA (512 threads, one per SM) takes work items
//   (1024-bin tile, range of reads).  The tile -- 4^q rows x 128 B of the
//   token-major table -- is staged in shared memory once per item and reused
//   by every read of the range.  Two extra rows follow it: all zeros (for a
//   q-gram holding a non-base: always a miss) and all ones (padding after a
//   read's last token: never a miss).
// * A warp holds four reads, one per quarter warp ("group" of 8 lanes).
//   Lane i of a group owns words 4i..4i+3 of the tile, i.e. 128 bins, and
//   fetches them for each token with one 16-byte shared load; a quarter warp
//   reads one whole 128-byte row, so the four groups' loads of four rows are
//   four conflict-free wavefronts.
// * Instead of p separate counters, each lane keeps bit-sliced vertical
//   counters: plane k of word w holds bit k of the counters of that word's 32
//   bins.  Counted are MISSES (tokens absent from the bin), started at
//   bias = 256 - (D'+1) with D' = min(q*e, L-q+1), so the 8-bit counter
//   overflows exactly when misses > D', i.e. when sum < T = (L-q+1) - q*e.
//   The overflow is kept in a sticky "dead" plane; a bin passes iff its dead
//   bit is clear at the end, and then its sum is (L-q+1) - (counter - bias).
// * Tokens are added 16 at a time with a carry-save (Harley-Seal) tree of
//   full adders (two 3-input LOP3s each), whose weight-16 carry ripples into
//   the upper four planes: ~2.4 logic ops per token per 32 bins.
// * Early exit: after each 16-token block the group stops a read once every
//   one of its 1024 bins is dead -- exact, since a dead bin can never pass.
// * Groups advance independently (a finished group takes the range's next
//   read) but stay converged: the per-block work is the same instruction
//   stream for all four groups, and every warp collective uses the full mask.
#include "grim_internal.cuh"

namespace grim {
namespace {

constexpr int kThreads = 512;
constexpr uint32_t kNone = 0xFFFFFFFFu;

#define LOP3(d, a, b, c, lut) \
  asm("lop3.b32 %0, %1, %2, %3, " #lut ";" : "=r"(d) : "r"(a), "r"(b), "r"(c))

// full adder of three planes of the same weight: sum (a^b^c), carry maj(a,b,c)
__device__ __forceinline__ void fa(uint32_t a, uint32_t b, uint32_t c, uint32_t& s, uint32_t& k) {
  LOP3(s, a, b, c, 0x96);
  LOP3(k, a, b, c, 0xE8);
}
// full adder where b and c are existence words whose complements (misses) are
// added: sum a^~b^~c = a^b^c, carry maj(a,~b,~c)
__device__ __forceinline__ void fa_miss(uint32_t a, uint32_t b, uint32_t c, uint32_t& s,
                                        uint32_t& k) {
  LOP3(s, a, b, c, 0x96);
  LOP3(k, a, b, c, 0x71);
}

struct Counters {
  // per word: s1 s2 s4 s8 (low planes), u[0..3] (weights 16..128), dead
  uint32_t s1[4], s2[4], s4[4], s8[4], u0[4], u1[4], u2[4], u3[4], dead[4];

  __device__ __forceinline__ void init(uint32_t bias) {
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      s1[w] = (bias & 1u) ? ~0u : 0u;
      s2[w] = (bias & 2u) ? ~0u : 0u;
      s4[w] = (bias & 4u) ? ~0u : 0u;
      s8[w] = (bias & 8u) ? ~0u : 0u;
      u0[w] = (bias & 16u) ? ~0u : 0u;
      u1[w] = (bias & 32u) ? ~0u : 0u;
      u2[w] = (bias & 64u) ? ~0u : 0u;
      u3[w] = (bias & 128u) ? ~0u : 0u;
      dead[w] = 0u;
    }
  }

  // counter value of bin `bit` of word w
  __device__ __forceinline__ uint32_t value(int w, uint32_t bit) const {
    return ((s1[w] >> bit) & 1u) | (((s2[w] >> bit) & 1u) << 1) | (((s4[w] >> bit) & 1u) << 2) |
           (((s8[w] >> bit) & 1u) << 3) | (((u0[w] >> bit) & 1u) << 4) |
           (((u1[w] >> bit) & 1u) << 5) | (((u2[w] >> bit) & 1u) << 6) |
           (((u3[w] >> bit) & 1u) << 7);
  }
};

// Add the misses of one 16-token block: tw holds 16 table row indices
// (uint16 pairs); lane_row points at this lane's 16 bytes of row 0.
__device__ __forceinline__ void add_block(Counters& c, const uint32_t (&tw)[8],
                                          const char* lane_row) {
  // the 4 words (this lane's 128 bins) of token j's row
#define ROW(j)                                                                          \
  (*reinterpret_cast<const uint4*>(                                                     \
      lane_row + (((j) & 1) ? (tw[(j) >> 1] >> 16) : (tw[(j) >> 1] & 0xFFFFu)) * 128u))
  uint32_t t2a[4], t2b[4], t4a[4], t4b[4], t8a[4], t8b[4], t16[4];
  {
    uint4 x0 = ROW(0), x1 = ROW(1), x2 = ROW(2), x3 = ROW(3);
    const uint32_t a0[4] = {x0.x, x0.y, x0.z, x0.w}, a1[4] = {x1.x, x1.y, x1.z, x1.w};
    const uint32_t a2[4] = {x2.x, x2.y, x2.z, x2.w}, a3[4] = {x3.x, x3.y, x3.z, x3.w};
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      fa_miss(c.s1[w], a0[w], a1[w], c.s1[w], t2a[w]);
      fa_miss(c.s1[w], a2[w], a3[w], c.s1[w], t2b[w]);
      fa(c.s2[w], t2a[w], t2b[w], c.s2[w], t4a[w]);
    }
  }
  {
    uint4 x0 = ROW(4), x1 = ROW(5), x2 = ROW(6), x3 = ROW(7);
    const uint32_t a0[4] = {x0.x, x0.y, x0.z, x0.w}, a1[4] = {x1.x, x1.y, x1.z, x1.w};
    const uint32_t a2[4] = {x2.x, x2.y, x2.z, x2.w}, a3[4] = {x3.x, x3.y, x3.z, x3.w};
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      fa_miss(c.s1[w], a0[w], a1[w], c.s1[w], t2a[w]);
      fa_miss(c.s1[w], a2[w], a3[w], c.s1[w], t2b[w]);
      fa(c.s2[w], t2a[w], t2b[w], c.s2[w], t4b[w]);
      fa(c.s4[w], t4a[w], t4b[w], c.s4[w], t8a[w]);
    }
  }
  {
    uint4 x0 = ROW(8), x1 = ROW(9), x2 = ROW(10), x3 = ROW(11);
    const uint32_t a0[4] = {x0.x, x0.y, x0.z, x0.w}, a1[4] = {x1.x, x1.y, x1.z, x1.w};
    const uint32_t a2[4] = {x2.x, x2.y, x2.z, x2.w}, a3[4] = {x3.x, x3.y, x3.z, x3.w};
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      fa_miss(c.s1[w], a0[w], a1[w], c.s1[w], t2a[w]);
      fa_miss(c.s1[w], a2[w], a3[w], c.s1[w], t2b[w]);
      fa(c.s2[w], t2a[w], t2b[w], c.s2[w], t4a[w]);
    }
  }
  {
    uint4 x0 = ROW(12), x1 = ROW(13), x2 = ROW(14), x3 = ROW(15);
    const uint32_t a0[4] = {x0.x, x0.y, x0.z, x0.w}, a1[4] = {x1.x, x1.y, x1.z, x1.w};
    const uint32_t a2[4] = {x2.x, x2.y, x2.z, x2.w}, a3[4] = {x3.x, x3.y, x3.z, x3.w};
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      fa_miss(c.s1[w], a0[w], a1[w], c.s1[w], t2a[w]);
      fa_miss(c.s1[w], a2[w], a3[w], c.s1[w], t2b[w]);
      fa(c.s2[w], t2a[w], t2b[w], c.s2[w], t4b[w]);
      fa(c.s4[w], t4a[w], t4b[w], c.s4[w], t8b[w]);
      fa(c.s8[w], t8a[w], t8b[w], c.s8[w], t16[w]);
      // ripple the weight-16 carry through the upper planes; the carry out of
      // weight 128 (counter >= 256: misses > D') sticks in `dead`
      uint32_t k = t16[w], nk;
      nk = c.u0[w] & k; c.u0[w] ^= k; k = nk;
      nk = c.u1[w] & k; c.u1[w] ^= k; k = nk;
      nk = c.u2[w] & k; c.u2[w] ^= k; k = nk;
      uint32_t d;
      LOP3(d, c.dead[w], c.u3[w], k, 0xF8);  // dead | (u3 & k)
      c.u3[w] ^= k;
      c.dead[w] = d;
    }
  }
#undef ROW
}

struct ExhArgs {
  IndexView ix;
  ReadsView rv;
  RecordsView rec;
  uint32_t bin_bits;
  uint32_t n_ranges, reads_per_range, n_items;
  Ctl* ctl;
};

__global__ void __launch_bounds__(kThreads, 1) k_exhaustive(ExhArgs a) {
  extern __shared__ __align__(16) uint32_t s_tile[];  // (r4 + 2) rows x 32 words
  __shared__ uint32_t s_item, s_next;
  const uint32_t tid = threadIdx.x, lane = tid & 31, grp = lane >> 3, li = lane & 7;
  const uint32_t r4 = a.ix.r4;
  if (*(volatile uint32_t*)&a.ctl->status) return;  // set by the tokeniser before launch

  for (uint32_t i = tid; i < kTileWords; i += kThreads) {
    s_tile[rowInvalid(r4) * kTileWords + i] = 0u;
    s_tile[rowPad(r4) * kTileWords + i] = ~0u;
  }
  const char* lane_row = reinterpret_cast<const char*>(s_tile) + li * 16u;

  for (;;) {
    __syncthreads();  // previous item finished with the tile
    if (tid == 0) {
      s_item = atomicAdd(&a.ctl->item, 1u);
      s_next = 0;
    }
    __syncthreads();
    const uint32_t item = s_item;
    if (item >= a.n_items) break;
    const uint32_t tile = item / a.n_ranges, range = item % a.n_ranges;
    const uint32_t r0 = range * a.reads_per_range;
    const uint32_t nr = min(a.reads_per_range, a.rv.n_reads - r0);

    // stage the tile: rows [0, r4), words [tile*32, tile*32+32)
    {
      const uint32_t* src = a.ix.tm + (uint64_t)tile * kTileWords;
      const uint32_t s0 = (uint32_t)__cvta_generic_to_shared(s_tile);
      for (uint32_t i = tid; i < r4 * 8u; i += kThreads) {
        const uint32_t row = i >> 3, chunk = i & 7u;
        const uint32_t* g = src + (uint64_t)row * a.ix.wpad + chunk * 4u;
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s0 + (row * 32u + chunk * 4u) * 4u),
                     "l"(g));
      }
      asm volatile("cp.async.commit_group;");
      asm volatile("cp.async.wait_all;" ::: "memory");
    }
    __syncthreads();

    // which of this lane's 128 bins exist (only the last tile is ragged)
    uint32_t vmask[4];
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      const uint64_t b0 = (uint64_t)tile * kTileBins + (li * 4u + w) * 32u;
      const uint64_t left = b0 < a.ix.num_bins ? a.ix.num_bins - b0 : 0;
      vmask[w] = left >= 32 ? ~0u : ((1u << left) - 1u);
    }

    // per-group state (identical in the group's 8 lanes)
    uint32_t cur = kNone, blk = 0, nblk = 0, ntok = 0, bias = 0;
    uint32_t executed = 0;  // blocks this group applied to real reads
    bool fin = false;
    const uint16_t* tk = a.rv.tokens + (uint64_t)r0 * a.rv.ts;  // any in-bounds block
    Counters c;
    c.init(0);

    for (;;) {
      // (1) groups without a read take the range's next one
      const bool need = !fin && cur == kNone;
      if (__any_sync(0xFFFFFFFFu, need)) {
        uint32_t k = 0;
        if (need && li == 0) k = atomicAdd(&s_next, 1u);
        k = __shfl_sync(0xFFFFFFFFu, k, grp * 8);
        if (need) {
          if (k >= nr) {
            fin = true;
            blk = 0;  // keep re-reading an in-bounds block
          } else {
            cur = r0 + k;
            const uint32_t m = a.rv.meta[cur];
            ntok = m & 0xFFu;
            const uint32_t d = (m >> 8) & 0xFFu;
            bias = 256u - (d + 1u);
            nblk = (ntok + kBlockTokens - 1) / kBlockTokens;
            blk = 0;
            tk = a.rv.tokens + (uint64_t)cur * a.rv.ts;
            c.init(bias);
          }
        }
      }
      if (__all_sync(0xFFFFFFFFu, fin)) break;

      // (2) one 16-token block for all four groups (finished groups repeat
      //     an in-bounds block; their results are ignored)
      {
        const uint4* tp = reinterpret_cast<const uint4*>(tk + blk * kBlockTokens);
        const uint4 t0 = __ldg(tp), t1 = __ldg(tp + 1);
        const uint32_t tw[8] = {t0.x, t0.y, t0.z, t0.w, t1.x, t1.y, t1.z, t1.w};
        add_block(c, tw, lane_row);
      }
      if (!fin) {
        ++blk;
        ++executed;
      }

      // (3) a read ends when every bin of its tile is dead or its tokens are used up
      const uint32_t all_dead = c.dead[0] & c.dead[1] & c.dead[2] & c.dead[3];
      const uint32_t bal = __ballot_sync(0xFFFFFFFFu, all_dead == ~0u);
      const bool gdead = ((bal >> (grp * 8)) & 0xFFu) == 0xFFu;
      const bool done = !fin && cur != kNone && (gdead || blk >= nblk);
      const bool emit = done && !gdead;
      if (__any_sync(0xFFFFFFFFu, emit)) {
        uint32_t pm[4], cnt = 0;
#pragma unroll
        for (int w = 0; w < 4; ++w) {
          pm[w] = emit ? (~c.dead[w] & vmask[w]) : 0u;
          cnt += __popc(pm[w]);
        }
        uint32_t incl = cnt;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
          const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, incl, d);
          if (lane >= (uint32_t)d) incl += t;
        }
        const uint32_t tot = __shfl_sync(0xFFFFFFFFu, incl, 31);
        unsigned long long base = 0;
        if (lane == 0 && tot) base = atomicAdd(&a.ctl->n_rec, (unsigned long long)tot);
        base = __shfl_sync(0xFFFFFFFFu, base, 0);
        unsigned long long pos = base + incl - cnt;
#pragma unroll
        for (int w = 0; w < 4; ++w) {
          uint32_t m = pm[w];
          while (m) {
            const uint32_t bit = __ffs(m) - 1;
            m &= m - 1;
            const uint32_t misses = c.value(w, bit) - bias;
            const uint64_t bin = (uint64_t)tile * kTileBins + (li * 4u + w) * 32u + bit;
            if (pos < a.rec.cap) {
              a.rec.keys[pos] = ((unsigned long long)cur << a.bin_bits) | bin;
              a.rec.counts[pos] = (uint8_t)(ntok - misses);
            }
            ++pos;
          }
        }
      }
      if (done) cur = kNone;
    }
    // one count per group (its 8 lanes agree), one atomic per warp and item
    uint32_t ex = li == 0 ? executed : 0u;
    ex = __reduce_add_sync(0xFFFFFFFFu, ex);
    if (lane == 0 && ex) atomicAdd(&a.ctl->blocks, (unsigned long long)ex);
  }
}

}  // namespace

void launch_exhaustive(const IndexView& ix, const ReadsView& rv, RecordsView rec, uint32_t bin_bits,
                       Ctl* ctl, cudaStream_t st) {
  if (rv.n_reads == 0) return;
  const uint32_t n_tiles = (uint32_t)(ix.num_bins_pad / kTileBins);
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (sms <= 0) sms = 1;
  // enough items to balance the persistent grid, each range at least 64 reads
  uint32_t n_ranges = (uint32_t)((4u * (uint32_t)sms + n_tiles - 1) / n_tiles);
  const uint32_t max_ranges = (rv.n_reads + 63) / 64;
  if (n_ranges > max_ranges) n_ranges = max_ranges;
  if (n_ranges < 1) n_ranges = 1;
  const uint32_t per = (rv.n_reads + n_ranges - 1) / n_ranges;
  n_ranges = (rv.n_reads + per - 1) / per;
  ExhArgs a{ix, rv, rec, bin_bits, n_ranges, per, n_tiles * n_ranges, ctl};
  const size_t smem = (size_t)(ix.r4 + 2) * kTileWords * sizeof(uint32_t);
  cudaFuncSetAttribute(k_exhaustive, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  uint32_t grid = (uint32_t)sms;
  if (grid > a.n_items) grid = a.n_items;
  ProfScope ps("exhaustive", st);
  k_exhaustive<<<grid, kThreads, smem, st>>>(a);
}

}  // namespace grim
