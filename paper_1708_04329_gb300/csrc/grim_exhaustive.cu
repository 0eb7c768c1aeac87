// All-bins filter over the token-major table (§GRIM-Filter steps 2-3;
// §Mapping GRIM-Filter: a row of p bins' existence bits per token is fetched
// and p counters are incremented, then p comparators give a pass bit per bin).
//
// GB300 mapping
// -------------
// * A persistent CTA (one per SM, 512 to 768 threads) takes work items (tile
//   of TW*32 bins, range of reads).  The tile -- 4^q rows x TW words of the
//   token-major table -- is staged in shared memory once per item and reused
//   by every read of the range.  TW = 32 (1024 bins, 128 KB at q = 5) up to q = 5 and
//   TW = 8 (256 bins, 128 KB) at q = 6.  Two extra rows follow the tile: all
//   zeros (for a q-gram holding a non-base: always a miss) and all ones
//   (padding after a read's last token: never a miss).
// * A warp holds 32/GL reads, one per group of GL = TW/4 lanes.  Lane i of a
//   group owns words 4i..4i+3 of the tile, i.e. 128 bins, and fetches them
//   for each token with one 16-byte shared load.  At TW = 32 a quarter warp
//   is one group reading one whole 128-byte row, so the four groups' loads of
//   four rows are four conflict-free wavefronts; at TW = 8 sixteen groups
//   load 32-byte rows whose bank group is row mod 4, and each group reads a
//   block-rotated copy of its read's class-cyclic token order (see
//   k_tokenise) so that every load covers the four bank groups evenly.
// * Each group copies the token row of the read it will take next into its
//   own shared-memory slot with cp.async while it works on the current one,
//   so the inner loop does not wait on global memory.  At TW = 8 a slot
//   holds a read's first blocks (up to four, as many as fit beside the tile
//   at the CTA size) and later blocks are loaded from L2.
// * Reads are swept in ranges whose token rows fit in L2, range by range,
//   so concurrent CTAs on different tiles share the same token rows.
// * Instead of p separate counters, each lane keeps bit-sliced vertical
//   counters: plane k of word w holds bit k of the counters of that word's 32
//   bins.  Counted are MISSES (tokens absent from the bin), started at
//   bias = 2^P - (D'+1) with D' = min(q*e, L-q+1), so the P-bit counter
//   overflows exactly when misses > D', i.e. when sum < T = (L-q+1) - q*e.
//   The overflow is kept in a sticky "dead" plane; a bin passes iff its dead
//   bit is clear at the end, and then its sum is (L-q+1) - (counter - bias).
//   P (5..8) is the smallest depth that holds the batch's largest D'.
// * Tokens are added 16 at a time with a carry-save (Harley-Seal) tree of
//   full adders (two 3-input LOP3s each), whose weight-16 carry ripples
//   through the P-4 upper planes: 2 logic ops per token per 32 bins at P = 5.
//   The logic ops run on the integer pipe, which bounds this kernel; the
//   token-to-address arithmetic is written as integer multiply-adds so that
//   it runs on the FMA pipe instead.
// * Early exit: after each 16-token block the group stops a read once every
//   one of its 1024 bins is dead -- exact, since a dead bin can never pass.
//   With the warp switch and 1024-bin tiles the test is one warp vote per
//   block: the warp takes new reads once every lane has no live bin or is
//   past its read's last block.  A group that ended reads on through its
//   token row's padding (the tokeniser fills each row to its stride with
//   the never-miss token), so its counters hold; a per-lane count of the
//   blocks that left a live bin gives each read's useful blocks.
// * Groups stay converged: the per-block work is the same instruction stream
//   for all groups of a warp, and every warp collective uses the full mask.
//   Taking a next read (new counters, the claim, the prefetch of the read
//   after it) runs for the whole warp whenever any group needs it, so the
//   launch chooses how groups switch reads (WS): each as soon as its read
//   ends (a switch for every read that ends), or all groups of a warp
//   together once every one of them has ended (one switch per warp per
//   round of reads; a group that ends early applies padding tokens, which
//   change nothing, until the others end).  With sixteen groups (256-bin
//   tiles) the warp switch comes once 14 of them wait; the other two keep
//   their reads.
// * One-word tail (1024-bin tiles, warp switch): after four blocks of a
//   round, if no lane of the warp has more than one word with a live bin,
//   the warp keeps that word's counters and applies the round's remaining
//   blocks to it alone (one 4-byte load and a quarter of the logic ops per
//   token).  Past the first blocks the live bins of a tile usually sit in
//   one or two words near the read's true position.  Register pressure
//   decides whether this pays: the tail runs as its own inner loop so that
//   the four-word loop stays as it was (a variant that chose the word count
//   per block spilled and ran slower than no tail at all).
#include "grim_internal.cuh"

namespace grim {
namespace {

// CTA sizes built (the register cap follows from one CTA per SM): 512
// threads (128 registers), 640 (96) and 768 (80).  640 is the default: on
// GB300 it beat 768 threads (which spill a few words) by 4.7% at q = 5 and
// 2.4% at q = 6, and 512 by 2.6%; the autotuner can pick another.
constexpr uint32_t kDefaultThreads = 640;
constexpr uint32_t kNone = 0xFFFFFFFFu;
constexpr size_t kSmemLimit = 227 * 1024;  // dynamic shared memory per CTA
// token rows of one read range: small enough to stay in L2 while every CTA
// sweeps its tiles against the range
constexpr uint64_t kDefaultRangeBytes = 48ull << 20;
constexpr uint32_t kSlotBlocksNarrow = 4;  // most slot blocks per read, 256-bin tiles
// WS, 256-bin tiles: groups of the sixteen that wait before the warp switches
constexpr uint32_t kSwitchGroupsNarrow = 14;
// blocks a warp applies to all four words of its lanes before it checks for
// the one-word tail (1024-bin tiles, warp-synchronous read switch)
constexpr uint32_t kTailAfter = 4;

template <int N>
struct Words {
  static constexpr int value = N;
};

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

// integer multiply-adds (FMA pipe); the multipliers come from kernel
// arguments so they are not strength-reduced into shifts
__device__ __forceinline__ uint32_t imad(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t d;
  asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}
__device__ __forceinline__ uint32_t imul_hi(uint32_t a, uint32_t b) {
  uint32_t d;
  asm("mul.hi.u32 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
  return d;
}
__device__ __forceinline__ uint4 lds128(uint32_t addr) {
  uint4 v;
  asm volatile("ld.shared.v4.u32 {%0,%1,%2,%3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "r"(addr));
  return v;
}

__device__ __forceinline__ uint32_t lds32(uint32_t addr) {
  uint32_t v;
  asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(addr));
  return v;
}

template <int P>
struct Counters {
  // per word: s1 s2 s4 s8 (weights 1..8), up[i] (weight 16 << i), dead
  uint32_t s1[4], s2[4], s4[4], s8[4], up[P - 4][4], dead[4];

  __device__ __forceinline__ void init(uint32_t bias) {
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      s1[w] = 0u - (bias & 1u);
      s2[w] = 0u - ((bias >> 1) & 1u);
      s4[w] = 0u - ((bias >> 2) & 1u);
      s8[w] = 0u - ((bias >> 3) & 1u);
#pragma unroll
      for (int i = 0; i < P - 4; ++i) up[i][w] = 0u - ((bias >> (4 + i)) & 1u);
      dead[w] = 0u;
    }
  }

  // One-word tail: keep only the counters of word k in slot 0 (dead unless
  // `live`); slots 1..3 die.
  __device__ __forceinline__ void keep_one(uint32_t k, bool live) {
    auto sel = [k](const uint32_t(&x)[4]) {
      return k == 0 ? x[0] : k == 1 ? x[1] : k == 2 ? x[2] : x[3];
    };
    s1[0] = sel(s1);
    s2[0] = sel(s2);
    s4[0] = sel(s4);
    s8[0] = sel(s8);
#pragma unroll
    for (int i = 0; i < P - 4; ++i) up[i][0] = sel(up[i]);
    dead[0] = live ? sel(dead) : ~0u;
    dead[1] = dead[2] = dead[3] = ~0u;
  }

  // counter value of bin `bit` of word w
  __device__ __forceinline__ uint32_t value(int w, uint32_t bit) const {
    uint32_t v = ((s1[w] >> bit) & 1u) | (((s2[w] >> bit) & 1u) << 1) |
                 (((s4[w] >> bit) & 1u) << 2) | (((s8[w] >> bit) & 1u) << 3);
#pragma unroll
    for (int i = 0; i < P - 4; ++i) v |= ((up[i][w] >> bit) & 1u) << (4 + i);
    return v;
  }
};

struct ExhArgs {
  IndexView ix;
  ReadsView rv;
  RecordsView rec;
  uint32_t bin_bits;
  uint32_t n_tiles, sms;
  Live live;
  uint32_t row_stride;  // bytes of one token row in a group slot (multiple of 32)
  uint32_t slot_bytes;  // bytes of a group slot: two token rows
  uint32_t slot_blocks; // 16-token blocks a slot row holds; later blocks come from L2
  uint32_t c_row, c_hi, c_lo;  // TW*4, 65536, -65536: multipliers of the address math
  uint64_t range_bytes;        // token-row bytes of one read range (the read tile)
  uint32_t switch_lanes;       // WS, 256-bin tiles: waiting lanes that make the warp switch
  Ctl* ctl;
};

// Add the misses of one 16-token block.  tw holds 16 table row indices as
// uint16 pairs; base is the shared address of this lane's words in row 0.
// NW = 4: all four words of the lane (one 16-byte load per token); NW = 1:
// the one-word tail, counter slot 0 only, its word at `base`.
template <int P, int NW>
__device__ __forceinline__ void add_block(Counters<P>& c, const uint32_t (&tw)[8], uint32_t base,
                                          const ExhArgs& a) {
  static_assert(NW == 4 || NW == 1, "four words or one");
  uint32_t addr[16];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const uint32_t hi = imul_hi(tw[j], a.c_hi);     // token 2j+1
    const uint32_t lo = imad(hi, a.c_lo, tw[j]);    // token 2j
    addr[2 * j] = imad(lo, a.c_row, base);
    addr[2 * j + 1] = imad(hi, a.c_row, base);
  }
  uint32_t t2a[NW], t2b[NW], t4a[NW], t4b[NW], t8a[NW], t8b[NW], t16[NW];
#pragma unroll
  for (int quad = 0; quad < 4; ++quad) {
    uint32_t a0[NW], a1[NW], a2[NW], a3[NW];
    if constexpr (NW == 4) {
      const uint4 x0 = lds128(addr[4 * quad]), x1 = lds128(addr[4 * quad + 1]);
      const uint4 x2 = lds128(addr[4 * quad + 2]), x3 = lds128(addr[4 * quad + 3]);
      a0[0] = x0.x; a0[1] = x0.y; a0[2] = x0.z; a0[3] = x0.w;
      a1[0] = x1.x; a1[1] = x1.y; a1[2] = x1.z; a1[3] = x1.w;
      a2[0] = x2.x; a2[1] = x2.y; a2[2] = x2.z; a2[3] = x2.w;
      a3[0] = x3.x; a3[1] = x3.y; a3[2] = x3.z; a3[3] = x3.w;
    } else {
      a0[0] = lds32(addr[4 * quad]);
      a1[0] = lds32(addr[4 * quad + 1]);
      a2[0] = lds32(addr[4 * quad + 2]);
      a3[0] = lds32(addr[4 * quad + 3]);
    }
#pragma unroll
    for (int w = 0; w < NW; ++w) {
      uint32_t* t4 = (quad & 1) ? t4b : t4a;
      fa_miss(c.s1[w], a0[w], a1[w], c.s1[w], t2a[w]);
      fa_miss(c.s1[w], a2[w], a3[w], c.s1[w], t2b[w]);
      fa(c.s2[w], t2a[w], t2b[w], c.s2[w], t4[w]);
      if (quad == 1) fa(c.s4[w], t4a[w], t4b[w], c.s4[w], t8a[w]);
      if (quad == 3) {
        fa(c.s4[w], t4a[w], t4b[w], c.s4[w], t8b[w]);
        fa(c.s8[w], t8a[w], t8b[w], c.s8[w], t16[w]);
        // ripple the weight-16 carry through the upper planes; the carry out
        // of the top plane (counter >= 2^P: misses > D') sticks in `dead`
        uint32_t k = t16[w];
#pragma unroll
        for (int i = 0; i < P - 5; ++i) {
          const uint32_t nk = c.up[i][w] & k;
          c.up[i][w] ^= k;
          k = nk;
        }
        uint32_t d;
        LOP3(d, c.dead[w], c.up[P - 5][w], k, 0xF8);  // dead | (top & k)
        c.up[P - 5][w] ^= k;
        c.dead[w] = d;
      }
    }
  }
}

template <int P, int TW, int NT, bool WS>
__global__ void __launch_bounds__(NT, 1) k_exhaustive(ExhArgs a) {
  constexpr uint32_t kRowBytes = TW * 4;     // one token's row of a tile
  constexpr uint32_t GL = TW / 4;            // lanes per group (one read)
  constexpr uint32_t kGroupMask = (1u << GL) - 1u;
  constexpr uint32_t kTileBinsT = TW * 32;
  // [tile: (r4 + 2) rows x TW words][group slots][16 padding tokens]
  extern __shared__ __align__(128) uint8_t smem[];
  __shared__ uint32_t s_item, s_next;
  const uint32_t tid = threadIdx.x, lane = tid & 31, grp = lane / GL, li = lane % GL;
  const uint32_t nthreads = blockDim.x;
  const uint32_t r4 = a.ix.r4;
  if (*(volatile uint32_t*)&a.ctl->status) return;  // set by the tokeniser before launch
  if (gated_off(a.ctl, a.live)) return;             // the batch takes the other path
  // work items: (tile, range of reads); enough of them to balance the
  // persistent grid, each range at least 64 reads
  const uint32_t n_reads = live_reads(a.ctl, a.live, a.rv.n_reads);
  if (n_reads == 0) return;
  // enough ranges to balance the persistent grid when tiles are few, and
  // ranges whose token rows fit in L2 when there are many reads: items are
  // then taken range by range, so the CTAs sweeping different tiles at the
  // same time share one range's token rows in L2 instead of each streaming
  // every read's tokens from DRAM
  uint32_t n_ranges = (4u * a.sms + a.n_tiles - 1) / a.n_tiles;
  const uint64_t token_bytes = (uint64_t)n_reads * a.rv.ts * 2u * a.rv.copies;
  const uint32_t l2_ranges = (uint32_t)((token_bytes + a.range_bytes - 1) / a.range_bytes);
  n_ranges = max(n_ranges, l2_ranges);
  n_ranges = min(n_ranges, (n_reads + 63) / 64);
  n_ranges = max(n_ranges, 1u);
  const uint32_t per = (n_reads + n_ranges - 1) / n_ranges;
  n_ranges = (n_reads + per - 1) / per;
  const uint32_t n_items = a.n_tiles * n_ranges;
  const bool range_major = a.n_tiles >= 4u * a.sms;

  uint32_t* s_tile = reinterpret_cast<uint32_t*>(smem);
  const uint32_t tile_bytes = (r4 + 2) * kRowBytes;
  const uint32_t sh_base = (uint32_t)__cvta_generic_to_shared(smem);
  const uint32_t slot = sh_base + tile_bytes + (tid / GL) * a.slot_bytes;
  const uint32_t pad_tokens = sh_base + tile_bytes + (nthreads / GL) * a.slot_bytes;
  for (uint32_t i = tid; i < (uint32_t)TW; i += nthreads) {
    s_tile[rowInvalid(r4) * TW + i] = 0u;
    s_tile[rowPad(r4) * TW + i] = ~0u;
  }
  if (tid < 2) {  // 16 padding tokens = 32 bytes
    const uint32_t pp = rowPad(r4) | (rowPad(r4) << 16);
    asm volatile("st.shared.v4.u32 [%0], {%1,%1,%1,%1};" ::"r"(pad_tokens + tid * 16u), "r"(pp));
  }
  const uint32_t lane_base = sh_base + li * 16u;
  // the token copy this group reads (block-rotated copies spread the groups'
  // 32-byte rows over the bank groups at q = 6)
  const uint32_t copy = a.rv.copies > 1 ? grp % a.rv.copies : 0u;
  const uint32_t row_chunks = a.row_stride / 16u;  // 16-byte chunks of a slot row

  for (;;) {
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();  // previous item finished with the tile and the slots
    if (tid == 0) {
      s_item = atomicAdd(&a.ctl->item, 1u);
      s_next = 0;
    }
    __syncthreads();
    const uint32_t item = s_item;
    if (item >= n_items) break;
    const uint32_t tile = range_major ? item % a.n_tiles : item / n_ranges;
    const uint32_t range = range_major ? item / a.n_tiles : item % n_ranges;
    const uint32_t r0 = range * per;
    const uint32_t nr = min(per, n_reads - r0);

    // stage the tile: rows [0, r4), words [tile*TW, tile*TW+TW)
    {
      constexpr uint32_t kChunks = TW / 4;  // 16-byte chunks per row
      const uint32_t* src = a.ix.tm + (uint64_t)tile * TW;
      for (uint32_t i = tid; i < r4 * kChunks; i += nthreads) {
        const uint32_t row = i / kChunks, chunk = i % kChunks;
        const uint32_t* g = src + (uint64_t)row * a.ix.wpad + chunk * 4u;
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sh_base + row * kRowBytes +
                                                                      chunk * 16u),
                     "l"(g));
      }
      asm volatile("cp.async.commit_group;");
    }

    // which bins of this lane's words exist (only the last tile is ragged)
    uint32_t vm[4];
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      const uint64_t b0 = (uint64_t)tile * kTileBinsT + (li * 4u + w) * 32u;
      const uint64_t left = b0 < a.ix.num_bins ? a.ix.num_bins - b0 : 0;
      vm[w] = left >= 32 ? ~0u : ((1u << left) - 1u);
    }
    auto vmask = [&](uint32_t w) -> uint32_t {
      return w == 0 ? vm[0] : w == 1 ? vm[1] : w == 2 ? vm[2] : vm[3];
    };

    // per-group state (identical in the group's 8 lanes); the group's slot
    // holds two token rows: `buf` is the current read's, buf^1 the next's
    uint32_t cur = kNone, nxt = kNone, nxt_meta = 0, buf = 1;
    uint32_t nblk = 0, ntok = 0, bias = 0, executed = 0, tail_exec = 0;
    // WS, 1024-bin tiles: blocks since the warp's last switch, and the word
    // kept in the one-word tail
    uint32_t bk = 0, kt = 0;
    uint32_t alive = 0;  // WS, 1024-bin tiles: blocks after which this lane had a live bin
    bool fin = false;
    Counters<P> c;
    c.init(0);

    // take the first read and start copying its tokens
    {
      uint32_t k = 0;
      if (li == 0) k = atomicAdd(&s_next, 1u);
      k = __shfl_sync(0xFFFFFFFFu, k, grp * GL);
      if (k < nr) {
        nxt = r0 + k;
        nxt_meta = __ldg(a.rv.meta + nxt);
        const char* src = reinterpret_cast<const char*>(
            a.rv.tokens + ((uint64_t)nxt * a.rv.copies + copy) * a.rv.ts);
        for (uint32_t ch = li; ch < row_chunks; ch += GL)
          asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(slot + ch * 16u),
                       "l"(src + ch * 16u));
      }
      asm volatile("cp.async.commit_group;");
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();  // tile staged

    // (1) groups without a read switch to the one whose tokens were copied
    //     ahead, and start copying the read after it; `tp` is the shared
    //     address of a group's next 16-token block, `left` its blocks left
    //     (finished groups apply padding tokens, their results ignored)
    uint32_t tp = pad_tokens, step = 0, left = 0;
    auto switch_reads = [&](bool need) {
      asm volatile("cp.async.wait_all;" ::: "memory");
      __syncwarp();
      if (need) {
        if (nxt == kNone) {
          fin = true;
        } else {
          cur = nxt;
          buf ^= 1u;
          ntok = nxt_meta & 0xFFu;
          const uint32_t d = (nxt_meta >> 8) & 0xFFu;
          bias = (1u << P) - (d + 1u);
          nblk = (ntok + kBlockTokens - 1) / kBlockTokens;
          c.init(bias);
        }
        tp = fin ? pad_tokens : slot + buf * a.row_stride;
        step = fin ? 0u : 32u;
        left = fin ? ~0u : nblk;
      }
      const bool take = need && !fin;
      uint32_t k = 0;
      if (take && li == 0) k = atomicAdd(&s_next, 1u);
      k = __shfl_sync(0xFFFFFFFFu, k, grp * GL);
      if (take) {
        nxt = k < nr ? r0 + k : kNone;
        if (nxt != kNone) {
          nxt_meta = __ldg(a.rv.meta + nxt);
          const char* src = reinterpret_cast<const char*>(
              a.rv.tokens + ((uint64_t)nxt * a.rv.copies + copy) * a.rv.ts);
          const uint32_t dst = slot + (buf ^ 1u) * a.row_stride;
          for (uint32_t ch = li; ch < row_chunks; ch += GL)
            asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(dst + ch * 16u),
                         "l"(src + ch * 16u));
        }
      }
      asm volatile("cp.async.commit_group;");
    };
    switch_reads(true);
    const uint32_t gmask = kGroupMask << (grp * GL);
    bool active = __any_sync(0xFFFFFFFFu, !fin);
    bool waiting = false;  // WS, 256-bin tiles: the group's read has ended; it waits for a switch

    // the passing bins of the groups whose reads ended (emit), then new
    // reads for them (done); the warp runs this together
    auto emit_and_switch = [&](bool done, bool emit, auto words) {
      constexpr int NW = decltype(words)::value;
      if (__any_sync(0xFFFFFFFFu, emit)) {
        // in the one-word tail slot 0 holds word kt and slots 1..3 are dead
        uint32_t pm[4], cnt = 0;
#pragma unroll
        for (int w = 0; w < 4; ++w) {
          pm[w] = emit ? (~c.dead[w] & vmask((NW == 1 && w == 0) ? kt : (uint32_t)w)) : 0u;
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
            const uint32_t wi = (NW == 1 && w == 0) ? kt : (uint32_t)w;
            const uint64_t bin = (uint64_t)tile * kTileBinsT + (li * 4u + wi) * 32u + bit;
            if (pos < a.rec.cap) {
              a.rec.keys[pos] = ((unsigned long long)cur << a.bin_bits) | bin;
              a.rec.counts[pos] = (uint8_t)(ntok - misses);
            }
            ++pos;
          }
        }
      }
      if (done) cur = kNone;
      switch_reads(done);
      waiting = false;
      active = __any_sync(0xFFFFFFFFu, !fin);
    };

    // (2) one 16-token block for all groups, to NW words per lane: from the
    //     slot, or for the blocks past the slot's rows (long reads at q = 6)
    //     from L2; (3) then the end-of-read test.  True when the warp took
    //     new reads.
    auto run_block = [&](auto words) -> bool {
      constexpr int NW = decltype(words)::value;
      {
        uint4 t0, t1;
        const uint32_t bi = nblk - left;  // this read's block index
        // (1024-bin tiles: whole reads in slots; waiting groups read padding)
        if (TW == 32 || fin || waiting || bi < a.slot_blocks) {
          t0 = lds128(tp);
          t1 = lds128(tp + 16u);
        } else {
          const uint4* g = reinterpret_cast<const uint4*>(
              a.rv.tokens + ((uint64_t)cur * a.rv.copies + copy) * a.rv.ts + bi * kBlockTokens);
          t0 = __ldg(g);
          t1 = __ldg(g + 1);
        }
        const uint32_t tw[8] = {t0.x, t0.y, t0.z, t0.w, t1.x, t1.y, t1.z, t1.w};
        if constexpr (NW == 1) add_block<P, 1>(c, tw, lane_base + kt * 4u, a);
        else add_block<P, 4>(c, tw, lane_base, a);
      }
      tp += step;
      --left;

      // a read ends when every bin of its tile is dead or its tokens are
      // used up
      const uint32_t all_dead = c.dead[0] & c.dead[1] & c.dead[2] & c.dead[3];
      if constexpr (WS && TW == 32) {
        // lockstep: one vote per block.  The warp takes new reads once every
        // lane has no live bin or is past its read's last block (a group
        // without a read has left = ~0).  A group whose read ended reads on
        // through its token row's padding (never a miss), so its counters
        // keep their values; a dead group may apply its remaining tokens
        // (dead bins stay dead).
        const bool ldead = all_dead == ~0u;
        alive += ldead ? 0u : 1u;
        if (!__all_sync(0xFFFFFFFFu, ldead || (int)left <= 0)) return false;
        const bool gdead = (__ballot_sync(0xFFFFFFFFu, ldead) & gmask) == gmask;
        // blocks the read needed: up to the one after which its last live
        // lane died, or all of them
        uint32_t m = alive;
        m = max(m, __shfl_xor_sync(0xFFFFFFFFu, m, 1));
        m = max(m, __shfl_xor_sync(0xFFFFFFFFu, m, 2));
        m = max(m, __shfl_xor_sync(0xFFFFFFFFu, m, 4));
        const uint32_t used = min(nblk, m + 1u);
        const bool done = !fin;
        if (done) {
          executed += used;
          if (NW == 1 && used > kTailAfter) tail_exec += used - kTailAfter;
        }
        alive = 0;
        emit_and_switch(done, done && !gdead, Words<NW>{});
        return true;
      }
      const uint32_t bal = __ballot_sync(0xFFFFFFFFu, all_dead == ~0u);
      const bool gdead = (bal & gmask) == gmask;
      bool done = !fin && !waiting && (gdead || left == 0);
      if (WS && done) {
        // freeze the group's counters (padding adds no misses) until the
        // warp switches
        executed += nblk - left;
        if (NW == 1) tail_exec += nblk - left;
        waiting = true;
        tp = pad_tokens;
        step = 0;
      }
      bool take_next;
      if constexpr (!WS) {
        take_next = __any_sync(0xFFFFFFFFu, done);
      } else if constexpr (TW == 32) {
        take_next = __all_sync(0xFFFFFFFFu, fin || waiting);
      } else {
        // sixteen groups: switch once enough of them wait, so that a few
        // long reads do not hold the rest (the others keep their reads)
        take_next = __popc(__ballot_sync(0xFFFFFFFFu, fin || waiting)) >= a.switch_lanes;
      }
      if (!take_next) return false;
      if (WS) {
        done = waiting;
      } else if (done) {
        executed += nblk - left;
      }
      emit_and_switch(done, done && !gdead, Words<NW>{});
      return true;
    };

    while (active) {
      if (run_block(Words<4>{})) {
        bk = 0;
        continue;
      }
      if constexpr (WS && TW == 32) {
        if (++bk != kTailAfter) continue;
        // one-word tail: once every lane of the warp has at most one word
        // with a live bin (typically only near a read's true position), the
        // warp applies the rest of the round's blocks to that word alone: a
        // quarter of the logic ops, one 4-byte load per token.  Exact: a
        // word dropped here has no live bin (or only bins past the table's
        // end), and dead bins never pass.
        uint32_t lm = 0;
        if (!fin) {
#pragma unroll
          for (int w = 0; w < 4; ++w)
            if (~c.dead[w] & vmask(w)) lm |= 1u << w;
        }
        if (__all_sync(0xFFFFFFFFu, (lm & (lm - 1u)) == 0u)) {
          kt = lm ? (uint32_t)__ffs(lm) - 1u : 0u;
          c.keep_one(kt, lm != 0u);
          while (!run_block(Words<1>{})) {
          }
          bk = 0;
        }
      }
    }
    // one count per group (its lanes agree), one atomic per warp and item
    uint32_t ex = li == 0 ? executed : 0u;
    ex = __reduce_add_sync(0xFFFFFFFFu, ex);
    if (lane == 0 && ex) atomicAdd(&a.ctl->blocks, (unsigned long long)ex);
    if constexpr (WS && TW == 32) {
      uint32_t tx = li == 0 ? tail_exec : 0u;
      tx = __reduce_add_sync(0xFFFFFFFFu, tx);
      if (lane == 0 && tx) atomicAdd(&a.ctl->tail_blocks, (unsigned long long)tx);
    }
  }
}

template <int P, int TW, int NT, bool WS>
void launch_p(const ExhArgs& a, size_t smem, uint32_t threads, uint32_t grid, cudaStream_t st,
              const char* name) {
  cudaFuncSetAttribute(k_exhaustive<P, TW, NT, WS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)smem);
  ProfScope ps(name, st);
  k_exhaustive<P, TW, NT, WS><<<grid, threads, smem, st>>>(a);
}

template <int TW, int NT, bool WS>
void launch_ws(const ExhArgs& a, size_t smem, uint32_t threads, uint32_t grid, uint32_t max_d,
               cudaStream_t st, const char* name) {
  // the counters need 2^P > D' (D' <= 255)
  if (max_d < 32) launch_p<5, TW, NT, WS>(a, smem, threads, grid, st, name);
  else if (max_d < 64) launch_p<6, TW, NT, WS>(a, smem, threads, grid, st, name);
  else if (max_d < 128) launch_p<7, TW, NT, WS>(a, smem, threads, grid, st, name);
  else launch_p<8, TW, NT, WS>(a, smem, threads, grid, st, name);
}

template <int TW, int NT>
void launch_nt(const ExhArgs& a, size_t smem, uint32_t threads, uint32_t grid, uint32_t max_d,
               bool warp_switch, cudaStream_t st, const char* name) {
  if (warp_switch) launch_ws<TW, NT, true>(a, smem, threads, grid, max_d, st, name);
  else launch_ws<TW, NT, false>(a, smem, threads, grid, max_d, st, name);
}

template <int TW>
void launch_tw(ExhArgs& a, const IndexView& ix, uint32_t max_d, uint32_t sms, uint32_t nt,
               bool warp_switch, cudaStream_t st, const char* name) {
  constexpr uint32_t kRowBytes = TW * 4, GL = TW / 4, kTileBinsT = TW * 32;
  a.n_tiles = (uint32_t)(ix.num_bins_pad / kTileBinsT);
  a.sms = sms;
  a.c_row = kRowBytes;
  // the largest CTA up to the built size whose tile and group slots fit in
  // shared memory
  const size_t tile_bytes = (size_t)(ix.r4 + 2) * kRowBytes;
  uint32_t threads = nt;
  while (threads > 64 && tile_bytes + (size_t)(threads / GL) * a.slot_bytes + 32 > kSmemLimit)
    threads -= 32;
  const size_t smem = tile_bytes + (size_t)(threads / GL) * a.slot_bytes + 32;
  // small batches on few tiles need fewer CTAs (graph launches size for the
  // largest batch and let surplus CTAs find no work)
  uint32_t grid = sms;
  if (!a.live.on) {
    const uint32_t per_item = 64;
    const uint64_t items = (uint64_t)a.n_tiles * ((a.rv.n_reads + per_item - 1) / per_item);
    if (items < grid) grid = (uint32_t)(items ? items : 1);
  }
  if (nt == 512) launch_nt<TW, 512>(a, smem, threads, grid, max_d, warp_switch, st, name);
  else if (nt == 768) launch_nt<TW, 768>(a, smem, threads, grid, max_d, warp_switch, st, name);
  else launch_nt<TW, 640>(a, smem, threads, grid, max_d, warp_switch, st, name);
}

}  // namespace

uint32_t exhaustive_tile_bins(uint32_t r4) { return r4 <= 1024 ? 32u * 32u : 8u * 32u; }

bool exhaustive_shape_ok(const ExhShape& s) {
  const bool t_ok = s.threads == 0 || s.threads == 512 || s.threads == 640 || s.threads == 768;
  const bool r_ok = s.range_kb == 0 || (s.range_kb >= 1024 && s.range_kb <= (4u << 20));
  const bool w_ok = s.read_switch <= 2;
  return t_ok && r_ok && w_ok;
}

void launch_exhaustive(const IndexView& ix, const ReadsView& rv, RecordsView rec, uint32_t bin_bits,
                       uint32_t max_d, Ctl* ctl, cudaStream_t st, const char* prof_name,
                       Live live, ExhShape shape) {
  if (rv.n_reads == 0) return;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (sms <= 0) sms = 1;
  ExhArgs a{};
  a.ix = ix;
  a.rv = rv;
  a.rec = rec;
  a.bin_bits = bin_bits;
  a.live = live;
  // a slot row holds a read's first blocks: all of them for the 1024-bin
  // tiles; for the 256-bin tiles of q = 6, whose 128 KB tile leaves little
  // room for the sixteen groups' slots of a warp, as many (up to
  // kSlotBlocksNarrow) as fit beside the tile at the CTA size -- the later
  // blocks come from L2 (warps matter more than slot blocks: at 768-thread
  // CTAs 1 block let 24 warps per SM fit, 7 blocks 11)
  const uint32_t nt = shape.threads ? shape.threads : kDefaultThreads;
  const uint32_t blocks = rv.ts / kBlockTokens;
  // slots of consecutive groups start 32 bytes apart modulo 128, so the
  // groups of a warp mostly read their tokens from different banks
  auto slot_bytes_of = [](uint32_t slot_blocks) {
    return (2u * slot_blocks * kBlockTokens * 2u + 127u) / 128u * 128u + 32u;
  };
  if (ix.r4 <= 1024) {
    a.slot_blocks = blocks;
  } else {
    const size_t tile_bytes = (size_t)(ix.r4 + 2) * 8u * 4u;
    const uint32_t groups = nt / 2u;  // 2-lane groups
    a.slot_blocks = 1;
    for (uint32_t sb = min(blocks, kSlotBlocksNarrow); sb > 1; --sb)
      if (tile_bytes + (size_t)groups * slot_bytes_of(sb) + 32 <= kSmemLimit) {
        a.slot_blocks = sb;
        break;
      }
  }
  a.row_stride = a.slot_blocks * kBlockTokens * 2u;
  a.slot_bytes = slot_bytes_of(a.slot_blocks);
  a.switch_lanes = kSwitchGroupsNarrow * 2u;
  a.c_hi = 65536u;
  a.c_lo = 0u - 65536u;
  a.range_bytes = shape.range_kb ? (uint64_t)shape.range_kb << 10 : kDefaultRangeBytes;
  a.ctl = ctl;
  const bool ws = shape.read_switch == GRIM_SWITCH_WARP;
  if (ix.r4 <= 1024) launch_tw<32>(a, ix, max_d, (uint32_t)sms, nt, ws, st, prof_name);
  else launch_tw<8>(a, ix, max_d, (uint32_t)sms, nt, ws, st, prof_name);
}

}  // namespace grim
