// Candidate-list filter over the bin-major table (§GRIM-Filter: for each
// candidate location the mapper asks whether the bin holding it can possibly
// match; steps 2-3 and Fig. 5).
//
// GB300 mapping
// -------------
// * Warps claim chunks of 256-4096 consecutive candidates of the flattened lists
//   from a global counter (a chunk may hold many short lists; a long list is
//   spread over many warps, so no single 20,000-candidate list is left
//   running alone at the end).  For each read in its chunk the warp turns the
//   read's tokens into a multiplicity histogram (a byte per token value) and
//   then into bit planes P_k = {t : bit k of mult(t) is 1}, held in
//   registers, so that for any bin vector v the token sum is
//       sum = sum_k 2^k * popcount(v & P_k)
//   -- every position counts, repeats included, with a handful of AND +
//   POPC per 32 bits instead of one bit test per token.
// * A bin vector (4^q bits) is gathered by G lanes with 16-byte loads
//   (q = 5: 8 lanes x 16 B = 128 B, four candidates per warp step; q = 6:
//   32 lanes x 16 B = 512 B).  The U vectors of a step are reduced over the
//   lane group together (a butterfly that halves the sums at each exchange;
//   for a whole-warp group, one redux.sync per vector), compared with
//   T = (L-q+1) - q*e, and one ballot places the passes.
// * The path is a random 128/512-byte gather per (read, bin) pair: bound by
//   HBM, not by arithmetic.
#include "grim_internal.cuh"

namespace grim {
namespace {

template <int WPB>
struct Cfg {
  static constexpr int WL = WPB >= 4 ? 4 : WPB;  // words per lane
  static constexpr int G = WPB / WL;             // lanes per candidate
  static constexpr int CPW = 32 / G;             // candidates per warp step
};

template <int WL>
__device__ __forceinline__ void load_words(const uint32_t* p, uint32_t (&v)[WL]) {
  if constexpr (WL == 4) {
    const uint4 x = __ldg(reinterpret_cast<const uint4*>(p));
    v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
  } else if constexpr (WL == 2) {
    const uint2 x = __ldg(reinterpret_cast<const uint2*>(p));
    v[0] = x.x; v[1] = x.y;
  } else {
    v[0] = __ldg(p);
  }
}

struct CandArgs {
  IndexView ix;
  ReadsView rv;
  const int32_t* cand;
  const uint64_t* cand_off;
  RecordsView rec;
  Ctl* ctl;
  Live live;
  bool check_ids;  // caller's lists: an id outside [0, num_bins) is an error
};

constexpr int kWarps = 8;
// gathers in flight per lane group when the caller leaves it to the library
// (the autotuner's choice on GB300 for both 128- and 512-byte vectors)
constexpr uint32_t kDefaultCandUnroll = 2;
constexpr int kRegPlanes = 2;  // bit planes held in registers: multiplicities up to 3

// Multiplicities of 4 and more (bits kRegPlanes.. of a token's count) are
// rare.  Up to 128-byte vectors they are kept as further bit planes in shared
// memory (xplanes[k - kRegPlanes][word]).  For 512-byte vectors those planes
// would take 3 KB a warp beside the 4 KB histogram and limit the kernel to
// 32 warps per SM; instead the read's tokens of multiplicity >= 4 are listed
// (token | (mult & ~3) << 16; at most 255 / 4 < 64 of them) and added one by
// one, which makes room for 48 warps.
template <int WPB> __host__ __device__ constexpr bool heavy_list() { return WPB >= 128; }
constexpr uint32_t kMaxHeavy = 64;

// per-warp shared memory: the multiplicity histogram, then the higher bit
// planes or the list of heavy tokens
__host__ __device__ constexpr uint32_t hist_words_of(uint32_t r4) { return r4 >= 4 ? r4 / 4 : 1; }
__host__ __device__ constexpr uint32_t warp_smem_words(uint32_t r4, uint32_t wpb) {
  return hist_words_of(r4) + (wpb >= 128 ? kMaxHeavy : (8 - kRegPlanes) * wpb);
}

// The read's multiplicity histogram (byte t = how many of its positions hold
// token t) and its bit planes P_k = {t : bit k of mult(t)} for this lane's WL
// words of a bin vector: planes below kRegPlanes in registers, the rest in
// shared memory, or (heavy_list) the heavy tokens in xplanes[0, *nh).
// Returns K, the number of planes in use, and the read's threshold in *thr.
// Warp-collective.
template <int WPB, int WL>
__device__ __forceinline__ uint32_t build_planes(const ReadsView& rv, uint32_t r, uint32_t r4,
                                                 uint32_t* hist, uint32_t* xplanes, uint32_t lane,
                                                 uint32_t sub, uint32_t (&P)[kRegPlanes][WL],
                                                 uint32_t* thr, uint32_t* nh) {
  constexpr int kPlanesBuilt = heavy_list<WPB>() ? kRegPlanes : 8;
  const uint32_t hist_words = hist_words_of(r4);
  // the warp has finished reading the previous read's histogram
  __syncwarp();
  for (uint32_t i = lane; i < hist_words; i += 32) hist[i] = 0;
  __syncwarp();
  const uint32_t m = rv.meta[r];
  const uint32_t ntok = m & 0xFFu, dmax = (m >> 8) & 0xFFu;
  const uint16_t* tk = rv.tokens + (uint64_t)r * rv.copies * rv.ts;
  for (uint32_t j = lane; j < ntok; j += 32) {
    const uint32_t t = tk[j];
    if (t < r4) atomicAdd(hist + (t >> 2), 1u << (8 * (t & 3u)));
  }
  __syncwarp();
  // the largest multiplicity decides how many bit planes the sums need
  // (almost always 1 or 2)
  uint32_t mx = 0;
  for (uint32_t i = lane; i < hist_words; i += 32) {
    const uint32_t h = hist[i];
    mx = max(mx, max(max(h & 0xFFu, (h >> 8) & 0xFFu), max((h >> 16) & 0xFFu, h >> 24)));
  }
  mx = __reduce_max_sync(0xFFFFFFFFu, mx);
  const uint32_t K = 32 - __clz(mx);  // planes in use
#pragma unroll
  for (int w = 0; w < WL; ++w) {
    const uint32_t wi = sub * WL + w;  // word index in the vector: tokens wi*32 .. wi*32+31
    uint32_t hw[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const uint32_t h = wi * 8 + j;
      hw[j] = h < hist_words && (wi * 32 + 4 * j) < r4 ? hist[h] : 0u;
    }
#pragma unroll
    for (int k = 0; k < kPlanesBuilt; ++k) {
      if ((uint32_t)k < K) {
        uint32_t pk = 0;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          uint32_t x = (hw[j] >> k) & 0x01010101u;  // bit k of 4 byte counters
          x |= x >> 7;
          x |= x >> 14;
          pk |= (x & 0xFu) << (4 * j);
        }
        if (k < kRegPlanes) P[k < kRegPlanes ? k : 0][w] = pk;
        else xplanes[(k - kRegPlanes) * WPB + wi] = pk;
      } else if (k < kRegPlanes) {
        P[k < kRegPlanes ? k : 0][w] = 0;
      }
    }
  }
  if constexpr (heavy_list<WPB>()) {
    uint32_t count = 0;
    if (K > (uint32_t)kRegPlanes) {
      // list the tokens of multiplicity >= 4 with the part of their count
      // above the register planes; each lane takes its histogram words
      uint32_t mine = 0;
      for (uint32_t i = lane; i < hist_words; i += 32) {
        const uint32_t h = hist[i];
        mine += ((h & 0xFCu) != 0) + ((h & 0xFC00u) != 0) + ((h & 0xFC0000u) != 0) +
                ((h & 0xFC000000u) != 0);
      }
      uint32_t incl = mine;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, incl, d);
        if (lane >= (uint32_t)d) incl += t;
      }
      count = __shfl_sync(0xFFFFFFFFu, incl, 31);
      uint32_t pos = incl - mine;
      for (uint32_t i = lane; i < hist_words; i += 32) {
        const uint32_t h = hist[i];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const uint32_t mult = (h >> (8 * j)) & 0xFFu;
          if (mult >= 4 && pos < kMaxHeavy) xplanes[pos++] = (4 * i + j) | ((mult & ~3u) << 16);
        }
      }
      __syncwarp();
    }
    *nh = min(count, kMaxHeavy);
  }
  *thr = ntok - dmax;  // pass iff sum >= (L-q+1) - min(q*e, L-q+1)
  return K;
}

// sum_k 2^k popc(v & P_k) over this lane's WL words (with heavy_list: the
// two register planes, then the listed heavy tokens that fall in this
// lane's words, nh of them)
template <int WPB, int WL>
__device__ __forceinline__ uint32_t plane_sum(const uint32_t (&v)[WL],
                                              const uint32_t (&P)[kRegPlanes][WL], uint32_t K,
                                              const uint32_t* xplanes, uint32_t sub, uint32_t nh) {
  static_assert(!heavy_list<WPB>() || (WL == 4 && kRegPlanes == 2), "heavy list layout");
  if constexpr (WL == 4 && kRegPlanes == 2) {
    if (heavy_list<WPB>() || K <= 2) {
      // the eight masked words (four of weight 1, four of weight 2) summed
      // bit-wise with a carry-save tree first: 4 POPC instead of 8
      const uint32_t a0 = v[0] & P[0][0], a1 = v[1] & P[0][1], a2 = v[2] & P[0][2],
                     a3 = v[3] & P[0][3];
      const uint32_t b0 = v[0] & P[1][0], b1 = v[1] & P[1][1], b2 = v[2] & P[1][2],
                     b3 = v[3] & P[1][3];
      const uint32_t s1 = a0 ^ a1 ^ a2, c1 = (a0 & a1) | (a2 & (a0 ^ a1));  // weights 1, 2
      const uint32_t s2 = s1 ^ a3, c2 = s1 & a3;                              // weights 1, 2
      const uint32_t s3 = c1 ^ c2 ^ b0, c3 = (c1 & c2) | (b0 & (c1 ^ c2));   // weights 2, 4
      const uint32_t s4 = b1 ^ b2 ^ b3, c4 = (b1 & b2) | (b3 & (b1 ^ b2));   // weights 2, 4
      const uint32_t s5 = s3 ^ s4, c5 = s3 & s4;                              // weights 2, 4
      const uint32_t s6 = c3 ^ c4 ^ c5, c6 = (c3 & c4) | (c5 & (c3 ^ c4));   // weights 4, 8
      uint32_t sum = __popc(s2) + 2u * __popc(s5) + 4u * __popc(s6) + 8u * __popc(c6);
      if constexpr (heavy_list<WPB>()) {
        for (uint32_t i = 0; i < nh; ++i) {
          const uint32_t ent = xplanes[i];
          const uint32_t t = ent & 0xFFFFu, wi = t >> 5;  // token, word of the vector
          if (wi / WL == sub) {
            const uint32_t w = wi % WL;
            const uint32_t word = w == 0 ? v[0] : w == 1 ? v[1] : w == 2 ? v[2] : v[3];
            sum += ((word >> (t & 31u)) & 1u) * (ent >> 16);
          }
        }
      }
      return sum;
    }
  }
  uint32_t sum = 0;
#pragma unroll
  for (int p = 0; p < kRegPlanes; ++p) {
    if ((uint32_t)p < K) {
      uint32_t s = 0;
#pragma unroll
      for (int w = 0; w < WL; ++w) s += __popc(v[w] & P[p][w]);
      sum += s << p;
    }
  }
  for (uint32_t p = kRegPlanes; p < K; ++p) {
    uint32_t s = 0;
#pragma unroll
    for (int w = 0; w < WL; ++w) s += __popc(v[w] & xplanes[(p - kRegPlanes) * WPB + sub * WL + w]);
    sum += s << p;
  }
  return sum;
}

// Sums of U candidates over a lane group of G lanes (U <= G, powers of two):
// at each of the first log2(U) butterfly steps a lane keeps half of its
// sums and adds its partner's copy of them, sending the other half; the
// remaining steps reduce the one sum left.  Lane `sub` of the group returns
// the group total of candidate sub / (G / U).  log2(U) + log2(G/U) shuffles
// instead of U * log2(G).
template <int G, int U>
__device__ __forceinline__ uint32_t reduce_scatter(uint32_t (&s)[U], uint32_t sub) {
#pragma unroll
  for (int n = U, m = G / 2; n > 1; n >>= 1, m >>= 1) {
    const bool upper = (sub & (uint32_t)m) != 0;  // keep the upper half of the n sums
#pragma unroll
    for (int i = 0; i < n / 2; ++i) {
      const uint32_t lo = s[i], hi = s[i + n / 2];
      s[i] = (upper ? hi : lo) + __shfl_xor_sync(0xFFFFFFFFu, upper ? lo : hi, m);
    }
  }
#pragma unroll
  for (int m = G / (2 * U); m >= 1; m >>= 1) s[0] += __shfl_xor_sync(0xFFFFFFFFu, s[0], m);
  return s[0];
}

// ids of candidates seg[off + u*CPW + slot] (u < U) of a segment of n
// candidates, 0 past its end; 32-bit offsets within the segment
template <int U, int CPW>
__device__ __forceinline__ void load_ids(const int32_t* __restrict__ seg, uint32_t off, uint32_t n,
                                         uint32_t slot, uint32_t (&b)[U]) {
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const uint32_t k = off + u * CPW + slot;
    b[u] = k < n ? (uint32_t)__ldg(seg + k) : 0u;
  }
}

// Candidates per work claim: large enough that the search for a chunk's
// first read and the planes of the reads split at chunk edges stay cheap,
// small enough that every warp gets about 16 chunks (an even finish).
constexpr uint64_t kChunkMin = 256, kChunkMax = 4096, kChunksPerWarp = 16;
__device__ __forceinline__ uint64_t chunk_size(uint64_t n_cand, uint64_t warps) {
  uint64_t c = kChunkMax;
  while (c > kChunkMin && c * kChunksPerWarp * warps > n_cand) c >>= 1;
  return c;
}

// The read holding candidate x: the largest r < n_reads with cand_off[r] <= x
// (empty lists in between are skipped), by a 32-way search.
__device__ __forceinline__ uint32_t read_of(const uint64_t* __restrict__ cand_off, uint32_t n_reads,
                                            uint64_t x, uint32_t lane) {
  uint32_t lo = 0, hi = n_reads;  // cand_off[lo] <= x < cand_off[hi]
  while (hi - lo > 1) {
    const uint32_t step = (hi - lo + 31) / 32;
    const uint32_t p = lo + lane * step;
    const bool le = p < hi && cand_off[p] <= x;
    const uint32_t bal = __ballot_sync(0xFFFFFFFFu, le);  // lane 0 always (cand_off[lo] <= x)
    const uint32_t last = 31 - __clz(bal);
    lo = lo + last * step;
    hi = min(hi, lo + step);
  }
  return lo;
}

// CTAs per SM.  Up to 128-byte vectors: eight (64 warps, 32 registers a
// thread); the gathers are latency-bound, and the extra warps outweigh a few
// spilled words.  512-byte vectors (q = 6): six (40 registers), where the
// spills of the 32-register layout cost more than the warps gain.
__host__ __device__ constexpr int cand_ctas_per_sm(int wpb) { return wpb >= 128 ? 6 : 8; }

template <int WPB, int U>
__global__ void __launch_bounds__(kWarps * 32, cand_ctas_per_sm(WPB)) k_candidates(CandArgs a) {
  using C = Cfg<WPB>;
  constexpr int WL = C::WL, G = C::G, CPW = C::CPW;
  extern __shared__ uint32_t s_warp[];
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t r4 = a.ix.r4;
  uint32_t* hist = s_warp + warp * warp_smem_words(r4, WPB);  // byte t = multiplicity of token t
  uint32_t* xplanes = hist + hist_words_of(r4);  // higher planes or heavy tokens
  const uint32_t sub = lane % G;     // this lane's slice of a bin vector
  const uint32_t slot = lane / G;    // which of the warp's CPW candidates
  if (*(volatile uint32_t*)&a.ctl->status) return;
  if (gated_off(a.ctl, a.live)) return;  // the batch takes the other path
  const uint32_t n_reads = live_reads(a.ctl, a.live, a.rv.n_reads);
  if (n_reads == 0) return;
  // the batch's lists span candidates [c_begin, c_end); warps claim chunks
  // of `chunk` consecutive candidates, so a long list is shared by many warps
  const uint64_t c_begin = a.cand_off[0], c_end = a.cand_off[n_reads];
  const uint64_t chunk =
      c_end > c_begin ? chunk_size(c_end - c_begin, (uint64_t)gridDim.x * kWarps) : kChunkMin;
  const uint64_t n_chunks = c_end > c_begin ? (c_end - c_begin + chunk - 1) / chunk : 0;

  uint32_t cur = 0xFFFFFFFFu, K = 0, thr = 0, nh = 0;  // the read whose planes are built
  const bool check = a.check_ids;
  const uint32_t last_row = (uint32_t)(a.ix.bm_rows - 1);
  const uint32_t num_bins = (uint32_t)a.ix.num_bins;  // bins are uint32 (checked at build)
  bool bad = false;  // this lane saw a candidate id outside [0, num_bins)
  uint32_t P[kRegPlanes][WL];
  // the next chunk is claimed one chunk ahead, so the atomic's latency
  // overlaps the current chunk's work
  uint32_t cj_next = 0;
  if (lane == 0) cj_next = atomicAdd(&a.ctl->item, 1u);
  for (;;) {
    const uint32_t cj = __shfl_sync(0xFFFFFFFFu, cj_next, 0);
    if (cj >= n_chunks) break;
    if (lane == 0) cj_next = atomicAdd(&a.ctl->item, 1u);
    // positions inside the chunk are 32-bit, relative to its first candidate
    const uint64_t base = c_begin + (uint64_t)cj * chunk;
    const uint32_t clen = (uint32_t)min(chunk, c_end - base);
    uint32_t r = read_of(a.cand_off, n_reads, base, lane);
    // the end of read r's list, clipped to the chunk (> 0: r's list holds base)
    uint32_t c1 = (uint32_t)min(a.cand_off[r + 1] - base, (uint64_t)clen);
    uint32_t p = 0;
    while (p < clen) {
      // the segment [p, c1) of read r's list inside this chunk; the end of the
      // next read's list is fetched while this one is scored
      const uint32_t c1_next = r + 2 <= n_reads && c1 < clen
                                   ? (uint32_t)min(a.cand_off[r + 2] - base, (uint64_t)clen)
                                   : c1;
      if (c1 > p) {
        // the segment's candidates seg[0, n)
        const int32_t* seg = a.cand + base + p;
        const uint32_t n = c1 - p;
        // the first candidate ids are fetched while the planes are built
        uint32_t bc[U];
        load_ids<U, CPW>(seg, 0, n, slot, bc);
        if (r != cur) {
          cur = r;
          K = build_planes<WPB, WL>(a.rv, r, r4, hist, xplanes, lane, sub, P, &thr, &nh);
        }
        // U independent gathers in flight per lane group; the ids of the
        // next step are fetched before this step's vectors are used
        for (uint32_t off = 0; off < n; off += CPW * U) {
          uint32_t bn[U];
          load_ids<U, CPW>(seg, off + CPW * U, n, slot, bn);
          // the caller's ids are checked here, where they are read anyway: an
          // id outside [0, num_bins) fails the call, never passes, and its
          // gather is clamped inside the table
          uint32_t v[U][WL];
#pragma unroll
          for (int u = 0; u < U; ++u) {
            const bool in = off + u * CPW + slot < n;
            bad |= check && in && bc[u] >= num_bins;
            const uint32_t row = min(bc[u], last_row);
            if (in) load_words<WL>(a.ix.bm + (uint64_t)row * WPB + sub * WL, v[u]);
          }
          // passing candidates of the warp get consecutive record slots
          auto emit = [&](bool pass, uint32_t c, uint32_t sum) {
            const uint32_t bal = __ballot_sync(0xFFFFFFFFu, pass);
            if (bal) {
              unsigned long long first = 0;  // the warp's first record slot
              if (lane == 0) first = atomicAdd(&a.ctl->n_rec, (unsigned long long)__popc(bal));
              first = __shfl_sync(0xFFFFFFFFu, first, 0);
              if (pass) {
                const unsigned long long pos = first + __popc(bal & ((1u << lane) - 1u));
                if (pos < a.rec.cap) {
                  a.rec.keys[pos] = base + p + c;
                  a.rec.counts[pos] = (uint8_t)sum;
                }
              }
            }
          };
          uint32_t sums[U];
#pragma unroll
          for (int u = 0; u < U; ++u)
            sums[u] = off + u * CPW + slot < n ? plane_sum<WPB, WL>(v[u], P, K, xplanes, sub, nh) : 0u;
          // bins past num_bins exist only as zero padding of the table
          // (members of the last super-bin); they never pass
          if constexpr (G == 32) {
            // a lane group is the whole warp (512-byte vectors): one
            // full-warp reduction per candidate, and lane u emits candidate u
            uint32_t total = 0, id = 0;
#pragma unroll
            for (int u = 0; u < U; ++u) {
              const uint32_t t = __reduce_add_sync(0xFFFFFFFFu, sums[u]);
              total = lane == (uint32_t)u ? t : total;
              id = lane == (uint32_t)u ? bc[u] : id;
            }
            const uint32_t c = off + lane;
            emit(lane < (uint32_t)U && c < n && id < num_bins && total >= thr, c, total);
          } else if constexpr (U > 1 && U <= G) {
            // the U sums reduced over the lane group at once: each lane ends
            // with the total of candidate uq, held by G/U lanes
            const uint32_t total = reduce_scatter<G, U>(sums, sub);
            const uint32_t uq = sub / (G / U);
            uint32_t id = bc[0];
#pragma unroll
            for (int u = 1; u < U; ++u) id = uq == (uint32_t)u ? bc[u] : id;
            const uint32_t c = off + uq * CPW + slot;
            emit(sub % (G / U) == 0 && c < n && id < num_bins && total >= thr, c, total);
          } else {
#pragma unroll
            for (int u = 0; u < U; ++u) {
              const uint32_t c = off + u * CPW + slot;
              uint32_t sum = sums[u];
#pragma unroll
              for (int o = G / 2; o >= 1; o >>= 1) sum += __shfl_xor_sync(0xFFFFFFFFu, sum, o);
              emit(c < n && bc[u] < num_bins && sub == 0 && sum >= thr, c, sum);
            }
          }
#pragma unroll
          for (int u = 0; u < U; ++u) bc[u] = bn[u];
        }
      }
      p = c1;
      ++r;
      c1 = c1_next;
    }
  }
  if (__any_sync(0xFFFFFFFFu, bad) && lane == 0) atomicOr(&a.ctl->status, kStatusBadCand);
}

template <int WPB, int U>
void launch_u(const CandArgs& a, cudaStream_t st, const char* name) {
  const size_t smem = (size_t)kWarps * warp_smem_words(a.ix.r4, WPB) * sizeof(uint32_t);
  cudaFuncSetAttribute(k_candidates<WPB, U>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_candidates<WPB, U>, kWarps * 32, smem);
  if (per_sm < 1) per_sm = 1;
  // persistent: warps that find no chunk left exit at once
  const uint64_t grid = (uint64_t)sms * per_sm;
  ProfScope ps(name, st);
  k_candidates<WPB, U><<<(unsigned)grid, kWarps * 32, smem, st>>>(a);
}

template <int WPB>
void launch_t(const CandArgs& a, cudaStream_t st, const char* name, uint32_t unroll) {
  if (unroll >= 8) launch_u<WPB, 8>(a, st, name);
  else if (unroll >= 4) launch_u<WPB, 4>(a, st, name);
  else if (unroll >= 2) launch_u<WPB, 2>(a, st, name);
  else launch_u<WPB, 1>(a, st, name);
}

}  // namespace

void launch_candidates(const IndexView& ix, const ReadsView& rv, const int32_t* cand,
                       const uint64_t* cand_off, RecordsView rec, Ctl* ctl, cudaStream_t st,
                       const char* prof_name, Live live, uint32_t unroll, bool check_ids) {
  if (unroll == 0) unroll = kDefaultCandUnroll;
  if (rv.n_reads == 0) return;
  CandArgs a{ix, rv, cand, cand_off, rec, ctl, live, check_ids};
  switch (ix.wpb) {
    case 1: launch_t<1>(a, st, prof_name, unroll); break;
    case 2: launch_t<2>(a, st, prof_name, unroll); break;
    case 8: launch_t<8>(a, st, prof_name, unroll); break;
    case 32: launch_t<32>(a, st, prof_name, unroll); break;
    case 128: launch_t<128>(a, st, prof_name, unroll); break;
    default: break;  // q outside 2..6 is rejected by grim_build
  }
}

}  // namespace grim
