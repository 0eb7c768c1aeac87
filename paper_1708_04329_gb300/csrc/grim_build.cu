// Index build (§GRIM-Filter: the reference is scanned once and every bin's
// bit vector is set from the tokens that occur in it; Fig. 2):
//   k_pack_ref          ASCII -> 2-bit codes + not-a-base mask
//   k_build_bin_major   one warp per bin, bit vector in shared memory
//   k_build_token_major one CTA per 1024-bin tile, the tile's [4^q rows x tile
//                       words] bitmap in shared memory (q <= 4)
//   k_tm_from_bm        q = 5, 6: token-major (and coarse token-major) tiles
//                       as bit transposes of the bin-major vectors, ORed over
//                       the members of each super-bin for the coarse table
#include "grim_internal.cuh"

namespace grim {
namespace {

// A/C/G/T (either case) -> 0/1/2/3; `ok` false for any other byte.
// Clearing bit 5 folds lowercase letters only ('a' 0x61 -> 'A' 0x41); the
// 2-bit code of the folded letter is ((u >> 1) ^ (u >> 2)) & 3 for exactly
// A (0x41), C (0x43), G (0x47) and T (0x54).
__device__ __forceinline__ uint32_t base_code(uint32_t c, bool& ok) {
  uint32_t u = c & 0xDFu;
  ok = (u == 0x41u) | (u == 0x43u) | (u == 0x47u) | (u == 0x54u);
  return ((u >> 1) ^ (u >> 2)) & 3u;
}

// Thread t packs bases [32t, 32t+32): two code words and one mask word.
__global__ void k_pack_ref(const char* __restrict__ ref, uint64_t n, uint32_t* __restrict__ codes,
                           uint32_t* __restrict__ invalid, uint64_t n32) {
  uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (t >= n32) return;
  uint64_t base = t * 32;
  uint8_t b[32];
  if (base + 32 <= n && ((reinterpret_cast<uintptr_t>(ref) & 15u) == 0)) {
    const uint4* p = reinterpret_cast<const uint4*>(ref + base);
    uint4 v0 = __ldg(p), v1 = __ldg(p + 1);
    uint32_t w[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
#pragma unroll
    for (int i = 0; i < 32; ++i) b[i] = (uint8_t)(w[i >> 2] >> (8 * (i & 3)));
  } else {
#pragma unroll
    for (int i = 0; i < 32; ++i) b[i] = (base + i < n) ? (uint8_t)ref[base + i] : (uint8_t)'N';
  }
  uint32_t c0 = 0, c1 = 0, inv = 0;
#pragma unroll
  for (int i = 0; i < 32; ++i) {
    bool ok;
    uint32_t c = base_code(b[i], ok);
    if (!ok) { inv |= 1u << i; c = 0; }
    if (i < 16) c0 |= c << (30 - 2 * i);
    else c1 |= c << (30 - 2 * (i - 16));
  }
  codes[2 * t] = c0;
  codes[2 * t + 1] = c1;
  invalid[t] = inv;
}

// Token starting at reference position p, or -1 if one of its q bases is not
// a base.  Needs p + q <= n (the packed arrays carry one spare word).
__device__ __forceinline__ int32_t token_at(const uint32_t* __restrict__ codes,
                                            const uint32_t* __restrict__ invalid, uint64_t p,
                                            uint32_t q) {
  uint64_t k = p >> 4;
  uint64_t w = ((uint64_t)__ldg(codes + k) << 32) | __ldg(codes + k + 1);
  uint32_t tok = (uint32_t)((w << (2 * (p & 15))) >> (64 - 2 * q));
  uint64_t m = p >> 5;
  uint64_t iw = (uint64_t)__ldg(invalid + m) | ((uint64_t)__ldg(invalid + m + 1) << 32);
  uint32_t bad = (uint32_t)(iw >> (p & 31)) & ((1u << q) - 1u);
  return bad ? -1 : (int32_t)tok;
}

// One warp per bin: set bit t of the bin's vector for every token wholly
// inside window [bB, min(bB+B+ext, n)).
__global__ void k_build_bin_major(const uint32_t* __restrict__ codes,
                                  const uint32_t* __restrict__ invalid, IndexView ix,
                                  uint32_t* __restrict__ bm) {
  extern __shared__ uint32_t s_vec[];  // [warps][wpb]
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint64_t b = blockIdx.x * (uint64_t)(blockDim.x >> 5) + warp;
  uint32_t* v = s_vec + warp * ix.wpb;
  for (uint32_t i = lane; i < ix.wpb; i += 32) v[i] = 0;
  __syncwarp();
  if (b < ix.num_bins) {
    uint64_t lo = b * ix.B;
    uint64_t hi = lo + ix.B + ix.ext;
    if (hi > ix.n) hi = ix.n;
    for (uint64_t p = lo + lane; p + ix.q <= hi; p += 32) {
      int32_t t = token_at(codes, invalid, p, ix.q);
      if (t >= 0) atomicOr(v + (t >> 5), 1u << (t & 31));
    }
  }
  __syncwarp();
  if (b < ix.num_bins)
    for (uint32_t i = lane; i < ix.wpb; i += 32) bm[b * ix.wpb + i] = v[i];
}

// One CTA per tile of tile_words*32 bins: every q-gram start p that lies in a
// window of the tile's bins sets its token's bit in each bin b whose window
// holds it, i.e. b*B <= p and p+q <= b*B+B+ext.
__global__ void __launch_bounds__(512) k_build_token_major(const uint32_t* __restrict__ codes,
                                                           const uint32_t* __restrict__ invalid,
                                                           IndexView ix, uint32_t tile_words,
                                                           uint32_t* __restrict__ tm) {
  extern __shared__ uint32_t s_tile[];  // [r4][tile_words]
  const uint32_t nwords = ix.r4 * tile_words;
  for (uint32_t i = threadIdx.x; i < nwords; i += blockDim.x) s_tile[i] = 0;
  __syncthreads();
  const uint64_t b0 = (uint64_t)blockIdx.x * tile_words * 32;
  uint64_t b1 = b0 + (uint64_t)tile_words * 32;
  if (b1 > ix.num_bins) b1 = ix.num_bins;
  if (b0 < b1) {
    const uint64_t p_lo = b0 * ix.B;
    // last start: p + q <= min(n, (b1-1)*B + B + ext)
    uint64_t end = b1 * ix.B + ix.ext;
    if (end > ix.n) end = ix.n;
    for (uint64_t p = p_lo + threadIdx.x; p + ix.q <= end; p += blockDim.x) {
      int32_t t = token_at(codes, invalid, p, ix.q);
      if (t < 0) continue;
      const uint64_t x = p + ix.q;
      uint64_t lo = x >= (uint64_t)ix.ext + 1 ? (x - ix.ext - 1) / ix.B : 0;
      uint64_t hi = p / ix.B;
      if (lo < b0) lo = b0;
      if (hi > b1 - 1) hi = b1 - 1;
      for (uint64_t b = lo; b <= hi; ++b) {
        uint32_t rel = (uint32_t)(b - b0);
        atomicOr(s_tile + (uint32_t)t * tile_words + (rel >> 5), 1u << (rel & 31));
      }
    }
  }
  __syncthreads();
  const uint64_t w0 = (uint64_t)blockIdx.x * tile_words;
  for (uint32_t i = threadIdx.x; i < nwords; i += blockDim.x) {
    uint32_t t = i / tile_words, w = i % tile_words;
    tm[(uint64_t)t * ix.wpad + w0 + w] = s_tile[i];
  }
}

template <int J>
__device__ __forceinline__ void transpose_round(uint32_t (&x)[32], uint32_t m) {
#pragma unroll
  for (int k = 0; k < 32; ++k) {
    if ((k & J) == 0) {
      const uint32_t t = ((x[k] >> J) ^ x[k + J]) & m;
      x[k + J] ^= t;
      x[k] ^= t << J;
    }
  }
}

// In-register transpose of a 32x32 bit matrix: on entry bit j of x[k] is
// element (k, j); on exit bit k of x[j] is.  Five rounds swap the
// off-diagonal halves of ever smaller diagonal blocks.
__device__ __forceinline__ void transpose32(uint32_t (&x)[32]) {
  transpose_round<16>(x, 0x0000FFFFu);
  transpose_round<8>(x, 0x00FF00FFu);
  transpose_round<4>(x, 0x0F0F0F0Fu);
  transpose_round<2>(x, 0x33333333u);
  transpose_round<1>(x, 0x55555555u);
}

// Token-major tile from the bin-major table (q >= 5, so a bin vector is a
// whole number of 32-word chunks).  One CTA of 32 warps per tile of TW*32
// (super-)bins; warp u takes bin group g = u % TW (32 bins) and token chunk
// c = u / TW (1024 tokens).  Lane l loads word 32c + l of each of the
// group's 32 vectors -- for a super-bin the OR of its f member bins, which
// is exactly the super-bin's vector (its window is the union of theirs) --
// transposes the 32x32 bits in registers, and leaves token rows in shared
// memory (row t at t*TW + (t >> 5): one padding word per 32 rows keeps the
// lanes' stores in distinct banks); the CTA then writes each token row's TW
// words to the token-major table.
template <int TW>
__global__ void __launch_bounds__(1024) k_tm_from_bm(const uint32_t* __restrict__ bm,
                                                     uint32_t wpb, uint32_t f, uint64_t units,
                                                     uint32_t r4, uint64_t wpad,
                                                     uint32_t* __restrict__ tm) {
  extern __shared__ uint32_t s_rows[];
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t g = warp % TW, c = warp / TW;
  const uint64_t u0 = (uint64_t)blockIdx.x * TW * 32 + g * 32;  // first unit of the group
  uint32_t x[32];
#pragma unroll
  for (int k = 0; k < 32; ++k) {
    const uint64_t u = u0 + k;
    uint32_t w = 0;
    if (u < units)
      for (uint32_t m = 0; m < f; ++m) w |= __ldg(bm + (u * f + m) * wpb + c * 32 + lane);
    x[k] = w;
  }
  transpose32(x);  // x[j]: token 32*(32c + lane) + j, bit k = unit u0 + k
#pragma unroll
  for (int j = 0; j < 32; ++j) {
    const uint32_t t = 32u * (32u * c + lane) + j;
    s_rows[t * TW + g + (t >> 5)] = x[j];
  }
  __syncthreads();
  const uint64_t col0 = (uint64_t)blockIdx.x * TW;
  for (uint32_t i = threadIdx.x; i < r4 * TW; i += blockDim.x) {
    const uint32_t t = i / TW, col = i % TW;
    tm[(uint64_t)t * wpad + col0 + col] = s_rows[t * TW + col + (t >> 5)];
  }
}

// One CTA per token row: the number of set bits, i.e. how many (super-)bins
// hold the token.
__global__ void k_row_popcount(const uint32_t* __restrict__ tm, uint64_t words,
                               uint32_t* __restrict__ presence) {
  __shared__ unsigned long long part[32];
  const uint32_t* row = tm + (uint64_t)blockIdx.x * words;
  unsigned long long c = 0;
  for (uint64_t i = threadIdx.x; i < words; i += blockDim.x) c += __popc(__ldg(row + i));
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xFFFFFFFFu, c, o);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x < 32) {
    c = threadIdx.x < blockDim.x / 32 ? part[threadIdx.x] : 0ull;
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xFFFFFFFFu, c, o);
    if (threadIdx.x == 0) presence[blockIdx.x] = (uint32_t)(c > 0xFFFFFFFFull ? 0xFFFFFFFFull : c);
  }
}

}  // namespace

void launch_tm_from_bm(const uint32_t* bm, const IndexView& unit_view, uint32_t wpb, uint32_t f,
                       uint32_t* tm, cudaStream_t st) {
  if (unit_view.num_bins == 0) return;
  const uint32_t r4 = unit_view.r4;
  const uint32_t tw = r4 <= 1024 ? 32u : 32768u / r4;  // tile words, as the filter's tiles
  const size_t smem = ((size_t)r4 * tw + r4 / 32) * sizeof(uint32_t);
  const uint64_t grid = unit_view.num_bins_pad / (tw * 32);
  ProfScope ps("transpose_token_major", st);
  if (tw == 32) {
    cudaFuncSetAttribute(k_tm_from_bm<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_tm_from_bm<32><<<(unsigned)grid, 1024, smem, st>>>(bm, wpb, f, unit_view.num_bins, r4,
                                                         unit_view.wpad, tm);
  } else {
    cudaFuncSetAttribute(k_tm_from_bm<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_tm_from_bm<8><<<(unsigned)grid, 1024, smem, st>>>(bm, wpb, f, unit_view.num_bins, r4,
                                                        unit_view.wpad, tm);
  }
}

void launch_row_popcount(const uint32_t* tm, uint32_t rows, uint64_t words_per_row,
                         uint32_t* presence, cudaStream_t st) {
  ProfScope ps("row_popcount", st);
  k_row_popcount<<<rows, 512, 0, st>>>(tm, words_per_row, presence);
}

void launch_pack_ref(const char* ref, uint64_t n, uint32_t* codes, uint32_t* invalid,
                     cudaStream_t st) {
  uint64_t n32 = (n + 31) / 32;
  if (n32 == 0) return;
  ProfScope ps("pack_ref", st);
  k_pack_ref<<<(unsigned)((n32 + 255) / 256), 256, 0, st>>>(ref, n, codes, invalid, n32);
}

void launch_build_bin_major(const uint32_t* codes, const uint32_t* invalid, const IndexView& ix,
                            uint32_t* bm, cudaStream_t st) {
  if (ix.num_bins == 0) return;
  const uint32_t warps = 8;
  uint64_t grid = (ix.num_bins + warps - 1) / warps;
  ProfScope ps("build_bin_major", st);
  k_build_bin_major<<<(unsigned)grid, warps * 32, warps * ix.wpb * sizeof(uint32_t), st>>>(
      codes, invalid, ix, bm);
}

void launch_build_token_major(const uint32_t* codes, const uint32_t* invalid, const IndexView& ix,
                              uint32_t* tm, cudaStream_t st) {
  if (ix.num_bins == 0) return;
  // 128 KB of shared memory per tile: 32 words (1024 bins) up to q = 5,
  // 8 words (256 bins) at q = 6
  uint32_t tile_words = ix.r4 <= 1024 ? 32u : 32768u / ix.r4;
  size_t smem = (size_t)ix.r4 * tile_words * sizeof(uint32_t);
  cudaFuncSetAttribute(k_build_token_major, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)smem);
  uint64_t grid = (ix.num_bins_pad / 32) / tile_words;
  ProfScope ps("build_token_major", st);
  k_build_token_major<<<(unsigned)grid, 512, smem, st>>>(codes, invalid, ix, tile_words, tm);
}

}  // namespace grim
