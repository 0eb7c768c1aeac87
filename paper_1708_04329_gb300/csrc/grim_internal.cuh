// Internal definitions shared by the CUDA translation units of libgrim.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "grim.h"

namespace grim {

// ---------------------------------------------------------------------------
// Packed reference: base i is 2 bits at [30-2(i%16), 31-2(i%16)] of word i/16
// (first base in the top bits, so a q-gram is one funnel shift); the
// not-a-base mask has bit i%32 of word i/32 set for a non-ACGT byte.
// ---------------------------------------------------------------------------
constexpr uint32_t kTileWords = 32;      // token-major tile: 32 words = 1024 bins
constexpr uint32_t kTileBins = kTileWords * 32;
constexpr uint32_t kBlockTokens = 16;    // tokens per carry-save block
constexpr uint32_t kMaxTokens = 255;     // counts are uint8

// Device control block at the start of the filter workspace.
struct Ctl {
  unsigned long long n_rec;   // passing records found (may exceed cap)
  uint32_t status;            // kStatus* bits
  uint32_t item;              // work-item counter of the persistent filter kernels
  unsigned long long blocks;  // 16-token blocks applied to 1024-bin tiles (all-bins mode)
  uint32_t max_d;             // largest miss budget D' = min(q*e, L-q+1) of the batch
  uint32_t max_tight;         // 255 - the smallest slack (L-q+1) - D' of the batch
  uint32_t pad[56];
};
static_assert(sizeof(Ctl) == 256, "Ctl is one 256-byte slot");

constexpr uint32_t kStatusShort = 1u;     // read with L < q
constexpr uint32_t kStatusLong = 2u;      // read with L > max_read_len or > 255 tokens
constexpr uint32_t kStatusBadCand = 4u;   // candidate outside [0, num_bins)
constexpr uint32_t kStatusBadCsr = 8u;    // CSR offsets decreasing or not ending at n_cand
constexpr uint32_t kStatusTimeout = 16u;  // bounded wait gave up

// Token buffer entries are table row indices: a token value t < 4^q, or
// rowInvalid(q) for a q-gram with a non-base (adds a miss: the zero row), or
// rowPad(q) past the read's last token (adds nothing: the all-ones row).
__host__ __device__ inline uint32_t rowInvalid(uint32_t r4) { return r4; }
__host__ __device__ inline uint32_t rowPad(uint32_t r4) { return r4 + 1; }

struct IndexView {
  uint64_t n, num_bins, num_bins_pad, wpad;  // wpad = num_bins_pad / 32 words per row
  uint32_t B, q, ext, max_read_len, r4, wpb;
  const uint32_t* tm;  // token-major [r4][wpad]
  const uint32_t* bm;  // bin-major [num_bins][wpb]
  // [r4] number of (super-)bins holding each token, or null; the tokeniser
  // orders each read's tokens by it so that the all-bins kernels apply the
  // rarest tokens first and every bin of a tile fails as early as possible
  const uint32_t* presence;
};

// Reads after tokenising: tokens[r * ts + j], meta[r] = ntok | D' << 8 where
// D' = min(q*e, ntok) is the number of misses a passing bin may have.
struct ReadsView {
  const uint16_t* tokens;
  const uint32_t* meta;
  uint32_t n_reads, ts;
};

struct RecordsView {
  unsigned long long* keys;  // sort keys of passing records
  uint8_t* counts;           // their sums
  uint64_t cap;
};

// ---------------------------------------------------------------------------
// launchers (each enqueues on `st`; errors surface through cudaGetLastError)
// ---------------------------------------------------------------------------
void launch_pack_ref(const char* ref, uint64_t n, uint32_t* codes, uint32_t* invalid,
                     cudaStream_t st);
void launch_build_bin_major(const uint32_t* codes, const uint32_t* invalid, const IndexView& ix,
                            uint32_t* bm, cudaStream_t st);
void launch_build_token_major(const uint32_t* codes, const uint32_t* invalid, const IndexView& ix,
                              uint32_t* tm, cudaStream_t st);
// presence[t] = popcount of row t of a token-major table
void launch_row_popcount(const uint32_t* tm, uint32_t rows, uint64_t words_per_row,
                         uint32_t* presence, cudaStream_t st);

void launch_tokenise(const char* reads, const uint64_t* offsets, const uint32_t* lens,
                     const uint16_t* e, const IndexView& ix, ReadsView rv, uint16_t* tokens,
                     uint32_t* meta, Ctl* ctl, cudaStream_t st);
void launch_check_candidates(const int32_t* cand, const uint64_t* cand_off, uint32_t n_reads,
                             uint64_t n_cand, uint64_t num_bins, Ctl* ctl, cudaStream_t st);

// bins per tile of the all-bins kernel for a table of r4 = 4^q rows
uint32_t exhaustive_tile_bins(uint32_t r4);
// max_d: the batch's largest miss budget (sizes the bit-sliced counters)
void launch_exhaustive(const IndexView& ix, const ReadsView& rv, RecordsView rec, uint32_t bin_bits,
                       uint32_t max_d, Ctl* ctl, cudaStream_t st,
                       const char* prof_name = "exhaustive");
void launch_candidates(const IndexView& ix, const ReadsView& rv, const int32_t* cand,
                       const uint64_t* cand_off, RecordsView rec, Ctl* ctl, cudaStream_t st,
                       const char* prof_name = "candidates");

// Radix sort of n (key, count) records by the low key_bits bits of the key,
// followed by the split into the caller's (read, bin, count) arrays.
uint64_t sort_workspace_bytes(uint64_t cap);
RecordsView sort_records(RecordsView a, RecordsView b, uint64_t n, uint32_t key_bits, void* hist,
                         cudaStream_t st);  // returns whichever of a, b holds the sorted keys
void expand_survivors(const unsigned long long* keys, uint64_t n_surv, uint32_t cbits, uint32_t f,
                      uint32_t n_reads, int32_t* cand, uint64_t* cand_off, cudaStream_t st);
void sort_and_emit(RecordsView a, RecordsView b, uint64_t n, uint32_t key_bits, void* hist,
                   bool candidate_mode, uint32_t bin_bits, const int32_t* cand,
                   const uint64_t* cand_off, uint32_t n_reads, uint32_t* out_read,
                   uint32_t* out_bin, uint8_t* out_count, cudaStream_t st);

// ---------------------------------------------------------------------------
// per-kernel timing (grim_profile): wraps one launch in events on `st`
// ---------------------------------------------------------------------------
struct ProfScope {
  ProfScope(const char* name, cudaStream_t st);
  ~ProfScope();
  int slot;
  cudaStream_t st;
};
void prof_collect();  // resolve finished events into the totals (after a sync)

inline uint32_t bit_length(uint64_t v) {
  uint32_t b = 0;
  while (v) { ++b; v >>= 1; }
  return b;
}

}  // namespace grim
