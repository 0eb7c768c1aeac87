// Internal definitions shared by the CUDA translation units of libgrim.so.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
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
  unsigned long long blocks;  // 16-token blocks applied to (super-)bin tiles (all-bins mode)
  uint32_t max_d;             // largest miss budget D' = min(q*e, L-q+1) of the batch
  uint32_t max_tight;         // 255 - the smallest slack (L-q+1) - D' of the batch
  // graph launches (grim_plan): the batch's counts and the path taken live
  // on the device, so no launch depends on a host read-back
  uint32_t live_reads;             // reads in this batch
  uint32_t path;                   // kPathCoarse / kPathExact
  unsigned long long live_cand;    // candidates in this batch
  unsigned long long live_bases;   // read bytes in this batch (host-memory plans)
  unsigned long long n_surv;       // survivors of the coarse pass
  unsigned long long n_final;      // passing records of the batch
  uint32_t blk_max;                // most 16-token blocks of a read in the batch
  uint32_t blk_lo;                 // 32 - the fewest 16-token blocks of a read
  unsigned long long tail_blocks;  // of `blocks`: applied to one word per lane (256 bins)
  uint32_t d_lo;                   // 255 - the smallest miss budget D' of the batch
  uint32_t pad[41];
};
static_assert(sizeof(Ctl) == 256, "Ctl is one 256-byte slot");
static_assert(offsetof(Ctl, live_reads) == 32, "live counts follow the per-pass counters");
constexpr uint32_t kPathCoarse = 1u;  // coarse pass, then exact check of the survivors
constexpr uint32_t kPathExact = 2u;   // one exact pass over every bin

// Counts a kernel works on: fixed by the host (grim_filter), or read from
// the control block at run time (graph launches).  `gate`, when nonzero, is
// the path the kernel belongs to: it returns at once unless ctl->path == gate.
struct Live {
  bool on;
  uint32_t gate;
};
// (plain loads: the fields are written by earlier kernels of the stream and
// do not change while the reading kernel runs)
__device__ __forceinline__ uint32_t live_reads(const Ctl* c, const Live& l, uint32_t host_n) {
  return l.on ? c->live_reads : host_n;
}
__device__ __forceinline__ bool gated_off(const Ctl* c, const Live& l) {
  return l.on && l.gate && c->path != l.gate;
}

constexpr uint32_t kStatusShort = 1u;     // read with L < q
constexpr uint32_t kStatusLong = 2u;      // read with L > max_read_len or > 255 tokens
constexpr uint32_t kStatusBadCand = 4u;   // candidate outside [0, num_bins)
constexpr uint32_t kStatusBadCsr = 8u;    // CSR offsets decreasing or not ending at n_cand
constexpr uint32_t kStatusTimeout = 16u;  // bounded wait gave up
constexpr uint32_t kStatusArg = 32u;      // a read's e exceeds the plan's declared maximum
constexpr uint32_t kStatusSurv = 64u;     // coarse survivors exceed their capacity (no exact table)

// Token buffer entries are table row indices: a token value t < 4^q, or
// rowInvalid(q) for a q-gram with a non-base (adds a miss: the zero row), or
// rowPad(q) past the read's last token (adds nothing: the all-ones row).
__host__ __device__ inline uint32_t rowInvalid(uint32_t r4) { return r4; }
__host__ __device__ inline uint32_t rowPad(uint32_t r4) { return r4 + 1; }

struct IndexView {
  uint64_t n, num_bins, num_bins_pad, wpad;  // wpad = num_bins_pad / 32 words per row
  uint64_t bm_rows;  // rows of the bin-major table: num_bins padded to whole super-bins
  uint32_t B, q, ext, max_read_len, r4, wpb;
  const uint32_t* tm;  // token-major [r4][wpad]
  const uint32_t* bm;  // bin-major [num_bins][wpb]
  // [r4] number of (super-)bins holding each token, or null; the tokeniser
  // orders each read's tokens by it so that the all-bins kernels apply the
  // rarest tokens first and every bin of a tile fails as early as possible
  const uint32_t* presence;
};

// Reads after tokenising: token j of read r (copy k) at
// tokens[(r * copies + k) * ts + j], meta[r] = ntok | D' << 8 where
// D' = min(q*e, ntok) is the number of misses a passing bin may have.
struct ReadsView {
  const uint16_t* tokens;  // read r, copy k: tokens + (r * copies + k) * ts
  const uint32_t* meta;
  uint32_t n_reads, ts;
  uint32_t copies;  // 1, or 4 block-rotated copies for the 256-bin tiles (q = 6)
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
// Token-major table of `unit_view` (bins, or super-bins of f bins) from the
// bin-major table bm [units * f][wpb]; q >= 5
void launch_tm_from_bm(const uint32_t* bm, const IndexView& unit_view, uint32_t wpb, uint32_t f,
                       uint32_t* tm, cudaStream_t st);
// presence[t] = popcount of row t of a token-major table
void launch_row_popcount(const uint32_t* tm, uint32_t rows, uint64_t words_per_row,
                         uint32_t* presence, cudaStream_t st);

void launch_reverse_complement(const char* reads, const uint64_t* offsets, const uint32_t* lens,
                               uint32_t n_reads, char* out, cudaStream_t st);
// max_e: reads with a larger budget are an argument error (graph launches
// fix the counter depth from it); 0xFFFF = no limit.  max_bases: size of the
// reads buffer when known (a read ending past it fails the batch with
// kStatusArg), else ~0.  rv.copies token copies per read are written.
void launch_tokenise(const char* reads, const uint64_t* offsets, const uint32_t* lens,
                     const uint16_t* e, const IndexView& ix, ReadsView rv, uint16_t* tokens,
                     uint32_t* meta, Ctl* ctl, cudaStream_t st, Live live = {false, 0},
                     uint32_t max_e = 0xFFFFu, uint64_t max_bases = ~0ull);
// ctl->blk_max / blk_lo: the most 16-token blocks of a read of the batch, and
// 32 - the fewest
void launch_block_spread(const uint32_t* lens, uint32_t n_reads, uint32_t q, Ctl* ctl,
                         cudaStream_t st);
// CSR offsets of the caller's lists: non-decreasing, ending at n_cand
// (kStatusBadCsr otherwise); the ids themselves are checked by the
// candidate kernel
void launch_check_candidates(const uint64_t* cand_off, uint32_t n_reads, uint64_t n_cand, Ctl* ctl,
                             cudaStream_t st, Live live = {false, 0});

// bins per tile of the all-bins kernel for a table of r4 = 4^q rows
uint32_t exhaustive_tile_bins(uint32_t r4);
// Launch shape of the all-bins kernel (0 = the default): CTA threads (512,
// 640 or 768; one persistent CTA per SM), the token-row bytes of one read
// range in KiB (reads are swept range by range so a range's token rows stay
// in L2 while the CTAs sweep their tiles), and how the lane groups of a warp
// take their next reads (GRIM_SWITCH_GROUP: each group as its read ends;
// GRIM_SWITCH_WARP: all groups of the warp together; 0 at launch = GROUP).
// `path` (GRIM_PATH_*) is the index's all-bins path: coarse-then-exact or
// one exact pass (0 = chosen per index, see all_bins_path).
struct ExhShape {
  uint32_t threads;
  uint32_t range_kb;
  uint32_t read_switch;
  uint32_t path;
};
// the launch shape's threads, range and read switch are ones the kernel builds
bool exhaustive_shape_ok(const ExhShape& s);
// max_d: the batch's largest miss budget (sizes the bit-sliced counters)
void launch_exhaustive(const IndexView& ix, const ReadsView& rv, RecordsView rec, uint32_t bin_bits,
                       uint32_t max_d, Ctl* ctl, cudaStream_t st,
                       const char* prof_name = "exhaustive", Live live = {false, 0},
                       ExhShape shape = {0, 0, 0, 0});
// unroll: candidate gathers in flight per lane group (1, 2, 4 or 8; 0 =
// default).  check_ids: the lists are the caller's; an id outside
// [0, num_bins) sets kStatusBadCand (and is not gathered).  Internal lists
// (survivor members) may hold zero-padding bins past num_bins: they are
// gathered and never pass.
void launch_candidates(const IndexView& ix, const ReadsView& rv, const int32_t* cand,
                       const uint64_t* cand_off, RecordsView rec, Ctl* ctl, cudaStream_t st,
                       const char* prof_name = "candidates", Live live = {false, 0},
                       uint32_t unroll = 0, bool check_ids = false);

// Radix sort of n (key, count) records by the low key_bits bits of the key,
// followed by the split into the caller's (read, bin, count) arrays.
uint64_t sort_workspace_bytes(uint64_t cap);
// n_live (nullable): the record count is read on the device from *n_live,
// capped at n; n then only sizes the launches
RecordsView sort_records(RecordsView a, RecordsView b, uint64_t n, uint32_t key_bits, void* hist,
                         cudaStream_t st, const unsigned long long* n_live = nullptr,
                         const Ctl* gate_ctl = nullptr, uint32_t gate = 0);
void expand_survivors(const unsigned long long* keys, uint64_t n_surv, uint32_t cbits, uint32_t f,
                      uint32_t n_reads, int32_t* cand, uint64_t* cand_off, cudaStream_t st,
                      const Ctl* live_ctl = nullptr, uint32_t gate = 0);
void sort_and_emit(RecordsView a, RecordsView b, uint64_t n, uint32_t key_bits, void* hist,
                   bool candidate_mode, uint32_t bin_bits, const int32_t* cand,
                   const uint64_t* cand_off, uint32_t n_reads, uint32_t* out_read,
                   uint32_t* out_bin, uint8_t* out_count, cudaStream_t st,
                   const unsigned long long* n_live = nullptr, const uint32_t* n_reads_live = nullptr,
                   const Ctl* gate_ctl = nullptr, uint32_t gate = 0);

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
void prof_suspend(bool on);  // no event timing while a graph is being captured

inline uint32_t bit_length(uint64_t v) {
  uint32_t b = 0;
  while (v) { ++b; v >>= 1; }
  return b;
}

// ---------------------------------------------------------------------------
// the index and the filter workspace (shared by grim_api.cu and grim_plan.cu)
// ---------------------------------------------------------------------------
inline uint64_t align256(uint64_t x) { return (x + 255) & ~255ull; }

// token stride: the longest read's token count rounded up to a 16-token block
inline uint32_t token_stride(const IndexView& v) {
  const uint32_t nt = v.max_read_len - v.q + 1;
  return (nt + kBlockTokens - 1) / kBlockTokens * kBlockTokens;
}

struct Layout {
  uint64_t tok, meta, keys_a, keys_b, cnt_a, cnt_b, hist, cand, cand_off, total;
};

// Survivors of the coarse pass get their own capacity: reads from repeat
// families survive in many super-bins that then fail the exact check.  On
// the 3.1 Gbp synthetic genome: 27 a read for 100 bp reads with e = 5 and
// ext = 99; against an index with ext = 249, 132 for the serving mix of
// 100-250 bp reads and 263 for 100 bp reads with e uniform in 0..5.  A call
// whose survivors do not fit takes the exact pass.
constexpr uint64_t kSurvivorsPerRead = 320;

inline uint64_t record_capacity(uint32_t n_reads, uint64_t cap, uint32_t coarse_factor) {
  const uint64_t s = coarse_factor ? kSurvivorsPerRead * n_reads : 0;
  return s > cap ? s : cap;
}

// coarse_factor > 0: room for the coarse pass's survivors and for the
// candidate lists they expand into (coarse_factor per survivor)
// Token copies per read: the all-bins kernel's 256-bin tiles (q = 6) read
// one of 4 block-rotated copies per lane group (see k_tokenise).
inline uint32_t token_copies(const IndexView& v, bool cand_mode) {
  return !cand_mode && v.r4 > 1024 ? 4u : 1u;
}

inline Layout layout(const IndexView& v, uint32_t n_reads, uint64_t cap, uint32_t coarse_factor,
                     uint32_t copies) {
  Layout L{};
  const uint64_t rcap = record_capacity(n_reads, cap, coarse_factor);
  uint64_t o = sizeof(Ctl);
  L.tok = o;
  o = align256(o + (uint64_t)n_reads * copies * token_stride(v) * sizeof(uint16_t));
  L.meta = o;
  o = align256(o + (uint64_t)n_reads * sizeof(uint32_t));
  L.keys_a = o;
  o = align256(o + rcap * sizeof(unsigned long long));
  L.keys_b = o;
  o = align256(o + rcap * sizeof(unsigned long long));
  L.cnt_a = o;
  o = align256(o + rcap);
  L.cnt_b = o;
  o = align256(o + rcap);
  L.hist = o;
  o = align256(o + sort_workspace_bytes(rcap));
  L.cand = o;
  o = align256(o + (coarse_factor ? rcap * coarse_factor * sizeof(int32_t) : 0));
  L.cand_off = o;
  o = align256(o + (coarse_factor ? ((uint64_t)n_reads + 1) * sizeof(uint64_t) : 0));
  L.total = o;
  return L;
}

inline int status_to_code(uint32_t s) {
  if (s & kStatusShort) return GRIM_E_READ_TOO_SHORT;
  if (s & kStatusLong) return GRIM_E_READ_TOO_LONG;
  if ((s & kStatusBadCsr) || (s & kStatusArg)) return GRIM_E_ARG;
  if (s & kStatusBadCand) return GRIM_E_BAD_CANDIDATE;
  if (s & kStatusTimeout) return GRIM_E_TIMEOUT;
  return GRIM_OK;
}

}  // namespace grim

struct grim_index {
  grim::IndexView v;   // bins: token-major and bin-major tables
  grim::IndexView cv;  // super-bins of `factor` bins: coarse token-major table
  uint32_t factor;
  uint32_t layouts;
  grim::ExhShape shape;  // launch shape of the all-bins kernel (grim_index_set_shape)
  // the coarse table is sparse enough for the coarse pass to pay: its
  // super-bin window would hold at most 40% of the 4^q tokens in a uniform
  // random sequence (the rule that picks the default coarse factor)
  bool coarse_pays;
  uint32_t* tm;
  uint32_t* bm;
  uint32_t* ctm;
  uint32_t* presence;
  // the allocator the tables came from (grim_set_allocator), or null for
  // cudaMalloc / cudaFree
  grim_free_fn free_fn;
  void* alloc_ctx;
};

namespace grim {
// Validate an index's parameters and allocate its (unwritten) tables; the
// views of the returned index point at them.  GRIM_* status.
int index_alloc(uint64_t len, uint32_t B, uint32_t q, uint32_t max_read_len, uint32_t layouts,
                uint32_t f, grim_index** out);
// Keep the CUDA error string for grim_last_cuda_error; the matching status.
int record_cuda_error(cudaError_t e);

// the all-bins filter can run coarse-then-exact when the index has both the
// coarse table and the bin-major table
inline bool two_level_capable(const grim_index* idx) {
  return (idx->layouts & GRIM_LAYOUT_COARSE) && (idx->layouts & GRIM_LAYOUT_BIN_MAJOR);
}

// The all-bins path of an index's calls before the per-batch rules (a
// batch with less than 24 tokens of slack takes the exact pass, and so do
// coarse survivors that overflow their room): kPathCoarse or kPathExact.
// *forced: the index leaves no choice, or the caller fixed the path
// (GRIM_PATH_*), so the slack rule does not apply.
inline uint32_t all_bins_path(const grim_index* idx, bool* forced) {
  *forced = true;
  if (!two_level_capable(idx)) return kPathExact;
  if (!(idx->layouts & GRIM_LAYOUT_TOKEN_MAJOR)) return kPathCoarse;
  if (idx->shape.path == GRIM_PATH_EXACT) return kPathExact;
  if (idx->shape.path == GRIM_PATH_TWO_LEVEL) return kPathCoarse;
  *forced = false;
  return idx->coarse_pays ? kPathCoarse : kPathExact;
}
}  // namespace grim
