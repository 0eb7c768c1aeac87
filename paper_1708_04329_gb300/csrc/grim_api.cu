// C-ABI of libgrim.so (include/grim.h): argument checks, index ownership,
// workspace layout, the order of kernel launches, status reporting and the
// optional per-kernel event timing.
#include <math.h>
#include <mutex>
#include <stddef.h>
#include <string.h>
#include <string>
#include <vector>

#include "grim_internal.cuh"

namespace grim {
namespace {

thread_local std::string g_cuda_err;
thread_local grim_filter_stats g_last_stats{};

int cuda_fail(cudaError_t e) {
  g_cuda_err = cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? GRIM_E_NOMEM : GRIM_E_CUDA;
}

#define CK(call)                                 \
  do {                                           \
    cudaError_t e_ = (call);                     \
    if (e_ != cudaSuccess) return cuda_fail(e_); \
  } while (0)

// Default bins per super-bin: the largest power of two (2..64) whose
// super-bin window of f*B + ext bases would hold at most 50% of the 4^q
// tokens if the sequence were uniform random (1 - exp(-q-grams / 4^q)); a
// denser coarse table lets too many super-bins pass.  q = 5, B = 200,
// ext = 99 or 249 gives 2 (38% and 47%); q = 6, B = 100, ext = 149 gives 16.
// The same bound decides whether the coarse pass is taken automatically:
// measured on GB300, f = 2 with ext = 249 (47%) beat one exact pass by 39%
// on 100-250 bp reads once its survivors had room, and f = 4 with ext = 99
// (58%) lost to f = 2 by 2.4x.
// Fraction of the 4^q tokens a super-bin window of f bins (f*B + ext bases)
// would hold in a uniform random sequence.
double coarse_density(uint32_t B, uint32_t q, uint32_t ext, uint32_t f) {
  const double tokens = (double)(1u << (2 * q));
  const double grams = (double)f * B + ext - q + 1;
  return 1.0 - exp(-grams / tokens);
}
constexpr double kCoarseDensityMax = 0.50;

uint32_t default_coarse_factor(uint32_t B, uint32_t q, uint32_t ext) {
  uint32_t best = 2;
  for (uint32_t f = 2; f <= 64; f *= 2)
    if (coarse_density(B, q, ext, f) <= kCoarseDensityMax) best = f;
  return best;
}

// A launch shape the index can run: an explicit path needs its tables.
int shape_fits(const grim_index* idx, const ExhShape& s) {
  if (!exhaustive_shape_ok(s) || s.path > GRIM_PATH_EXACT) return GRIM_E_ARG;
  if (s.path == GRIM_PATH_EXACT && !(idx->layouts & GRIM_LAYOUT_TOKEN_MAJOR))
    return GRIM_E_NO_LAYOUT;
  if (s.path == GRIM_PATH_TWO_LEVEL && !two_level_capable(idx)) return GRIM_E_NO_LAYOUT;
  return GRIM_OK;
}

// ---------------------------------------------------------------------------
// per-kernel timing
// ---------------------------------------------------------------------------
struct ProfEntry {
  std::string name;
  uint64_t launches = 0;
  double ms = 0.0;
};
struct Pending {
  int slot;
  cudaEvent_t a, b;
};
std::mutex g_prof_mu;
bool g_prof_on = false;
thread_local bool g_prof_suspended = false;
std::vector<ProfEntry> g_prof;
std::vector<Pending> g_pending;
std::vector<cudaEvent_t> g_event_pool;

cudaEvent_t take_event() {
  if (!g_event_pool.empty()) {
    cudaEvent_t e = g_event_pool.back();
    g_event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

}  // namespace

// The caller's device allocator for index tables (grim_set_allocator).
std::mutex g_alloc_mu;
grim_alloc_fn g_alloc = nullptr;
grim_free_fn g_free = nullptr;
void* g_alloc_ctx = nullptr;

// Validate an index's parameters and allocate its tables (contents not yet
// written): token-major [4^q][num_bins_pad/32], bin-major padded with zero
// vectors to whole super-bins, coarse token-major over super-bins of f bins,
// and the per-token presence counts.
int index_alloc(uint64_t len, uint32_t B, uint32_t q, uint32_t max_read_len, uint32_t layouts,
                uint32_t f, grim_index** out) {
  *out = nullptr;
  if (f == 0 || f > 64) return GRIM_E_ARG;
  if (len == 0 || B == 0 || max_read_len < q || layouts == 0 || (layouts & ~GRIM_LAYOUT_ALL))
    return GRIM_E_ARG;
  if (q < 2 || q > 6 || max_read_len - q + 1 > kMaxTokens) return GRIM_E_UNSUPPORTED;
  IndexView v{};
  v.n = len;
  v.B = B;
  v.q = q;
  v.ext = max_read_len - 1;
  v.max_read_len = max_read_len;
  v.r4 = 1u << (2 * q);
  v.wpb = v.r4 >= 32 ? v.r4 / 32 : 1;
  v.num_bins = (len + B - 1) / B;
  v.num_bins_pad = (v.num_bins + kTileBins - 1) / kTileBins * kTileBins;
  v.wpad = v.num_bins_pad / 32;
  if (v.num_bins > 0xFFFFFFFFull) return GRIM_E_UNSUPPORTED;  // bins are uint32 in the output
  // super-bins: core f*B, the same extension (window = union of f bins' windows)
  IndexView cv = v;
  cv.B = v.B * f;
  cv.num_bins = (len + cv.B - 1) / cv.B;
  cv.num_bins_pad = (cv.num_bins + kTileBins - 1) / kTileBins * kTileBins;
  cv.wpad = cv.num_bins_pad / 32;
  // bin-major vectors padded with zero vectors to whole super-bins
  const uint64_t bm_bins = cv.num_bins * f;

  grim_index* ix = new (std::nothrow) grim_index{};
  if (!ix) return GRIM_E_NOMEM;
  ix->layouts = layouts;
  ix->factor = f;
  grim_alloc_fn alloc_fn;
  {
    std::lock_guard<std::mutex> g(g_alloc_mu);
    alloc_fn = g_alloc;
    ix->free_fn = g_free;
    ix->alloc_ctx = g_alloc_ctx;
  }
  auto fail = [&](cudaError_t e) {
    grim_free(ix);
    return cuda_fail(e);
  };
  auto table = [&](uint32_t** p, uint64_t bytes) -> cudaError_t {
    if (!alloc_fn) return cudaMalloc(p, bytes);
    *p = static_cast<uint32_t*>(alloc_fn(bytes, ix->alloc_ctx));
    return *p ? cudaSuccess : cudaErrorMemoryAllocation;
  };
  cudaError_t e;
  if (layouts & GRIM_LAYOUT_TOKEN_MAJOR) {
    e = table(&ix->tm, (uint64_t)v.r4 * v.wpad * sizeof(uint32_t));
    if (e != cudaSuccess) return fail(e);
  }
  if (layouts & GRIM_LAYOUT_BIN_MAJOR) {
    e = table(&ix->bm, bm_bins * v.wpb * sizeof(uint32_t));
    if (e != cudaSuccess) return fail(e);
  }
  if (layouts & GRIM_LAYOUT_COARSE) {
    e = table(&ix->ctm, (uint64_t)cv.r4 * cv.wpad * sizeof(uint32_t));
    if (e != cudaSuccess) return fail(e);
  }
  if (layouts & (GRIM_LAYOUT_COARSE | GRIM_LAYOUT_TOKEN_MAJOR)) {
    e = table(&ix->presence, (uint64_t)v.r4 * sizeof(uint32_t));
    if (e != cudaSuccess) return fail(e);
  }
  ix->coarse_pays = coarse_density(B, q, v.ext, f) <= kCoarseDensityMax;
  v.tm = ix->tm;
  v.bm = ix->bm;
  v.bm_rows = bm_bins;
  v.presence = ix->presence;
  ix->v = v;
  cv.tm = ix->ctm;
  cv.bm = nullptr;
  cv.presence = ix->presence;
  ix->cv = cv;
  *out = ix;
  return GRIM_OK;
}

int record_cuda_error(cudaError_t e) { return cuda_fail(e); }

// A library-owned stream-ordered pool per device for the scratch of the
// build and of the host-buffer entry points (packed reference, device copies
// of host inputs, workspaces).  Its release threshold keeps freed memory
// cached, so repeated calls do not map and unmap gigabytes each time, and it
// leaves the process's default pool and its settings alone.
cudaMemPool_t scratch_pool() {
  static std::mutex mu;
  static cudaMemPool_t pools[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> g(mu);
  if (!pools[dev]) {
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t p = nullptr;
    if (cudaMemPoolCreate(&p, &props) != cudaSuccess) return nullptr;
    uint64_t keep = ~0ull;
    cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
    pools[dev] = p;
  }
  return pools[dev];
}

cudaError_t scratch_alloc(void** p, size_t bytes, cudaStream_t st) {
  cudaMemPool_t pool = scratch_pool();
  if (!pool) return cudaMallocAsync(p, bytes, st);
  return cudaMallocFromPoolAsync(p, bytes, pool, st);
}


void prof_suspend(bool on) { g_prof_suspended = on; }

ProfScope::ProfScope(const char* name, cudaStream_t s) : slot(-1), st(s) {
  if (g_prof_suspended) return;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (!g_prof_on) return;
  int idx = -1;
  for (size_t i = 0; i < g_prof.size(); ++i)
    if (g_prof[i].name == name) idx = (int)i;
  if (idx < 0) {
    g_prof.push_back(ProfEntry{name});
    idx = (int)g_prof.size() - 1;
  }
  Pending p{idx, take_event(), take_event()};
  cudaEventRecord(p.a, st);
  g_pending.push_back(p);
  slot = (int)g_pending.size() - 1;
}

ProfScope::~ProfScope() {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (slot < 0 || slot >= (int)g_pending.size()) return;
  cudaEventRecord(g_pending[slot].b, st);
}

void prof_collect() {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  for (const Pending& p : g_pending) {
    float ms = 0.f;
    if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess &&
        p.slot < (int)g_prof.size()) {
      g_prof[p.slot].launches += 1;
      g_prof[p.slot].ms += ms;
    }
    g_event_pool.push_back(p.a);
    g_event_pool.push_back(p.b);
  }
  g_pending.clear();
}

}  // namespace grim

using namespace grim;

extern "C" {

const char* grim_strerror(int s) {
  switch (s) {
    case GRIM_OK: return "ok";
    case GRIM_E_ARG: return "bad argument";
    case GRIM_E_NOMEM: return "out of memory";
    case GRIM_E_CUDA: return "CUDA error";
    case GRIM_E_READ_TOO_SHORT: return "read shorter than q";
    case GRIM_E_READ_TOO_LONG: return "read longer than max_read_len or more than 255 tokens";
    case GRIM_E_BAD_CANDIDATE: return "candidate bin out of range";
    case GRIM_E_OVERFLOW: return "more passing records than the output capacity";
    case GRIM_E_TIMEOUT: return "bounded device wait gave up";
    case GRIM_E_WORKSPACE: return "workspace too small";
    case GRIM_E_NO_LAYOUT: return "index lacks the table layout this call needs";
    case GRIM_E_UNSUPPORTED: return "parameter outside what this build implements";
    case GRIM_E_NOT_READY: return "not finished yet";
    case GRIM_E_BUSY: return "the server's queue is full";
    case GRIM_E_IO: return "file could not be opened, read or written";
    case GRIM_E_FORMAT: return "not an index file of this library, or damaged";
    case GRIM_E_CANCELLED: return "request cancelled before it ran";
    default: return "unknown status";
  }
}

const char* grim_last_cuda_error(void) { return g_cuda_err.c_str(); }

int grim_set_allocator(grim_alloc_fn alloc, grim_free_fn free_fn, void* ctx) {
  if ((alloc == nullptr) != (free_fn == nullptr)) return GRIM_E_ARG;
  std::lock_guard<std::mutex> g(g_alloc_mu);
  g_alloc = alloc;
  g_free = free_fn;
  g_alloc_ctx = alloc ? ctx : nullptr;
  return GRIM_OK;
}

int grim_trim_scratch(void) {
  cudaMemPool_t pool = scratch_pool();
  if (!pool) return GRIM_OK;
  const cudaError_t e = cudaMemPoolTrimTo(pool, 0);
  return e == cudaSuccess ? GRIM_OK : cuda_fail(e);
}

int grim_build(const char* ref, uint64_t len, uint32_t B, uint32_t q, uint32_t max_read_len,
               uint32_t layouts, void* stream, grim_index** out) {
  return grim_build_ex(ref, len, B, q, max_read_len, layouts, nullptr, stream, out);
}

uint32_t grim_default_coarse_factor(uint32_t B, uint32_t q, uint32_t max_read_len) {
  if (B == 0 || q < 2 || q > 6 || max_read_len < q) return 0;
  return default_coarse_factor(B, q, max_read_len - 1);
}

int grim_build_ex(const char* ref, uint64_t len, uint32_t B, uint32_t q, uint32_t max_read_len,
                  uint32_t layouts, const grim_build_opts* opts, void* stream, grim_index** out) {
  if (!out) return GRIM_E_ARG;
  *out = nullptr;
  if (!ref || B == 0 || max_read_len < q) return GRIM_E_ARG;
  const ExhShape shape = opts ? ExhShape{opts->cta_threads, opts->read_range_kb, opts->read_switch,
                                          opts->all_bins_path}
                              : ExhShape{0, 0, 0, 0};
  if (!exhaustive_shape_ok(shape) || shape.path > GRIM_PATH_EXACT) return GRIM_E_ARG;
  const uint32_t f = (opts && opts->coarse_factor) ? opts->coarse_factor
                     : (q >= 2 && q <= 6)              ? default_coarse_factor(B, q, max_read_len - 1)
                                                       : 2u;  // q is refused by index_alloc
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  grim_index* ix = nullptr;
  const int rc = index_alloc(len, B, q, max_read_len, layouts, f, &ix);
  if (rc != GRIM_OK) return rc;
  {
    const int fit = shape_fits(ix, shape);
    if (fit != GRIM_OK) {
      grim_free(ix);
      return fit;
    }
    ix->shape = shape;
  }
  const IndexView& v = ix->v;
  const IndexView& cv = ix->cv;
  const uint64_t bm_bins = cv.num_bins * f;
  auto fail = [&](int code) {
    grim_free(ix);
    return code;
  };
  cudaError_t e;
  // packed reference (one spare word at the end of each array for the
  // two-word reads of the token extraction)
  const uint64_t n32 = (len + 31) / 32;
  uint32_t *codes = nullptr, *invalid = nullptr;
  e = scratch_alloc(reinterpret_cast<void**>(&codes), (2 * n32 + 2) * sizeof(uint32_t), st);
  if (e != cudaSuccess) return fail(cuda_fail(e));
  e = scratch_alloc(reinterpret_cast<void**>(&invalid), (n32 + 2) * sizeof(uint32_t), st);
  if (e != cudaSuccess) {
    cudaFreeAsync(codes, st);
    return fail(cuda_fail(e));
  }
  cudaMemsetAsync(codes + 2 * n32, 0, 2 * sizeof(uint32_t), st);
  cudaMemsetAsync(invalid + n32, 0xFF, 2 * sizeof(uint32_t), st);
  launch_pack_ref(ref, len, codes, invalid, st);
  // q >= 5: the token-major tables are bit transposes of the bin-major one
  // (a scratch copy when the index keeps no bin-major table)
  const bool transpose = v.q >= 5 && (ix->tm || ix->ctm);
  uint32_t* bm = ix->bm;
  if (!bm && transpose) {
    e = scratch_alloc(reinterpret_cast<void**>(&bm), bm_bins * v.wpb * sizeof(uint32_t), st);
    if (e != cudaSuccess) {
      cudaFreeAsync(codes, st);
      cudaFreeAsync(invalid, st);
      return fail(cuda_fail(e));
    }
  }
  if (bm) {
    if (bm_bins > v.num_bins)
      cudaMemsetAsync(bm + v.num_bins * v.wpb, 0, (bm_bins - v.num_bins) * v.wpb * sizeof(uint32_t),
                      st);
    launch_build_bin_major(codes, invalid, v, bm, st);
  }
  if (transpose) {
    if (ix->tm) launch_tm_from_bm(bm, v, v.wpb, 1, ix->tm, st);
    if (ix->ctm) launch_tm_from_bm(bm, cv, v.wpb, f, ix->ctm, st);
  } else {
    if (ix->tm) launch_build_token_major(codes, invalid, v, ix->tm, st);
    if (ix->ctm) launch_build_token_major(codes, invalid, cv, ix->ctm, st);
  }
  if (bm != ix->bm) cudaFreeAsync(bm, st);
  // token presence from the table the all-bins filter sweeps first
  if (ix->ctm) launch_row_popcount(ix->ctm, cv.r4, cv.wpad, ix->presence, st);
  else if (ix->tm) launch_row_popcount(ix->tm, v.r4, v.wpad, ix->presence, st);
  cudaFreeAsync(codes, st);
  cudaFreeAsync(invalid, st);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  prof_collect();
  if (e != cudaSuccess) return fail(cuda_fail(e));
  *out = ix;
  return GRIM_OK;
}

int grim_build_host(const char* ref, uint64_t len, uint32_t B, uint32_t q, uint32_t max_read_len,
                    uint32_t layouts, void* stream, grim_index** out) {
  return grim_build_host_ex(ref, len, B, q, max_read_len, layouts, nullptr, stream, out);
}

int grim_build_host_ex(const char* ref, uint64_t len, uint32_t B, uint32_t q,
                       uint32_t max_read_len, uint32_t layouts, const grim_build_opts* opts,
                       void* stream, grim_index** out) {
  if (!out) return GRIM_E_ARG;
  *out = nullptr;
  if (!ref || len == 0) return GRIM_E_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  char* d = nullptr;
  CK(scratch_alloc(reinterpret_cast<void**>(&d), len, st));
  cudaError_t e = cudaMemcpyAsync(d, ref, len, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) {
    cudaFreeAsync(d, st);
    return cuda_fail(e);
  }
  int rc = grim_build_ex(d, len, B, q, max_read_len, layouts, opts, stream, out);
  cudaFreeAsync(d, st);
  e = cudaStreamSynchronize(st);
  if (rc == GRIM_OK && e != cudaSuccess) {
    grim_free(*out);
    *out = nullptr;
    return cuda_fail(e);
  }
  return rc;
}

int grim_index_info(const grim_index* idx, grim_index_desc* out) {
  if (!idx || !out) return GRIM_E_ARG;
  const IndexView& v = idx->v;
  memset(out, 0, sizeof(*out));
  out->ref_len = v.n;
  out->num_bins = v.num_bins;
  out->num_bins_pad = v.num_bins_pad;
  out->B = v.B;
  out->q = v.q;
  out->ext = v.ext;
  out->max_read_len = v.max_read_len;
  out->layouts = idx->layouts;
  out->words_per_bin = v.wpb;
  out->token_major = idx->tm;
  out->bin_major = idx->bm;
  out->token_major_bytes = idx->tm ? (uint64_t)v.r4 * v.wpad * sizeof(uint32_t) : 0;
  out->bin_major_bytes = idx->bm ? v.num_bins * v.wpb * sizeof(uint32_t) : 0;
  out->coarse_token_major = idx->ctm;
  out->num_coarse = idx->cv.num_bins;
  out->num_coarse_pad = idx->cv.num_bins_pad;
  out->coarse_token_major_bytes =
      idx->ctm ? (uint64_t)idx->cv.r4 * idx->cv.wpad * sizeof(uint32_t) : 0;
  out->coarse_factor = idx->factor;
  out->cta_threads = idx->shape.threads ? idx->shape.threads : 640u;
  out->read_range_kb = idx->shape.range_kb ? idx->shape.range_kb : (48u << 10);
  out->read_switch = idx->shape.read_switch;
  out->all_bins_path = idx->shape.path;
  bool forced = false;
  out->two_level = all_bins_path(idx, &forced) == kPathCoarse ? 1u : 0u;
  return GRIM_OK;
}

int grim_index_set_shape(grim_index* idx, const grim_shape* shape) {
  if (!idx) return GRIM_E_ARG;
  const ExhShape s = shape ? ExhShape{shape->cta_threads, shape->read_range_kb,
                                      shape->read_switch, shape->all_bins_path}
                           : ExhShape{0, 0, 0, 0};
  const int rc = shape_fits(idx, s);
  if (rc != GRIM_OK) return rc;
  idx->shape = s;
  return GRIM_OK;
}

void grim_free(grim_index* idx) {
  if (!idx) return;
  for (uint32_t* p : {idx->tm, idx->bm, idx->ctm, idx->presence}) {
    if (!p) continue;
    if (idx->free_fn) idx->free_fn(p, idx->alloc_ctx);
    else cudaFree(p);
  }
  delete idx;
}

uint64_t grim_filter_workspace_size(const grim_index* idx, uint32_t n_reads, uint64_t n_cand,
                                    uint64_t cap) {
  if (!idx) return 0;
  // room for coarse survivors only in all-bins mode (n_cand == 0); a
  // candidate-mode call with no candidates gets the larger all-bins figure
  const bool all_bins = n_cand == 0;
  return layout(idx->v, n_reads, cap, all_bins && two_level_capable(idx) ? idx->factor : 0,
                token_copies(idx->v, !all_bins))
      .total;
}

int grim_filter(const grim_index* idx, const char* reads, const uint64_t* offsets,
                const uint32_t* lens, uint32_t n_reads, const uint16_t* e, const int32_t* cand,
                const uint64_t* cand_off, uint64_t n_cand, uint32_t* out_read, uint32_t* out_bin,
                uint8_t* out_count, uint64_t cap, uint64_t* n_out, void* workspace,
                uint64_t workspace_bytes, void* stream) {
  if (!idx || !n_out) return GRIM_E_ARG;
  *n_out = 0;
  const bool cand_mode = cand != nullptr || cand_off != nullptr;
  if (cand_mode && !cand_off) return GRIM_E_ARG;
  if (cand_mode && n_cand && !cand) return GRIM_E_ARG;
  const bool capable = two_level_capable(idx);
  if (cand_mode && !(idx->layouts & GRIM_LAYOUT_BIN_MAJOR)) return GRIM_E_NO_LAYOUT;
  if (!cand_mode && !(idx->layouts & GRIM_LAYOUT_TOKEN_MAJOR) && !capable) return GRIM_E_NO_LAYOUT;
  if (n_reads == 0) return GRIM_OK;
  if (!reads || !offsets || !lens || !e) return GRIM_E_ARG;
  if (cap && (!out_read || !out_bin || !out_count)) return GRIM_E_ARG;
  if (cap > 0xFFFFFFFFull) return GRIM_E_ARG;
  const IndexView& v = idx->v;
  const uint32_t f = capable && !cand_mode ? idx->factor : 0;  // survivors: all-bins mode
  const uint32_t copies = token_copies(v, cand_mode);
  const Layout L = layout(v, n_reads, cap, f, copies);
  if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255)) return GRIM_E_ARG;
  if (workspace_bytes < L.total) return GRIM_E_WORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  char* ws = static_cast<char*>(workspace);
  Ctl* ctl = reinterpret_cast<Ctl*>(ws);
  uint16_t* tokens = reinterpret_cast<uint16_t*>(ws + L.tok);
  uint32_t* meta = reinterpret_cast<uint32_t*>(ws + L.meta);
  // record buffers hold rcap >= cap records; more than cap final records is
  // still an overflow of the caller's arrays
  const uint64_t rcap = record_capacity(n_reads, cap, f);
  RecordsView ra{reinterpret_cast<unsigned long long*>(ws + L.keys_a),
                 reinterpret_cast<uint8_t*>(ws + L.cnt_a), rcap};
  RecordsView rb{reinterpret_cast<unsigned long long*>(ws + L.keys_b),
                 reinterpret_cast<uint8_t*>(ws + L.cnt_b), rcap};
  ReadsView rv{tokens, meta, n_reads, token_stride(v), copies};
  const uint32_t bin_bits = v.num_bins > 1 ? bit_length(v.num_bins - 1) : 0;
  uint64_t survivors = 0;
  uint32_t switch_used = 0, path_used = 0;  // all-bins mode: what the call took
  const uint32_t read_bits = n_reads > 1 ? bit_length((uint64_t)n_reads - 1) : 0;

  CK(cudaMemsetAsync(ctl, 0, sizeof(Ctl), st));
  launch_tokenise(reads, offsets, lens, e, v, rv, tokens, meta, ctl, st);
  if (cand_mode) launch_check_candidates(cand_off, n_reads, n_cand, ctl, st);
  else if (!idx->shape.read_switch) launch_block_spread(lens, n_reads, v.q, ctl, st);
  CK(cudaGetLastError());
  // input errors end the call before the filter runs; the batch's largest
  // miss budget sizes the all-bins kernel's counters
  Ctl h{};
  CK(cudaMemcpyAsync(&h, ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  int sc = status_to_code(h.status);
  if (sc != GRIM_OK) {
    prof_collect();
    return sc;
  }

  // what the final sort and split work from
  const int32_t* lists = cand;
  const uint64_t* lists_off = cand_off;
  uint64_t n_lists = n_cand;
  bool list_mode = cand_mode;

  if (cand_mode) {
    launch_candidates(v, rv, cand, cand_off, ra, ctl, st, "candidates", {false, 0}, 0, true);
  } else {
    // all bins: coarse-then-exact when the index allows it and every read
    // needs enough of its tokens present for super-bins to fail early;
    // otherwise (some read passes almost anywhere) one exact pass
    const uint32_t min_slack = 255u - h.max_tight;
    bool forced = false;
    bool two = all_bins_path(idx, &forced) == kPathCoarse && (forced || min_slack >= 24);
    // automatic read switch: a warp's lane groups take their next reads
    // together when every read has as many 16-token blocks and the same miss
    // budget D' (reads then leave a tile at similar blocks, so no group
    // waits long for the others), each on its own otherwise
    ExhShape shape = idx->shape;
    if (!shape.read_switch)
      shape.read_switch = h.blk_max + h.blk_lo == 32u && h.max_d + h.d_lo == 255u
                              ? GRIM_SWITCH_WARP
                              : GRIM_SWITCH_GROUP;
    switch_used = shape.read_switch;
    if (two) {
      const IndexView& cv = idx->cv;
      const uint32_t cbits = cv.num_bins > 1 ? bit_length(cv.num_bins - 1) : 0;
      launch_exhaustive(cv, rv, ra, cbits, h.max_d, ctl, st, "exhaustive_coarse", {false, 0},
                        shape);
      CK(cudaGetLastError());
      CK(cudaMemcpyAsync(&h, ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      prof_collect();
      const uint64_t n_surv = h.n_rec;
      survivors = n_surv;
      if (n_surv > rcap && (idx->layouts & GRIM_LAYOUT_TOKEN_MAJOR)) {
        two = false;  // too many survivors to hold: one exact pass instead
      } else if (n_surv > rcap) {
        // every passing record lies in a surviving super-bin, so f times the
        // survivors bounds the total from above
        *n_out = n_surv * f;
        return GRIM_E_OVERFLOW;
      } else {
        int32_t* icand = reinterpret_cast<int32_t*>(ws + L.cand);
        uint64_t* ioff = reinterpret_cast<uint64_t*>(ws + L.cand_off);
        const RecordsView surv = sort_records(ra, rb, n_surv, read_bits + cbits, ws + L.hist, st);
        expand_survivors(surv.keys, n_surv, cbits, f, n_reads, icand, ioff, st);
        lists = icand;
        lists_off = ioff;
        n_lists = n_surv * f;
        list_mode = true;
      }
      // restart the record and work counters for the next pass
      CK(cudaMemsetAsync(ctl, 0, offsetof(Ctl, blocks), st));
    }
    path_used = two ? GRIM_PATH_TWO_LEVEL : GRIM_PATH_EXACT;
    if (two) launch_candidates(v, rv, lists, lists_off, ra, ctl, st, "candidates_refine");
    else launch_exhaustive(v, rv, ra, bin_bits, h.max_d, ctl, st, "exhaustive", {false, 0},
                           shape);
  }
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(&h, ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  prof_collect();
  sc = status_to_code(h.status);
  if (sc != GRIM_OK) return sc;
  *n_out = h.n_rec;
  if (h.n_rec > cap) return GRIM_E_OVERFLOW;
  const uint32_t key_bits =
      list_mode ? bit_length(n_lists ? n_lists - 1 : 0) : bin_bits + read_bits;
  sort_and_emit(ra, rb, h.n_rec, key_bits, ws + L.hist, list_mode, bin_bits, lists, lists_off,
                n_reads, out_read, out_bin, out_count, st);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(st));
  prof_collect();
  g_last_stats.n_reads = n_reads;
  g_last_stats.n_records = h.n_rec;
  g_last_stats.pairs = cand_mode ? n_cand : (uint64_t)n_reads * v.num_bins;
  g_last_stats.tokens_executed = h.blocks * kBlockTokens;
  // blocks of the one-word tail test a quarter of the tile's bins
  g_last_stats.bit_tests_executed =
      (h.blocks - h.tail_blocks) * kBlockTokens * exhaustive_tile_bins(v.r4) +
      h.tail_blocks * kBlockTokens * (exhaustive_tile_bins(v.r4) / 4);
  g_last_stats.survivors = survivors;
  g_last_stats.read_switch = switch_used;
  g_last_stats.all_bins_path = path_used;
  return GRIM_OK;
}

int grim_filter_host(const grim_index* idx, const char* reads, const uint64_t* offsets,
                     const uint32_t* lens, uint32_t n_reads, const uint16_t* e,
                     const int32_t* cand, const uint64_t* cand_off, uint64_t n_cand,
                     uint32_t* out_read, uint32_t* out_bin, uint8_t* out_count, uint64_t cap,
                     uint64_t* n_out, void* stream) {
  if (!idx || !n_out) return GRIM_E_ARG;
  *n_out = 0;
  const bool cand_mode = cand != nullptr || cand_off != nullptr;
  if (n_reads == 0) return GRIM_OK;
  if (!reads || !offsets || !lens || !e) return GRIM_E_ARG;
  if (cand_mode && (!cand_off || (n_cand && !cand))) return GRIM_E_ARG;
  if (cap && (!out_read || !out_bin || !out_count)) return GRIM_E_ARG;
  uint64_t bytes = 0;
  for (uint32_t r = 0; r < n_reads; ++r)
    if (offsets[r] + lens[r] > bytes) bytes = offsets[r] + lens[r];
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const uint64_t ws_bytes = grim_filter_workspace_size(idx, n_reads, n_cand, cap);
  // one stream-ordered allocation holds every device copy
  const uint64_t o_reads = 0;
  const uint64_t o_off = align256(o_reads + (bytes ? bytes : 1));
  const uint64_t o_lens = align256(o_off + (uint64_t)n_reads * 8);
  const uint64_t o_e = align256(o_lens + (uint64_t)n_reads * 4);
  const uint64_t o_cand = align256(o_e + (uint64_t)n_reads * 2);
  const uint64_t o_coff = align256(o_cand + (cand_mode ? n_cand * 4 : 0));
  const uint64_t o_or = align256(o_coff + (cand_mode ? ((uint64_t)n_reads + 1) * 8 : 0));
  const uint64_t o_ob = align256(o_or + cap * 4);
  const uint64_t o_oc = align256(o_ob + cap * 4);
  const uint64_t o_ws = align256(o_oc + cap);
  const uint64_t total = o_ws + ws_bytes;
  char* d = nullptr;
  CK(scratch_alloc(reinterpret_cast<void**>(&d), total, st));
  auto h2d = [&](uint64_t o, const void* src, uint64_t n) {
    return n ? cudaMemcpyAsync(d + o, src, n, cudaMemcpyHostToDevice, st) : cudaSuccess;
  };
  cudaError_t ce = h2d(o_reads, reads, bytes);
  if (ce == cudaSuccess) ce = h2d(o_off, offsets, (uint64_t)n_reads * 8);
  if (ce == cudaSuccess) ce = h2d(o_lens, lens, (uint64_t)n_reads * 4);
  if (ce == cudaSuccess) ce = h2d(o_e, e, (uint64_t)n_reads * 2);
  if (ce == cudaSuccess && cand_mode) ce = h2d(o_cand, cand, n_cand * 4);
  if (ce == cudaSuccess && cand_mode) ce = h2d(o_coff, cand_off, ((uint64_t)n_reads + 1) * 8);
  if (ce != cudaSuccess) {
    cudaFreeAsync(d, st);
    return cuda_fail(ce);
  }
  int rc = grim_filter(idx, d + o_reads, reinterpret_cast<const uint64_t*>(d + o_off),
                       reinterpret_cast<const uint32_t*>(d + o_lens), n_reads,
                       reinterpret_cast<const uint16_t*>(d + o_e),
                       cand_mode ? reinterpret_cast<const int32_t*>(d + o_cand) : nullptr,
                       cand_mode ? reinterpret_cast<const uint64_t*>(d + o_coff) : nullptr, n_cand,
                       reinterpret_cast<uint32_t*>(d + o_or), reinterpret_cast<uint32_t*>(d + o_ob),
                       reinterpret_cast<uint8_t*>(d + o_oc), cap, n_out, d + o_ws, ws_bytes, stream);
  if (rc == GRIM_OK && *n_out) {
    const uint64_t n = *n_out;
    ce = cudaMemcpyAsync(out_read, d + o_or, n * 4, cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(out_bin, d + o_ob, n * 4, cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(out_count, d + o_oc, n, cudaMemcpyDeviceToHost, st);
    if (ce != cudaSuccess) rc = cuda_fail(ce);
  }
  cudaFreeAsync(d, st);
  ce = cudaStreamSynchronize(st);
  if (rc == GRIM_OK && ce != cudaSuccess) rc = cuda_fail(ce);
  return rc;
}

int grim_reverse_complement(const char* reads, const uint64_t* offsets, const uint32_t* lens,
                            uint32_t n_reads, char* out, void* stream) {
  if (n_reads == 0) return GRIM_OK;
  if (!reads || !offsets || !lens || !out || out == reads) return GRIM_E_ARG;
  launch_reverse_complement(reads, offsets, lens, n_reads, out, static_cast<cudaStream_t>(stream));
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GRIM_OK : cuda_fail(e);
}

uint64_t grim_loc_to_bin(const grim_index* idx, uint64_t loc) { return idx ? loc / idx->v.B : 0; }

uint32_t grim_edits_for_rate(uint32_t L, uint32_t num, uint32_t den) {
  if (den == 0) return 0;
  return (uint32_t)(((uint64_t)L * num + den - 1) / den);
}

int grim_last_filter_stats(grim_filter_stats* out) {
  if (!out) return GRIM_E_ARG;
  *out = g_last_stats;
  return GRIM_OK;
}

int grim_profile(int enable) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  g_prof_on = enable != 0;
  if (g_prof_on) g_prof.clear();
  return GRIM_OK;
}

int grim_profile_get(grim_kernel_time* out, int max) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  const int n = (int)g_prof.size();
  for (int i = 0; i < n && i < max && out; ++i) {
    memset(&out[i], 0, sizeof(out[i]));
    strncpy(out[i].name, g_prof[i].name.c_str(), sizeof(out[i].name) - 1);
    out[i].launches = g_prof[i].launches;
    out[i].total_ms = g_prof[i].ms;
  }
  return n;
}

}  // extern "C"
