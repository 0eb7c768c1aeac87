/*
 * grim.h -- C-ABI of libgrim.so, a GB300 (sm_103a) implementation of the
 * bin-level q-gram filter of GRIM-Filter (Kim et al., arXiv 1708.04329).
 *
 * The filter (§GRIM-Filter, Fig. 2, Fig. 3, Fig. 5):
 *   - the reference of N bases is cut into bins of B bases; bin b's window is
 *     [b*B, min(b*B + B + ext, N)) with ext = max_read_len - 1, so any read
 *     whose first base lies in bin b's B-base core fits inside the window;
 *   - each bin has a 4^q-bit vector: bit t is 1 iff token t (the base-4
 *     number of q consecutive bases, A=0 C=1 G=2 T=3, first base most
 *     significant, case folded) occurs wholly inside the window with no
 *     other character in it;
 *   - for a read of length L the L-q+1 tokens are extracted and, for each
 *     candidate bin, their existence bits are summed (every position counts,
 *     repeats included; a q-gram holding a non-ACGT character adds 0);
 *   - the bin passes iff sum >= T = (L-q+1) - q*e (e = the read's edit
 *     budget); T <= 0 makes every bin pass.
 *
 * Conventions for every call below:
 *   - "device" pointers are CUDA device memory of the current device (for
 *     example torch tensors' data_ptr()); "host" pointers are CPU memory
 *     (page-locked memory gives the fastest copies);
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream); work is
 *     enqueued on it, and the calls that return results synchronise it;
 *   - the caller owns every buffer it passes; the library keeps no caller
 *     pointer after a call returns;
 *   - errors are reported by the return value only (GRIM_OK = 0, negatives
 *     below); nothing is thrown across the ABI and nothing aborts.
 */
#ifndef GRIM_H
#define GRIM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes -------------------------------------------------------- */
#define GRIM_OK 0
#define GRIM_E_ARG (-1)            /* bad argument (null pointer, bad size, bad CSR offsets)   */
#define GRIM_E_NOMEM (-2)          /* device or host allocation failed                         */
#define GRIM_E_CUDA (-3)           /* a CUDA call failed; grim_last_cuda_error() says which    */
#define GRIM_E_READ_TOO_SHORT (-4) /* a read has L < q                                          */
#define GRIM_E_READ_TOO_LONG (-5)  /* a read has L > max_read_len or L-q+1 > 255               */
#define GRIM_E_BAD_CANDIDATE (-6)  /* a candidate bin is outside [0, num_bins)                  */
#define GRIM_E_OVERFLOW (-7)       /* more passing records than `cap`; *n_out holds the total   */
#define GRIM_E_TIMEOUT (-8)        /* a bounded device wait gave up                             */
#define GRIM_E_WORKSPACE (-9)      /* workspace smaller than grim_filter_workspace_size()       */
#define GRIM_E_NO_LAYOUT (-10)     /* the index lacks the table layout this call needs          */
#define GRIM_E_UNSUPPORTED (-11)   /* parameter outside what this build implements              */
#define GRIM_E_NOT_READY (-12)     /* a plan launch or server request has not finished yet     */
#define GRIM_E_BUSY (-13)          /* grim_server_submit: the server's queue is full            */
#define GRIM_E_IO (-14)            /* a file could not be opened, read or written               */
#define GRIM_E_FORMAT (-15)        /* not an index file of this library, or damaged             */
#define GRIM_E_CANCELLED (-16)     /* a server request was cancelled before it ran              */

/* ---- table layouts (bit mask for grim_build) ----------------------------- */
/* Token-major: row t holds token t's bit for every bin, contiguous
 * (§Mapping GRIM-Filter: one token's existence bits across all bins share a
 * contiguous region, a bin's bits across tokens share a column).  Used by the
 * all-bins filter. */
#define GRIM_LAYOUT_TOKEN_MAJOR 1u
/* Bin-major: bin b's 4^q-bit vector is contiguous (Fig. 2 column).  Used by
 * the candidate-list filter. */
#define GRIM_LAYOUT_BIN_MAJOR 2u
/* Coarse token-major: the token-major layout over super-bins of f adjacent
 * bins (f = grim_build_opts.coarse_factor; see there for the default).  A super-bin's window is the union of its
 * bins' windows, and because ext >= q-1 every q-gram of that union lies wholly
 * inside one member's window, so a super-bin's vector is exactly the OR of its
 * members' vectors and its token sum bounds each member's from above.  With
 * this layout and the bin-major one, the all-bins filter first discards
 * super-bins whose sum is below T, then checks the members of the rest
 * exactly against the bin-major table; the result is identical. */
#define GRIM_LAYOUT_COARSE 4u
#define GRIM_LAYOUT_ALL 7u


typedef struct grim_index grim_index; /* opaque; owns its device tables */

/* Description of a built index (all sizes in the units named). */
typedef struct {
  uint64_t ref_len;          /* N                                                   */
  uint64_t num_bins;         /* ceil(N / B)                                         */
  uint64_t num_bins_pad;     /* num_bins rounded up to a multiple of 1024           */
  uint32_t B, q, ext;        /* bin core size, token length, extension (L_max - 1)  */
  uint32_t max_read_len;     /* longest read the index accepts                      */
  uint32_t layouts;          /* GRIM_LAYOUT_* bits present                          */
  uint32_t words_per_bin;    /* uint32 words of one bin-major vector: max(1, 4^q/32) */
  /* token-major table, device, uint32[4^q][num_bins_pad / 32]; bin b of row t
   * is bit (b % 32) of word b / 32; padded bins are 0.  NULL if absent. */
  const uint32_t* token_major;
  /* bin-major table, device, uint32[num_bins][words_per_bin]; token t of bin
   * b is bit (t % 32) of word t / 32.  NULL if absent. */
  const uint32_t* bin_major;
  uint64_t token_major_bytes, bin_major_bytes;
  /* coarse token-major table, device, uint32[4^q][num_coarse_pad / 32] over
   * super-bins s = bins [s*coarse_factor, (s+1)*coarse_factor); NULL if absent */
  const uint32_t* coarse_token_major;
  uint64_t num_coarse, num_coarse_pad, coarse_token_major_bytes;
  uint32_t coarse_factor;
  /* launch shape of the all-bins kernel (grim_build_opts, grim_index_set_shape) */
  uint32_t cta_threads;      /* threads of its one persistent CTA per SM        */
  uint32_t read_range_kb;    /* token-row KiB of one read range (the read tile) */
  uint32_t read_switch;      /* GRIM_SWITCH_GROUP, GRIM_SWITCH_WARP, 0 = automatic */
  uint32_t all_bins_path;    /* GRIM_PATH_* as set (0 = automatic)              */
  uint32_t two_level;        /* 1: all-bins calls take coarse-then-exact (before
                                the per-batch rules), 0: one exact pass         */
} grim_index_desc;

/*
 * Build the bin bit vectors of a reference (§GRIM-Filter: the genome is
 * scanned once, bit vectors are kept for reuse; Fig. 2).
 *   ref           device, `len` ASCII bytes; A/C/G/T in either case are bases,
 *                 any other byte is "not a base"
 *   B             bin core size in bases, >= 1
 *   q             token length, 2..6 (4^q bits per bin)
 *   max_read_len  longest read to be filtered, >= q; ext = max_read_len - 1
 *   layouts       nonzero mask of GRIM_LAYOUT_* to build
 *   out           receives the index; free it with grim_free
 * The index's tables are allocated by the library with cudaMalloc on the
 * current device.  Synchronises `stream` before returning.
 * Errors: GRIM_E_ARG, GRIM_E_UNSUPPORTED (q outside 2..6), GRIM_E_NOMEM,
 * GRIM_E_CUDA.
 */
int grim_build(const char* ref, uint64_t len, uint32_t B, uint32_t q, uint32_t max_read_len,
               uint32_t layouts, void* stream, grim_index** out);

/* As grim_build, with `ref` in host memory; the copy to the device is part of
 * the call. */
int grim_build_host(const char* ref, uint64_t len, uint32_t B, uint32_t q, uint32_t max_read_len,
                    uint32_t layouts, void* stream, grim_index** out);

/* How the lane groups of a warp in the all-bins kernel take their next read
 * (grim_shape). */
#define GRIM_SWITCH_GROUP 1u /* each group as soon as its read ends             */
#define GRIM_SWITCH_WARP 2u  /* all groups of a warp together, once all ended   */

/* The all-bins path (grim_shape).  Automatic (0): coarse-then-exact when the
 * index has the coarse and bin-major tables and its super-bin window would
 * hold at most 50% of the 4^q tokens in a uniform random sequence (denser
 * coarse tables let too many super-bins pass: at q = 5, B = 200 that is an
 * index for reads up to about 300 bp), else one exact pass; a batch whose
 * tightest read has fewer than 24 tokens of slack takes the exact pass too,
 * and so does a call whose coarse survivors exceed its record room (320 a
 * read, or the output capacity if larger).  An index with only one of the
 * two paths' tables always takes that path. */
#define GRIM_PATH_TWO_LEVEL 1u /* coarse pass over super-bins, then exact checks */
#define GRIM_PATH_EXACT 2u     /* one exact pass over every bin                  */

/* Build options.  Zero-initialise and set what you need. */
typedef struct {
  /* bins per super-bin of the coarse table (1..64).  0 chooses the largest
   * power of two up to 64 whose super-bin window (f*B + ext bases) would
   * hold at most 50% of all 4^q tokens in a uniform random sequence: 2 at
   * q = 5, B = 200, ext = 99 or 249 and 16 at q = 6, B = 100, ext = 149.  Larger
   * factors shrink the coarse pass but let more super-bins pass it; the best
   * value depends on the genome too (the package's autotuner measures it). */
  uint32_t coarse_factor;
  /* Launch shape of the all-bins kernel (0 = default; see
   * grim_index_set_shape): CTA threads (512, 640 or 768) and the read tile,
   * in KiB of token rows per read range (1024 .. 4194304). */
  uint32_t cta_threads;
  uint32_t read_range_kb;
  uint32_t read_switch;    /* GRIM_SWITCH_* (0 = automatic) */
  uint32_t all_bins_path;  /* GRIM_PATH_* (0 = automatic)   */
  uint32_t reserved[3];
} grim_build_opts;

/* The coarse factor grim_build_ex chooses when opts->coarse_factor is 0. */
uint32_t grim_default_coarse_factor(uint32_t B, uint32_t q, uint32_t max_read_len);

/* grim_build / grim_build_host with options (opts may be NULL).
 * Errors: as grim_build, and GRIM_E_ARG for an option out of range. */
int grim_build_ex(const char* ref, uint64_t len, uint32_t B, uint32_t q, uint32_t max_read_len,
                  uint32_t layouts, const grim_build_opts* opts, void* stream, grim_index** out);
int grim_build_host_ex(const char* ref, uint64_t len, uint32_t B, uint32_t q,
                       uint32_t max_read_len, uint32_t layouts, const grim_build_opts* opts,
                       void* stream, grim_index** out);

/* Fill *out with the index's sizes and device table pointers. */
int grim_index_info(const grim_index* idx, grim_index_desc* out);

/*
 * Launch shape of the all-bins filter for later calls with this index (the
 * tile sizes the paper ties to its parallel width p, §Parameter Evaluation
 * Results: how many bins' bits one fetch covers and how many reads reuse
 * it).  The bin tile is fixed by shared memory (1024 bins up to q = 5, 256
 * at q = 6; the coarse factor of grim_build_opts sets how many bins a
 * super-bin holds); a grim_shape sets the rest (zero fields: the default;
 * shape NULL: every default):
 *   cta_threads    threads of the one persistent CTA per SM: 512, 640 or 768
 *                  (more warps, fewer registers each); 0 = 640
 *   read_range_kb  read tile: reads are swept in ranges of about this many
 *                  KiB of token rows, range by range, so that a range stays
 *                  in L2 while every CTA sweeps its tiles against it;
 *                  1024 .. 4194304, 0 = 49152 (48 MiB)
 *   read_switch    GRIM_SWITCH_GROUP, GRIM_SWITCH_WARP, or 0 (automatic):
 *                  a warp's lane groups each hold one read; taking the next
 *                  read costs the whole warp the same instructions whether
 *                  one group or all take one, so WARP lets a group whose read
 *                  ended early idle until every group's read has ended, and
 *                  then switches all of them at once (fewer switches, some
 *                  idle blocks).  Automatic: WARP when every read of the
 *                  batch spans the same number of 16-token blocks and has
 *                  the same miss budget D' (so reads leave a tile at similar
 *                  blocks and no group idles for long), GROUP otherwise;
 *                  graph plans, whose batches are not known when they are
 *                  captured, use GROUP
 *   all_bins_path  GRIM_PATH_TWO_LEVEL, GRIM_PATH_EXACT, or 0 (automatic; see
 *                  GRIM_PATH_*)
 * Results do not depend on the shape.  Graph plans take the shape when they
 * are created.  Not to be called while a filter call with this index runs.
 * Errors: GRIM_E_ARG (NULL index, a value outside the ranges above),
 * GRIM_E_NO_LAYOUT (a path whose tables the index lacks).
 */
typedef struct {
  uint32_t cta_threads;
  uint32_t read_range_kb;
  uint32_t read_switch;
  uint32_t all_bins_path;
  uint32_t reserved[4];
} grim_shape;
int grim_index_set_shape(grim_index* idx, const grim_shape* shape);

/*
 * Index persistence (§GRIM-Filter: the bit vectors are generated once per
 * reference and stored for later runs).  grim_save writes the build
 * parameters and every table the index holds to `path` (a 256-byte header,
 * then the tables exactly as in device memory, with a checksum); grim_load
 * reads such a file into new device tables on the current device.
 *   layouts  the tables to load (a subset of those in the file), 0 = all
 *   flags    GRIM_LOAD_VERIFY: recompute the checksum while reading
 * A loaded index is identical to the one saved (same parameters, coarse
 * factor and table bits) and gives identical filter results.  Both calls
 * synchronise.  Errors: GRIM_E_ARG, GRIM_E_IO (open/read/write failed),
 * GRIM_E_FORMAT (bad magic, version, sizes or checksum; truncated file),
 * GRIM_E_NO_LAYOUT (a requested table is not in the file), GRIM_E_NOMEM,
 * GRIM_E_CUDA.
 */
#define GRIM_LOAD_VERIFY 1u
int grim_save(const grim_index* idx, const char* path);
int grim_load(const char* path, uint32_t layouts, uint32_t flags, grim_index** out);

/* Release an index and its device tables (NULL is ignored). */
void grim_free(grim_index* idx);

/* Static description of a status code. */
const char* grim_strerror(int status);

/* The CUDA error string behind the last GRIM_E_CUDA of the calling thread. */
const char* grim_last_cuda_error(void);

/* Device allocations of index tables through the caller's allocator (for
 * example a framework's caching allocator, so the tables show in its
 * accounting).  alloc returns `bytes` of device memory on the current
 * device, or NULL (the build then fails with GRIM_E_NOMEM); free releases
 * what alloc returned.  Both NULL restores cudaMalloc / cudaFree.  An index
 * keeps the functions and ctx it was built with and frees its tables with
 * them in grim_free.  Errors: GRIM_E_ARG (only one of the two given). */
typedef void* (*grim_alloc_fn)(uint64_t bytes, void* ctx);
typedef void (*grim_free_fn)(void* ptr, void* ctx);
int grim_set_allocator(grim_alloc_fn alloc, grim_free_fn free, void* ctx);

/* The build's scratch (packed reference) and the host-buffer entry points'
 * device copies come from a library-owned stream-ordered memory pool per
 * device that keeps freed memory for the next call.  This releases that
 * cached memory of the current device (cudaMemPoolTrimTo).  Errors:
 * GRIM_E_CUDA. */
int grim_trim_scratch(void);

/*
 * Bytes of device workspace grim_filter needs for n_reads reads, n_cand
 * candidates (0 in all-bins mode) and an output capacity of cap records.
 * All-bins mode on an index with the coarse table also holds room for the
 * coarse pass's survivors (320 records a read); candidate mode does not.
 */
uint64_t grim_filter_workspace_size(const grim_index* idx, uint32_t n_reads, uint64_t n_cand,
                                    uint64_t cap);

/*
 * Filter reads against the index (§GRIM-Filter steps 1-3: tokenise,
 * accumulate existence bits, compare with the threshold of Fig. 3; the
 * mapper's per-location check of Fig. 5 is the candidate-list mode).
 *
 *   reads      device, ASCII; read r is reads[offsets[r] .. offsets[r]+lens[r])
 *   offsets    device, uint64[n_reads]
 *   lens       device, uint32[n_reads]; every q <= lens[r] <= max_read_len
 *   n_reads    number of reads (0 gives *n_out = 0)
 *   e          device, uint16[n_reads], per-read absolute edit budget
 *   cand       device, int32[n_cand] candidate bins, or NULL for every bin
 *              (all-bins mode, needs the token-major layout)
 *   cand_off   device, uint64[n_reads+1] CSR offsets into cand: read r's
 *              candidates are cand[cand_off[r] .. cand_off[r+1]); must be
 *              non-decreasing with cand_off[n_reads] == n_cand (candidate
 *              mode needs the bin-major layout)
 *   out_read, out_bin, out_count
 *              device, uint32/uint32/uint8 [cap]: the passing records
 *              (read, bin, sum), ordered by read, then by bin (all-bins
 *              mode) or by position in the read's candidate list
 *   cap        capacity of the three output arrays, in records
 *   n_out      host; receives the number of passing records
 *   workspace  device, >= grim_filter_workspace_size(idx, n_reads, n_cand, cap)
 *              bytes, 256-byte aligned; contents need not be initialised
 * Synchronises `stream` before returning.
 * Errors: GRIM_E_ARG, GRIM_E_NO_LAYOUT, GRIM_E_WORKSPACE,
 * GRIM_E_READ_TOO_SHORT, GRIM_E_READ_TOO_LONG, GRIM_E_BAD_CANDIDATE (these
 * three in that order of precedence; output contents then unspecified),
 * GRIM_E_OVERFLOW (*n_out = total passing records; outputs unspecified, call
 * again with cap >= *n_out), GRIM_E_CUDA.
 */
int grim_filter(const grim_index* idx, const char* reads, const uint64_t* offsets,
                const uint32_t* lens, uint32_t n_reads, const uint16_t* e, const int32_t* cand,
                const uint64_t* cand_off, uint64_t n_cand, uint32_t* out_read, uint32_t* out_bin,
                uint8_t* out_count, uint64_t cap, uint64_t* n_out, void* workspace,
                uint64_t workspace_bytes, void* stream);

/*
 * As grim_filter with every array in host memory.  The library allocates
 * device staging (stream-ordered, returned to the pool before the call
 * returns) and the host<->device copies are part of the call.
 */
int grim_filter_host(const grim_index* idx, const char* reads, const uint64_t* offsets,
                     const uint32_t* lens, uint32_t n_reads, const uint16_t* e,
                     const int32_t* cand, const uint64_t* cand_off, uint64_t n_cand,
                     uint32_t* out_read, uint32_t* out_bin, uint8_t* out_count, uint64_t cap,
                     uint64_t* n_out, void* stream);

/*
 * As grim_filter, for callers that cannot allocate device memory: a host
 * process whose memory manager owns the whole GPU, or a serving loop that
 * keeps cudaMalloc / cudaFree (which can synchronise the device) off its
 * request path.  The paper has no counterpart to this entry point.
 *
 * The scratch the filter needs lives in one fixed device array of
 * GRIM_NOALLOC_SCRATCH_BYTES inside the library, which every GPU that loads
 * the library holds until the process exits; the call allocates nothing.
 * The caller still passes the inputs and the output arrays (device memory),
 * exactly as for grim_filter.
 *   - Size limit: a call whose scratch (grim_filter_workspace_size(idx,
 *     n_reads, n_cand, cap), the exact figure to check a batch against)
 *     exceeds GRIM_NOALLOC_SCRATCH_BYTES (also returned by
 *     grim_noalloc_scratch_bytes) is rejected with GRIM_E_WORKSPACE before
 *     any device work.  The per-read part depends on the index, not on the
 *     reads' own lengths: 2*ts + 4 bytes per read, with ts = the index's
 *     max_read_len - q + 1 rounded up to a multiple of 16 (196 bytes for an
 *     index built for 100 bp reads at q = 5, 484 bytes for 250 bp), times 4
 *     for the token copies of the all-bins mode at q = 6; then 18 bytes per
 *     record of capacity, which is cap, or max(cap, 320 * n_reads) for an
 *     index with the coarse layout (room for the coarse pass's survivors),
 *     whose records take another 4 * coarse_factor bytes each for the
 *     survivors' expanded candidate lists.
 *   - First call on a device: it looks up the array's device address (once
 *     per device, with that device current) and keeps it for the life of the
 *     process; make that first call before any stream capture.  The kept
 *     address assumes one CUDA context per device for the whole process:
 *     after cudaDeviceReset the library must be reloaded before this entry
 *     point is used again.
 *   - Sharing: all calls share the one array and it keeps the last call's
 *     contents (each call clears what must start at zero).  Calls that
 *     overlap on the GPU -- from several host threads, or on several
 *     streams -- race on it; serialise them.
 * Errors: as grim_filter.
 */
#define GRIM_NOALLOC_SCRATCH_BYTES (32u << 20)
/* GRIM_NOALLOC_SCRATCH_BYTES as compiled into the library. */
uint64_t grim_noalloc_scratch_bytes(void);
int grim_filter_noalloc(const grim_index* idx, const char* reads, const uint64_t* offsets,
                        const uint32_t* lens, uint32_t n_reads, const uint16_t* e,
                        const int32_t* cand, const uint64_t* cand_off, uint64_t n_cand,
                        uint32_t* out_read, uint32_t* out_bin, uint8_t* out_count, uint64_t cap,
                        uint64_t* n_out, void* stream);

/* ---- graph-captured plans for ragged batches ---------------------------- */
/*
 * A plan runs grim_filter's work for batches of up to declared maximum sizes
 * as one CUDA graph: every launch shape is fixed at creation, the batch's
 * counts are copied to the device at the start of each run, and the choices
 * grim_filter makes on the host between launches (coarse-then-exact or one
 * exact pass, survivor overflow, sort sizes) are made by the kernels from
 * device-resident counts.  Reads of any lengths up to the index's
 * max_read_len and, in candidate mode, ragged candidate lists are handled in
 * that single graph launch per batch.  Results are identical to grim_filter.
 *
 * The plan owns device buffers for one batch's inputs and outputs
 * (grim_plan_buffers_get); the caller fills them (for example with
 * cudaMemcpyAsync on the launch stream) before grim_plan_launch.  One launch
 * of a plan may be in flight at a time: grim_plan_launch waits for the
 * previous one to finish; use several plans to overlap batches.
 */
typedef struct grim_plan grim_plan;

#define GRIM_PLAN_CANDIDATES 1u /* candidate-list mode (else all bins) */
/* Host-memory plan: the buffers of grim_plan_buffers_get are mapped pinned
 * HOST memory.  The caller writes a batch's inputs there; the graph copies
 * them to the device itself (only the bytes the batch uses: reads up to the
 * largest offset + length, which grim_plan_launch checks against max_bases)
 * and writes the pass list straight back into the host output buffers, so a
 * batch costs one graph launch and no separate copies.  Inputs and outputs
 * must not be touched while a launch of the plan is in flight. */
#define GRIM_PLAN_HOST_IO 2u

typedef struct {
  uint32_t max_reads;   /* reads per batch, >= 1                                    */
  uint32_t max_e;       /* largest per-read edit budget (sizes the counters); a read
                           with a larger e makes that batch fail with GRIM_E_ARG    */
  uint64_t max_bases;   /* bytes of read sequence per batch, >= 1                   */
  uint64_t max_cand;    /* candidate mode: candidates per batch                     */
  uint64_t cap;         /* output records per batch                                 */
  uint32_t flags;       /* GRIM_PLAN_*                                              */
  uint32_t cand_unroll; /* candidate gathers in flight per lane group: 1, 2, 4 or 8;
                           0 = the library default (tuned by the package's autotuner) */
  uint32_t reserved[6];
} grim_plan_desc;

/* Buffers owned by a plan (layouts as for grim_filter): device memory, or
 * mapped pinned host memory for a GRIM_PLAN_HOST_IO plan. */
typedef struct {
  char* reads;          /* [max_bases]                                 */
  uint64_t* offsets;    /* [max_reads]                                 */
  uint32_t* lens;       /* [max_reads]                                 */
  uint16_t* e;          /* [max_reads]                                 */
  int32_t* cand;        /* [max_cand], candidate mode only, else NULL  */
  uint64_t* cand_off;   /* [max_reads + 1], candidate mode only        */
  uint32_t* out_read;   /* [cap]                                       */
  uint32_t* out_bin;    /* [cap]                                       */
  uint8_t* out_count;   /* [cap]                                       */
} grim_plan_buffers;

/* Allocate a plan's buffers (cudaMalloc, pinned host memory) and capture its
 * graph.  The index must outlive the plan.
 * Errors: GRIM_E_ARG (zero maxima, unknown flags, cand_unroll > 8),
 * GRIM_E_NO_LAYOUT, GRIM_E_NOMEM, GRIM_E_CUDA. */
int grim_plan_create(const grim_index* idx, const grim_plan_desc* desc, grim_plan** out);
int grim_plan_buffers_get(const grim_plan* plan, grim_plan_buffers* out);
/* Enqueue one run on `stream` for a batch of n_reads reads (and n_cand
 * candidates) already in the plan's buffers.  Asynchronous.  A read ending
 * past max_bases fails the batch with GRIM_E_ARG (a host-memory plan refuses
 * the launch with GRIM_E_ARG instead). */
int grim_plan_launch(grim_plan* plan, uint32_t n_reads, uint64_t n_cand, void* stream);
/* GRIM_OK if the last launch has finished (or none was made),
 * GRIM_E_NOT_READY if it is still running. */
int grim_plan_query(const grim_plan* plan);
/* Wait for the last launch; *n_out = passing records in the output buffers.
 * Errors of the batch as for grim_filter (GRIM_E_OVERFLOW: *n_out = total). */
int grim_plan_wait(grim_plan* plan, uint64_t* n_out);
/* Device bytes the plan holds (inputs, outputs and workspace). */
uint64_t grim_plan_device_bytes(const grim_plan* plan);
void grim_plan_free(grim_plan* plan);

/* ---- serving: continuous batching over a resident index ---------------- */
/*
 * A server keeps an index resident and filters requests -- read batches of
 * any size, read lengths and per-read edit budgets (and, in candidate mode,
 * candidate lists) -- as they arrive.  The paper filters each read on its
 * own (§GRIM-Filter, Fig. 5); a server is this library's way of feeding
 * many independent callers to the device at once, and has no counterpart
 * in the paper.
 *
 * A scheduler thread owns `slots` host-memory plans (GRIM_PLAN_HOST_IO), each
 * on its own stream.  Whenever a slot is free it merges the queued requests,
 * oldest first, into one batch within the slot's limits (max_reads,
 * max_bases, max_cand) and launches it; requests that arrive meanwhile wait
 * for the next free slot, and the batches of different slots overlap on the
 * device.  The slots' device memory (batch buffers, workspace, pass lists)
 * is bounded by mem_budget.  A request's result is the same as grim_filter
 * of that request alone: the filter works read by read, and each request's
 * records are handed back with its own read numbering.  With
 * max_chunk_reads, large requests are cut into chunks of consecutive reads
 * that are queued and batched like requests of their own.  A merged batch
 * whose pass list exceeds `cap` is split and its requests (or chunks) rerun
 * one per batch; one over `cap` alone completes its request with
 * GRIM_E_OVERFLOW and the request's total.
 *
 * Requests are validated at submission (read lengths against the index,
 * e <= max_e, sizes against the slot limits, candidate ids and offsets), so
 * one bad request cannot fail the batch it would have joined.
 */
typedef struct grim_server grim_server;

typedef struct {
  uint32_t slots;            /* batches in flight on the device, >= 1 (reduced to fit mem_budget) */
  uint32_t max_reads;        /* reads per merged batch, >= 1; a larger request is refused */
  uint64_t max_bases;        /* read bytes per merged batch, >= 1 */
  uint64_t max_cand;         /* candidate mode: candidates per merged batch                */
  uint64_t cap;              /* pass-list records per merged batch, >= 1                   */
  uint32_t max_e;            /* largest per-read edit budget a request may carry          */
  uint32_t flags;            /* GRIM_PLAN_CANDIDATES, or 0 for all bins                    */
  uint64_t mem_budget;       /* device bytes the slots may hold together (0: no limit)     */
  uint64_t max_queued_reads; /* submit returns GRIM_E_BUSY past this many waiting reads
                                (0: no limit; a request is always taken into an empty queue) */
  uint32_t cand_unroll;      /* as grim_plan_desc                                          */
  /* 0: each request runs whole, in one batch (a request larger than a slot
   * is refused).  N >= 1 (at most max_reads): a request is cut into chunks
   * of up to N consecutive reads (and within max_bases and max_cand), which
   * may run in different slots and batches; the request completes when its
   * last chunk does, and a request larger than a slot is accepted. */
  uint32_t max_chunk_reads;
  uint32_t reserved[6];
} grim_server_desc;

typedef struct {
  int32_t status;           /* GRIM_OK or the request's error                        */
  uint32_t n_reads;
  uint64_t n_out;           /* passing records (the total, on GRIM_E_OVERFLOW)       */
  uint64_t batch;           /* sequence number (from 1) of the batch that served it  */
  uint32_t batch_requests;  /* requests merged into that batch                       */
  uint32_t batch_reads;     /* reads in that batch                                   */
  uint64_t t_submit_ns;     /* steady-clock times: submission, launch, completion    */
  uint64_t t_launch_ns;
  uint64_t t_done_ns;
} grim_request_info;

typedef struct {
  uint32_t slots;           /* slots created (after the memory budget)   */
  uint32_t reserved;
  uint64_t device_bytes;    /* device bytes the slots hold                */
  uint64_t submitted, completed, batches, batch_reads, reads_done, records;
  uint64_t overflow_splits; /* merged batches rerun one request at a time */
  uint64_t queued_requests;   /* requests (or chunks of split requests) waiting */
  uint64_t queued_reads;
  uint64_t cancelled;       /* requests cancelled before they ran         */
} grim_server_stats;

/* Create the slots' plans and start the scheduler.  The index must outlive
 * the server.  Errors: GRIM_E_ARG, GRIM_E_NO_LAYOUT, GRIM_E_NOMEM (not even
 * one slot fits mem_budget), GRIM_E_CUDA. */
int grim_server_create(const grim_index* idx, const grim_server_desc* desc, grim_server** out);
/* Queue a request; every pointer is HOST memory and is copied before the
 * call returns.  reads/offsets/lens/e as grim_filter; cand/cand_off (CSR
 * from 0) in candidate mode, both NULL in all-bins mode.  *ticket names the
 * request.  Errors: GRIM_E_ARG, GRIM_E_READ_TOO_SHORT, GRIM_E_READ_TOO_LONG,
 * GRIM_E_BAD_CANDIDATE, GRIM_E_BUSY (queue full), GRIM_E_NOMEM, or the CUDA
 * failure that stopped the server. */
int grim_server_submit(grim_server* s, const char* reads, const uint64_t* offsets,
                       const uint32_t* lens, uint32_t n_reads, const uint16_t* e,
                       const int32_t* cand, const uint64_t* cand_off, uint64_t* ticket);
/* Block until the request has completed (timeout_us < 0: no limit).
 * GRIM_OK when it has, GRIM_E_NOT_READY on timeout, GRIM_E_ARG for an
 * unknown ticket. */
int grim_server_wait(grim_server* s, uint64_t ticket, int64_t timeout_us);
/* Copy a completed request's pass list (sorted by read, then bin or
 * candidate order) into host buffers of `cap` records and release it.
 * `info` (may be NULL) receives its status, sizes and times.
 * GRIM_E_NOT_READY: still running.  GRIM_E_OVERFLOW: cap < info->n_out; the
 * request is kept, take again with more room.  A failed request returns its
 * error and is released. */
int grim_server_take(grim_server* s, uint64_t ticket, uint32_t* out_read, uint32_t* out_bin,
                     uint8_t* out_count, uint64_t cap, grim_request_info* info);
/* Cancel a request still in the queue: it completes at once with
 * GRIM_E_CANCELLED (grim_server_take returns that and releases it).
 * GRIM_E_NOT_READY: it is already on the device and will complete normally.
 * GRIM_E_ARG: unknown ticket, or the request has completed. */
int grim_server_cancel(grim_server* s, uint64_t ticket);
int grim_server_stats_get(grim_server* s, grim_server_stats* out);
/* Cancel queued requests, let batches on the device finish, stop, release.
 * No other call on the server may be running or follow. */
void grim_server_free(grim_server* s);

/* ---- helpers of the mapper around the filter (§GRIM-Filter, Fig. 5) ----- */

/* Reverse complement of reads (device pointers, grim_filter's layout): `out`
 * receives, at the same offsets, each read reversed with A<->T and C<->G in
 * either case (case kept; any other byte is moved unchanged).  The filter
 * reads the forward strand only; a mapper that tests both strands submits
 * these as further reads.  `out` must not overlap `reads`.  Asynchronous on
 * `stream`.  Errors: GRIM_E_ARG, GRIM_E_CUDA. */
int grim_reverse_complement(const char* reads, const uint64_t* offsets, const uint32_t* lens,
                            uint32_t n_reads, char* out, void* stream);

/* Bin whose core holds reference position `loc`: loc / B. */
uint64_t grim_loc_to_bin(const grim_index* idx, uint64_t loc);

/* Edit budget for an error rate num/den of read length L, rounded up
 * (Fig. 4 caption: the ceiling of read length times the error rate). */
uint32_t grim_edits_for_rate(uint32_t L, uint32_t num, uint32_t den);

/* ---- work counters of the last filter call ------------------------------ */
typedef struct {
  uint64_t n_reads;          /* reads in the call                                     */
  uint64_t n_records;        /* passing records found (may exceed the call's cap)     */
  uint64_t pairs;            /* (read, bin) pairs decided: reads x bins, or n_cand    */
  uint64_t tokens_executed;  /* all-bins mode: read tokens applied to (super-)bin tiles
                                (1024 wide up to q = 5, 256 at q = 6), counting padding
                                up to a 16-token block; stops early for a read once
                                every bin of the tile has failed                       */
  uint64_t survivors;        /* all-bins mode, coarse-then-exact: (read, super-bin)
                                pairs that passed the coarse pass (0 otherwise)       */
  uint64_t bit_tests_executed; /* all-bins mode: tokens_executed x (super-)bins per tile,
                                  except that a token of the one-word tail (1024-bin tiles,
                                  warp read switch: the last blocks of a read once every
                                  lane of the warp has at most one 32-bin word with a live
                                  bin) tests 256 of the tile's bins                       */
  uint32_t read_switch;        /* all-bins mode: GRIM_SWITCH_GROUP or GRIM_SWITCH_WARP, as
                                  chosen for the call (automatic: WARP when every read
                                  spans as many 16-token blocks and has the same miss
                                  budget D' = min(q*e, L-q+1)); 0 in candidate mode      */
  uint32_t all_bins_path;      /* all-bins mode: GRIM_PATH_TWO_LEVEL or GRIM_PATH_EXACT,
                                  the path the call took (after any fallback); 0 in
                                  candidate mode                                          */
} grim_filter_stats;

/* Counters of the calling thread's last successful grim_filter /
 * grim_filter_host / grim_filter_noalloc call. */
int grim_last_filter_stats(grim_filter_stats* out);

/* ---- per-kernel timing -------------------------------------------------- */
typedef struct {
  char name[32];      /* kernel name                                 */
  uint64_t launches;  /* launches timed since grim_profile(1)         */
  double total_ms;    /* summed CUDA-event time on the launch stream  */
} grim_kernel_time;

/* Turn per-kernel CUDA-event timing on (1) or off (0); turning it on clears
 * the counters.  Timing brackets each kernel launch with events recorded on
 * the launch stream. */
int grim_profile(int enable);

/* Copy up to `max` per-kernel totals into out; returns how many there are. */
int grim_profile_get(grim_kernel_time* out, int max);

#ifdef __cplusplus
}
#endif

#endif /* GRIM_H */
