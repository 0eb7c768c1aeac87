/*
 * CPU oracle for the GRIM-Filter bin-level q-gram filter.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file: only the tests, the package smoke check and the benchmark's
 * CPU-baseline leg use it.  It shares no code, header, table or helper with
 * the CUDA library.
 *
 * It computes the plain definition, without bit slicing, tiling or early exit:
 *
 *   code(A)=0 code(C)=1 code(G)=2 code(T)=3 (case folded), anything else is
 *   not a base.  A token (the paper's "token" of n bases, written q here) is
 *   the base-4 number of q consecutive bases, first base most significant
 *   (§GRIM-Filter, Fig. 2: rows indexed by the token value).
 *
 *   Bins (§GRIM-Filter, Fig. 2): bin b covers core [b*B, b*B+B) and is
 *   extended by ext = L_max-1 bases so a read starting in the core fits
 *   wholly inside it; window W_b = ref[b*B, min(b*B+B+ext, N)).
 *   numBins = ceil(N/B).
 *
 *   Bit vector (§GRIM-Filter; 4^q bits per bin as the 4^5 = 1024 sizing in
 *   §Parameter Evaluation Results fixes): bit t of bin b is 1 iff token t
 *   occurs as a q-gram lying wholly inside W_b with only A/C/G/T bases.
 *
 *   Filter (§GRIM-Filter steps 1-3, Fig. 5): the read's L-q+1 tokens are
 *   extracted; the existence bits of all of them are summed (every position
 *   counts, repeats included; a token with a non-base character adds 0);
 *   the sum is compared with T = (L-q+1) - q*e (the threshold of Fig. 3:
 *   each edit can spoil at most q tokens) and the bin passes iff
 *   sum >= T.  Passing (read, bin, sum) records are emitted read by read,
 *   bins ascending (all-bins mode) or in the given candidate order.
 *
 * Error codes mirror the library's: -1 bad argument, -4 read shorter than
 * q, -5 read longer than max_read_len or with more than 255 tokens,
 * -6 candidate bin out of range, -2 out of memory.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_E_ARG (-1)
#define ORC_E_NOMEM (-2)
#define ORC_E_SHORT (-4)
#define ORC_E_LONG (-5)
#define ORC_E_CAND (-6)

/* base code, or -1 for a character that is not A/C/G/T in either case */
static int base_code(unsigned char c) {
  switch (c) {
    case 'A': case 'a': return 0;
    case 'C': case 'c': return 1;
    case 'G': case 'g': return 2;
    case 'T': case 't': return 3;
    default: return -1;
  }
}

/* token value of s[0..q), or -1 if one of its characters is not a base */
static int64_t token_of(const unsigned char* s, uint32_t q) {
  int64_t v = 0;
  for (uint32_t i = 0; i < q; ++i) {
    int c = base_code(s[i]);
    if (c < 0) return -1;
    v = v * 4 + c;
  }
  return v;
}

uint64_t oracle_num_bins(uint64_t n, uint32_t B) { return B ? (n + B - 1) / B : 0; }

/* bytes of one bin's bit vector: 4^q bits, at least one byte */
uint64_t oracle_vector_bytes(uint32_t q) {
  uint64_t bits = 1ull << (2 * q);
  return bits < 8 ? 1 : bits / 8;
}

/*
 * Bit vectors of all bins, bin-major: bin b's 4^q bits start at byte
 * b*oracle_vector_bytes(q); token t is bit (t % 8) of byte t / 8.
 * out must hold numBins * oracle_vector_bytes(q) bytes.
 */
int oracle_bin_vectors(const unsigned char* ref, uint64_t n, uint32_t B, uint32_t ext, uint32_t q,
                       unsigned char* out) {
  if (!ref || !out || B == 0 || q == 0 || q > 8) return ORC_E_ARG;
  uint64_t nb = oracle_num_bins(n, B), vb = oracle_vector_bytes(q);
  int64_t nbi = (int64_t)nb;
#pragma omp parallel for schedule(dynamic, 1024)
  for (int64_t b = 0; b < nbi; ++b) {
    unsigned char* v = out + (uint64_t)b * vb;
    memset(v, 0, vb);
    uint64_t lo = (uint64_t)b * B;
    uint64_t hi = lo + B + ext;
    if (hi > n) hi = n;
    /* every q-gram start p with p + q <= hi */
    for (uint64_t p = lo; p + q <= hi; ++p) {
      int64_t t = token_of(ref + p, q);
      if (t >= 0) v[t / 8] |= (unsigned char)(1u << (t % 8));
    }
  }
  return 0;
}

/* tokens of one read: out[j] = token_of(read + j) for j < L-q+1 (-1 = not counted) */
int oracle_read_tokens(const unsigned char* read, uint32_t L, uint32_t q, int64_t* out) {
  if (L < q) return ORC_E_SHORT;
  for (uint32_t j = 0; j + q <= L; ++j) out[j] = token_of(read + j, q);
  return 0;
}

static int vec_bit(const unsigned char* v, int64_t t) { return (v[t / 8] >> (t % 8)) & 1; }

typedef struct {
  uint32_t* read;
  uint32_t* bin;
  uint8_t* count;
  uint64_t n, cap;
} rec_list;

static int rec_push(rec_list* l, uint32_t r, uint32_t b, uint8_t c) {
  if (l->n == l->cap) {
    uint64_t nc = l->cap ? l->cap * 2 : 16;
    uint32_t* a = (uint32_t*)realloc(l->read, nc * sizeof(uint32_t));
    if (a) l->read = a;
    uint32_t* bb = (uint32_t*)realloc(l->bin, nc * sizeof(uint32_t));
    if (bb) l->bin = bb;
    uint8_t* cc = (uint8_t*)realloc(l->count, nc);
    if (cc) l->count = cc;
    if (!a || !bb || !cc) return ORC_E_NOMEM;
    l->cap = nc;
  }
  l->read[l->n] = r;
  l->bin[l->n] = b;
  l->count[l->n] = c;
  l->n++;
  return 0;
}

/* result handed back to the caller; free with oracle_free */
typedef struct {
  uint32_t* read;
  uint32_t* bin;
  uint8_t* count;
  uint64_t n;
} oracle_out;

void oracle_free(oracle_out* o) {
  if (!o) return;
  free(o->read);
  free(o->bin);
  free(o->count);
  o->read = o->bin = NULL;
  o->count = NULL;
  o->n = 0;
}

/*
 * The filter.
 *   vecs, num_bins, q : bit vectors from oracle_bin_vectors
 *   reads/offsets/lens/n_reads : read r is reads[offsets[r] .. +lens[r])
 *   e : per-read absolute edit budget
 *   cand/cand_off : CSR candidate lists (cand_off has n_reads+1 entries);
 *                   cand == NULL means every bin in [bin_lo, bin_hi)
 *   max_read_len : reads longer than this are an error (as in the library)
 * On success returns 0 and fills *out with the passing records.
 */
int oracle_filter(const unsigned char* vecs, uint64_t num_bins, uint32_t q,
                  const unsigned char* reads, const uint64_t* offsets, const uint32_t* lens,
                  uint64_t n_reads, const uint16_t* e, const int32_t* cand,
                  const uint64_t* cand_off, uint64_t bin_lo, uint64_t bin_hi,
                  uint32_t max_read_len, oracle_out* out) {
  if (!out || (n_reads && (!vecs || !reads || !offsets || !lens || !e))) return ORC_E_ARG;
  if (cand && !cand_off) return ORC_E_ARG;
  if (!cand && (bin_hi > num_bins || bin_lo > bin_hi)) return ORC_E_ARG;
  memset(out, 0, sizeof(*out));
  uint64_t vb = oracle_vector_bytes(q);
  /* argument errors first; when several kinds occur, short reads are
   * reported before long reads, and both before bad candidates */
  for (uint64_t r = 0; r < n_reads; ++r)
    if (lens[r] < q) return ORC_E_SHORT;
  for (uint64_t r = 0; r < n_reads; ++r)
    if (lens[r] > max_read_len || lens[r] - q + 1 > 255) return ORC_E_LONG;
  if (cand) {
    for (uint64_t k = 0; k < cand_off[n_reads]; ++k)
      if (cand[k] < 0 || (uint64_t)cand[k] >= num_bins) return ORC_E_CAND;
  }
  rec_list* per = (rec_list*)calloc(n_reads ? n_reads : 1, sizeof(rec_list));
  if (!per) return ORC_E_NOMEM;
  int err = 0;
  int64_t nr = (int64_t)n_reads;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : err)
  for (int64_t r = 0; r < nr; ++r) {
    uint32_t L = lens[r];
    uint32_t ntok = L - q + 1;
    int64_t tok[256];
    oracle_read_tokens(reads + offsets[r], L, q, tok);
    int64_t T = (int64_t)ntok - (int64_t)q * (int64_t)e[r];
    uint64_t k0, k1;
    if (cand) { k0 = cand_off[r]; k1 = cand_off[r + 1]; }
    else { k0 = bin_lo; k1 = bin_hi; }
    for (uint64_t k = k0; k < k1; ++k) {
      uint64_t b = cand ? (uint64_t)cand[k] : k;
      const unsigned char* v = vecs + b * vb;
      int64_t sum = 0;
      for (uint32_t j = 0; j < ntok; ++j)
        if (tok[j] >= 0) sum += vec_bit(v, tok[j]);
      if (sum >= T) err |= rec_push(&per[r], (uint32_t)r, (uint32_t)b, (uint8_t)sum) != 0;
    }
  }
  uint64_t total = 0;
  for (uint64_t r = 0; r < n_reads; ++r) total += per[r].n;
  if (!err) {
    out->read = (uint32_t*)malloc((total ? total : 1) * sizeof(uint32_t));
    out->bin = (uint32_t*)malloc((total ? total : 1) * sizeof(uint32_t));
    out->count = (uint8_t*)malloc(total ? total : 1);
    if (!out->read || !out->bin || !out->count) err = 1;
  }
  if (!err) {
    uint64_t w = 0;
    for (uint64_t r = 0; r < n_reads; ++r) {
      memcpy(out->read + w, per[r].read, per[r].n * sizeof(uint32_t));
      memcpy(out->bin + w, per[r].bin, per[r].n * sizeof(uint32_t));
      memcpy(out->count + w, per[r].count, per[r].n);
      w += per[r].n;
    }
    out->n = total;
  }
  for (uint64_t r = 0; r < n_reads; ++r) {
    free(per[r].read);
    free(per[r].bin);
    free(per[r].count);
  }
  free(per);
  if (err) {
    oracle_free(out);
    return ORC_E_NOMEM;
  }
  return 0;
}

int oracle_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Sets the OpenMP thread count of the oracle's parallel loops (n >= 1). */
void oracle_set_threads(int n) {
#ifdef _OPENMP
  if (n >= 1) omp_set_num_threads(n);
#else
  (void)n;
#endif
}
