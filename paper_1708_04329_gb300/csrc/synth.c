/*
 * Seeded synthetic inputs for the bin-level q-gram filter: genomes, reads with
 * planted edits, and per-read candidate bin lists.
 *
 * This file is the one input source shared by the CPU oracle and the CUDA
 * path.  It holds none of the filter's arithmetic (no tokens, no bit vectors,
 * no thresholds); it only draws bases and positions.
 *
 * Randomness is counter based, so the output does not depend on the number of
 * threads:
 *   - mix64() is the SplitMix64 output function (Steele, Lea and Flood,
 *     "Fast splittable pseudorandom number generators", OOPSLA 2014);
 *   - ctr(seed, stream, i) hashes a (seed, stream, index) triple through it
 *     twice, so every base / copy / read has its own independent draw;
 *   - per-object sequential draws (one read's edits, one read's candidate
 *     list) use a SplitMix64 sequence seeded by ctr().
 *
 * Workload shapes follow the paper's data (100 bp reads of a human-sized
 * genome, Table 1) without reproducing any record of it.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define GOLDEN 0x9E3779B97F4A7C15ull

enum {
  ST_BG = 1,        /* background base draws, 4 bases per draw            */
  ST_FAMLEN = 2,    /* family consensus lengths                           */
  ST_FAMSEQ = 3,    /* family consensus bases, 4 per draw                 */
  ST_GAP = 4,       /* gap before each repeat copy                        */
  ST_FAMPICK = 5,   /* family of each copy                                */
  ST_DIV = 6,       /* divergence of each copy                            */
  ST_SUB = 7,       /* per-base substitution draws inside copies          */
  ST_READ = 8,      /* per-read sequential stream                         */
  ST_READLEN = 9,   /* per-read length                                    */
  ST_CAND = 10,     /* per-read candidate stream                          */
};

static inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

static inline uint64_t ctr(uint64_t seed, uint64_t stream, uint64_t i) {
  return mix64(mix64(seed * GOLDEN + stream) + (i + 1) * GOLDEN);
}

typedef struct { uint64_t s; } seq64;
static inline uint64_t seq_next(seq64* g) { g->s += GOLDEN; return mix64(g->s); }
/* uniform integer in [0, n) by 64x64->128 multiply (Lemire); n > 0 */
static inline uint64_t seq_below(seq64* g, uint64_t n) {
  return (uint64_t)(((unsigned __int128)seq_next(g) * n) >> 64);
}
static inline double seq_u01(seq64* g) { return (double)(seq_next(g) >> 11) * 0x1.0p-53; }

static const char LETTER[4] = {'A', 'C', 'G', 'T'};

/* 16-bit thresholds for a base composition with GC fraction gc:
 * P(A)=P(T)=(1-gc)/2, P(C)=P(G)=gc/2. */
static void gc_thresholds(double gc, uint32_t th[3]) {
  double pa = (1.0 - gc) * 0.5, pc = gc * 0.5;
  th[0] = (uint32_t)(pa * 65536.0 + 0.5);
  th[1] = (uint32_t)((pa + pc) * 65536.0 + 0.5);
  th[2] = (uint32_t)((pa + 2.0 * pc) * 65536.0 + 0.5);
}
static inline uint8_t draw_base(uint32_t u16, const uint32_t th[3]) {
  return (uint8_t)((u16 >= th[0]) + (u16 >= th[1]) + (u16 >= th[2]));
}

/* Background of i.i.d. bases: base i uses 16 bits of ctr(seed, ST_BG, i/4). */
static void fill_iid(uint64_t seed, uint64_t stream, uint8_t* out, uint64_t n, double gc) {
  uint32_t th[3];
  gc_thresholds(gc, th);
  int64_t nw = (int64_t)((n + 3) / 4);
#pragma omp parallel for schedule(static)
  for (int64_t w = 0; w < nw; ++w) {
    uint64_t r = ctr(seed, stream, (uint64_t)w);
    for (int k = 0; k < 4; ++k) {
      uint64_t i = (uint64_t)w * 4 + k;
      if (i < n) out[i] = draw_base((uint32_t)(r >> (16 * k)) & 0xFFFF, th);
    }
  }
}

/*
 * Genome of n bases, written as ASCII 'A','C','G','T' into out[0..n).
 *
 * n_fam == 0: i.i.d. bases with GC fraction gc.
 * n_fam  > 0: repeat-rich genome.  n_fam family consensus sequences of length
 *   U[len_min, len_max] (i.i.d., same GC) are drawn; then the genome is laid
 *   out left to right as gap, copy, gap, copy, ...  Each copy is a whole copy
 *   of a uniformly chosen family, clipped only at the genome end, with every
 *   base independently substituted (to one of the 3 other bases) with
 *   probability d ~ U[div_min, div_max] drawn per copy.  Gaps are i.i.d.
 *   background of length U[0, 2*g) with g chosen so that the expected repeat
 *   fraction is repeat_frac.  Copies therefore never overlap.
 *
 * Returns the number of copies placed, or -1 on bad arguments / no memory.
 */
int64_t synth_genome(uint64_t seed, uint64_t n, double gc, uint32_t n_fam, uint32_t len_min,
                     uint32_t len_max, double div_min, double div_max, double repeat_frac,
                     uint8_t* out) {
  if (!out || gc < 0 || gc > 1) return -1;
  uint8_t* codes = out; /* generate 2-bit codes in place, convert to ASCII at the end */
  fill_iid(seed, ST_BG, codes, n, gc);
  int64_t n_copies = 0;
  if (n_fam > 0) {
    if (len_min == 0 || len_max < len_min || len_max > 65535 || repeat_frac <= 0 ||
        repeat_frac >= 1 || div_max >= 1.0)
      return -1;
    uint64_t* fam_off = (uint64_t*)malloc(sizeof(uint64_t) * (n_fam + 1));
    uint32_t* fam_len = (uint32_t*)malloc(sizeof(uint32_t) * n_fam);
    if (!fam_off || !fam_len) { free(fam_off); free(fam_len); return -1; }
    fam_off[0] = 0;
    for (uint32_t f = 0; f < n_fam; ++f) {
      seq64 g = {ctr(seed, ST_FAMLEN, f)};
      fam_len[f] = len_min + (uint32_t)seq_below(&g, (uint64_t)(len_max - len_min + 1));
      fam_off[f + 1] = fam_off[f] + fam_len[f];
    }
    uint8_t* fam_seq = (uint8_t*)malloc(fam_off[n_fam] + 4);
    if (!fam_seq) { free(fam_off); free(fam_len); return -1; }
    fill_iid(seed, ST_FAMSEQ, fam_seq, fam_off[n_fam], gc);
    double mean_copy = (double)fam_off[n_fam] / n_fam;
    double mean_gap = mean_copy * (1.0 - repeat_frac) / repeat_frac;

    /* lay out copies sequentially (cheap: ~n / mean_copy copies) */
    uint64_t cap = 1024;
    uint64_t* c_pos = (uint64_t*)malloc(cap * sizeof(uint64_t));
    uint32_t* c_len = (uint32_t*)malloc(cap * sizeof(uint32_t));
    uint32_t* c_fam = (uint32_t*)malloc(cap * sizeof(uint32_t));
    uint64_t pos = 0, c = 0;
    while (c_pos && c_len && c_fam) {
      seq64 gg = {ctr(seed, ST_GAP, c)};
      uint64_t gap = (uint64_t)(seq_u01(&gg) * 2.0 * mean_gap);
      pos += gap;
      if (pos >= n) break;
      seq64 gf = {ctr(seed, ST_FAMPICK, c)};
      uint32_t f = (uint32_t)seq_below(&gf, n_fam);
      uint64_t len = fam_len[f];
      if (pos + len > n) len = n - pos;
      if (c == cap) {
        cap *= 2;
        uint64_t* p1 = (uint64_t*)realloc(c_pos, cap * sizeof(uint64_t));
        uint32_t* p2 = (uint32_t*)realloc(c_len, cap * sizeof(uint32_t));
        uint32_t* p3 = (uint32_t*)realloc(c_fam, cap * sizeof(uint32_t));
        if (p1) c_pos = p1;
        if (p2) c_len = p2;
        if (p3) c_fam = p3;
        if (!p1 || !p2 || !p3) { n_copies = -1; break; }
      }
      c_pos[c] = pos;
      c_len[c] = (uint32_t)len;
      c_fam[c] = f;
      ++c;
      pos += len;
    }
    if (!c_pos || !c_len || !c_fam) n_copies = -1;
    if (n_copies == 0) {
      n_copies = (int64_t)c;
#pragma omp parallel for schedule(dynamic, 64)
      for (int64_t k = 0; k < n_copies; ++k) {
        seq64 gd = {ctr(seed, ST_DIV, (uint64_t)k)};
        double d = div_min + (div_max - div_min) * seq_u01(&gd);
        uint64_t dth = (uint64_t)(d * 18446744073709551616.0); /* d * 2^64 */
        const uint8_t* src = fam_seq + fam_off[c_fam[k]];
        uint8_t* dst = codes + c_pos[k];
        for (uint32_t i = 0; i < c_len[k]; ++i) {
          uint64_t u = ctr(seed, ST_SUB, ((uint64_t)k << 16) | i);
          uint8_t b = src[i];
          if ((u >> 8) < (dth >> 8)) b = (uint8_t)((b + 1 + (u & 0xFF) % 3) & 3);
          dst[i] = b;
        }
      }
    }
    free(c_pos); free(c_len); free(c_fam);
    free(fam_seq); free(fam_off); free(fam_len);
    if (n_copies < 0) return -1;
  }
  int64_t nn = (int64_t)n;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < nn; ++i) out[i] = (uint8_t)LETTER[codes[i] & 3];
  return n_copies;
}

/*
 * Per-read lengths.  Read r has length lens_choice[k] with probability
 * probs[k] (k < n_choice), drawn from ctr(seed, ST_READLEN, r).
 */
void synth_read_lengths(uint64_t seed, uint64_t n_reads, uint32_t n_choice,
                        const uint32_t* lens_choice, const double* probs, uint32_t* lens_out) {
  int64_t nr = (int64_t)n_reads;
#pragma omp parallel for schedule(static)
  for (int64_t r = 0; r < nr; ++r) {
    double u = (double)(ctr(seed, ST_READLEN, (uint64_t)r) >> 11) * 0x1.0p-53;
    double acc = 0.0;
    uint32_t L = lens_choice[n_choice - 1];
    for (uint32_t k = 0; k + 1 < n_choice; ++k) {
      acc += probs[k];
      if (u < acc) { L = lens_choice[k]; break; }
    }
    lens_out[r] = L;
  }
}

/*
 * Reads with planted edits.
 *
 * For read r (length lens[r], already drawn, offsets[r] its start in
 * reads_out):
 *   - its edit budget e_r is e_fixed, or, when e_den > 0, uniform in
 *     {0, ..., floor(lens[r] * e_num / e_den)};
 *   - its number of planted edits k is uniform in {0..kmax_fixed}, or in
 *     {0..e_r} when kmax_fixed < 0;
 *   - its source start s is uniform in [0, n - L - k_cap], k_cap the largest
 *     k it could have drawn, so the source plus all deletions stay inside;
 *   - k edits are applied one after another to the source run
 *     genome[s, s + L + k) at positions uniform in [0, L): a substitution
 *     (prob p_sub) to one of the 3 other bases, a 1-base insertion of a
 *     random base (prob p_ins), or a 1-base deletion (the rest);
 *   - the read is the first L bases of the edited run.
 * true_pos[r] = s, n_edits[r] = k, e_out[r] = e_r.
 * Returns 0, or -1 if some read does not fit in the genome.
 */
int synth_reads(uint64_t seed, const uint8_t* genome, uint64_t n, uint64_t n_reads,
                const uint32_t* lens, const uint64_t* offsets, uint32_t e_fixed, uint32_t e_num,
                uint32_t e_den, int32_t kmax_fixed, double p_sub, double p_ins, uint8_t* reads_out,
                uint64_t* true_pos, uint16_t* n_edits, uint16_t* e_out) {
  int bad = 0;
  int64_t nr = (int64_t)n_reads;
#pragma omp parallel for schedule(dynamic, 256) reduction(| : bad)
  for (int64_t r = 0; r < nr; ++r) {
    uint32_t L = lens[r];
    uint32_t e = e_den ? (uint32_t)(((uint64_t)L * e_num) / e_den) : e_fixed;
    seq64 g = {ctr(seed, ST_READ, (uint64_t)r)};
    if (e_den) e = (uint32_t)seq_below(&g, (uint64_t)e + 1);
    uint32_t kcap = kmax_fixed >= 0 ? (uint32_t)kmax_fixed : e;
    uint32_t k = (uint32_t)seq_below(&g, (uint64_t)kcap + 1);
    if ((uint64_t)L + kcap >= n) { bad = 1; continue; }
    uint64_t s = seq_below(&g, n - L - kcap + 1); /* uniform in [0, n-L-kcap] */
    /* edited run lives in a small local buffer: length <= L + 2k */
    uint8_t buf[4096 + 256];
    uint32_t blen = L + k;
    if (blen + k > sizeof(buf)) { bad = 1; continue; }
    memcpy(buf, genome + s, blen);
    for (uint32_t j = 0; j < k; ++j) {
      double t = seq_u01(&g);
      uint32_t p = (uint32_t)seq_below(&g, L);
      if (t < p_sub) {
        uint8_t cur = buf[p];
        int ci = cur == 'A' ? 0 : cur == 'C' ? 1 : cur == 'G' ? 2 : 3;
        buf[p] = (uint8_t)LETTER[(ci + 1 + (int)seq_below(&g, 3)) & 3];
      } else if (t < p_sub + p_ins) {
        memmove(buf + p + 1, buf + p, blen - p);
        buf[p] = (uint8_t)LETTER[seq_below(&g, 4)];
        ++blen;
      } else {
        memmove(buf + p, buf + p + 1, blen - p - 1);
        --blen;
      }
    }
    memcpy(reads_out + offsets[r], buf, L);
    true_pos[r] = s;
    n_edits[r] = (uint16_t)k;
    e_out[r] = (uint16_t)e;
  }
  return bad ? -1 : 0;
}

/*
 * Candidate-list sizes: count_r = min(clip, max(1, round(exp(ln(median) +
 * sigma * Z)))) with Z standard normal (Box-Muller), further capped at
 * num_bins so every list can hold distinct bins.
 */
void synth_candidate_counts(uint64_t seed, uint64_t n_reads, uint64_t num_bins, double median,
                            double sigma, uint32_t clip, uint32_t* counts) {
  int64_t nr = (int64_t)n_reads;
#pragma omp parallel for schedule(static)
  for (int64_t r = 0; r < nr; ++r) {
    seq64 g = {ctr(seed, ST_CAND, (uint64_t)r)};
    double u1 = seq_u01(&g), u2 = seq_u01(&g);
    double z = sqrt(-2.0 * log(1.0 - u1)) * cos(6.283185307179586 * u2);
    double v = round(exp(log(median) + sigma * z));
    uint64_t c = v < 1.0 ? 1 : (v > (double)clip ? clip : (uint64_t)v);
    if (c > num_bins) c = num_bins;
    counts[r] = (uint32_t)c;
  }
}

static int cmp_i32(const void* a, const void* b) {
  int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
  return (x > y) - (x < y);
}

/*
 * Candidate lists (CSR, offsets from the counts above): list r holds
 * true_bin[r] plus count_r - 1 distinct other bins drawn uniformly from
 * [0, num_bins), sorted ascending.
 */
int synth_candidates(uint64_t seed, uint64_t n_reads, const int32_t* true_bin, uint64_t num_bins,
                     const uint64_t* off, int32_t* cand) {
  int bad = 0;
  int64_t nr = (int64_t)n_reads;
#pragma omp parallel for schedule(dynamic, 64) reduction(| : bad)
  for (int64_t r = 0; r < nr; ++r) {
    seq64 g = {ctr(seed, ST_CAND, (uint64_t)r) ^ 0x5bd1e995ull};
    uint64_t c = off[r + 1] - off[r];
    int32_t* lst = cand + off[r];
    if (c == 0) continue;
    if ((uint64_t)true_bin[r] >= num_bins || c > num_bins) { bad = 1; continue; }
    if (c * 2 > num_bins) {
      /* dense: partial Fisher-Yates over all bins, true bin forced first */
      int32_t* all = (int32_t*)malloc(num_bins * sizeof(int32_t));
      if (!all) { bad = 1; continue; }
      for (uint64_t i = 0; i < num_bins; ++i) all[i] = (int32_t)i;
      all[true_bin[r]] = 0;
      all[0] = true_bin[r];
      for (uint64_t i = 1; i < c; ++i) {
        uint64_t j = i + seq_below(&g, num_bins - i);
        int32_t t = all[i]; all[i] = all[j]; all[j] = t;
      }
      memcpy(lst, all, c * sizeof(int32_t));
      free(all);
      qsort(lst, c, sizeof(int32_t), cmp_i32);
      continue;
    }
    /* sparse: draw, sort, drop duplicates, redraw the shortfall */
    lst[0] = true_bin[r];
    uint64_t have = 1;
    while (have < c) {
      for (uint64_t i = have; i < c; ++i) lst[i] = (int32_t)seq_below(&g, num_bins);
      qsort(lst, c, sizeof(int32_t), cmp_i32);
      uint64_t w = 1;
      for (uint64_t i = 1; i < c; ++i)
        if (lst[i] != lst[w - 1]) lst[w++] = lst[i];
      have = w;
    }
  }
  return bad ? -1 : 0;
}
