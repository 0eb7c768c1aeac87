"""Seeded synthetic inputs (genomes, reads, candidate lists).

This module is the only input source that the CPU oracle and the CUDA path
share.  It draws bases and positions and nothing else: it computes no tokens,
bit vectors, counts or thresholds.  The heavy lifting is ``csrc/synth.c``
(counter-based SplitMix64 draws, so results do not depend on thread count).

Workload recipes mirror the paper's evaluation data (100 bp reads against a
~3.1 Gbp human-like reference, Table 1 and the methodology section) with
synthetic stand-ins; no record of the real data sets is reproduced.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass, field

import numpy as np

from . import _build

_lib = None


def _load():
    global _lib
    if _lib is None:
        path = _build.build_synth()
        lib = C.CDLL(str(path))
        u64, u32, i32, dbl, vp = C.c_uint64, C.c_uint32, C.c_int32, C.c_double, C.c_void_p
        lib.synth_genome.restype = C.c_int64
        lib.synth_genome.argtypes = [u64, u64, dbl, u32, u32, u32, dbl, dbl, dbl, vp]
        lib.synth_read_lengths.restype = None
        lib.synth_read_lengths.argtypes = [u64, u64, u32, vp, vp, vp]
        lib.synth_reads.restype = C.c_int
        lib.synth_reads.argtypes = [u64, vp, u64, u64, vp, vp, u32, u32, u32, i32, dbl, dbl,
                                    vp, vp, vp, vp]
        lib.synth_candidate_counts.restype = None
        lib.synth_candidate_counts.argtypes = [u64, u64, u64, dbl, dbl, u32, vp]
        lib.synth_candidates.restype = C.c_int
        lib.synth_candidates.argtypes = [u64, u64, vp, u64, vp, vp]
        _lib = lib
    return _lib


def _p(a: np.ndarray) -> int:
    return a.ctypes.data


def genome(n: int, seed: int, gc: float = 0.5, families: int = 0,
           fam_len: tuple[int, int] = (300, 6000), divergence: tuple[float, float] = (0.05, 0.20),
           repeat_frac: float = 0.5) -> np.ndarray:
    """ASCII genome (uint8 'A','C','G','T') of ``n`` bases.

    ``families == 0``: i.i.d. bases with GC fraction ``gc``.  Otherwise about
    ``repeat_frac`` of the genome is whole copies of ``families`` consensus
    sequences (lengths uniform in ``fam_len``), each copy with uniform
    substitutions at a per-copy rate uniform in ``divergence``.
    """
    out = np.empty(n, dtype=np.uint8)
    rc = _load().synth_genome(seed, n, gc, families, fam_len[0], fam_len[1], divergence[0],
                              divergence[1], repeat_frac, _p(out))
    if rc < 0:
        raise ValueError("synth_genome: bad arguments or out of memory")
    return out


@dataclass
class ReadSet:
    """Reads concatenated in ``seq`` (ASCII), read r = seq[offsets[r]:offsets[r]+lens[r]]."""

    seq: np.ndarray          # uint8, all reads back to back
    offsets: np.ndarray      # uint64 [n]
    lens: np.ndarray         # uint32 [n]
    e: np.ndarray            # uint16 [n], per-read absolute edit budget
    true_pos: np.ndarray     # uint64 [n], source start in the genome
    n_edits: np.ndarray      # uint16 [n], planted edits (<= e for planted workloads)
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.lens.shape[0])

    def read(self, r: int) -> bytes:
        o = int(self.offsets[r])
        return self.seq[o:o + int(self.lens[r])].tobytes()

    def subset(self, idx) -> "ReadSet":
        """Reads ``idx`` (in that order), repacked back to back."""
        idx = np.asarray(idx, dtype=np.int64)
        lens = self.lens[idx].copy()
        offs = np.zeros(len(idx), dtype=np.uint64)
        if len(idx) > 1:
            offs[1:] = np.cumsum(lens[:-1], dtype=np.uint64)
        seq = np.empty(int(lens.sum()), dtype=np.uint8)
        for j, r in enumerate(idx):
            o = int(self.offsets[r])
            seq[int(offs[j]):int(offs[j]) + int(lens[j])] = self.seq[o:o + int(lens[j])]
        return ReadSet(seq, offs, lens, self.e[idx].copy(), self.true_pos[idx].copy(),
                       self.n_edits[idx].copy(), dict(self.meta))


def reads(g: np.ndarray, n_reads: int, seed: int, lengths=(100,), probs=(1.0,), e: int = 5,
          e_frac: tuple[int, int] | None = None, max_edits: int | None = 5,
          p_sub: float = 0.70, p_ins: float = 0.15) -> ReadSet:
    """Reads sampled from genome ``g`` with planted edits.

    Read length is drawn from ``lengths`` with ``probs``.  The edit budget is
    ``e`` for every read, or, with ``e_frac=(num, den)``, uniform in
    ``{0..floor(L*num/den)}`` per read.  The number of planted edits is
    uniform in ``{0..max_edits}`` (``None``: in ``{0..e_r}``).  Each edit is a
    substitution (``p_sub``), a 1-base insertion (``p_ins``) or a 1-base
    deletion, at a uniform position; the read is the first L bases of the
    edited source run.
    """
    lib = _load()
    lens_choice = np.asarray(lengths, dtype=np.uint32)
    pr = np.asarray(probs, dtype=np.float64)
    lens = np.empty(n_reads, dtype=np.uint32)
    if n_reads:
        lib.synth_read_lengths(seed, n_reads, len(lens_choice), _p(lens_choice), _p(pr), _p(lens))
    offs = np.zeros(n_reads, dtype=np.uint64)
    if n_reads > 1:
        offs[1:] = np.cumsum(lens[:-1], dtype=np.uint64)
    seq = np.empty(int(lens.sum(dtype=np.uint64)), dtype=np.uint8)
    pos = np.empty(n_reads, dtype=np.uint64)
    ned = np.empty(n_reads, dtype=np.uint16)
    ee = np.empty(n_reads, dtype=np.uint16)
    num, den = e_frac if e_frac else (0, 0)
    kmax = -1 if max_edits is None else int(max_edits)
    if n_reads:
        rc = lib.synth_reads(seed, _p(g), len(g), n_reads, _p(lens), _p(offs), e, num, den, kmax,
                             p_sub, p_ins, _p(seq), _p(pos), _p(ned), _p(ee))
        if rc != 0:
            raise ValueError("synth_reads: a read does not fit in the genome")
    return ReadSet(seq, offs, lens, ee, pos, ned)


def candidates(true_bin: np.ndarray, num_bins: int, seed: int, median: float = 200.0,
               sigma: float = 1.0, clip: int = 20000) -> tuple[np.ndarray, np.ndarray]:
    """Per-read candidate bin lists in CSR form ``(off uint64[n+1], cand int32[off[-1]])``.

    List r has min(clip, max(1, round(LogNormal(ln median, sigma)))) entries
    (capped at ``num_bins``): ``true_bin[r]`` plus distinct uniform bins,
    sorted ascending.
    """
    lib = _load()
    tb = np.ascontiguousarray(true_bin, dtype=np.int32)
    n = len(tb)
    counts = np.empty(n, dtype=np.uint32)
    if n:
        lib.synth_candidate_counts(seed, n, num_bins, median, sigma, clip, _p(counts))
    off = np.zeros(n + 1, dtype=np.uint64)
    np.cumsum(counts, dtype=np.uint64, out=off[1:])
    cand = np.empty(int(off[-1]), dtype=np.int32)
    if n:
        rc = lib.synth_candidates(seed, n, _p(tb), num_bins, _p(off), _p(cand))
        if rc != 0:
            raise ValueError("synth_candidates: bad true bin or list longer than num_bins")
    return off, cand


# ---------------------------------------------------------------------------
# Workload recipes.  Each returns a dict with the genome, index parameters,
# reads and (where the workload has them) candidate lists.
# ---------------------------------------------------------------------------

HUMAN_N = 3_100_000_000


def tiny_plain(n_reads: int = 2000) -> dict:
    """1 Mbp uniform i.i.d. genome (seed 1); B=200, ext=99, q=5 (5,000 bins);
    2,000 reads of L=100 with 0-5 planted edits (70/15/15), e=5; all bins."""
    g = genome(1_000_000, seed=1, gc=0.5)
    rs = reads(g, n_reads, seed=11, lengths=(100,), e=5, max_edits=5)
    return dict(name="tiny_plain", genome=g, B=200, q=5, max_read_len=100, reads=rs)


def human_genome(n: int = HUMAN_N, seed: int = 2) -> np.ndarray:
    """41% GC genome, ~50% whole copies of 500 repeat families (consensus 300-6,000 bp,
    copies diverged by 5-20% uniform substitutions), the rest i.i.d."""
    return genome(n, seed=seed, gc=0.41, families=500, fam_len=(300, 6000),
                  divergence=(0.05, 0.20), repeat_frac=0.5)


def human_exhaustive(n_reads: int = 1_000_000, n: int = HUMAN_N, g: np.ndarray | None = None) -> dict:
    """Human-scale exhaustive workload: B=200, q=5, 1M reads of L=100, 0-5 edits, e=5."""
    g = human_genome(n) if g is None else g
    rs = reads(g, n_reads, seed=3, lengths=(100,), e=5, max_edits=5)
    return dict(name="human_exhaustive", genome=g, B=200, q=5, max_read_len=100, reads=rs)


def ragged_candidates(n_reads: int = 4_000_000, n: int = HUMAN_N, g: np.ndarray | None = None,
                      B: int = 200) -> dict:
    """Ragged candidate workload: L in {100,150,250} w.p. .5/.3/.2, e_r uniform in
    {0..floor(0.05 L)} with <= e_r planted edits; LogNormal(ln 200, 1.0) candidate
    counts clipped at 20,000, true bin plus distinct random bins.  Index built with
    max_read_len=250."""
    g = human_genome(n) if g is None else g
    rs = reads(g, n_reads, seed=4, lengths=(100, 150, 250), probs=(0.5, 0.3, 0.2), e_frac=(5, 100),
               max_edits=None)
    num_bins = (len(g) + B - 1) // B
    off, cand = candidates((rs.true_pos // B).astype(np.int32), num_bins, seed=4)
    return dict(name="ragged_candidates", genome=g, B=B, q=5, max_read_len=250, reads=rs,
                cand_off=off, cand=cand)


def finer_index(n_reads: int = 1_000_000, n: int = HUMAN_N, g: np.ndarray | None = None) -> dict:
    """Finer index: q=6, B=100, 1M reads of L=150 with 0-7 planted edits, e=7."""
    g = human_genome(n) if g is None else g
    rs = reads(g, n_reads, seed=5, lengths=(150,), e=7, max_edits=7)
    num_bins = (len(g) + 100 - 1) // 100
    off, cand = candidates((rs.true_pos // 100).astype(np.int32), num_bins, seed=5)
    return dict(name="finer_index", genome=g, B=100, q=6, max_read_len=150, reads=rs,
                cand_off=off, cand=cand)


def serving(pool_reads: int = 2_000_000, n: int = HUMAN_N, g: np.ndarray | None = None) -> dict:
    """Serving workload: the human-scale genome (B=200, q=5, index built with
    max_read_len=250) and a pool of reads with L in {100,150,250} w.p.
    .5/.3/.2 and e_r uniform in {0..floor(0.05 L)} (seed 6), from which the
    requests of a trace are cut."""
    g = human_genome(n) if g is None else g
    rs = reads(g, pool_reads, seed=6, lengths=(100, 150, 250), probs=(0.5, 0.3, 0.2),
               e_frac=(5, 100), max_edits=None)
    return dict(name="serving", genome=g, B=200, q=5, max_read_len=250, reads=rs)


def request_trace(duration_s: float, rate: float, pool: int, seed: int = 6,
                  max_batch: int = 8192) -> dict:
    """Poisson arrivals of read batches: exponential gaps of mean 1/rate
    seconds over ``duration_s``; batch sizes log-uniform in [1, max_batch]
    (floor(exp(U(0, ln(max_batch+1))))); each batch is the reads
    [start, start+size) of a pool of ``pool`` reads, start uniform."""
    rng = np.random.default_rng(seed)
    n = max(1, int(duration_s * rate * 1.5) + 16)
    t = np.cumsum(rng.exponential(1.0 / rate, n))
    t = t[t < duration_s]
    size = np.floor(np.exp(rng.uniform(0.0, np.log(max_batch + 1), len(t)))).astype(np.int64)
    size = np.clip(size, 1, max_batch)
    start = (rng.random(len(t)) * (pool - size + 1)).astype(np.int64)
    return dict(t=t, size=size, start=start)
