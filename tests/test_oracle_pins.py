"""Pins for the CPU oracle: things the paper and plain mathematics fix.

None of these re-types the oracle's own formula.  They check it against
(a) hand-worked fixtures, (b) an independent brute force that uses substring
search instead of bit vectors and token codes, (c) closed forms the paper
prints, and (d) invariants of the method (the q-gram lemma behind Fig. 3's
threshold, monotonicity in e, T <= 0, relabelling of the alphabet).
"""
import numpy as np
import pytest

import oracle
from oracle import bruteforce
from tests.conftest import Reads, load_fixture, random_case


def _as_triples(res):
    r, b, c = res
    return [(int(x), int(y), int(z)) for x, y, z in zip(r, b, c)]


def _run_oracle(ref: str, B: int, max_read_len: int, q: int, reads: list[str], e: list[int],
                cands=None):
    idx = oracle.bin_vectors(np.frombuffer(ref.encode(), dtype=np.uint8), B, q, max_read_len)
    rs = Reads(reads, e)
    if cands is None:
        return _as_triples(oracle.filter(idx, rs))
    off = np.zeros(len(cands) + 1, dtype=np.uint64)
    off[1:] = np.cumsum([len(c) for c in cands])
    flat = np.array([b for c in cands for b in c], dtype=np.int32)
    return _as_triples(oracle.filter(idx, rs, cand_off=off, cand=flat))


# --------------------------------------------------------------------------
# (a) hand-worked fixtures
# --------------------------------------------------------------------------

def test_handworked_fixture_oracle():
    fx = load_fixture("handworked_q3.txt")
    reads = [r for r, _ in fx["read"]]
    e = [x for _, x in fx["read"]]
    got = _run_oracle(fx["ref"], fx["B"], fx["max_read_len"], fx["q"], reads, e)
    assert got == fx["pass"]


def test_handworked_fixture_bruteforce():
    fx = load_fixture("handworked_q3.txt")
    reads = [r for r, _ in fx["read"]]
    e = [x for _, x in fx["read"]]
    got = bruteforce.filter(fx["ref"], fx["B"], fx["max_read_len"] - 1, fx["q"], reads, e)
    assert got == fx["pass"]


def test_fig2_token_bits():
    """Fig. 2: the bin's vector has GACAG's bit set and TTTTT's clear."""
    fx = load_fixture("fig2_q5.txt")
    idx = oracle.bin_vectors(np.frombuffer(fx["ref"].encode(), dtype=np.uint8), fx["B"], fx["q"],
                             fx["max_read_len"])
    bits = np.unpackbits(idx.vecs[0], bitorder="little")
    assert sorted(np.flatnonzero(bits).tolist()) == sorted(fx["set"])
    for t in fx["clear"]:
        assert bits[t] == 0
    # and the read tokens use the same values
    assert oracle.read_tokens(b"GACAG", 5).tolist() == [530]
    assert oracle.read_tokens(b"TTTTT", 5).tolist() == [1023]


# --------------------------------------------------------------------------
# (b) brute force on random tiny inputs
# --------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(12))
def test_bruteforce_random_all_bins(seed):
    rng = np.random.default_rng(1000 + seed)
    q = int(rng.choice([2, 3, 4, 5]))
    B = int(rng.integers(5, 60))
    mrl = int(rng.integers(max(q, 6), 40))
    n = int(rng.integers(50, 1500))
    ref, reads, e = random_case(rng, q, n, B, mrl, 25)
    got = _run_oracle(ref, B, mrl, q, reads, e)
    want = bruteforce.filter(ref, B, mrl - 1, q, reads, e)
    assert got == want


@pytest.mark.parametrize("seed", range(6))
def test_bruteforce_random_candidates(seed):
    """Candidate mode: unsorted lists with duplicates keep the given order."""
    rng = np.random.default_rng(2000 + seed)
    q = int(rng.choice([3, 4, 5]))
    B = int(rng.integers(5, 60))
    mrl = int(rng.integers(max(q, 6), 40))
    n = int(rng.integers(50, 1500))
    ref, reads, e = random_case(rng, q, n, B, mrl, 25)
    nb = -(-n // B)
    cands = [list(rng.integers(0, nb, int(rng.integers(0, 12)))) for _ in reads]
    cands = [[int(b) for b in c] for c in cands]
    got = _run_oracle(ref, B, mrl, q, reads, e, cands)
    want = bruteforce.filter(ref, B, mrl - 1, q, reads, e, cands)
    assert got == want


@pytest.mark.parametrize("q", [4, 5, 6])
def test_bruteforce_repeated_tokens(q):
    """Homopolymers and short tandem repeats: a read position counts every
    time its token occurs, so one token can contribute up to L-q+1 to a sum
    (the multiset reading).  The brute force counts positions by substring
    search."""
    rng = np.random.default_rng(3000 + q)
    alpha = "ACGT"
    parts = []
    for _ in range(12):
        if rng.random() < 0.5:
            unit = "".join(alpha[i] for i in rng.integers(0, 4, int(rng.integers(1, 8))))
            parts.append((unit * 80)[: int(rng.integers(30, 90))])
        else:
            parts.append("".join(alpha[i] for i in rng.integers(0, 4, int(rng.integers(20, 80)))))
    ref = "".join(parts)
    B, mrl = int(rng.integers(20, 50)), 60
    reads, e = [], []
    for _ in range(30):
        L = int(rng.integers(q + 4, mrl + 1))
        if rng.random() < 0.6:
            s = int(rng.integers(0, len(ref) - L))
            reads.append(ref[s:s + L])
        else:
            unit = "".join(alpha[i] for i in rng.integers(0, 4, int(rng.integers(1, 4))))
            reads.append((unit * L)[:L])
        e.append(int(rng.integers(0, 3)))
    got = _run_oracle(ref, B, mrl, q, reads, e)
    assert got == bruteforce.filter(ref, B, mrl - 1, q, reads, e)
    # some pass counts exceed the number of distinct tokens of their read
    distinct = {i: len({r[j:j + q] for j in range(len(r) - q + 1)}) for i, r in enumerate(reads)}
    assert any(c > distinct[r] for r, _, c in got)


@pytest.mark.parametrize("q", [3, 4, 5])
def test_vector_popcount_is_distinct_qgrams(q):
    """Each bin's bits are exactly the distinct clean q-grams of its window."""
    rng = np.random.default_rng(q)
    ref, _, _ = random_case(rng, q, 700, 37, 30, 0)
    idx = oracle.bin_vectors(np.frombuffer(ref.encode(), dtype=np.uint8), 37, q, 30)
    for b in range(idx.num_bins):
        bits = np.unpackbits(idx.vecs[b], bitorder="little")[: 4 ** q]
        want = bruteforce.present_set(ref, 37, 29, q, b)
        assert int(bits.sum()) == len(want)
        for g in want:
            assert bits[int(oracle.read_tokens(g.encode(), q)[0])] == 1


def test_token_major_is_transpose():
    rng = np.random.default_rng(5)
    ref, _, _ = random_case(rng, 4, 3000, 23, 20, 0)
    idx = oracle.bin_vectors(np.frombuffer(ref.encode(), dtype=np.uint8), 23, 4, 20)
    tm = oracle.token_major(idx)
    assert tm.shape == (256, 1024 // 32 * (-(-idx.num_bins // 1024)))
    bm = np.unpackbits(idx.vecs, axis=1, bitorder="little")
    tmb = np.unpackbits(tm.view(np.uint8), axis=1, bitorder="little")
    assert np.array_equal(tmb[:, : idx.num_bins], bm.T)
    assert not tmb[:, idx.num_bins:].any()


# --------------------------------------------------------------------------
# (c) closed forms the paper prints
# --------------------------------------------------------------------------

def test_table_size_closed_form():
    """§Parameter Evaluation Results: q=5 gives 4^5 = 1024-bit vectors, and
    450 x 64k bins need about 3.8 GB."""
    assert oracle.vector_bytes(5) * 8 == 1024
    total = 450 * 65536 * oracle.vector_bytes(5)
    assert round(total / 1e9, 1) == 3.8


def test_counter_width_for_100bp(tiny_plain_oracle):
    """§Mapping GRIM-Filter: 7-bit counters suffice for 100 bp reads, since a
    sum never exceeds the number of tokens (96 at q=5)."""
    _, _, c = tiny_plain_oracle
    assert c.max() <= 96 < 2 ** 7


# --------------------------------------------------------------------------
# (d) invariants
# --------------------------------------------------------------------------

def test_qgram_lemma_true_bin_passes(tiny_plain, tiny_plain_oracle):
    """Fig. 3's threshold is the q-gram lemma: a read with <= e edits against
    the window holding it keeps >= (L-q+1) - q*e tokens, so its true bin passes."""
    rs = tiny_plain["reads"]
    B = tiny_plain["B"]
    r, b, c = tiny_plain_oracle
    got = set(zip(r.tolist(), b.tolist()))
    assert (rs.n_edits <= rs.e).all()
    for i in range(rs.n):
        assert (i, int(rs.true_pos[i]) // B) in got


@pytest.mark.parametrize("q,B,lengths,e_fixed", [
    (6, 100, (150,), 7),              # the finer index: T = 145 - 42 = 103
    (5, 200, (100, 150, 250), None),  # mixed lengths, e up to 0.05 L, ext = 249
])
def test_qgram_lemma_other_configurations(q, B, lengths, e_fixed):
    """The same lemma at the other index shapes: q = 6 with B = 100, and
    reads of 100-250 bp with per-read budgets against an index extended by
    249 bases.  Reads are planted with up to e edits (substitutions,
    insertions, deletions) on a repeat-rich genome; every true bin passes,
    and edit-free reads count all L-q+1 tokens there."""
    from paper_1708_04329_gb300 import synth

    g = synth.human_genome(300_000, seed=12)
    mrl = max(lengths)
    if e_fixed is None:
        rs = synth.reads(g, 400, seed=13, lengths=lengths, probs=(0.5, 0.3, 0.2), e_frac=(5, 100),
                         max_edits=None)
    else:
        rs = synth.reads(g, 400, seed=13, lengths=lengths, e=e_fixed, max_edits=e_fixed)
    idx = oracle.bin_vectors(g, B, q, mrl)
    true_bin = (rs.true_pos // B).astype(np.int32)
    off = np.arange(rs.n + 1, dtype=np.uint64)
    r, b, c = oracle.filter(idx, rs, cand_off=off, cand=true_bin)
    assert (rs.n_edits <= rs.e).all()
    assert r.tolist() == list(range(rs.n))  # every read passes its true bin
    exact = rs.n_edits == 0
    assert exact.sum() > 20
    assert (c[exact] == rs.lens[exact] - q + 1).all()


def test_exact_reads_full_count(tiny_plain, tiny_plain_oracle):
    """Reads with 0 edits find all L-q+1 tokens in their true bin."""
    rs = tiny_plain["reads"]
    B = tiny_plain["B"]
    r, b, c = tiny_plain_oracle
    d = {(int(x), int(y)): int(z) for x, y, z in zip(r, b, c)}
    exact = np.flatnonzero(rs.n_edits == 0)
    assert len(exact) > 100
    for i in exact:
        assert d[(int(i), int(rs.true_pos[i]) // B)] == 96


def test_random_bins_rarely_pass(tiny_plain, tiny_plain_oracle):
    """Sanity (not parity): on i.i.d. bins a 96-token read finds ~25% of its
    tokens, far below T = 71, so passes are the true bin and its neighbours
    (a read starting late in its core also lies mostly inside the next bin's
    window, one starting early mostly inside the previous bin's)."""
    rs = tiny_plain["reads"]
    r, b, _ = tiny_plain_oracle
    true_bin = (rs.true_pos // tiny_plain["B"]).astype(np.int64)
    dist = b.astype(np.int64) - true_bin[r]
    assert np.isin(dist, [-1, 0, 1]).all()
    assert 1.0 <= len(r) / rs.n < 1.5


def test_monotone_in_e(tiny_plain, tiny_plain_index):
    rs = tiny_plain["reads"].subset(range(60))
    prev = None
    for e in range(0, 8):
        rs.e[:] = e
        cur = dict(((x, y), z) for x, y, z in _as_triples(oracle.filter(tiny_plain_index, rs)))
        if prev is not None:
            for k, v in prev.items():
                assert cur[k] == v
        prev = cur


def test_threshold_nonpositive_passes_everything(tiny_plain, tiny_plain_index):
    """T <= 0 (e >= 20 at L=100, q=5) makes every bin pass."""
    rs = tiny_plain["reads"].subset(range(4))
    rs.e[:] = 20
    r, b, c = oracle.filter(tiny_plain_index, rs)
    nb = tiny_plain_index.num_bins
    assert len(r) == 4 * nb
    assert np.array_equal(b, np.tile(np.arange(nb, dtype=np.uint32), 4))
    # and the counts are the plain token-hit sums of the windows
    g = tiny_plain["genome"].tobytes().decode()
    for j in range(0, nb, 997):
        assert int(c[j]) == bruteforce.count(rs.read(0).decode(), bruteforce.windows(g, 200, 99)[j], 5)


def test_alphabet_relabelling_invariant():
    """Relabelling A/C/G/T consistently in reference and reads changes no count."""
    rng = np.random.default_rng(77)
    ref, reads, e = random_case(rng, 4, 2000, 50, 30, 40)
    perm = str.maketrans("ACGTacgt", "GTCAgtca")
    a = _run_oracle(ref, 50, 30, 4, reads, e)
    b = _run_oracle(ref.translate(perm), 50, 30, 4, [x.translate(perm) for x in reads], e)
    assert a == b and len(a) > 0


def test_degenerate_genomes_and_reads():
    """Degenerate inputs against the brute force and the plain facts they
    imply: a genome of non-bases has no q-gram in any bin, so only reads
    whose threshold is <= 0 pass, with count 0; a genome shorter than q is
    one bin with an empty vector; a read of non-bases only counts nothing
    anywhere but still has L-q+1 tokens (it passes only when q*e >= L-q+1)."""
    q, B, mrl = 4, 10, 20
    reads = ["ACGTACGTAC", "NNNNNNNNNN", "ACGTNACGTA", "acgtacgtac"]
    # all non-bases
    ref = "N" * 95
    for e in ([0, 0, 0, 0], [2, 2, 2, 2], [3, 1, 2, 3]):
        got = _run_oracle(ref, B, mrl, q, reads, e)
        assert got == bruteforce.filter(ref, B, mrl - 1, q, reads, e)
        for r, _, c in got:
            assert c == 0 and (len(reads[r]) - q + 1) - q * e[r] <= 0
        nb = -(-len(ref) // B)
        passing = [i for i in range(len(reads)) if (len(reads[i]) - q + 1) - q * e[i] <= 0]
        assert sorted({r for r, _, _ in got}) == passing
        assert len(got) == nb * len(passing)
    # shorter than q: one bin, nothing in it
    idx = oracle.bin_vectors(np.frombuffer(b"ACG", dtype=np.uint8), B, q, mrl)
    assert idx.num_bins == 1 and not idx.vecs.any()
    # a read of non-bases against a clean genome
    ref = "ACGTTGCAAC" * 12
    for e in (1, 2):
        got = _run_oracle(ref, B, mrl, q, ["NNNNNNNNNN"], [e])
        assert got == bruteforce.filter(ref, B, mrl - 1, q, ["NNNNNNNNNN"], [e])
        assert bool(got) == (q * e >= 10 - q + 1)


def test_errors():
    idx = oracle.bin_vectors(np.frombuffer(b"ACGTACGTAC", dtype=np.uint8), 4, 3, 6)
    with pytest.raises(oracle.OracleError) as ei:
        oracle.filter(idx, Reads(["AC"], [0]))
    assert ei.value.code == -4
    with pytest.raises(oracle.OracleError) as ei:
        oracle.filter(idx, Reads(["ACGTACG"], [0]))
    assert ei.value.code == -5
    off = np.array([0, 1], dtype=np.uint64)
    with pytest.raises(oracle.OracleError) as ei:
        oracle.filter(idx, Reads(["ACGT"], [0]), cand_off=off, cand=np.array([3], np.int32))
    assert ei.value.code == -6
