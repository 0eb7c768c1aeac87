"""Parity of the CUDA path (through the C-ABI) with the CPU oracle.

Integer work: every comparison is bit-exact -- tables byte for byte, pass
lists record for record (read, bin, count) in order.
"""
import numpy as np
import pytest

import oracle
from tests.conftest import Reads, load_fixture, random_case
from tests.gpu_helpers import assert_same, build, dev_reads, gpu_filter

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def _np(s: str) -> np.ndarray:
    return np.frombuffer(s.encode(), dtype=np.uint8).copy()


def _gpu_tables(idx, q):
    tm = idx.token_major()
    bm = idx.bin_major()
    return (None if tm is None else tm.cpu().numpy().view(np.uint32),
            None if bm is None else bm.cpu().numpy().view(np.uint32))


def _check_tables(ref: np.ndarray, B: int, q: int, mrl: int, layouts: int = 7, factor: int = 0):
    idx = build(ref, B, q, mrl, layouts, factor)
    tm, bm = _gpu_tables(idx, q)
    oix = oracle.bin_vectors(ref, B, q, mrl)
    vb = oracle.vector_bytes(q)
    if bm is not None:
        got = bm.view(np.uint8).reshape(oix.num_bins, -1)
        assert np.array_equal(got[:, :vb], oix.vecs)
        assert not got[:, vb:].any()
    if tm is not None:
        assert np.array_equal(tm, oracle.token_major(oix))
    ctm = idx.coarse_token_major()
    if ctm is not None:
        # super-bins of f bins: the oracle's vectors with core f*B, same extension
        f = idx.desc.coarse_factor
        coarse = oracle.bin_vectors(ref, f * B, q, mrl)
        assert np.array_equal(ctm.cpu().numpy().view(np.uint32), oracle.token_major(coarse))
        assert idx.desc.num_coarse == coarse.num_bins
    d = idx.desc
    assert d.num_bins == oix.num_bins and d.num_bins_pad % 1024 == 0
    return idx, oix


# ---------------------------------------------------------------------------
# tables (a1-a3)
# ---------------------------------------------------------------------------

def test_fig2_bits_on_gpu():
    fx = load_fixture("fig2_q5.txt")
    idx = build(_np(fx["ref"]), fx["B"], fx["q"], fx["max_read_len"])
    tm, bm = _gpu_tables(idx, 5)
    bits = np.unpackbits(bm.view(np.uint8)[0], bitorder="little")
    assert sorted(np.flatnonzero(bits).tolist()) == sorted(fx["set"])
    for t in fx["set"]:
        assert tm[t, 0] & 1
    for t in fx["clear"]:
        assert not tm[t, 0] & 1


@pytest.mark.parametrize("q", [2, 3, 4, 5, 6])
def test_tables_match_oracle(q):
    rng = np.random.default_rng(100 + q)
    n = int(rng.integers(20_000, 60_000))
    B = int(rng.integers(7, 40))
    ref, _, _ = random_case(rng, q, n, B, 50, 0)
    _check_tables(_np(ref), B, q, int(rng.integers(q, 80)))


def test_tables_ragged_and_tiny():
    # one base shorter than q, a single bin, a window clipped at N
    for ref, B, q, mrl in [("ACG", 5, 4, 4), ("ACGTA", 5, 4, 10), ("ACGTACGTNNacgtTT", 3, 3, 5)]:
        _check_tables(_np(ref), B, q, mrl)


def test_build_host_equals_build():
    from paper_1708_04329_gb300 import grim

    g = np.frombuffer(b"ACGT", np.uint8)[np.random.default_rng(3).integers(0, 4, 70_001)]
    a = build(g, 50, 5, 100)
    b = grim.grim_build_host(g, 50, 5, 100)
    assert np.array_equal(a.token_major().cpu().numpy(), b.token_major().cpu().numpy())
    assert np.array_equal(a.bin_major().cpu().numpy(), b.bin_major().cpu().numpy())


# ---------------------------------------------------------------------------
# filter (a4-a8)
# ---------------------------------------------------------------------------

def test_handworked_fixture_gpu():
    fx = load_fixture("handworked_q3.txt")
    rs = Reads([r for r, _ in fx["read"]], [x for _, x in fx["read"]])
    idx = build(_np(fx["ref"]), fx["B"], fx["q"], fx["max_read_len"])
    r, b, c = gpu_filter(idx, rs)
    assert list(zip(r.tolist(), b.tolist(), c.tolist())) == fx["pass"]


@pytest.mark.parametrize("layouts", [1, 6, 7])
@pytest.mark.parametrize("seed", range(8))
def test_random_all_bins(seed, layouts):
    """Several 1024-bin tiles plus a ragged one, mixed read lengths, non-bases,
    per-read e including T <= 0; one exact pass over the token-major table
    (layouts 1), coarse-then-exact (6), or whichever the batch suits (7)."""
    rng = np.random.default_rng(500 + seed)
    q = int(rng.choice([2, 3, 4, 5, 6]))
    B = int(rng.integers(5, 40))
    mrl = int(rng.integers(max(q, 20), 120))
    n = int(rng.integers(30_000, 90_000))
    ref, reads, e = random_case(rng, q, n, B, mrl, 300)
    if seed % 2:  # half the cases with some T <= 0 reads
        e = [int(x) if rng.random() < 0.9 else 40 for x in e]
    rs = Reads(reads, e)
    idx, oix = _check_tables(_np(ref), B, q, mrl, layouts)
    assert_same(gpu_filter(idx, rs), oracle.filter(oix, rs))


@pytest.mark.parametrize("seed", range(6))
def test_random_candidates(seed):
    """Unsorted lists with duplicates and empty lists keep the given order."""
    rng = np.random.default_rng(700 + seed)
    q = int(rng.choice([2, 3, 4, 5, 6]))
    B = int(rng.integers(5, 40))
    mrl = int(rng.integers(max(q, 20), 120))
    n = int(rng.integers(20_000, 60_000))
    ref, reads, e = random_case(rng, q, n, B, mrl, 300)
    rs = Reads(reads, e)
    idx, oix = _check_tables(_np(ref), B, q, mrl)
    nb = oix.num_bins
    counts = rng.integers(0, 40, len(reads))
    counts[rng.random(len(reads)) < 0.1] = 0
    off = np.zeros(len(reads) + 1, np.uint64)
    off[1:] = np.cumsum(counts)
    cand = rng.integers(0, nb, int(off[-1])).astype(np.int32)
    assert_same(gpu_filter(idx, rs, off, cand), oracle.filter(oix, rs, cand_off=off, cand=cand))


def test_tiny_plain_full(tiny_plain, tiny_plain_index, tiny_plain_oracle):
    """The 1 Mbp / 5,000-bin / 2,000-read workload: the whole pass list."""
    w = tiny_plain
    idx = build(w["genome"], w["B"], w["q"], w["max_read_len"])
    assert_same(gpu_filter(idx, w["reads"]), tiny_plain_oracle)
    from paper_1708_04329_gb300 import synth

    off, cand = synth.candidates((w["reads"].true_pos // w["B"]).astype(np.int32),
                                 tiny_plain_index.num_bins, seed=4)
    assert_same(gpu_filter(idx, w["reads"], off, cand),
                oracle.filter(tiny_plain_index, w["reads"], cand_off=off, cand=cand))


def test_many_ranges_per_tile():
    """Few tiles, many reads: each tile is split into read ranges."""
    from paper_1708_04329_gb300 import synth

    g = synth.genome(250_000, seed=9)
    rs = synth.reads(g, 6000, seed=10, e=5, max_edits=5)
    idx = build(g, 200, 5, 100)
    oix = oracle.bin_vectors(g, 200, 5, 100)
    assert_same(gpu_filter(idx, rs), oracle.filter(oix, rs))


def test_threshold_nonpositive_passes_everything():
    from paper_1708_04329_gb300 import synth

    g = synth.genome(40_000, seed=5)
    rs = synth.reads(g, 7, seed=6, e=20, max_edits=5)
    idx = build(g, 100, 5, 100)
    oix = oracle.bin_vectors(g, 100, 5, 100)
    got = gpu_filter(idx, rs)
    assert len(got[0]) == 7 * oix.num_bins
    assert_same(got, oracle.filter(oix, rs))


def test_reads_of_every_length_in_one_call():
    rng = np.random.default_rng(11)
    ref, _, _ = random_case(rng, 5, 50_000, 64, 0, 0, dirty=False)
    g = _np(ref)
    reads = []
    for L in range(5, 256):
        s = int(rng.integers(0, len(ref) - L))
        reads.append(ref[s:s + L])
    rs = Reads(reads, [int(x) for x in rng.integers(0, 6, len(reads))])
    idx = build(g, 64, 5, 255)
    oix = oracle.bin_vectors(g, 64, 5, 255)
    want = oracle.filter(oix, rs)
    assert_same(gpu_filter(idx, rs), want)
    # and with every read switch and both all-bins paths forced: under the
    # warp switch the groups of a warp end 1 to 16 blocks apart, so groups
    # whose read ended read on through their token rows' padding
    from paper_1708_04329_gb300 import grim

    for path in (grim.GRIM_PATH_TWO_LEVEL, grim.GRIM_PATH_EXACT):
        for switch in (grim.GRIM_SWITCH_GROUP, grim.GRIM_SWITCH_WARP):
            grim.grim_index_set_shape(idx, read_switch=switch, all_bins_path=path)
            assert_same(gpu_filter(idx, rs), want)
    # reversed length order: long and short reads share every warp
    back = Reads(reads[::-1], list(rs.e[::-1]))
    grim.grim_index_set_shape(idx, read_switch=grim.GRIM_SWITCH_WARP)
    assert_same(gpu_filter(idx, back), oracle.filter(oix, back))
    idx.close()


def test_zero_reads():
    from paper_1708_04329_gb300 import grim

    idx = build(_np("ACGTACGTAC" * 10), 10, 3, 10)
    z = torch.zeros(0, dtype=torch.int64, device="cuda")
    r, b, c = grim.grim_filter(idx, torch.zeros(0, dtype=torch.uint8, device="cuda"), z,
                               z.to(torch.int32), z.to(torch.int16))
    assert r.numel() == 0


@pytest.mark.parametrize("reads,code", [(["ACGTAC", "AC"], -4), (["ACGTACGTACGT"], -5),
                                        (["AC", "ACGTACGTACGT"], -4)])
def test_read_length_errors(reads, code):
    from paper_1708_04329_gb300 import grim

    idx = build(_np("ACGTACGTAC" * 10), 10, 3, 10)
    with pytest.raises(grim.GrimError) as ei:
        gpu_filter(idx, Reads(reads, [0] * len(reads)))
    assert ei.value.code == code


def test_candidate_errors():
    from paper_1708_04329_gb300 import grim

    idx = build(_np("ACGTACGTAC" * 10), 10, 3, 10)
    rs = Reads(["ACGTAC", "CGTACG"], [0, 0])
    with pytest.raises(grim.GrimError) as ei:
        gpu_filter(idx, rs, np.array([0, 1, 2], np.uint64), np.array([3, 10], np.int32))
    assert ei.value.code == grim.GRIM_E_BAD_CANDIDATE
    with pytest.raises(grim.GrimError) as ei:  # decreasing offsets
        gpu_filter(idx, rs, np.array([0, 2, 1], np.uint64), np.array([3, 4], np.int32))
    assert ei.value.code == grim.GRIM_E_ARG
    # an index with only the token-major table cannot serve candidate lists
    tmo = build(_np("ACGTACGTAC" * 10), 10, 3, 10, layouts=1)
    with pytest.raises(grim.GrimError) as ei:
        gpu_filter(tmo, rs, np.array([0, 1, 2], np.uint64), np.array([3, 4], np.int32))
    assert ei.value.code == grim.GRIM_E_NO_LAYOUT


def test_overflow_reports_total_and_count_only():
    from paper_1708_04329_gb300 import grim, synth
    from tests.gpu_helpers import dev_reads

    g = synth.genome(40_000, seed=5)
    rs = synth.reads(g, 50, seed=6, e=5, max_edits=5)
    idx = build(g, 100, 5, 100)
    want = oracle.filter(oracle.bin_vectors(g, 100, 5, 100), rs)
    n = len(want[0])
    assert n > 3
    for cap in (0, 3):
        out = tuple(torch.empty(cap, dtype=dt, device="cuda")
                    for dt in (torch.int32, torch.int32, torch.uint8))
        with pytest.raises(grim.GrimError) as ei:
            grim.grim_filter(idx, **dev_reads(rs), out=out)
        assert ei.value.code == grim.GRIM_E_OVERFLOW and ei.value.n_out == n
    # the binding's retry returns the full list
    assert_same(gpu_filter(idx, rs, cap=1), want)
    # coarse-then-exact without a token-major table: an overflow of the
    # survivors reports an upper bound, and the retry with it succeeds
    cto = build(g, 100, 5, 100, layouts=6)
    out = tuple(torch.empty(3, dtype=dt, device="cuda") for dt in (torch.int32, torch.int32, torch.uint8))
    with pytest.raises(grim.GrimError) as ei:
        grim.grim_filter(cto, **dev_reads(rs), out=out)
    assert ei.value.code == grim.GRIM_E_OVERFLOW and ei.value.n_out >= n
    assert_same(gpu_filter(cto, rs, cap=3), want)


def test_workspace_reuse_is_clean():
    from paper_1708_04329_gb300 import grim, synth

    g = synth.genome(80_000, seed=7)
    a = synth.reads(g, 500, seed=8, e=5, max_edits=5)
    b = synth.reads(g, 300, seed=9, e=3, max_edits=3)
    idx = build(g, 200, 5, 100)
    oix = oracle.bin_vectors(g, 200, 5, 100)
    ws = grim.Workspace()
    for rs in (a, b, a):
        assert_same(gpu_filter(idx, rs, workspace=ws), oracle.filter(oix, rs))


def test_filter_host_equals_oracle():
    from paper_1708_04329_gb300 import grim, synth

    g = synth.genome(80_000, seed=12)
    rs = synth.reads(g, 400, seed=13, e=5, max_edits=5)
    idx = build(g, 200, 5, 100)
    oix = oracle.bin_vectors(g, 200, 5, 100)
    got = grim.grim_filter_host(idx, rs.seq, rs.offsets, rs.lens, rs.e)
    assert_same(got, oracle.filter(oix, rs))
    off, cand = synth.candidates((rs.true_pos // 200).astype(np.int32), oix.num_bins, seed=3)
    got = grim.grim_filter_host(idx, rs.seq, rs.offsets, rs.lens, rs.e, cand=cand, cand_off=off)
    assert_same(got, oracle.filter(oix, rs, cand_off=off, cand=cand))


@pytest.mark.parametrize("layouts", [1, 6, 7])
def test_q6_all_bins(layouts):
    """q = 6 (4096-row table, 256-bin tiles): several tiles plus a ragged one."""
    from paper_1708_04329_gb300 import synth

    g = synth.human_genome(400_000, seed=8)
    rs = synth.reads(g, 700, seed=9, lengths=(150,), e=7, max_edits=7)
    idx, oix = _check_tables(g, 100, 6, 150, layouts)
    if layouts & 4:  # default factor: the largest power of two keeping a window near 40% full
        assert idx.desc.coarse_factor == 16
    assert_same(gpu_filter(idx, rs), oracle.filter(oix, rs))


@pytest.mark.parametrize("lengths", [(150,), (60, 150, 250)])
def test_q6_read_switch_modes(lengths):
    """q = 6, every read switch: with sixteen 2-lane groups per warp the warp
    switch takes new reads once 14 groups wait, so the others keep reads that
    started earlier (groups out of phase, token blocks past the slot read
    from L2).  2,400 reads span several read ranges of a 1 MiB read tile;
    uniform and mixed lengths; both all-bins paths; equal to the oracle."""
    from paper_1708_04329_gb300 import grim, synth

    g = synth.human_genome(600_000, seed=12)
    rs = synth.reads(g, 2400, seed=13, lengths=lengths, probs=(1.0,) if len(lengths) == 1 else (0.3, 0.4, 0.3),
                     e_frac=(5, 100), max_edits=None)
    idx = build(g, 100, 6, 250)
    want = oracle.filter(oracle.bin_vectors(g, 100, 6, 250), rs)
    for path in (grim.GRIM_PATH_TWO_LEVEL, grim.GRIM_PATH_EXACT):
        for switch in (grim.GRIM_SWITCH_GROUP, grim.GRIM_SWITCH_WARP, 0):
            grim.grim_index_set_shape(idx, read_range_kb=1024, read_switch=switch, all_bins_path=path)
            assert_same(gpu_filter(idx, rs), want)
    idx.close()


def test_default_coarse_factor_q5():
    from paper_1708_04329_gb300 import synth

    g = synth.genome(50_000, seed=2)
    assert build(g, 200, 5, 100).desc.coarse_factor == 2


@pytest.mark.parametrize("q,factor", [(4, 3), (5, 4), (5, 7), (6, 8), (6, 16)])
def test_coarse_factors(q, factor):
    """Coarse-then-exact with super-bins of 3..16 bins (ragged last super-bin)."""
    rng = np.random.default_rng(900 + factor)
    B = int(rng.integers(20, 60))
    mrl = 120
    ref, reads, e = random_case(rng, q, 90_001, B, mrl, 300)
    rs = Reads(reads, e)
    idx, oix = _check_tables(_np(ref), B, q, mrl, layouts=6, factor=factor)
    assert idx.desc.coarse_factor == factor
    assert_same(gpu_filter(idx, rs), oracle.filter(oix, rs))


def _low_complexity_case(rng, n: int, n_reads: int, mrl: int):
    """A genome with homopolymer and short tandem-repeat blocks, and reads
    drawn from them (or made of such repeats): tokens of high multiplicity,
    up to L-q+1 copies of one token."""
    alpha = np.frombuffer(b"ACGT", dtype=np.uint8)
    g = alpha[rng.integers(0, 4, n)].copy()
    blocks = []
    for period in (1, 1, 2, 3, 4, 6, 7, 8, 12):
        unit = alpha[rng.integers(0, 4, period)]
        size = int(rng.integers(150, 400))
        s = int(rng.integers(0, n - size))
        g[s:s + size] = np.resize(unit, size)
        blocks.append((s, size))
    ref = g.tobytes().decode()
    reads, es = [], []
    for _ in range(n_reads):
        L = int(rng.integers(max(20, mrl // 2), mrl + 1))
        kind = rng.random()
        if kind < 0.5:  # from (or across the edge of) a low-complexity block
            s0, size = blocks[int(rng.integers(0, len(blocks)))]
            s = int(np.clip(s0 + rng.integers(-L // 2, size), 0, n - L))
            rd = bytearray(ref[s:s + L].encode())
            for _k in range(int(rng.integers(0, 3))):
                rd[int(rng.integers(0, L))] = b"ACGT"[int(rng.integers(0, 4))]
        elif kind < 0.8:  # a pure tandem repeat, period 1..8
            unit = alpha[rng.integers(0, 4, int(rng.integers(1, 9)))]
            rd = bytearray(np.resize(unit, L).tobytes())
        else:
            rd = bytearray(alpha[rng.integers(0, 4, L)].tobytes())
        reads.append(rd.decode())
        es.append(int(rng.integers(0, 6)))
    return ref, reads, es, blocks


@pytest.mark.parametrize("q", [5, 6])
def test_repeated_tokens(q):
    """Reads whose tokens repeat many times (homopolymers, short tandem
    repeats): the multiplicity planes above the first two -- in shared
    memory for 128-byte vectors, the list of heavy tokens for 512-byte ones
    -- in candidate mode and in the coarse-then-exact all-bins mode."""
    rng = np.random.default_rng(1100 + q)
    B, mrl = 40, 150
    ref, reads, e, blocks = _low_complexity_case(rng, 60_000, 400, mrl)
    rs = Reads(reads, e)
    idx, oix = _check_tables(_np(ref), B, q, mrl, layouts=7)
    nb = oix.num_bins
    block_bins = np.concatenate([np.arange(s // B, min(nb, (s + size) // B + 1))
                                 for s, size in blocks]).astype(np.int32)
    lists = []
    for _ in reads:
        picks = [rng.integers(0, nb, int(rng.integers(0, 30))),
                 rng.choice(block_bins, int(rng.integers(0, 30)))]
        lists.append(np.concatenate(picks).astype(np.int32))
    off = np.zeros(len(reads) + 1, np.uint64)
    off[1:] = np.cumsum([len(x) for x in lists])
    cand = np.concatenate(lists).astype(np.int32)
    want = oracle.filter(oix, rs, cand_off=off, cand=cand)
    assert len(want[0]) > 100  # the repeats do pass somewhere
    assert_same(gpu_filter(idx, rs, off, cand), want)
    assert_same(gpu_filter(idx, rs), oracle.filter(oix, rs))


@pytest.mark.parametrize("layouts", [1, 6, 7])
def test_degenerate_genome_and_reads(layouts):
    """A genome of non-bases (no bin holds any q-gram: only reads with T <= 0
    pass, with count 0) and a read of non-bases against a clean genome, in
    the all-bins paths and in candidate mode."""
    q, B, mrl = 4, 10, 20
    reads = ["ACGTACGTAC", "NNNNNNNNNN", "ACGTNACGTA", "acgtacgtac", "NNNNNNNNNNNNNNNNNNNN"]
    for ref, e in (("N" * 2_095, [0, 2, 2, 3, 5]), ("ACGTTGCAAC" * 300, [1, 2, 0, 1, 5]),
                   ("ACGTTGCAAC" * 300, [0, 1, 1, 0, 4])):
        rs = Reads(reads, e)
        idx, oix = _check_tables(_np(ref), B, q, mrl, layouts)
        assert_same(gpu_filter(idx, rs), oracle.filter(oix, rs))
        if layouts & 2:
            nb = oix.num_bins
            off = np.array([0, 3, 3, 7, 9, 12], np.uint64)
            cand = np.array([0, 1, nb - 1, 5, 4, 3, 2, 0, nb - 1, 7, 8, 9], np.int32)
            assert_same(gpu_filter(idx, rs, off, cand), oracle.filter(oix, rs, cand_off=off, cand=cand))
        idx.close()


def test_filter_stats_are_per_thread():
    """grim_last_filter_stats reports the calling thread's own last call:
    two threads filtering different batches at the same time (each on its
    own stream and workspace) each read back the counters of their own call,
    identical to the same call made alone."""
    import threading

    from paper_1708_04329_gb300 import grim, synth

    torch.cuda.set_device(0)
    g = synth.human_genome(1_500_000, seed=91)
    idx = build(g, 200, 5, 100)
    batches = [synth.reads(g, 3000, seed=92, e=5, max_edits=5),
               synth.reads(g, 1200, seed=93, e=3, max_edits=3)]
    alone = []
    for rs in batches:
        grim.grim_filter(idx, **dev_reads(rs))
        alone.append(grim.grim_last_filter_stats())
    assert alone[0] != alone[1]
    got = [None, None]
    errors = []

    def work(i):
        try:
            st = torch.cuda.Stream()
            ws = grim.Workspace()
            kw = dev_reads(batches[i])
            for _ in range(5):
                with torch.cuda.stream(st):
                    grim.grim_filter(idx, **kw, workspace=ws, stream=st)
                s = grim.grim_last_filter_stats()
                if s != alone[i]:
                    errors.append((i, s))
            got[i] = s
        except Exception as e:  # surfaced below
            errors.append((i, repr(e)))

    threads = [threading.Thread(target=work, args=(i,)) for i in range(2)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors
    assert got == alone
    idx.close()


@pytest.mark.parametrize("path", ["exact", "two_level"])
def test_one_word_tail(path):
    """With the warp-synchronous read switch, a warp whose lanes each hold at
    most one word (32 bins) with a live bin after four blocks applies its
    remaining blocks to that word alone.  On repeat-rich 100 bp reads (6
    blocks each) most warps get there; the counters show it (fewer bit tests
    than tokens x tile bins) and the pass list stays exactly the oracle's, and
    equal to the group switch, which never takes the tail.  15,000 bins end
    in a ragged tile (15 x 1024 = 15,360)."""
    from paper_1708_04329_gb300 import grim, synth

    g = synth.human_genome(3_000_000, seed=95)
    rs = synth.reads(g, 4000, seed=96, lengths=(100,), e=5, max_edits=5)
    idx = build(g, 200, 5, 100)
    assert idx.desc.num_bins == 15000
    p = grim.GRIM_PATH_EXACT if path == "exact" else grim.GRIM_PATH_TWO_LEVEL
    want = oracle.filter(oracle.bin_vectors(g, 200, 5, 100), rs)
    got = {}
    for switch in (grim.GRIM_SWITCH_WARP, grim.GRIM_SWITCH_GROUP):
        grim.grim_index_set_shape(idx, read_switch=switch, all_bins_path=p)
        got[switch] = gpu_filter(idx, rs)
        st = grim.grim_last_filter_stats()
        full = st["tokens_executed"] * 1024
        if switch == grim.GRIM_SWITCH_WARP:
            assert st["bit_tests_executed"] < full  # the tail ran
        else:
            assert st["bit_tests_executed"] == full
    assert_same(got[grim.GRIM_SWITCH_WARP], want)
    assert_same(got[grim.GRIM_SWITCH_GROUP], want)
    idx.close()


def test_automatic_read_switch_and_path():
    """The choices a call makes on its own, reported by grim_last_filter_stats:
    the warp switch only when every read spans as many 16-token blocks and
    has the same miss budget D' (with budgets that differ, reads leave a tile
    blocks apart); coarse-then-exact unless a read has too little slack.  The
    pass list equals the oracle's in every case."""
    from paper_1708_04329_gb300 import grim, synth

    g = synth.human_genome(1_000_000, seed=97)
    idx = build(g, 200, 5, 150)
    oix = oracle.bin_vectors(g, 200, 5, 150)
    W, G = grim.GRIM_SWITCH_WARP, grim.GRIM_SWITCH_GROUP
    two, exact = grim.GRIM_PATH_TWO_LEVEL, grim.GRIM_PATH_EXACT
    cases = [
        (synth.reads(g, 1500, seed=98, lengths=(100,), e=5, max_edits=5), W, two),
        (synth.reads(g, 1500, seed=99, lengths=(100,), e_frac=(5, 100), max_edits=None), G, two),
        (synth.reads(g, 1500, seed=100, lengths=(100, 150), probs=(0.5, 0.5), e=5, max_edits=5), G, two),
        # 96 tokens, D' = 75: slack 21 < 24, so the exact pass
        (synth.reads(g, 600, seed=101, lengths=(100,), e=15, max_edits=3), W, exact),
    ]
    for rs, switch, path in cases:
        assert_same(gpu_filter(idx, rs), oracle.filter(oix, rs))
        st = grim.grim_last_filter_stats()
        assert (st["read_switch"], st["all_bins_path"]) == (switch, path)
    # candidate mode reports neither
    off, cand = synth.candidates((cases[0][0].true_pos // 200).astype(np.int32), oix.num_bins, seed=3)
    gpu_filter(idx, cases[0][0], off, cand)
    st = grim.grim_last_filter_stats()
    assert (st["read_switch"], st["all_bins_path"]) == (0, 0)
    idx.close()


def test_survivor_overflow_takes_the_exact_pass():
    """Coarse survivors beyond their room (the larger of the output capacity
    and 320 a read) with the token-major table present: the call drops the
    coarse result and takes the exact pass, reports that path, and still
    equals the oracle.  The genome repeats one random 127-base period: a
    super-bin window (2 x 24 + 79 = 127 bases) holds nearly every q-gram of
    the period, so ~998 super-bins pass per read, while a bin window (103
    bases) holds a read's q-grams only near its copies (~551 bins a read)."""
    from paper_1708_04329_gb300 import grim

    rng = np.random.default_rng(41)
    period = "".join("ACGT"[i] for i in rng.integers(0, 4, 127))
    ref = (period * (48_000 // 127 + 1))[:48_000]
    reads = []
    for _ in range(20):
        s = int(rng.integers(0, len(ref) - 80))
        reads.append(ref[s:s + 80])
    rs = Reads(reads, [1] * len(reads))
    g = _np(ref)
    want = oracle.filter(oracle.bin_vectors(g, 24, 5, 80), rs)
    n_surv = len(oracle.filter(oracle.bin_vectors(g, 48, 5, 80), rs)[0])
    assert n_surv > max(len(want[0]), 320 * rs.n)  # the survivors do not fit
    idx = build(g, 24, 5, 80, coarse_factor=2)
    grim.grim_index_set_shape(idx, all_bins_path=grim.GRIM_PATH_TWO_LEVEL)
    assert_same(gpu_filter(idx, rs, cap=len(want[0])), want)
    st = grim.grim_last_filter_stats()
    assert st["survivors"] == n_surv
    assert st["all_bins_path"] == grim.GRIM_PATH_EXACT
    # with room for every survivor the same call stays on the coarse path
    assert_same(gpu_filter(idx, rs, cap=n_surv), want)
    st = grim.grim_last_filter_stats()
    assert st["survivors"] == n_surv and st["all_bins_path"] == grim.GRIM_PATH_TWO_LEVEL
    idx.close()
