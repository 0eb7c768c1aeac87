"""Mapper front-end helpers on the GPU: reverse complements, both-strand
batches, count-only filtering and the read-existence measure of the
parameter sweep, each against the oracle or a plain restatement."""
import numpy as np
import pytest

import oracle
from tests.conftest import Reads
from tests.gpu_helpers import assert_same, build, dev_reads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

COMP = bytes.maketrans(b"ACGTacgt", b"TGCAtgca")


@pytest.fixture(scope="module")
def world():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    from paper_1708_04329_gb300 import synth

    g = synth.human_genome(300_000, seed=91)
    return g, oracle.bin_vectors(g, 100, 5, 100), build(g, 100, 5, 100, 7)


def _host(t):
    return t.cpu().numpy().view(np.uint32) if t.dtype != torch.uint8 else t.cpu().numpy()


def test_reverse_complement_matches_plain_restatement():
    from paper_1708_04329_gb300 import grim

    rng = np.random.default_rng(3)
    strs = ["".join(rng.choice(list("ACGTacgtN-"), int(n))) for n in rng.integers(0, 300, 200)]
    rs = Reads(strs, [0] * len(strs))
    kw = dev_reads(rs)
    out = grim.grim_reverse_complement(kw["reads"], kw["offsets"], kw["lens"])
    got = out.cpu().numpy().tobytes()
    want = b"".join(s.encode().translate(COMP)[::-1] for s in strs)
    assert got == want


def test_both_strands_filter(world):
    from paper_1708_04329_gb300 import grim, synth

    g, oix, idx = world
    rs = synth.reads(g, 400, seed=92, lengths=(100,), e=4, max_edits=4)
    strs = [rs.read(i).decode() for i in range(rs.n)]
    rc = [s.encode().translate(COMP)[::-1].decode() for s in strs]
    both = Reads(strs + rc, list(rs.e) * 2)
    kw = grim.both_strands(**dev_reads(rs))
    got = tuple(_host(x) for x in grim.grim_filter(idx, **kw))
    assert_same(got, oracle.filter(oix, both))


def test_count_and_existence(world):
    from paper_1708_04329_gb300 import existence, grim, synth

    g, oix, idx = world
    rs = synth.reads(g, 300, seed=93, lengths=(100,), e=3, max_edits=3)
    want = oracle.filter(oix, rs)
    kw = dev_reads(rs)
    assert grim.grim_filter_count(idx, **kw) == len(want[0])
    assert existence.read_existence(idx, kw) == len(want[0]) / (rs.n * oix.num_bins)
    # T <= 0: every bin passes
    kw["e"] = torch.full_like(kw["e"], 30)
    assert grim.grim_filter_count(idx, **kw) == rs.n * oix.num_bins


def test_existence_sweep_small(world):
    from paper_1708_04329_gb300 import existence

    g, _, _ = world
    rows = existence.sweep(g, qs=(4, 5), bins_k=(1,), rates_pct=(0, 3), n_sets=2,
                           reads_per_set=100, max_edits=0)
    assert len(rows) == 4
    for r in rows:
        assert 0 < r["min"] <= r["mean"] <= r["max"] <= 1
    # more tolerance never lowers existence; longer tokens never raise it
    by = {(r["q"], r["rate_pct"]): r["mean"] for r in rows}
    assert by[(4, 3)] >= by[(4, 0)] and by[(5, 3)] >= by[(5, 0)]
    assert by[(5, 0)] <= by[(4, 0)]


def test_host_entry_points_reuse_and_trim_scratch(world):
    """The host-buffer entry points give the same result call after call from
    the library's cached scratch pool, and after the cache is trimmed."""
    from paper_1708_04329_gb300 import grim, synth

    g, oix, idx = world
    rs = synth.reads(g, 200, seed=94, lengths=(100,), e=4, max_edits=4)
    want = oracle.filter(oix, rs)
    args = (np.frombuffer(rs.seq, np.uint8), rs.offsets, rs.lens, rs.e)
    for _ in range(3):
        assert_same(grim.grim_filter_host(idx, *args, cap=10_000), want)
    grim.grim_trim_scratch()
    assert_same(grim.grim_filter_host(idx, *args, cap=10_000), want)
    idx2 = grim.grim_build_host(g, 100, 5, 100)
    assert_same(grim.grim_filter_host(idx2, *args, cap=10_000), want)
    grim.grim_trim_scratch()
    idx2.close()


def test_index_tables_from_torch_allocator(world):
    """With the allocator hook the index tables come from PyTorch's caching
    allocator (they show in its accounting), filter identically, and go back
    to it when the index is freed."""
    from paper_1708_04329_gb300 import grim, synth

    g, oix, _ = world
    rs = synth.reads(g, 150, seed=95, lengths=(100,), e=4, max_edits=4)
    want = oracle.filter(oix, rs)
    ref = torch.from_numpy(g).cuda()
    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated()
    grim.use_torch_allocator()
    try:
        idx = grim.grim_build(ref, 100, 5, 100, 7)
        d = idx.desc
        tables = d.token_major_bytes + d.bin_major_bytes + d.coarse_token_major_bytes
        assert torch.cuda.memory_allocated() - before >= tables
        got = tuple(_host(x) for x in grim.grim_filter(idx, **dev_reads(rs)))
        assert_same(got, want)
        idx.close()
        torch.cuda.synchronize()
        assert torch.cuda.memory_allocated() == before
    finally:
        grim.use_torch_allocator(False)
    idx = grim.grim_build(ref, 100, 5, 100, 7)  # cudaMalloc again
    assert_same(tuple(_host(x) for x in grim.grim_filter(idx, **dev_reads(rs))), want)
    idx.close()


def test_concurrent_calls_on_streams(world):
    """The index is read-only: grim_filter calls from several host threads,
    each on its own stream with its own workspace, give each caller the
    same pass list as a call alone."""
    import threading

    from paper_1708_04329_gb300 import grim, synth

    g, oix, idx = world
    sets = [synth.reads(g, 120 + 40 * i, seed=96 + i, lengths=(100,), e=4, max_edits=4)
            for i in range(4)]
    want = [oracle.filter(oix, rs) for rs in sets]
    errors = []

    def worker(i):
        try:
            st = torch.cuda.Stream()
            ws = grim.Workspace()
            with torch.cuda.stream(st):
                kw = dev_reads(sets[i])
                for _ in range(5):
                    got = grim.grim_filter(idx, **kw, workspace=ws, stream=st)
                    st.synchronize()
                    assert_same(tuple(_host(x) for x in got), want[i])
        except Exception as exc:  # reported on the main thread
            errors.append(exc)

    threads = [threading.Thread(target=worker, args=(i,)) for i in range(4)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors
