"""Parity at the full sizes of the finer-index and ragged-candidate
workloads, in the launch configurations the benchmark times.

* Finer index: the 3.1 Gbp genome with q=6, B=100 (31M bins, 512-byte
  vectors, 15.9 GB per layout), 1,000,000 reads of L=150 with e=7, every
  read against every bin (coarse-then-exact), and candidate lists.
* Ragged candidates: 4,000,000 reads of L in {100,150,250} with per-read e
  and 1.32e9 candidates, through one graph-captured plan launch.
* Serving index: the same genome with max_read_len 250, its automatic
  coarse-then-exact path on reads of the serving pool.

The oracle checks what it can compute exactly (every bin for sampled reads,
every read for a bin range, the lists of the first reads) and properties
that hold at any size (sortedness, the q-gram lemma)."""
import numpy as np
import pytest

import oracle
from tests.gpu_helpers import build, dev_reads, gpu_filter

pytestmark = [pytest.mark.gpu]

torch = pytest.importorskip("torch")


def _check_slices(got, want_r, want_b, want_c, idx):
    r, b, c = got
    for j, ridx in enumerate(idx):
        sel = r == ridx
        ws = want_r == j
        assert np.array_equal(b[sel], want_b[ws]), ridx
        assert np.array_equal(c[sel], want_c[ws]), ridx


@pytest.fixture(scope="module")
def finer():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1708_04329_gb300 import synth

    w = synth.finer_index()
    idx = build(w["genome"], w["B"], w["q"], w["max_read_len"])
    got = gpu_filter(idx, w["reads"], cap=8 * w["reads"].n)
    oix = oracle.bin_vectors(w["genome"], w["B"], w["q"], w["max_read_len"])
    yield w, idx, got, oix
    idx.close()


def test_finer_every_bin_for_sampled_reads(finer):
    w, _, got, oix = finer
    rs = w["reads"]
    idx = np.linspace(0, rs.n - 1, 16).astype(np.int64)
    _check_slices(got, *oracle.filter(oix, rs.subset(idx)), idx)


def test_finer_every_read_for_a_bin_range(finer):
    w, _, got, oix = finer
    want = oracle.filter(oix, w["reads"], bin_range=(0, 2048))
    r, b, c = got
    sel = b < 2048
    assert np.array_equal(r[sel], want[0]) and np.array_equal(b[sel], want[1])
    assert np.array_equal(c[sel], want[2])


def test_finer_bin_major_sampled_rows(finer):
    w, idx, _, oix = finer
    bm = idx.bin_major()
    rng = np.random.default_rng(1)
    rows = np.unique(np.concatenate([rng.integers(0, oix.num_bins, 4000), [0, oix.num_bins - 1]]))
    got = bm[torch.from_numpy(rows).cuda()].cpu().numpy().view(np.uint8)
    assert np.array_equal(got, oix.vecs[rows])


def test_finer_properties(finer):
    w, _, got, _ = finer
    rs = w["reads"]
    r, b, c = got
    key = r.astype(np.uint64) << np.uint64(32) | b.astype(np.uint64)
    assert (np.diff(key.astype(np.int64)) > 0).all()
    assert c.max() <= 145
    true_key = np.arange(rs.n, dtype=np.uint64) << np.uint64(32) | (rs.true_pos // 100).astype(np.uint64)
    pos = np.searchsorted(key, true_key)
    assert (pos < len(key)).all() and (key[pos] == true_key).all()


def test_finer_candidate_lists(finer):
    w, idx, _, oix = finer
    rs, off, cand = w["reads"], w["cand_off"], w["cand"]
    got = gpu_filter(idx, rs, off, cand, cap=4 * rs.n)
    k = 2000
    want = oracle.filter(oix, rs.subset(range(k)), cand_off=off[: k + 1], cand=cand[: int(off[k])])
    r, b, c = got
    sel = r < k
    assert np.array_equal(r[sel], want[0]) and np.array_equal(b[sel], want[1])
    assert np.array_equal(c[sel], want[2])


def test_ragged_full_size_plan():
    """The 4M-read ragged workload in one plan launch (the benchmark's step)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1708_04329_gb300 import grim, synth

    w = synth.ragged_candidates()
    rs, off, cand = w["reads"], w["cand_off"], w["cand"]
    idx = build(w["genome"], w["B"], w["q"], w["max_read_len"], grim.GRIM_LAYOUT_BIN_MAJOR)
    kw = dev_reads(rs)
    kw["cand"] = torch.from_numpy(cand).cuda()
    kw["cand_off"] = torch.from_numpy(off.view(np.int64)).cuda()
    plan = grim.grim_plan_create(idx, max_reads=rs.n, max_bases=len(rs.seq), max_e=int(rs.e.max()),
                                 cap=4 * rs.n + 4096, max_cand=len(cand), candidates=True)
    r, b, c = (x.cpu().numpy() for x in plan.run(**kw))
    r, b = r.view(np.uint32), b.view(np.uint32)
    plan.close()
    k = 3000
    want = oracle.filter(oracle.bin_vectors(w["genome"], w["B"], w["q"], w["max_read_len"]),
                         rs.subset(range(k)), cand_off=off[: k + 1], cand=cand[: int(off[k])])
    sel = r < k
    assert np.array_equal(r[sel], want[0]) and np.array_equal(b[sel], want[1])
    assert np.array_equal(c[sel], want[2])
    # sorted by (read, candidate position); every read passes its true bin
    key = r.astype(np.uint64) << np.uint64(32) | b.astype(np.uint64)
    assert (np.diff(r.astype(np.int64)) >= 0).all()
    true_key = np.arange(rs.n, dtype=np.uint64) << np.uint64(32) | (rs.true_pos // w["B"]).astype(np.uint64)
    assert np.isin(true_key, key).all()
    idx.close()


def test_serving_index_two_level_at_full_size():
    """The serving index at full size: the 3.1 Gbp genome with B=200, q=5
    and max_read_len 250 (ext = 249, super-bin windows ~47% full), whose
    automatic all-bins path is coarse-then-exact.  50,000 reads of the
    serving pool (100-250 bp, e up to 5% of L): every bin for 24 sampled
    reads equals the oracle, and the exact pass gives the same pass list
    record for record."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1708_04329_gb300 import grim, synth

    w = synth.serving()
    rs = w["reads"].subset(np.arange(50_000))
    idx = build(w["genome"], w["B"], w["q"], w["max_read_len"])
    assert idx.desc.two_level == 1
    got = gpu_filter(idx, rs, cap=64 * rs.n)
    st = grim.grim_last_filter_stats()
    assert st["all_bins_path"] == grim.GRIM_PATH_TWO_LEVEL
    assert st["read_switch"] == grim.GRIM_SWITCH_GROUP  # mixed lengths and budgets
    oix = oracle.bin_vectors(w["genome"], w["B"], w["q"], w["max_read_len"])
    sample = np.linspace(0, rs.n - 1, 24).astype(np.int64)
    _check_slices(got, *oracle.filter(oix, rs.subset(sample)), sample)
    grim.grim_index_set_shape(idx, all_bins_path=grim.GRIM_PATH_EXACT)
    exact = gpu_filter(idx, rs, cap=64 * rs.n)
    assert grim.grim_last_filter_stats()["all_bins_path"] == grim.GRIM_PATH_EXACT
    for a, b in zip(exact, got):
        assert np.array_equal(a, b)
    idx.close()
