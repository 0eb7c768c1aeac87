"""Graph-captured plans: ragged batches (mixed read lengths, per-read e,
ragged candidate lists) replayed through one captured graph give exactly the
oracle's pass lists, batch after batch, on every path the device can choose."""
import numpy as np
import pytest

import oracle
from tests.conftest import Reads
from tests.gpu_helpers import assert_same, build, dev_reads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def world():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    from paper_1708_04329_gb300 import synth

    g = synth.human_genome(600_000, seed=31)
    oix = oracle.bin_vectors(g, 200, 5, 250)
    return g, oix


def _ragged(g, n, seed):
    from paper_1708_04329_gb300 import synth

    return synth.reads(g, n, seed=seed, lengths=(100, 150, 250), probs=(0.5, 0.3, 0.2),
                       e_frac=(5, 100), max_edits=None)


def _host(t):
    return t.cpu().numpy().view(np.uint32) if t.dtype != torch.uint8 else t.cpu().numpy()


@pytest.mark.parametrize("layouts,path", [(1, 0), (6, 0), (7, 0), (7, 1), (7, 2)])
def test_all_bins_plan_batches(world, layouts, path):
    """Every path a plan can capture: one exact pass (layouts 1, or path 2),
    coarse-then-exact (layouts 6, path 1, or automatic with layouts 7: the
    super-bin window of an index for 250 bp reads holds ~47% of the tokens,
    under the 50% bound), with the device's per-batch rules."""
    from paper_1708_04329_gb300 import grim

    g, oix = world
    idx = build(g, 200, 5, 250, layouts)
    grim.grim_index_set_shape(idx, all_bins_path=path)
    assert idx.desc.two_level == (path == 1 or (path == 0 and layouts in (6, 7)))
    plan = grim.grim_plan_create(idx, max_reads=900, max_bases=900 * 250, max_e=20, cap=40_000)
    batches = [_ragged(g, 900, 40), _ragged(g, 37, 41), _ragged(g, 500, 42)]
    t_le0 = _ragged(g, 20, 43)
    t_le0.e[:5] = 20  # T <= 0 for these: the device must take the exact pass (or keep all)
    batches.append(t_le0)
    for rs in batches:
        got = plan.run(**dev_reads(rs))
        assert_same(tuple(_host(x) for x in got), oracle.filter(oix, rs))
    # an empty batch
    z = Reads([], [])
    got = plan.run(**dev_reads(z))
    assert got[0].numel() == 0


def test_candidate_plan_batches(world):
    from paper_1708_04329_gb300 import grim, synth

    g, oix = world
    idx = build(g, 200, 5, 250, 2)
    plan = grim.grim_plan_create(idx, max_reads=800, max_bases=800 * 250, max_e=20, cap=50_000,
                                 max_cand=800 * 400, candidates=True)
    for n, seed in ((800, 50), (3, 51), (333, 52)):
        rs = _ragged(g, n, seed)
        off, cand = synth.candidates((rs.true_pos // 200).astype(np.int32), oix.num_bins, seed=seed,
                                     median=60)
        c = torch.from_numpy(cand).cuda()
        co = torch.from_numpy(off.view(np.int64)).cuda()
        got = plan.run(**dev_reads(rs), cand=c, cand_off=co)
        assert_same(tuple(_host(x) for x in got), oracle.filter(oix, rs, cand_off=off, cand=cand))


def test_plan_equals_filter_and_reports_errors(world):
    from paper_1708_04329_gb300 import grim

    g, oix = world
    idx = build(g, 200, 5, 250)
    rs = _ragged(g, 400, 60)
    plan = grim.grim_plan_create(idx, max_reads=400, max_bases=400 * 250, max_e=12, cap=5)
    kw = dev_reads(rs)
    want = oracle.filter(oix, rs)
    # too small an output capacity: the total comes back
    plan.stage(**kw)
    grim.grim_plan_launch(plan, rs.n)
    with pytest.raises(grim.GrimError) as ei:
        grim.grim_plan_wait(plan)
    assert ei.value.code == grim.GRIM_E_OVERFLOW and ei.value.n_out == len(want[0])
    # a read with e above the declared maximum fails the batch
    big = plan.buffers["e"]
    big[:rs.n].copy_(kw["e"])
    big[0] = 13
    grim.grim_plan_launch(plan, rs.n)
    with pytest.raises(grim.GrimError) as ei:
        grim.grim_plan_wait(plan)
    assert ei.value.code == grim.GRIM_E_ARG
    # a plan as large as the batch agrees with grim_filter
    plan2 = grim.grim_plan_create(idx, max_reads=400, max_bases=400 * 250, max_e=12, cap=20_000)
    got = tuple(_host(x) for x in plan2.run(**kw))
    assert_same(got, want)
    assert grim.grim_plan_query(plan2)
    assert grim.grim_plan_device_bytes(plan2) > 0
    with pytest.raises(grim.GrimError):
        grim.grim_plan_launch(plan2, 401)


def test_ragged_candidates_sampled_parity():
    """The ragged candidate workload at 200 Mbp / 200k reads (~66M pairs) in one
    plan launch; the oracle checks the first 3,000 reads' lists exactly."""
    from paper_1708_04329_gb300 import autotune, grim, synth

    w = synth.ragged_candidates(n_reads=200_000, n=200_000_000)
    rs, off, cand = w["reads"], w["cand_off"], w["cand"]
    idx = build(w["genome"], w["B"], w["q"], w["max_read_len"], 2)
    kw = dev_reads(rs)
    kw["cand"] = torch.from_numpy(cand).cuda()
    kw["cand_off"] = torch.from_numpy(off.view(np.int64)).cuda()
    ns = 20_000
    cs = int(off[ns])
    sample = dict(reads=kw["reads"][: int(rs.offsets[ns - 1] + rs.lens[ns - 1])],
                  offsets=kw["offsets"][:ns], lens=kw["lens"][:ns], e=kw["e"][:ns],
                  cand=kw["cand"][:cs], cand_off=kw["cand_off"][: ns + 1])
    tuned = autotune.tune_candidate_unroll(idx, sample, int(rs.e.max()), cache=None)
    assert tuned["unroll"] in (1, 2, 4, 8)
    plan = grim.grim_plan_create(idx, max_reads=rs.n, max_bases=len(rs.seq), max_e=int(rs.e.max()),
                                 cap=4 * rs.n, max_cand=len(cand), candidates=True,
                                 cand_unroll=tuned["unroll"])
    r, b, c = (_host(x) for x in plan.run(**kw))
    k = 3000
    sub = rs.subset(range(k))
    want = oracle.filter(oracle.bin_vectors(w["genome"], w["B"], w["q"], w["max_read_len"]), sub,
                         cand_off=off[: k + 1], cand=cand[: int(off[k])])
    sel = r < k
    assert_same((r[sel], b[sel], c[sel]), want)
    # every read passes its true bin (planted edits <= e)
    assert set(zip(r.tolist(), b.tolist())) >= {(i, int(rs.true_pos[i]) // w["B"]) for i in range(rs.n)}
