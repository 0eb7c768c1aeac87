"""The all-bins autotuner and the launch shapes it chooses from.

Every launch shape of the all-bins kernel (CTA size, read-range size, read
switch), both all-bins paths, and every bin tile the tuner tries (coarse
factors, one exact pass) must give
exactly the oracle's pass list; the tuner's pick, built into an index the way
a caller builds it, must too.  Reads are mixed in length (100-250 bp) with
per-read budgets, so the read ranges hold uneven reads.
"""
import numpy as np
import pytest

import oracle
from tests.gpu_helpers import assert_same, dev_reads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def world():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    from paper_1708_04329_gb300 import synth

    g = synth.human_genome(2_000_000, seed=51)
    rs = synth.reads(g, 6000, seed=52, lengths=(100, 150, 250), probs=(0.5, 0.3, 0.2),
                     e_frac=(5, 100), max_edits=None)
    oix = oracle.bin_vectors(g, 200, 5, 250)
    return g, rs, oracle.filter(oix, rs)


def _host(got):
    r, b, c = got
    return r.cpu().numpy().view(np.uint32), b.cpu().numpy().view(np.uint32), c.cpu().numpy()


def test_every_launch_shape_matches_oracle(world):
    from paper_1708_04329_gb300 import grim

    g, rs, want = world
    ref = torch.from_numpy(g).cuda()
    kw = dev_reads(rs)
    for layouts in (grim.GRIM_LAYOUT_ALL, grim.GRIM_LAYOUT_TOKEN_MAJOR):
        idx = grim.grim_build_ex(ref, 200, 5, 250, layouts, 0, cta_threads=512,
                                 read_range_kb=1024)
        d = idx.desc
        assert (d.cta_threads, d.read_range_kb) == (512, 1024)
        # 1 MiB ranges split the 6000 reads' 1.5 MB of token rows in two
        for threads in (512, 640, 768):
            for range_kb in (1024, 0):
                for switch in (0, grim.GRIM_SWITCH_GROUP, grim.GRIM_SWITCH_WARP):
                    grim.grim_index_set_shape(idx, threads, range_kb, switch)
                    assert_same(_host(grim.grim_filter(idx, **kw)), want)
        if layouts == grim.GRIM_LAYOUT_ALL:
            # both all-bins paths, forced
            for path in (grim.GRIM_PATH_TWO_LEVEL, grim.GRIM_PATH_EXACT):
                grim.grim_index_set_shape(idx, 640, 1024, 0, path)
                assert idx.desc.two_level == (path == grim.GRIM_PATH_TWO_LEVEL)
                assert_same(_host(grim.grim_filter(idx, **kw)), want)
        else:  # no coarse table: the two-level path cannot be forced
            with pytest.raises(grim.GrimError) as ei:
                grim.grim_index_set_shape(idx, all_bins_path=grim.GRIM_PATH_TWO_LEVEL)
            assert ei.value.code == grim.GRIM_E_NO_LAYOUT
        grim.grim_index_set_shape(idx)  # defaults
        d = idx.desc
        assert (d.cta_threads, d.read_range_kb, d.read_switch, d.all_bins_path) == (640, 48 << 10, 0, 0)
        # reads up to 250 bp: super-bins of 2 x 200 bp hold ~47% of all tokens,
        # under the 50% bound, so the automatic path is coarse-then-exact
        assert d.two_level == (layouts == grim.GRIM_LAYOUT_ALL)
        for bad in ((600, 0, 0), (0, 512, 0), (0, (4 << 20) + 1, 0), (0, 0, 3), (0, 0, 0, 3)):
            with pytest.raises(grim.GrimError) as ei:
                grim.grim_index_set_shape(idx, *bad)
            assert ei.value.code == grim.GRIM_E_ARG
        idx.close()


def test_tuned_shape_matches_oracle(world):
    from paper_1708_04329_gb300 import autotune, grim

    g, rs, want = world
    ref = torch.from_numpy(g).cuda()
    kw = dev_reads(rs)
    tuned = autotune.tune_all_bins(ref, 200, 5, 250, kw, ranges_kb=(1024,), repeats=1,
                                   cache=None)
    f0 = grim.grim_default_coarse_factor(200, 5, 250)
    assert set(tuned["ms"]) >= {"exact", f"f={f0}", "threads=512", "threads=640", "threads=768",
                                "range_kb=1024", "switch=1", "switch=2"}
    assert tuned["factor"] in (max(2, f0 // 2), f0, f0 * 2)
    assert tuned["all_bins_path"] in (grim.GRIM_PATH_TWO_LEVEL, grim.GRIM_PATH_EXACT)
    idx = grim.grim_build_ex(ref, 200, 5, 250, grim.GRIM_LAYOUT_ALL, tuned["factor"],
                             cta_threads=tuned["cta_threads"], read_range_kb=tuned["read_range_kb"],
                             read_switch=tuned["read_switch"],
                             all_bins_path=tuned["all_bins_path"])
    assert_same(_host(grim.grim_filter(idx, **kw)), want)
    # and through a graph-captured plan, which takes the index's shape when created
    plan = grim.grim_plan_create(idx, max_reads=rs.n, max_bases=len(rs.seq), max_e=int(rs.e.max()),
                                 cap=8 * rs.n)
    assert_same(_host(plan.run(**kw)), want)
    plan.close()
    idx.close()
