"""Index persistence: an index written by grim_save and read back by
grim_load holds the same table bits and gives the same pass lists; subsets
of the stored tables load alone; damaged files are refused."""
import numpy as np
import pytest

import oracle
from tests.gpu_helpers import assert_same, build, gpu_filter

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def world():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    from paper_1708_04329_gb300 import synth

    g = synth.human_genome(450_000, seed=81)
    return g, oracle.bin_vectors(g, 150, 5, 120)


def _tables(idx):
    out = {}
    for name in ("token_major", "bin_major", "coarse_token_major"):
        t = getattr(idx, name)()
        out[name] = None if t is None else t.cpu().numpy().copy()
    return out


def test_save_load_roundtrip(world, tmp_path):
    from paper_1708_04329_gb300 import grim, synth

    g, oix = world
    idx = build(g, 150, 5, 120, 7, coarse_factor=4)
    path = tmp_path / "g.grim"
    grim.grim_save(idx, path)
    back = grim.grim_load(path, verify=True)
    d0, d1 = idx.desc, back.desc
    for f in ("ref_len", "num_bins", "num_bins_pad", "B", "q", "ext", "max_read_len", "layouts",
              "coarse_factor", "num_coarse"):
        assert getattr(d0, f) == getattr(d1, f), f
    t0, t1 = _tables(idx), _tables(back)
    for k in t0:
        assert np.array_equal(t0[k], t1[k]), k
    rs = synth.reads(g, 300, seed=82, lengths=(80, 120), probs=(0.5, 0.5), e_frac=(5, 100),
                     max_edits=None)
    want = oracle.filter(oix, rs)
    assert_same(gpu_filter(back, rs), want)
    off, cand = synth.candidates((rs.true_pos // 150).astype(np.int32), oix.num_bins, seed=83,
                                 median=30)
    assert_same(gpu_filter(back, rs, off, cand), oracle.filter(oix, rs, cand_off=off, cand=cand))
    # one table alone
    bm = grim.grim_load(path, layouts=grim.GRIM_LAYOUT_BIN_MAJOR)
    assert bm.desc.layouts == grim.GRIM_LAYOUT_BIN_MAJOR
    assert np.array_equal(bm.bin_major().cpu().numpy(), t0["bin_major"])
    tm = grim.grim_load(path, layouts=grim.GRIM_LAYOUT_TOKEN_MAJOR)
    assert_same(gpu_filter(tm, rs), want)


def test_load_errors(world, tmp_path):
    from paper_1708_04329_gb300 import grim

    g, _ = world
    idx = build(g, 150, 5, 120, grim.GRIM_LAYOUT_BIN_MAJOR)
    path = tmp_path / "b.grim"
    grim.grim_save(idx, path)
    with pytest.raises(grim.GrimError) as ei:
        grim.grim_load(path, layouts=grim.GRIM_LAYOUT_TOKEN_MAJOR)
    assert ei.value.code == grim.GRIM_E_NO_LAYOUT
    raw = bytearray(path.read_bytes())
    raw[256 + 1000] ^= 0x10  # one flipped bit in the table
    bad = tmp_path / "bad.grim"
    bad.write_bytes(bytes(raw))
    grim.grim_load(bad)  # not verified: loads
    with pytest.raises(grim.GrimError) as ei:
        grim.grim_load(bad, verify=True)
    assert ei.value.code == grim.GRIM_E_FORMAT
    short = tmp_path / "short.grim"
    short.write_bytes(bytes(raw[:-4096]))
    with pytest.raises(grim.GrimError) as ei:
        grim.grim_load(short)
    assert ei.value.code == grim.GRIM_E_FORMAT
