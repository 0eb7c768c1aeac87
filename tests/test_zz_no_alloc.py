"""grim_filter_noalloc -- the filter for callers that cannot allocate device
memory (a process whose memory manager owns the GPU, or a serving loop that
keeps cudaMalloc off its request path) -- gives exactly what grim_filter gives.

Its scratch is one fixed array inside the library that every call reuses, so
the check runs two different calls in a row (the second must not see the
first one's leftovers), in both filter modes, and checks that a call too big
for the array is refused.  This file is collected last on purpose.
"""
import numpy as np
import pytest

from tests.gpu_helpers import build, dev_reads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    from paper_1708_04329_gb300 import synth

    g = synth.genome(400_000, seed=21)
    idx = build(g, 200, 5, 100)
    first = synth.reads(g, 3000, seed=22, e=5, max_edits=5)
    second = synth.reads(g, 700, seed=23, e=3, max_edits=3)
    return idx, first, second


def _np(t):
    return tuple(x.cpu().numpy() for x in t)


def _outs(cap):
    return tuple(torch.empty(cap, dtype=dt, device="cuda")
                 for dt in (torch.int32, torch.int32, torch.uint8))


def _cands(rs, nb, seed):
    from paper_1708_04329_gb300 import synth

    off, cand = synth.candidates((rs.true_pos // 200).astype(np.int32), nb, seed=seed, median=40)
    return dict(cand=torch.from_numpy(cand).cuda(),
                cand_off=torch.from_numpy(off.view(np.int64)).cuda())


def test_noalloc_equals_filter_on_two_calls_in_a_row(setup):
    from paper_1708_04329_gb300 import grim

    idx, first, second = setup
    nb = idx.desc.num_bins
    calls = []
    for rs, seed in ((first, 31), (second, 32)):
        kw = dev_reads(rs)
        cap = 8 * rs.n + 64
        calls.append((kw, cap, {}))
        calls.append((kw, cap, _cands(rs, nb, seed)))
    # the existing entry point's answers first ...
    wants = [_np(grim.grim_filter(idx, **kw, **ck, cap=cap)) for kw, cap, ck in calls]
    # ... then the no-allocation entry point, all-bins mode on the two read
    # sets back to back, then candidate mode on the two back to back
    order = [0, 2, 1, 3]
    for i in order:
        kw, cap, ck = calls[i]
        got = _np(grim.grim_filter_noalloc(idx, **kw, **ck, out=_outs(cap)))
        assert len(got[0]) == len(wants[i][0]) > 0
        for a, b in zip(got, wants[i]):
            assert np.array_equal(a, b)


def test_noalloc_refuses_calls_beyond_its_scratch(setup):
    from paper_1708_04329_gb300 import grim

    idx, first, _ = setup
    kw = dev_reads(first)
    limit = grim.grim_noalloc_scratch_bytes()
    too_big = limit // 18 + 1  # output capacity alone overflows it
    assert grim.grim_filter_workspace_size(idx, first.n, 0, too_big) > limit
    with pytest.raises(grim.GrimError) as ei:
        grim.grim_filter_noalloc(idx, **kw, out=_outs(too_big))
    assert ei.value.code == grim.GRIM_E_WORKSPACE
