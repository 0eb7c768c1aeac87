"""Helpers for the GPU tests: move seeded inputs to the device, call the C-ABI
through the binding, and bring results back as numpy arrays."""
from __future__ import annotations

import numpy as np


def dev_reads(rs):
    import torch

    return dict(reads=torch.from_numpy(np.ascontiguousarray(rs.seq)).cuda(),
                offsets=torch.from_numpy(np.ascontiguousarray(rs.offsets, np.uint64).view(np.int64)).cuda(),
                lens=torch.from_numpy(np.ascontiguousarray(rs.lens, np.uint32).view(np.int32)).cuda(),
                e=torch.from_numpy(np.ascontiguousarray(rs.e, np.uint16).view(np.int16)).cuda())


def build(genome: np.ndarray, B: int, q: int, mrl: int, layouts: int = 7, coarse_factor: int = 0):
    import torch

    from paper_1708_04329_gb300 import grim

    ref = torch.from_numpy(np.ascontiguousarray(genome)).cuda()
    if coarse_factor:
        return grim.grim_build_ex(ref, B, q, mrl, layouts, coarse_factor)
    return grim.grim_build(ref, B, q, mrl, layouts)


def gpu_filter(idx, rs, cand_off=None, cand=None, cap=None, workspace=None):
    import torch

    from paper_1708_04329_gb300 import grim

    kw = dev_reads(rs)
    if cand is not None:
        kw["cand"] = torch.from_numpy(np.ascontiguousarray(cand, np.int32)).cuda()
        kw["cand_off"] = torch.from_numpy(np.ascontiguousarray(cand_off, np.uint64).view(np.int64)).cuda()
    r, b, c = grim.grim_filter(idx, **kw, cap=cap, workspace=workspace)
    torch.cuda.synchronize()
    return (r.cpu().numpy().view(np.uint32), b.cpu().numpy().view(np.uint32), c.cpu().numpy())


def assert_same(got, want):
    gr, gb, gc = got
    wr, wb, wc = want
    assert len(gr) == len(wr), (len(gr), len(wr))
    assert np.array_equal(gr, wr)
    assert np.array_equal(gb, wb)
    assert np.array_equal(gc, wc)
