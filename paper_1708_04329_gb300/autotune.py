"""Autotuner for the filter's tile shapes, by measurement on the GPU.

Two shapes are tuned, each by timing real filter runs on a sample of the
caller's reads with CUDA events:

* the bin tile of the all-bins mode: the coarse factor f (bins per super-bin
  of the coarse table).  Candidates are the power-of-two neighbours of the
  presence-model default; each needs its own index build (~0.1 s at 3.1 Gbp).
* the read tile of the candidate mode: how many candidate gathers each lane
  group keeps in flight (1, 2, 4 or 8), timed through graph-captured plans.

Results are cached in a JSON file keyed by the problem's shape and the GPU,
so a service tunes once per (reference, parameters, device).
"""
from __future__ import annotations

import json
import os
import statistics
from pathlib import Path

from . import grim

DEFAULT_CACHE = Path(os.environ.get("GRIM_AUTOTUNE_CACHE",
                                    Path.home() / ".cache" / "grim_gb300" / "autotune.json"))


def _device_name() -> str:
    import torch

    return torch.cuda.get_device_name()


def _load(cache: Path | None) -> dict:
    if cache is None or not cache.exists():
        return {}
    try:
        return json.loads(cache.read_text())
    except (OSError, ValueError):
        return {}


def _store(cache: Path | None, table: dict) -> None:
    if cache is None:
        return
    cache.parent.mkdir(parents=True, exist_ok=True)
    tmp = cache.with_suffix(f".tmp{os.getpid()}")
    tmp.write_text(json.dumps(table, indent=1, sort_keys=True))
    os.replace(tmp, cache)


def _time(fn, repeats: int) -> float:
    """Median milliseconds of fn() over `repeats` runs after one warm-up."""
    import torch

    fn()
    torch.cuda.synchronize()
    times = []
    for _ in range(repeats):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        b.synchronize()
        times.append(a.elapsed_time(b))
    return statistics.median(times)


def tune_coarse_factor(ref, B: int, q: int, max_read_len: int, sample: dict,
                       factors: list[int] | None = None, repeats: int = 2,
                       cache: Path | None = DEFAULT_CACHE) -> dict:
    """Pick the coarse factor for all-bins filtering of reads like `sample`.

    ref: uint8 CUDA tensor of the reference; sample: the grim_filter keyword
    arguments (reads, offsets, lens, e) of a few thousand to a few hundred
    thousand representative reads.  Returns {"factor": f, "ms": {f: ms}}.
    """
    key = f"coarse|{int(ref.numel())}|{B}|{q}|{max_read_len}|{int(sample['lens'].numel())}|{_device_name()}"
    table = _load(cache)
    if key in table:
        return table[key]
    if factors is None:
        f0 = grim.grim_default_coarse_factor(B, q, max_read_len)
        factors = sorted({max(2, f0 // 2), f0, min(64, f0 * 2)})
    ws = grim.Workspace()
    ms = {}
    for f in factors:
        idx = grim.grim_build_ex(ref, B, q, max_read_len, grim.GRIM_LAYOUT_ALL, f)
        try:
            ms[f] = _time(lambda: grim.grim_filter(idx, **sample, workspace=ws), repeats)
        finally:
            idx.close()
    best = min(ms, key=ms.get)
    out = {"factor": int(best), "ms": {str(k): round(v, 3) for k, v in ms.items()}}
    table[key] = out
    _store(cache, table)
    return out


def tune_candidate_unroll(index, sample: dict, max_e: int, unrolls=(1, 2, 4, 8), repeats: int = 3,
                          cache: Path | None = DEFAULT_CACHE) -> dict:
    """Pick the number of candidate gathers in flight per lane group.

    sample: the candidate-mode grim_filter keyword arguments (reads, offsets,
    lens, e, cand, cand_off) as CUDA tensors.  Each setting is timed through
    a graph-captured plan sized for the sample.  Returns
    {"unroll": u, "ms": {u: ms}}.
    """
    n = int(sample["lens"].numel())
    nc = int(sample["cand"].numel())
    d = index.desc
    key = f"cand|{d.num_bins}|{d.q}|{n}|{nc}|{_device_name()}"
    table = _load(cache)
    if key in table:
        return table[key]
    ms = {}
    for u in unrolls:
        plan = grim.grim_plan_create(index, max_reads=n, max_bases=int(sample["reads"].numel()),
                                     max_e=max_e, cap=n * 8 + 1024, max_cand=nc, candidates=True,
                                     cand_unroll=u)
        try:
            plan.stage(**sample)

            def run():
                grim.grim_plan_launch(plan, n, nc)
                grim.grim_plan_wait(plan)

            ms[u] = _time(run, repeats)
        finally:
            plan.close()
    best = min(ms, key=ms.get)
    out = {"unroll": int(best), "ms": {str(k): round(v, 3) for k, v in ms.items()}}
    table[key] = out
    _store(cache, table)
    return out
