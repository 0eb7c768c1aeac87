"""Autotuner for the filter's tile shapes, by measurement on the GPU.

The shapes are tuned by timing real filter runs on a sample of the caller's
reads with CUDA events:

* all-bins mode (``tune_all_bins``), by coordinate descent:
  - the bin tile: the coarse factor f (bins per super-bin of the coarse
    table) among the power-of-two neighbours of the presence-model default,
    each with its own index build (~0.1 s at 3.1 Gbp) and the two-level path,
    or one exact pass over every bin;
  - the CTA size of the persistent kernel (512, 640 or 768 threads: warps
    per SM against registers per thread);
  - the read tile: KiB of token rows per read range (a range stays in L2
    while every CTA sweeps its tiles against it);
  - how a warp's lane groups take their next reads (each on its own, or
    all together).
  A trial replaces the current choice only if it is faster by more than
  ``min_gain`` (1%): smaller differences are run-to-run noise.
  The paper ties its throughput to the same two widths: how many bins one
  row fetch covers and how many reads share it (§Parameter Evaluation
  Results, parallel width p).
* candidate mode (``tune_candidate_unroll``): how many candidate gathers
  each lane group keeps in flight (1, 2, 4 or 8), timed through
  graph-captured plans.

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


def _token_bytes(n_reads: int, q: int, max_read_len: int) -> int:
    """Token-row bytes the all-bins kernel sweeps for n_reads reads: a 16-token
    aligned row of uint16 per read, in four copies at q = 6."""
    ts = (max_read_len - q + 1 + 15) // 16 * 16
    return n_reads * ts * 2 * (4 if q >= 6 else 1)


def tune_all_bins(ref, B: int, q: int, max_read_len: int, sample: dict,
                  factors: list[int] | None = None, threads=(512, 640, 768),
                  ranges_kb=(12 << 10, 24 << 10, 48 << 10, 96 << 10), switches=(1, 2),
                  repeats: int = 2, min_gain: float = 0.01,
                  cache: Path | None = DEFAULT_CACHE) -> dict:
    """Pick the all-bins mode's tile shapes for reads like `sample`.

    ref: uint8 CUDA tensor of the reference; sample: the grim_filter keyword
    arguments (reads, offsets, lens, e) of representative reads, enough to
    fill the GPU (tens of thousands or more).  Read ranges are only compared
    when the sample's token rows span more than one of them.  Returns
    {"factor": f, "all_bins_path": GRIM_PATH_TWO_LEVEL or GRIM_PATH_EXACT,
    "cta_threads": t, "read_range_kb": r, "read_switch": w, "ms": {trial: ms}};
    build the index with grim_build_ex(..., coarse_factor=f, cta_threads=t,
    read_range_kb=r, read_switch=w, all_bins_path=p).
    """
    n = int(sample["lens"].numel())
    key = (f"allbins|{int(ref.numel())}|{B}|{q}|{max_read_len}|{n}|"
           f"{tuple(threads)}|{tuple(ranges_kb)}|{tuple(switches)}|{_device_name()}")
    table = _load(cache)
    if key in table:
        return table[key]
    f0 = grim.grim_default_coarse_factor(B, q, max_read_len)
    if factors is None:
        factors = sorted({max(2, f0 // 2), f0, min(64, f0 * 2)})
    factors = [f0] + [f for f in factors if f != f0]
    two, exact = grim.GRIM_PATH_TWO_LEVEL, grim.GRIM_PATH_EXACT
    ws = grim.Workspace()
    ms = {}

    def build(f, path):
        return grim.grim_build_ex(ref, B, q, max_read_len, grim.GRIM_LAYOUT_ALL, f,
                                  all_bins_path=path)

    def run(index):
        return _time(lambda: grim.grim_filter(index, **sample, workspace=ws), repeats)

    def pick(cur, options, name):
        """The option to keep: the current one unless another beats it by more
        than min_gain."""
        best = cur
        for o in options:
            if ms[f"{name}={o}"] < ms[f"{name}={best}"] * (1.0 - min_gain):
                best = o
        return best

    # 1. bin tile: the two-level path at each coarse factor (the first is the
    #    default), and one exact pass, at the default launch shape
    for f in factors:
        index = build(f, two)
        try:
            ms[f"f={f}"] = run(index)
            if f == f0:
                grim.grim_index_set_shape(index, all_bins_path=exact)
                ms["exact"] = run(index)
        finally:
            index.close()
    best_f = pick(factors[0], factors, "f")
    path = exact if ms["exact"] < ms[f"f={best_f}"] * (1.0 - min_gain) else two
    if path == exact:
        best_f = f0
    index = build(best_f, path)
    try:
        d = index.desc
        best_t, best_r, best_w = d.cta_threads, d.read_range_kb, d.read_switch
        ms[f"threads={best_t}"] = ms["exact" if path == exact else f"f={best_f}"]
        # 2. CTA size
        for t in threads:
            if t != best_t:
                grim.grim_index_set_shape(index, t, best_r, best_w, path)
                ms[f"threads={t}"] = run(index)
        best_t = pick(best_t, threads, "threads")
        ms[f"switch={best_w}"] = ms[f"threads={best_t}"]
        # 3. read switch
        for w in switches:
            if w != best_w:
                grim.grim_index_set_shape(index, best_t, best_r, w, path)
                ms[f"switch={w}"] = run(index)
        best_w = pick(best_w, switches, "switch")
        ms[f"range_kb={best_r}"] = ms[f"switch={best_w}"]
        # 4. read tile: only sizes that split the sample into several ranges
        tb = _token_bytes(n, q, max_read_len)
        tried = [r for r in ranges_kb if (r << 10) < tb and r != best_r]
        for r in tried:
            grim.grim_index_set_shape(index, best_t, r, best_w, path)
            ms[f"range_kb={r}"] = run(index)
        best_r = pick(best_r, tried, "range_kb")
    finally:
        index.close()
    out = {"factor": int(best_f), "all_bins_path": int(path), "cta_threads": int(best_t),
           "read_range_kb": int(best_r), "read_switch": int(best_w),
           "ms": {k: round(v, 3) for k, v in ms.items()}, "sample_reads": n}
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
