"""Read existence sweep (§Parameter Evaluation Results, Fig. 4), on synthetic data.

The paper chooses its parameters from the *average read existence*: for a
representative set of reads, the fraction of all bins of the genome that pass
the filter, swept over the token length q (4-6), the number of bins
(multiples of 65,536) and the error tolerance (e = ceil(L x rate), Fig. 4
caption), with the mean and the min/max over several read sets.

This module runs the same sweep through the library's all-bins filter
(count-only calls: no pass list is materialised) on the seeded synthetic
genome and read sets of ``synth``; it needs the human reference and the
1000 Genomes read sets for nothing.

    python -m paper_1708_04329_gb300.existence --genome 3100000000 --json out.json
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import grim, synth

BINS_UNIT = 65536


def bin_size_for(n: int, bins_k: int) -> int:
    """Bin core size B giving about bins_k x 65,536 bins over n bases."""
    return max(1, math.ceil(n / (bins_k * BINS_UNIT)))


def read_existence(index: grim.GrimIndex, reads: dict, workspace=None) -> float:
    """Passing (read, bin) pairs / (reads x bins) for CUDA-resident reads."""
    n = int(reads["lens"].numel())
    if n == 0:
        return 0.0
    passing = grim.grim_filter_count(index, **reads, workspace=workspace)
    return passing / (n * index.desc.num_bins)


def _device_reads(rs, e: int):
    import torch

    return dict(reads=torch.from_numpy(rs.seq).cuda(),
                offsets=torch.from_numpy(rs.offsets.view(np.int64)).cuda(),
                lens=torch.from_numpy(rs.lens.view(np.int32)).cuda(),
                e=torch.full((rs.n,), e, dtype=torch.int16, device="cuda"))


def sweep(genome: np.ndarray, qs=(4, 5, 6), bins_k=(100, 200, 300, 450),
          rates_pct=(0, 1, 2, 3, 4, 5), n_sets: int = 4, reads_per_set: int = 2000,
          read_len: int = 100, max_edits: int = 3, seed: int = 9) -> list[dict]:
    """One row per (q, bins, rate): mean, min and max read existence over
    ``n_sets`` read sets of ``reads_per_set`` reads (L = read_len, 0..max_edits
    planted edits each)."""
    import torch

    sets = [synth.reads(genome, reads_per_set, seed=seed + 101 * k, lengths=(read_len,),
                        e=max_edits, max_edits=max_edits) for k in range(n_sets)]
    ref = torch.from_numpy(genome).cuda()
    ws = grim.Workspace()
    rows = []
    for q in qs:
        for k in bins_k:
            B = bin_size_for(len(genome), k)
            t0 = time.perf_counter()
            idx = grim.grim_build(ref, B, q, read_len,
                                  grim.GRIM_LAYOUT_TOKEN_MAJOR | grim.GRIM_LAYOUT_COARSE
                                  | grim.GRIM_LAYOUT_BIN_MAJOR)
            build_s = time.perf_counter() - t0
            for pct in rates_pct:
                e = grim.grim_edits_for_rate(read_len, pct, 100)
                vals = [read_existence(idx, _device_reads(rs, e), ws) for rs in sets]
                rows.append({"q": q, "bins_k": k, "bins": int(idx.desc.num_bins), "B": B,
                             "rate_pct": pct, "e": e, "mean": float(np.mean(vals)),
                             "min": float(np.min(vals)), "max": float(np.max(vals)),
                             "build_s": round(build_s, 3)})
            idx.close()
    return rows


def main():
    p = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    p.add_argument("--genome", type=int, default=synth.HUMAN_N)
    p.add_argument("--q", type=int, nargs="+", default=[4, 5, 6])
    p.add_argument("--bins-k", type=int, nargs="+", default=[100, 200, 300, 450])
    p.add_argument("--rates", type=int, nargs="+", default=[0, 1, 2, 3, 4, 5])
    p.add_argument("--sets", type=int, default=4)
    p.add_argument("--reads", type=int, default=2000)
    p.add_argument("--json", default=None)
    a = p.parse_args()
    g = synth.human_genome(a.genome)
    rows = sweep(g, a.q, a.bins_k, a.rates, a.sets, a.reads)
    for r in rows:
        print(f"q={r['q']} bins={r['bins_k']}x64k (B={r['B']}) rate={r['rate_pct']}% e={r['e']}: "
              f"existence mean {r['mean']:.3e} [{r['min']:.3e}, {r['max']:.3e}]")
    if a.json:
        with open(a.json, "w") as f:
            json.dump(rows, f, indent=1)


if __name__ == "__main__":
    main()
