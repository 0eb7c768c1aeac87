"""The multi-rank (weak scaling) host logic of bench.py on CPU: two gloo
ranks each filter their own reads, with no collective on the data path; the
step time is the slowest rank's and the job's throughput counts the units of
every rank.  The filtering here is the oracle (the CPU stand-in of one rank's
GPU work), so the test needs no GPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port() -> int:
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank: int, world: int, port: int, out_dir: str):
    import json
    import sys
    import time

    import torch.distributed as dist

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    import oracle
    from paper_1708_04329_gb300 import synth

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    g = synth.genome(200_000, seed=1)
    rs = synth.reads(g, 40, seed=bench.rank_seed(11, rank), lengths=(100,), e=5, max_edits=5)
    oix = oracle.bin_vectors(g, 200, 5, 100)
    dist.barrier()
    t0 = time.perf_counter()
    r, b, c = oracle.filter(oix, rs)
    ms = (time.perf_counter() - t0) * 1e3 + 50.0 * rank  # rank 1 is the slow one
    ms_max = bench.max_over_ranks(ms, dist, "cpu")
    value = bench.weak_value(rs.n, world, ms_max)
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump({"ms": ms, "ms_max": ms_max, "value": value, "n": rs.n,
                   "true_pos": rs.true_pos.tolist(), "pairs": len(r),
                   "hits_true_bin": int(sum(1 for i in range(rs.n)
                                            if ((r == i) & (b == rs.true_pos[i] // 200)).any()))},
                  f)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_weak_scaling(tmp_path):
    import json

    import torch.multiprocessing as mp

    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    res = [json.loads((tmp_path / f"rank{k}.json").read_text()) for k in range(2)]
    # each rank filtered its own reads
    assert res[0]["true_pos"] != res[1]["true_pos"]
    # rank 0's reads are the single-GPU workload's
    from paper_1708_04329_gb300 import synth

    import bench

    g = synth.genome(200_000, seed=1)
    solo = synth.reads(g, 40, seed=bench.rank_seed(11, 0), lengths=(100,), e=5, max_edits=5)
    assert res[0]["true_pos"] == solo.true_pos.tolist()
    # the job's time is the slowest rank's, seen identically by both ranks
    assert res[0]["ms_max"] == res[1]["ms_max"] == pytest.approx(max(r["ms"] for r in res))
    # throughput counts every rank's reads against that time
    assert res[0]["value"] == pytest.approx(80 / (res[0]["ms_max"] / 1e3))
    # the q-gram lemma on each shard: every read passes its true bin
    assert all(r["hits_true_bin"] == r["n"] for r in res)
