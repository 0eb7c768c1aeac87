"""bench.py's reference arm (the CPU oracle on the host cores) prints one
JSON line with the contract's keys; it needs no GPU."""
import json
import subprocess
import sys

from tests.conftest import ROOT


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, str(ROOT / "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "1"], capture_output=True, text=True,
                         timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config"):
        assert key in line, key
    assert line["value"] > 0 and line["higher_is_better"] is True
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert "workload" in line["config"]


def _fake_trace_parts(n=20):
    import numpy as np

    class Info:
        t_done_ns = t_launch_ns = t_submit_ns = 0
        batch_requests = batch_reads = 1

    class Pool:
        offsets = np.arange(n, dtype=np.uint64) * 10
        lens = np.full(n, 10, np.uint32)
        seq = np.zeros(10 * n, np.uint8)
        e = np.zeros(n, np.uint16)

    trace = dict(t=np.linspace(0, 0.01, n), size=np.ones(n, int), start=np.arange(n))
    return Info, Pool(), trace


def test_serve_trace_ends_with_a_failed_submit_or_result():
    """The serving bench's trace runner (host logic, a fake server): a request
    the server refuses, or a result that fails, ends the run with that error
    at once; no result thread is left waiting."""
    import threading

    import pytest

    sys.path.insert(0, str(ROOT))
    import bench

    Info, pool, trace = _fake_trace_parts()

    class Server:
        def __init__(self, bad_submit=0, bad_result=0):
            self.k, self.bad_submit, self.bad_result = 0, bad_submit, bad_result

        def submit(self, **kw):
            self.k += 1
            if self.k == self.bad_submit:
                raise ValueError("refused")
            return self.k

        def result(self, ticket):
            if ticket == self.bad_result:
                raise RuntimeError("failed")
            return (None, None, None), Info()

    before = threading.active_count()
    for paced in (False, True):
        with pytest.raises(ValueError):
            bench._serve_trace(Server(bad_submit=5), pool, trace, paced=paced)
        with pytest.raises(RuntimeError):
            bench._serve_trace(Server(bad_result=3), pool, trace, paced=paced)
        assert bench._serve_trace(Server(), pool, trace, paced=paced)["requests"] == 20
    assert threading.active_count() == before
