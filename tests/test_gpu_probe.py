"""The benchmark's random-gather probe (a measurement helper in bench_helpers/,
apart from the filter library) runs for both vector sizes and every unroll, and rejects bad
arguments on the host before any launch."""
import ctypes

import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def _lib():
    from bench_helpers import probe

    return probe()


def test_gather_probe_runs_and_checks_arguments():
    lib = _lib()
    table_bytes = 1 << 24
    table = torch.randint(-2 ** 31, 2 ** 31 - 1, (table_bytes // 4,), dtype=torch.int32,
                          device="cuda")
    words = int(lib.grim_probe_gather_sink_words())
    assert words > 0
    sink = torch.zeros(words, dtype=torch.int32, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for row_bytes in (128, 512):
        for unroll in (1, 2, 4):
            rc = lib.grim_probe_gather(table.data_ptr(), table_bytes // row_bytes, row_bytes,
                                       1 << 20, unroll, sink.data_ptr(), words, stream)
            assert rc == 0, (row_bytes, unroll, rc)
    torch.cuda.synchronize()
    assert bool(sink.ne(0).any())
    ok = dict(rows=table_bytes // 128, row_bytes=128, unroll=1, words=words)

    def call(**kw):
        a = {**ok, **kw}
        return lib.grim_probe_gather(a.get("table", table.data_ptr()), a["rows"], a["row_bytes"],
                                     1000, a["unroll"], sink.data_ptr(), a["words"], stream)

    assert call(row_bytes=64) == -1            # no probe for that row size
    assert call(unroll=3) == -1
    assert call(rows=0) == -1
    assert call(table=table.data_ptr() + 4) == -1  # not 16-byte aligned
    assert call(words=1) == -1                  # sink smaller than the launch
    torch.cuda.synchronize()
