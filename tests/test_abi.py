"""The C-ABI library builds, loads and exports every symbol include/grim.h
declares (no compute call: this runs without a GPU)."""
import re
import subprocess

import pytest

from tests.conftest import ROOT


def _declared() -> set[str]:
    text = (ROOT / "include" / "grim.h").read_text()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return set(re.findall(r"^[A-Za-z_][\w\s\*]*?\b(grim_\w+)\s*\(", text, flags=re.M))


def test_header_declares_the_binding_names():
    from paper_1708_04329_gb300 import grim

    assert _declared() == set(grim.EXPORTS)


def test_library_exports_every_declared_symbol():
    from paper_1708_04329_gb300 import grim

    lib = grim._lib()
    for name in _declared():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", grim.library_path()], capture_output=True,
                         text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    assert _declared() <= exported


def test_host_helpers_without_gpu():
    from paper_1708_04329_gb300 import grim

    # the no-allocation entry point's scratch size, as the header states it
    hdr = (ROOT / "include" / "grim.h").read_text()
    m = re.search(r"#define GRIM_NOALLOC_SCRATCH_BYTES \((\d+)u << (\d+)\)", hdr)
    assert m and grim.grim_noalloc_scratch_bytes() == int(m.group(1)) << int(m.group(2))

    assert grim.grim_strerror(grim.GRIM_E_OVERFLOW).startswith("more passing records")
    assert grim.grim_strerror(0) == "ok"
    # Fig. 4 caption: e = ceil(L * error rate)
    assert grim.grim_edits_for_rate(100, 5, 100) == 5
    assert grim.grim_edits_for_rate(150, 5, 100) == 8
    assert grim.grim_edits_for_rate(250, 5, 100) == 13


def test_binding_rejects_host_tensors_before_any_device_call():
    torch = pytest.importorskip("torch")
    from paper_1708_04329_gb300 import grim

    with pytest.raises(ValueError):
        grim._dptr(torch.zeros(4, dtype=torch.uint8), "ref", 1)


def test_index_file_errors_without_gpu(tmp_path):
    """grim_load checks the file before any device call: a missing file is an
    I/O error, a file that is not an index (or a truncated header) a format
    error, and a bad flag an argument error."""
    from paper_1708_04329_gb300 import grim

    with pytest.raises(grim.GrimError) as ei:
        grim.grim_load(tmp_path / "missing.grim")
    assert ei.value.code == grim.GRIM_E_IO
    junk = tmp_path / "junk.grim"
    junk.write_bytes(b"not an index" * 40)
    with pytest.raises(grim.GrimError) as ei:
        grim.grim_load(junk)
    assert ei.value.code == grim.GRIM_E_FORMAT
    junk.write_bytes(b"GRIMIDX1")
    with pytest.raises(grim.GrimError) as ei:
        grim.grim_load(junk)
    assert ei.value.code == grim.GRIM_E_FORMAT
    h = C_void()
    assert grim._lib().grim_load(str(junk).encode(), 0, 2, h) == grim.GRIM_E_ARG
    assert grim._lib().grim_load(str(junk).encode(), 8, 0, h) == grim.GRIM_E_ARG


def C_void():
    import ctypes

    return ctypes.byref(ctypes.c_void_p())


def test_gather_probe_library_exports():
    """The benchmark's random-gather probe (a measurement helper in
    bench_helpers/, apart from the filter library) builds and exports its two
    entry points."""
    import bench_helpers

    path = bench_helpers.build_probe()
    out = subprocess.run(["nm", "-D", "--defined-only", str(path)], capture_output=True, text=True,
                         check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    assert {"grim_probe_gather", "grim_probe_gather_sink_words"} <= exported


def test_launch_shape_options_checked_before_any_device_work():
    """grim_build_ex refuses an all-bins launch shape it does not build (CTA
    sizes other than 512/640/768, read ranges outside 1 MiB..4 GiB, an
    unknown read-switch mode or all-bins path) before it touches the
    reference pointer, and grim_index_set_shape refuses a NULL index."""
    import ctypes

    from paper_1708_04329_gb300 import grim

    lib = grim._lib()
    h = ctypes.c_void_p()
    fake_ref = ctypes.c_void_p(16)  # never dereferenced: the options fail first
    for threads, range_kb in ((600, 0), (1024, 0), (0, 512), (0, (4 << 20) + 1)):
        opts = grim._BuildOpts(0, threads, range_kb)
        rc = lib.grim_build_ex(fake_ref, 1000, 200, 5, 100, 7, ctypes.byref(opts), None,
                               ctypes.byref(h))
        assert rc == grim.GRIM_E_ARG, (threads, range_kb)
    assert lib.grim_index_set_shape(None, None) == grim.GRIM_E_ARG
    for bad in (grim._BuildOpts(0, 0, 0, 3), grim._BuildOpts(0, 0, 0, 0, 3)):  # no such modes
        assert lib.grim_build_ex(fake_ref, 1000, 200, 5, 100, 7, ctypes.byref(bad), None,
                                 ctypes.byref(h)) == grim.GRIM_E_ARG
