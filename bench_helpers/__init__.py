"""Measurement helpers of bench.py, kept apart from the filter library.

``probe_gather.cu`` (built into ``bench_helpers/_lib/libgrim_probe.so``) is
a random-gather probe: the rate at which this GPU reads random bin-vector-
sized rows from a table shaped like the bin-major table, the practical
ceiling of the candidate-list kernel.  It computes nothing of the filter.
"""
from __future__ import annotations

import ctypes
import os
import shutil
import subprocess
from pathlib import Path

HERE = Path(__file__).resolve().parent
LIBDIR = HERE / "_lib"
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

_probe = None


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and Path(cand).exists():
            return cand
    raise RuntimeError("nvcc not found: the gather probe cannot be built")


def build_probe(force: bool = False) -> Path:
    """nvcc the probe for sm_103a (skipped when the library is up to date)."""
    LIBDIR.mkdir(exist_ok=True)
    out = LIBDIR / "libgrim_probe.so"
    src = HERE / "probe_gather.cu"
    if force or not out.exists() or src.stat().st_mtime > out.stat().st_mtime:
        tmp = out.with_suffix(f".so.tmp{os.getpid()}")
        cmd = [_nvcc()] + ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                                  "-shared", "--cudart", "static", str(src), "-o", str(tmp)]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"build failed: {' '.join(cmd)}\n{res.stdout}\n{res.stderr}")
        os.replace(tmp, out)
    return out


def probe() -> ctypes.CDLL:
    """The probe library, with its two entry points typed."""
    global _probe
    if _probe is None:
        lib = ctypes.CDLL(str(build_probe()))
        lib.grim_probe_gather.restype = ctypes.c_int
        lib.grim_probe_gather.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32,
                                          ctypes.c_uint64, ctypes.c_uint32, ctypes.c_void_p,
                                          ctypes.c_uint64, ctypes.c_void_p]
        lib.grim_probe_gather_sink_words.restype = ctypes.c_uint64
        lib.grim_probe_gather_sink_words.argtypes = []
        _probe = lib
    return _probe
