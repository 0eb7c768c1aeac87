"""Compile the native parts of the package in-tree.

* ``libgrim.so``  -- the CUDA kernels and the C-ABI (``include/grim.h``), built
  by nvcc for sm_103a only.
* ``libsynth.so`` -- the seeded synthetic-input generator (plain C).

Both land in ``paper_1708_04329_gb300/_lib/``.  A build is skipped when the
library is newer than every source it depends on.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
from pathlib import Path

PKG = Path(__file__).resolve().parent
ROOT = PKG.parent
CSRC = PKG / "csrc"
LIBDIR = PKG / "_lib"
INCLUDE = ROOT / "include"

GRIM_SOURCES = [
    "grim_api.cu",
    "grim_build.cu",
    "grim_tokens.cu",
    "grim_exhaustive.cu",
    "grim_candidates.cu",
    "grim_compact.cu",
    "grim_noalloc.cu",
    "grim_plan.cu",
    "grim_serve.cu",
    "grim_io.cu",
]
GRIM_HEADERS = ["grim_internal.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and Path(cand).exists():
            return cand
    raise RuntimeError("nvcc not found: the CUDA library cannot be built")


def _stale(target: Path, deps: list[Path]) -> bool:
    if not target.exists():
        return True
    t = target.stat().st_mtime
    return any(d.stat().st_mtime > t for d in deps)


def _run(cmd: list[str]) -> None:
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"build failed: {' '.join(cmd)}\n{res.stdout}\n{res.stderr}")


def build_synth(force: bool = False) -> Path:
    LIBDIR.mkdir(exist_ok=True)
    out = LIBDIR / "libsynth.so"
    src = CSRC / "synth.c"
    if force or _stale(out, [src]):
        tmp = out.with_suffix(f".so.tmp{os.getpid()}")
        _run(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", str(src), "-o", str(tmp), "-lm"])
        os.replace(tmp, out)
    return out


def build_grim(force: bool = False, extra: list[str] | None = None) -> Path:
    """nvcc every translation unit in parallel, then link one shared library."""
    LIBDIR.mkdir(exist_ok=True)
    objdir = LIBDIR / "obj"
    objdir.mkdir(exist_ok=True)
    out = LIBDIR / "libgrim.so"
    headers = [CSRC / h for h in GRIM_HEADERS] + [INCLUDE / "grim.h"]
    nvcc = _nvcc()
    flags = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", str(INCLUDE),
                    "-I", str(CSRC)] + (extra or [])
    jobs = []
    objs = []
    for s in GRIM_SOURCES:
        src = CSRC / s
        obj = objdir / (Path(s).stem + ".o")
        objs.append(obj)
        if force or _stale(obj, [src] + headers):
            jobs.append([nvcc] + flags + ["-c", str(src), "-o", str(obj)])
    if jobs:
        with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            list(ex.map(_run, jobs))
    if force or jobs or _stale(out, objs):
        tmp = out.with_suffix(f".so.tmp{os.getpid()}")
        _run([nvcc] + ARCH + ["-shared", "--cudart", "static", "-o", str(tmp)] + [str(o) for o in objs]
             + ["-lpthread"])
        os.replace(tmp, out)
    return out


def build_all(force: bool = False) -> dict[str, Path]:
    with cf.ThreadPoolExecutor(max_workers=2) as ex:
        synth = ex.submit(build_synth, force)
        out = {"grim": build_grim(force)}
        out["synth"] = synth.result()
    return out


if __name__ == "__main__":
    import sys

    print(build_all(force="--force" in sys.argv))
