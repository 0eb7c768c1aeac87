"""CPU oracle for the bin-level q-gram filter (GRIM-Filter, arXiv 1708.04329).

TEST INFRASTRUCTURE ONLY: the tests, the package smoke check and the
benchmark's CPU-baseline / reference leg are the only users.  The product
path (the CUDA library and its binding) never imports this package, and this
package imports nothing from the product.

* ``grim_oracle.c`` -- the plain definition (bit vectors per bin, token sums,
  threshold), OpenMP over bins / reads, built here with gcc.
* ``bruteforce``     -- an independent re-statement for tiny inputs that uses
  no bit vectors and no token codes at all: substring search in each bin's
  window.

Every function cites the passage it follows; see ``grim_oracle.c``'s header
for the definitions and the readings taken where the paper is silent.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass
from pathlib import Path

import numpy as np

HERE = Path(__file__).resolve().parent
_LIB = HERE / "_lib" / "liboracle.so"
_lib = None

ERRORS = {-1: "bad argument", -2: "out of memory", -4: "read shorter than q",
          -5: "read too long", -6: "candidate bin out of range"}


class OracleError(RuntimeError):
    def __init__(self, code: int):
        super().__init__(f"oracle error {code}: {ERRORS.get(code, '?')}")
        self.code = code


def build(force: bool = False) -> Path:
    """Compile liboracle.so with gcc (plain C + OpenMP)."""
    src = HERE / "grim_oracle.c"
    _LIB.parent.mkdir(exist_ok=True)
    if force or not _LIB.exists() or _LIB.stat().st_mtime < src.stat().st_mtime:
        tmp = _LIB.with_suffix(f".so.tmp{os.getpid()}")
        cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", str(src), "-o", str(tmp)]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"oracle build failed:\n{res.stderr}")
        os.replace(tmp, _LIB)
    return _LIB


class _Out(C.Structure):
    _fields_ = [("read", C.POINTER(C.c_uint32)), ("bin", C.POINTER(C.c_uint32)),
                ("count", C.POINTER(C.c_uint8)), ("n", C.c_uint64)]


def _bind(path) -> C.CDLL:
    """Load a compiled oracle library and declare its entry points."""
    lib = C.CDLL(str(path))
    u64, u32, vp = C.c_uint64, C.c_uint32, C.c_void_p
    lib.oracle_num_bins.restype = u64
    lib.oracle_num_bins.argtypes = [u64, u32]
    lib.oracle_vector_bytes.restype = u64
    lib.oracle_vector_bytes.argtypes = [u32]
    lib.oracle_bin_vectors.restype = C.c_int
    lib.oracle_bin_vectors.argtypes = [vp, u64, u32, u32, u32, vp]
    lib.oracle_read_tokens.restype = C.c_int
    lib.oracle_read_tokens.argtypes = [vp, u32, u32, vp]
    lib.oracle_filter.restype = C.c_int
    lib.oracle_filter.argtypes = [vp, u64, u32, vp, vp, vp, u64, vp, vp, vp, u64, u64, u32,
                                  C.POINTER(_Out)]
    lib.oracle_free.restype = None
    lib.oracle_free.argtypes = [C.POINTER(_Out)]
    lib.oracle_threads.restype = C.c_int
    lib.oracle_set_threads.restype = None
    lib.oracle_set_threads.argtypes = [C.c_int]
    return lib


def _load():
    global _lib
    if _lib is None:
        _lib = _bind(build())
    return _lib


def _p(a: np.ndarray | None) -> int | None:
    return None if a is None else a.ctypes.data


def threads() -> int:
    """OpenMP threads the oracle uses (``OMP_NUM_THREADS`` or all cores)."""
    return int(_load().oracle_threads())


def set_threads(n: int) -> None:
    """Run the oracle's parallel loops on ``n`` OpenMP threads."""
    _load().oracle_set_threads(int(n))


def num_bins(n: int, B: int) -> int:
    """numBins = ceil(N / B) (§GRIM-Filter: contiguous bins of B bases)."""
    return int(_load().oracle_num_bins(n, B))


def vector_bytes(q: int) -> int:
    """4^q bits per bin vector (§Parameter Evaluation Results: 4^5 = 1024)."""
    return int(_load().oracle_vector_bytes(q))


@dataclass
class Index:
    """Bin-major bit vectors: ``vecs[b]`` holds bin b's 4^q bits, token t at
    bit t % 8 of byte t // 8."""

    vecs: np.ndarray  # uint8 [num_bins, vector_bytes(q)]
    n: int
    B: int
    ext: int
    q: int

    @property
    def num_bins(self) -> int:
        return int(self.vecs.shape[0])


def bin_vectors(ref: np.ndarray, B: int, q: int, max_read_len: int) -> Index:
    """Bit vector of every bin (§GRIM-Filter, Fig. 2), ext = max_read_len - 1."""
    ref = np.ascontiguousarray(ref, dtype=np.uint8)
    nb, vb = num_bins(len(ref), B), vector_bytes(q)
    out = np.empty((nb, vb), dtype=np.uint8)
    ext = max_read_len - 1
    rc = _load().oracle_bin_vectors(_p(ref), len(ref), B, ext, q, _p(out))
    if rc:
        raise OracleError(rc)
    return Index(out, len(ref), B, ext, q)


def read_tokens(read: bytes, q: int) -> np.ndarray:
    """Token values of the read's L-q+1 q-grams, -1 where a q-gram has a non-base."""
    a = np.frombuffer(read, dtype=np.uint8)
    if len(a) < q:
        raise OracleError(-4)
    out = np.empty(len(a) - q + 1, dtype=np.int64)
    rc = _load().oracle_read_tokens(_p(np.ascontiguousarray(a)), len(a), q, _p(out))
    if rc:
        raise OracleError(rc)
    return out


def filter(index: Index, reads, cand_off: np.ndarray | None = None, cand: np.ndarray | None = None,
           bin_range: tuple[int, int] | None = None, max_read_len: int | None = None):
    """Passing (read, bin, count) records (§GRIM-Filter steps 1-3, Fig. 3).

    ``reads`` carries ``seq`` (uint8), ``offsets`` (uint64), ``lens`` (uint32)
    and ``e`` (uint16).  ``cand``/``cand_off`` select candidate mode; otherwise
    every bin in ``bin_range`` (default: all bins).
    Returns three arrays ``(read uint32, bin uint32, count uint8)``.
    """
    lib = _load()
    seq = np.ascontiguousarray(reads.seq, dtype=np.uint8)
    offs = np.ascontiguousarray(reads.offsets, dtype=np.uint64)
    lens = np.ascontiguousarray(reads.lens, dtype=np.uint32)
    e = np.ascontiguousarray(reads.e, dtype=np.uint16)
    n_reads = len(lens)
    lo, hi = bin_range if bin_range is not None else (0, index.num_bins)
    if cand is not None:
        cand = np.ascontiguousarray(cand, dtype=np.int32)
        cand_off = np.ascontiguousarray(cand_off, dtype=np.uint64)
    mrl = index.ext + 1 if max_read_len is None else max_read_len
    out = _Out()
    rc = lib.oracle_filter(_p(index.vecs), index.num_bins, index.q, _p(seq) if len(seq) else None,
                           _p(offs), _p(lens), n_reads, _p(e), _p(cand), _p(cand_off), lo, hi, mrl,
                           C.byref(out))
    if rc:
        raise OracleError(rc)
    try:
        n = int(out.n)
        r = np.ctypeslib.as_array(out.read, (n,)).copy() if n else np.empty(0, np.uint32)
        b = np.ctypeslib.as_array(out.bin, (n,)).copy() if n else np.empty(0, np.uint32)
        c = np.ctypeslib.as_array(out.count, (n,)).copy() if n else np.empty(0, np.uint8)
    finally:
        lib.oracle_free(C.byref(out))
    return r, b, c


def token_major(index: Index, pad_to: int = 1024) -> np.ndarray:
    """The same bits transposed: row t lists token t's bit for every bin
    (§Mapping GRIM-Filter: one token's bits across all bins are contiguous),
    bin b at bit b % 32 of uint32 word b // 32, bins padded with zero bits to a
    multiple of ``pad_to``.  Plain numpy unpack / transpose / pack."""
    nb = index.num_bins
    bits = np.unpackbits(index.vecs, axis=1, bitorder="little")[:, : 4 ** index.q]  # [nb, 4^q]
    padded = -(-nb // pad_to) * pad_to
    full = np.zeros((4 ** index.q, padded), dtype=np.uint8)
    full[:, :nb] = bits.T
    return np.packbits(full, axis=1, bitorder="little").view(np.uint32)
