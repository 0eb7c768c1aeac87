"""Python binding of libgrim.so (``include/grim.h``), argument marshalling only.

Every entry point of the C-ABI has a function of the same name here.  Device
arrays are torch CUDA tensors (PyTorch supplies device memory and streams);
host arrays are numpy arrays or CPU tensors.  All computation happens in the
library's CUDA kernels; there is no CPU fallback: if ``libgrim.so`` cannot be
built or loaded, importing the library raises.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np

from . import _build

GRIM_OK = 0
GRIM_E_ARG = -1
GRIM_E_NOMEM = -2
GRIM_E_CUDA = -3
GRIM_E_READ_TOO_SHORT = -4
GRIM_E_READ_TOO_LONG = -5
GRIM_E_BAD_CANDIDATE = -6
GRIM_E_OVERFLOW = -7
GRIM_E_TIMEOUT = -8
GRIM_E_WORKSPACE = -9
GRIM_E_NO_LAYOUT = -10
GRIM_E_UNSUPPORTED = -11
GRIM_E_NOT_READY = -12
GRIM_E_BUSY = -13
GRIM_E_IO = -14
GRIM_E_FORMAT = -15
GRIM_E_CANCELLED = -16
GRIM_LOAD_VERIFY = 1
GRIM_SWITCH_GROUP = 1
GRIM_SWITCH_WARP = 2
GRIM_PATH_TWO_LEVEL = 1
GRIM_PATH_EXACT = 2
GRIM_PLAN_CANDIDATES = 1
GRIM_PLAN_HOST_IO = 2

GRIM_LAYOUT_TOKEN_MAJOR = 1
GRIM_LAYOUT_BIN_MAJOR = 2
GRIM_LAYOUT_BOTH = 3
GRIM_LAYOUT_COARSE = 4
GRIM_LAYOUT_ALL = 7

#: every symbol include/grim.h declares
EXPORTS = (
    "grim_build", "grim_build_host", "grim_index_info", "grim_free", "grim_strerror",
    "grim_last_cuda_error", "grim_filter_workspace_size", "grim_filter", "grim_filter_host",
    "grim_loc_to_bin", "grim_edits_for_rate", "grim_profile", "grim_profile_get",
    "grim_filter_noalloc", "grim_last_filter_stats", "grim_build_ex", "grim_build_host_ex",
    "grim_plan_create", "grim_plan_buffers_get", "grim_plan_launch", "grim_plan_query",
    "grim_plan_wait", "grim_plan_device_bytes", "grim_plan_free", "grim_default_coarse_factor",
    "grim_server_create", "grim_server_submit", "grim_server_wait", "grim_server_take",
    "grim_server_stats_get", "grim_server_free", "grim_save", "grim_load",
    "grim_reverse_complement", "grim_server_cancel", "grim_trim_scratch", "grim_set_allocator",
    "grim_noalloc_scratch_bytes", "grim_index_set_shape",
)


class GrimError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        msg = grim_strerror(code)
        if code == GRIM_E_CUDA:
            msg += f" ({_lib().grim_last_cuda_error().decode()})"
        super().__init__(f"{what}: {msg} [{code}]" if what else f"{msg} [{code}]")
        self.code = code


class _Desc(C.Structure):
    _fields_ = [("ref_len", C.c_uint64), ("num_bins", C.c_uint64), ("num_bins_pad", C.c_uint64),
                ("B", C.c_uint32), ("q", C.c_uint32), ("ext", C.c_uint32),
                ("max_read_len", C.c_uint32), ("layouts", C.c_uint32),
                ("words_per_bin", C.c_uint32), ("token_major", C.c_void_p),
                ("bin_major", C.c_void_p), ("token_major_bytes", C.c_uint64),
                ("bin_major_bytes", C.c_uint64), ("coarse_token_major", C.c_void_p),
                ("num_coarse", C.c_uint64), ("num_coarse_pad", C.c_uint64),
                ("coarse_token_major_bytes", C.c_uint64), ("coarse_factor", C.c_uint32),
                ("cta_threads", C.c_uint32), ("read_range_kb", C.c_uint32),
                ("read_switch", C.c_uint32), ("all_bins_path", C.c_uint32),
                ("two_level", C.c_uint32)]


class _Stats(C.Structure):
    _fields_ = [("n_reads", C.c_uint64), ("n_records", C.c_uint64), ("pairs", C.c_uint64),
                ("tokens_executed", C.c_uint64), ("survivors", C.c_uint64),
                ("bit_tests_executed", C.c_uint64), ("read_switch", C.c_uint32),
                ("all_bins_path", C.c_uint32)]


class _BuildOpts(C.Structure):
    _fields_ = [("coarse_factor", C.c_uint32), ("cta_threads", C.c_uint32),
                ("read_range_kb", C.c_uint32), ("read_switch", C.c_uint32),
                ("all_bins_path", C.c_uint32), ("reserved", C.c_uint32 * 3)]


class _Shape(C.Structure):
    _fields_ = [("cta_threads", C.c_uint32), ("read_range_kb", C.c_uint32),
                ("read_switch", C.c_uint32), ("all_bins_path", C.c_uint32),
                ("reserved", C.c_uint32 * 4)]


class _PlanDesc(C.Structure):
    _fields_ = [("max_reads", C.c_uint32), ("max_e", C.c_uint32), ("max_bases", C.c_uint64),
                ("max_cand", C.c_uint64), ("cap", C.c_uint64), ("flags", C.c_uint32),
                ("cand_unroll", C.c_uint32), ("reserved", C.c_uint32 * 6)]


class _PlanBuffers(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in ("reads", "offsets", "lens", "e", "cand", "cand_off",
                                           "out_read", "out_bin", "out_count")]


class _ServerDesc(C.Structure):
    _fields_ = [("slots", C.c_uint32), ("max_reads", C.c_uint32), ("max_bases", C.c_uint64),
                ("max_cand", C.c_uint64), ("cap", C.c_uint64), ("max_e", C.c_uint32),
                ("flags", C.c_uint32), ("mem_budget", C.c_uint64),
                ("max_queued_reads", C.c_uint64), ("cand_unroll", C.c_uint32),
                ("max_chunk_reads", C.c_uint32), ("reserved", C.c_uint32 * 6)]


class _RequestInfo(C.Structure):
    _fields_ = [("status", C.c_int32), ("n_reads", C.c_uint32), ("n_out", C.c_uint64),
                ("batch", C.c_uint64), ("batch_requests", C.c_uint32),
                ("batch_reads", C.c_uint32), ("t_submit_ns", C.c_uint64),
                ("t_launch_ns", C.c_uint64), ("t_done_ns", C.c_uint64)]


class _ServerStats(C.Structure):
    _fields_ = [("slots", C.c_uint32), ("reserved", C.c_uint32), ("device_bytes", C.c_uint64)] + [
        (n, C.c_uint64) for n in ("submitted", "completed", "batches", "batch_reads", "reads_done",
                                  "records", "overflow_splits", "queued_requests", "queued_reads",
                                  "cancelled")]


class _KTime(C.Structure):
    _fields_ = [("name", C.c_char * 32), ("launches", C.c_uint64), ("total_ms", C.c_double)]


_ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_uint64, C.c_void_p)
_FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)
_ALLOCATOR = None  # the ctypes callbacks in use (kept alive here)

_L = None


def _lib() -> C.CDLL:
    """Load libgrim.so (building it in-tree first if it is missing or stale)."""
    global _L
    if _L is None:
        path = _build.build_grim()
        lib = C.CDLL(str(path))
        u64, u32, i32, vp = C.c_uint64, C.c_uint32, C.c_int, C.c_void_p
        pp = C.POINTER(C.c_void_p)
        lib.grim_build.restype = i32
        lib.grim_build.argtypes = [vp, u64, u32, u32, u32, u32, vp, pp]
        lib.grim_build_host.restype = i32
        lib.grim_build_host.argtypes = [vp, u64, u32, u32, u32, u32, vp, pp]
        lib.grim_build_ex.restype = i32
        lib.grim_build_ex.argtypes = [vp, u64, u32, u32, u32, u32, C.POINTER(_BuildOpts), vp, pp]
        lib.grim_build_host_ex.restype = i32
        lib.grim_build_host_ex.argtypes = [vp, u64, u32, u32, u32, u32, C.POINTER(_BuildOpts), vp,
                                           pp]
        lib.grim_default_coarse_factor.restype = u32
        lib.grim_default_coarse_factor.argtypes = [u32, u32, u32]
        lib.grim_index_info.restype = i32
        lib.grim_index_info.argtypes = [vp, C.POINTER(_Desc)]
        lib.grim_index_set_shape.restype = i32
        lib.grim_index_set_shape.argtypes = [vp, C.POINTER(_Shape)]
        lib.grim_free.restype = None
        lib.grim_free.argtypes = [vp]
        lib.grim_strerror.restype = C.c_char_p
        lib.grim_strerror.argtypes = [i32]
        lib.grim_last_cuda_error.restype = C.c_char_p
        lib.grim_last_cuda_error.argtypes = []
        lib.grim_filter_workspace_size.restype = u64
        lib.grim_filter_workspace_size.argtypes = [vp, u32, u64, u64]
        fargs = [vp, vp, vp, vp, u32, vp, vp, vp, u64, vp, vp, vp, u64, C.POINTER(C.c_uint64)]
        lib.grim_filter.restype = i32
        lib.grim_filter.argtypes = fargs + [vp, u64, vp]
        lib.grim_filter_host.restype = i32
        lib.grim_filter_host.argtypes = fargs + [vp]
        lib.grim_filter_noalloc.restype = i32
        lib.grim_filter_noalloc.argtypes = fargs + [vp]
        lib.grim_noalloc_scratch_bytes.restype = u64
        lib.grim_noalloc_scratch_bytes.argtypes = []
        lib.grim_loc_to_bin.restype = u64
        lib.grim_loc_to_bin.argtypes = [vp, u64]
        lib.grim_edits_for_rate.restype = u32
        lib.grim_edits_for_rate.argtypes = [u32, u32, u32]
        lib.grim_last_filter_stats.restype = i32
        lib.grim_last_filter_stats.argtypes = [C.POINTER(_Stats)]
        lib.grim_plan_create.restype = i32
        lib.grim_plan_create.argtypes = [vp, C.POINTER(_PlanDesc), pp]
        lib.grim_plan_buffers_get.restype = i32
        lib.grim_plan_buffers_get.argtypes = [vp, C.POINTER(_PlanBuffers)]
        lib.grim_plan_launch.restype = i32
        lib.grim_plan_launch.argtypes = [vp, u32, u64, vp]
        lib.grim_plan_query.restype = i32
        lib.grim_plan_query.argtypes = [vp]
        lib.grim_plan_wait.restype = i32
        lib.grim_plan_wait.argtypes = [vp, C.POINTER(C.c_uint64)]
        lib.grim_plan_device_bytes.restype = u64
        lib.grim_plan_device_bytes.argtypes = [vp]
        lib.grim_plan_free.restype = None
        lib.grim_plan_free.argtypes = [vp]
        lib.grim_profile.restype = i32
        lib.grim_set_allocator.restype = i32
        lib.grim_set_allocator.argtypes = [_ALLOC_FN, _FREE_FN, vp]
        lib.grim_trim_scratch.restype = i32
        lib.grim_trim_scratch.argtypes = []
        lib.grim_reverse_complement.restype = i32
        lib.grim_reverse_complement.argtypes = [vp, vp, vp, u32, vp, vp]
        lib.grim_save.restype = i32
        lib.grim_save.argtypes = [vp, C.c_char_p]
        lib.grim_load.restype = i32
        lib.grim_load.argtypes = [C.c_char_p, u32, u32, pp]
        lib.grim_server_create.restype = i32
        lib.grim_server_create.argtypes = [vp, C.POINTER(_ServerDesc), pp]
        lib.grim_server_submit.restype = i32
        lib.grim_server_submit.argtypes = [vp, vp, vp, vp, u32, vp, vp, vp, C.POINTER(C.c_uint64)]
        lib.grim_server_wait.restype = i32
        lib.grim_server_wait.argtypes = [vp, u64, C.c_int64]
        lib.grim_server_take.restype = i32
        lib.grim_server_take.argtypes = [vp, u64, vp, vp, vp, u64, C.POINTER(_RequestInfo)]
        lib.grim_server_cancel.restype = i32
        lib.grim_server_cancel.argtypes = [vp, u64]
        lib.grim_server_stats_get.restype = i32
        lib.grim_server_stats_get.argtypes = [vp, C.POINTER(_ServerStats)]
        lib.grim_server_free.restype = None
        lib.grim_server_free.argtypes = [vp]
        lib.grim_profile.argtypes = [i32]
        lib.grim_profile_get.restype = i32
        lib.grim_profile_get.argtypes = [C.POINTER(_KTime), i32]
        _L = lib
    return _L


def library_path() -> str:
    return str(_build.LIBDIR / "libgrim.so")


# ---------------------------------------------------------------------------
# helpers
# ---------------------------------------------------------------------------

def _torch():
    import torch

    return torch


def _dptr(t, what: str, esize: int | None = None) -> int:
    """Device pointer of a contiguous CUDA tensor (or None -> 0)."""
    if t is None:
        return 0
    if not t.is_cuda:
        raise ValueError(f"{what} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{what} must be contiguous")
    if esize is not None and t.element_size() != esize:
        raise ValueError(f"{what} must have {esize}-byte elements")
    return t.data_ptr()


def _check_out(out, what: str) -> int:
    """Validate a caller's (read, bin, count) output triple of CUDA tensors and
    return its capacity.  The kernels write up to `cap` records into each of
    the three arrays, so all three must hold `cap` elements of the right
    width on the current device."""
    torch = _torch()
    if len(out) != 3:
        raise ValueError(f"{what}: out must be a (read, bin, count) triple")
    cap = int(out[0].numel())
    dev = torch.cuda.current_device()
    for t, name, es in zip(out, ("out_read", "out_bin", "out_count"), (4, 4, 1)):
        if not t.is_cuda or t.device.index != dev:
            raise ValueError(f"{what}: {name} must be a CUDA tensor on the current device")
        if t.element_size() != es or t.is_floating_point():
            raise ValueError(f"{what}: {name} must have {es}-byte integer elements")
        if not t.is_contiguous():
            raise ValueError(f"{what}: {name} must be contiguous")
        if int(t.numel()) != cap:
            raise ValueError(f"{what}: the three output arrays must have the same length")
    return cap


def _hptr(a, what: str, dtype) -> tuple[int, object]:
    """Host pointer of an array converted to dtype (keeps the buffer alive)."""
    if a is None:
        return 0, None
    if hasattr(a, "numpy") and not isinstance(a, np.ndarray):  # CPU tensor
        if a.is_cuda:
            raise ValueError(f"{what} must be host memory")
        a = a.contiguous()
        if a.element_size() != np.dtype(dtype).itemsize:
            raise ValueError(f"{what} must have {np.dtype(dtype).itemsize}-byte elements")
        return a.data_ptr(), a
    arr = np.ascontiguousarray(a, dtype=dtype)
    return arr.ctypes.data, arr


def _stream_ptr(stream) -> int:
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)


class _CudaArray:
    """__cuda_array_interface__ view of library-owned device memory."""

    def __init__(self, ptr: int, shape: tuple, typestr: str, owner):
        self.__cuda_array_interface__ = {"shape": shape, "typestr": typestr, "data": (ptr, False),
                                         "version": 3, "strides": None}
        self._owner = owner


# ---------------------------------------------------------------------------
# index
# ---------------------------------------------------------------------------

@dataclass
class IndexDesc:
    ref_len: int
    num_bins: int
    num_bins_pad: int
    B: int
    q: int
    ext: int
    max_read_len: int
    layouts: int
    words_per_bin: int
    token_major_ptr: int
    bin_major_ptr: int
    token_major_bytes: int
    bin_major_bytes: int
    coarse_token_major_ptr: int = 0
    num_coarse: int = 0
    num_coarse_pad: int = 0
    coarse_token_major_bytes: int = 0
    coarse_factor: int = 0
    cta_threads: int = 0
    read_range_kb: int = 0
    read_switch: int = 0
    all_bins_path: int = 0
    two_level: int = 0


class GrimIndex:
    """Owns a grim_index handle; grim_free runs when it is closed or collected."""

    def __init__(self, handle: int):
        self._h = handle

    @property
    def handle(self) -> int:
        if not self._h:
            raise ValueError("index already freed")
        return self._h

    def close(self) -> None:
        if self._h:
            grim_free(self)
            self._h = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def desc(self) -> IndexDesc:
        return grim_index_info(self)

    def token_major(self):
        """Zero-copy CUDA tensor [4^q, num_bins_pad/32] of the table's uint32
        words, typed int32 (torch's fully supported 32-bit type; view the host
        copy as uint32).  None if the index has no token-major table."""
        d = self.desc
        if not d.token_major_ptr:
            return None
        torch = _torch()
        shape = (4 ** d.q, d.num_bins_pad // 32)
        view = _CudaArray(d.token_major_ptr, shape, "<i4", self)
        return torch.as_tensor(view, device="cuda")

    def coarse_token_major(self):
        """Zero-copy int32-typed CUDA tensor [4^q, num_coarse_pad/32] of the
        super-bin table's words (None if absent)."""
        d = self.desc
        if not d.coarse_token_major_ptr:
            return None
        torch = _torch()
        view = _CudaArray(d.coarse_token_major_ptr, (4 ** d.q, d.num_coarse_pad // 32), "<i4", self)
        return torch.as_tensor(view, device="cuda")

    def bin_major(self):
        """Zero-copy CUDA tensor [num_bins, words_per_bin] of the table's uint32
        words, typed int32.  None if the index has no bin-major table."""
        d = self.desc
        if not d.bin_major_ptr:
            return None
        torch = _torch()
        view = _CudaArray(d.bin_major_ptr, (d.num_bins, d.words_per_bin), "<i4", self)
        return torch.as_tensor(view, device="cuda")


def grim_build(ref, B: int, q: int, max_read_len: int, layouts: int = GRIM_LAYOUT_ALL,
               stream=None) -> GrimIndex:
    """grim_build: ``ref`` is a uint8 CUDA tensor of ASCII bases."""
    h = C.c_void_p()
    rc = _lib().grim_build(_dptr(ref, "ref", 1), ref.numel(), B, q, max_read_len, layouts,
                           _stream_ptr(stream), C.byref(h))
    if rc != GRIM_OK:
        raise GrimError(rc, "grim_build")
    return GrimIndex(h.value)


def grim_build_host(ref, B: int, q: int, max_read_len: int, layouts: int = GRIM_LAYOUT_ALL,
                    stream=None) -> GrimIndex:
    """grim_build_host: ``ref`` is host memory (numpy uint8 / CPU tensor)."""
    p, keep = _hptr(ref, "ref", np.uint8)
    n = keep.numel() if hasattr(keep, "numel") else keep.size
    h = C.c_void_p()
    rc = _lib().grim_build_host(p, n, B, q, max_read_len, layouts, _stream_ptr(stream), C.byref(h))
    if rc != GRIM_OK:
        raise GrimError(rc, "grim_build_host")
    return GrimIndex(h.value)


def grim_build_ex(ref, B: int, q: int, max_read_len: int, layouts: int = GRIM_LAYOUT_ALL,
                  coarse_factor: int = 0, stream=None, cta_threads: int = 0,
                  read_range_kb: int = 0, read_switch: int = 0,
                  all_bins_path: int = 0) -> GrimIndex:
    """grim_build_ex: grim_build with build options (``coarse_factor``: bins per
    super-bin of the coarse table; ``cta_threads``, ``read_range_kb``: the
    all-bins kernel's launch shape; 0 = the library default)."""
    opts = _BuildOpts(coarse_factor, cta_threads, read_range_kb, read_switch, all_bins_path)
    h = C.c_void_p()
    rc = _lib().grim_build_ex(_dptr(ref, "ref", 1), ref.numel(), B, q, max_read_len, layouts,
                              C.byref(opts), _stream_ptr(stream), C.byref(h))
    if rc != GRIM_OK:
        raise GrimError(rc, "grim_build_ex")
    return GrimIndex(h.value)


def grim_build_host_ex(ref, B: int, q: int, max_read_len: int, layouts: int = GRIM_LAYOUT_ALL,
                       coarse_factor: int = 0, stream=None, cta_threads: int = 0,
                       read_range_kb: int = 0, read_switch: int = 0,
                       all_bins_path: int = 0) -> GrimIndex:
    """grim_build_host_ex: grim_build_host with build options."""
    p, keep = _hptr(ref, "ref", np.uint8)
    n = keep.numel() if hasattr(keep, "numel") else keep.size
    opts = _BuildOpts(coarse_factor, cta_threads, read_range_kb, read_switch, all_bins_path)
    h = C.c_void_p()
    rc = _lib().grim_build_host_ex(p, n, B, q, max_read_len, layouts, C.byref(opts),
                                   _stream_ptr(stream), C.byref(h))
    if rc != GRIM_OK:
        raise GrimError(rc, "grim_build_host_ex")
    return GrimIndex(h.value)


def grim_set_allocator(alloc=None, free=None) -> None:
    """Route index-table allocations through alloc(bytes) -> device pointer
    and free(pointer); no arguments restores cudaMalloc / cudaFree."""
    global _ALLOCATOR
    if (alloc is None) != (free is None):
        raise ValueError("give both alloc and free, or neither")
    if alloc is None:
        rc = _lib().grim_set_allocator(_ALLOC_FN(), _FREE_FN(), None)
        _ALLOCATOR = None
    else:
        def _a(nbytes, _ctx):
            try:
                return int(alloc(int(nbytes))) or None
            except Exception:
                return None

        def _f(ptr, _ctx):
            free(int(ptr))

        cbs = (_ALLOC_FN(_a), _FREE_FN(_f))
        rc = _lib().grim_set_allocator(cbs[0], cbs[1], None)
        if rc == GRIM_OK:
            _ALLOCATOR = cbs
    if rc != GRIM_OK:
        raise GrimError(rc, "grim_set_allocator")


def use_torch_allocator(enable: bool = True) -> None:
    """Index tables from PyTorch's caching allocator (they then count in
    torch.cuda.memory_allocated), or back to cudaMalloc."""
    if not enable:
        grim_set_allocator()
        return
    torch = _torch()
    grim_set_allocator(lambda n: torch.cuda.caching_allocator_alloc(n),
                       lambda p: torch.cuda.caching_allocator_delete(p))


def grim_trim_scratch() -> None:
    """Return the library's cached scratch memory of the current device."""
    rc = _lib().grim_trim_scratch()
    if rc != GRIM_OK:
        raise GrimError(rc, "grim_trim_scratch")


def grim_save(index: GrimIndex, path) -> None:
    """Write the index (parameters and every table it holds) to a file."""
    rc = _lib().grim_save(index.handle, str(path).encode())
    if rc != GRIM_OK:
        raise GrimError(rc, "grim_save")


def grim_load(path, layouts: int = 0, verify: bool = False) -> GrimIndex:
    """Read an index written by grim_save (``layouts``: tables to load, 0 = all)."""
    h = C.c_void_p()
    rc = _lib().grim_load(str(path).encode(), layouts, GRIM_LOAD_VERIFY if verify else 0,
                          C.byref(h))
    if rc != GRIM_OK:
        raise GrimError(rc, "grim_load")
    return GrimIndex(h.value)


def grim_default_coarse_factor(B: int, q: int, max_read_len: int) -> int:
    return int(_lib().grim_default_coarse_factor(B, q, max_read_len))


def grim_index_info(index: GrimIndex) -> IndexDesc:
    d = _Desc()
    rc = _lib().grim_index_info(index.handle, C.byref(d))
    if rc != GRIM_OK:
        raise GrimError(rc, "grim_index_info")
    return IndexDesc(d.ref_len, d.num_bins, d.num_bins_pad, d.B, d.q, d.ext, d.max_read_len,
                     d.layouts, d.words_per_bin, d.token_major or 0, d.bin_major or 0,
                     d.token_major_bytes, d.bin_major_bytes, d.coarse_token_major or 0,
                     d.num_coarse, d.num_coarse_pad, d.coarse_token_major_bytes, d.coarse_factor,
                     d.cta_threads, d.read_range_kb, d.read_switch, d.all_bins_path,
                     d.two_level)


def grim_index_set_shape(index: GrimIndex, cta_threads: int = 0, read_range_kb: int = 0,
                         read_switch: int = 0, all_bins_path: int = 0) -> None:
    """Launch shape of the all-bins filter for later calls with this index:
    CTA threads (512, 640 or 768), the read tile in KiB of token rows per
    read range, GRIM_SWITCH_GROUP / GRIM_SWITCH_WARP, and GRIM_PATH_TWO_LEVEL
    / GRIM_PATH_EXACT; 0 restores a default (automatic)."""
    shape = _Shape(cta_threads, read_range_kb, read_switch, all_bins_path)
    rc = _lib().grim_index_set_shape(index.handle, C.byref(shape))
    if rc != GRIM_OK:
        raise GrimError(rc, "grim_index_set_shape")


def grim_free(index: GrimIndex) -> None:
    if index._h:
        _lib().grim_free(index._h)


def grim_strerror(code: int) -> str:
    return _lib().grim_strerror(code).decode()


def grim_filter_workspace_size(index: GrimIndex, n_reads: int, n_cand: int = 0, cap: int = 0) -> int:
    return int(_lib().grim_filter_workspace_size(index.handle, n_reads, n_cand, cap))


def grim_loc_to_bin(index: GrimIndex, loc: int) -> int:
    return int(_lib().grim_loc_to_bin(index.handle, loc))


def grim_edits_for_rate(L: int, num: int, den: int) -> int:
    return int(_lib().grim_edits_for_rate(L, num, den))


def grim_last_filter_stats() -> dict:
    """Work counters of this thread's last successful filter call."""
    st = _Stats()
    rc = _lib().grim_last_filter_stats(C.byref(st))
    if rc != GRIM_OK:
        raise GrimError(rc, "grim_last_filter_stats")
    return {f: int(getattr(st, f)) for f, _ in _Stats._fields_}


def grim_profile(enable: bool) -> None:
    _lib().grim_profile(1 if enable else 0)


def grim_profile_get() -> dict[str, tuple[int, float]]:
    """{kernel name: (launches, total ms)} since grim_profile(True)."""
    lib = _lib()
    n = lib.grim_profile_get(None, 0)
    arr = (_KTime * max(n, 1))()
    n = lib.grim_profile_get(arr, n)
    return {arr[i].name.decode(): (int(arr[i].launches), float(arr[i].total_ms)) for i in range(n)}


# ---------------------------------------------------------------------------
# filter
# ---------------------------------------------------------------------------

class Workspace:
    """A reusable device workspace (a uint8 CUDA tensor, 256-byte aligned)."""

    def __init__(self, nbytes: int = 0):
        self.buf = None
        self.ensure(nbytes)

    def ensure(self, nbytes: int):
        torch = _torch()
        if self.buf is None or self.buf.numel() < nbytes + 256:
            self.buf = torch.empty(max(nbytes, 1) + 256, dtype=torch.uint8, device="cuda")
        return self

    def ptr(self) -> int:
        p = self.buf.data_ptr()
        return (p + 255) & ~255

    def nbytes(self) -> int:
        return self.buf.numel() - (self.ptr() - self.buf.data_ptr())


def grim_filter(index: GrimIndex, reads, offsets, lens, e, cand=None, cand_off=None,
                out=None, cap: int | None = None, workspace: Workspace | None = None, stream=None,
                retry: bool = True):
    """grim_filter on CUDA tensors.

    reads uint8 [bytes], offsets int64/uint64 [n], lens int32/uint32 [n],
    e int16/uint16 [n]; cand int32 [n_cand] and cand_off int64/uint64 [n+1]
    for candidate mode.  ``out`` may be a preallocated (read, bin, count)
    triple of CUDA tensors of length cap.  Returns (read, bin, count) views of
    the first n_out records.  With ``retry`` an overflow is retried once with
    a capacity of exactly n_out.
    """
    torch = _torch()
    n_reads = int(lens.numel())
    n_cand = int(cand.numel()) if cand is not None else 0
    user_out = out is not None
    if out is not None:
        cap = _check_out(out, "grim_filter")
    elif cap is None:
        cap = 4 * n_reads + 1024
    if out is None:
        out = (torch.empty(cap, dtype=torch.int32, device="cuda"),
               torch.empty(cap, dtype=torch.int32, device="cuda"),
               torch.empty(cap, dtype=torch.uint8, device="cuda"))
    ws = workspace or Workspace()
    ws.ensure(grim_filter_workspace_size(index, n_reads, n_cand, cap))
    n_out = C.c_uint64(0)
    rc = _lib().grim_filter(
        index.handle, _dptr(reads, "reads", 1) if reads.numel() else 0, _dptr(offsets, "offsets", 8),
        _dptr(lens, "lens", 4), n_reads, _dptr(e, "e", 2), _dptr(cand, "cand", 4),
        _dptr(cand_off, "cand_off", 8), n_cand, _dptr(out[0], "out_read", 4),
        _dptr(out[1], "out_bin", 4), _dptr(out[2], "out_count", 1), cap, C.byref(n_out),
        ws.ptr(), ws.nbytes(), _stream_ptr(stream))
    if rc == GRIM_E_OVERFLOW and retry and not user_out:
        return grim_filter(index, reads, offsets, lens, e, cand, cand_off, cap=int(n_out.value),
                           workspace=ws, stream=stream, retry=False)
    if rc != GRIM_OK:
        err = GrimError(rc, "grim_filter")
        err.n_out = int(n_out.value)
        raise err
    n = int(n_out.value)
    return out[0][:n], out[1][:n], out[2][:n]


def grim_filter_count(index: GrimIndex, reads, offsets, lens, e, cand=None, cand_off=None,
                      workspace: Workspace | None = None, stream=None) -> int:
    """Number of passing (read, bin) pairs, without the pass list (a
    grim_filter call with no output capacity)."""
    n_reads = int(lens.numel())
    n_cand = int(cand.numel()) if cand is not None else 0
    ws = workspace or Workspace()
    ws.ensure(grim_filter_workspace_size(index, n_reads, n_cand, 0))
    n_out = C.c_uint64(0)
    rc = _lib().grim_filter(
        index.handle, _dptr(reads, "reads", 1) if reads.numel() else 0, _dptr(offsets, "offsets", 8),
        _dptr(lens, "lens", 4), n_reads, _dptr(e, "e", 2), _dptr(cand, "cand", 4),
        _dptr(cand_off, "cand_off", 8), n_cand, None, None, None, 0, C.byref(n_out),
        ws.ptr(), ws.nbytes(), _stream_ptr(stream))
    if rc not in (GRIM_OK, GRIM_E_OVERFLOW):
        raise GrimError(rc, "grim_filter")
    return int(n_out.value)


def grim_reverse_complement(reads, offsets, lens, out=None, stream=None):
    """Reverse complements of CUDA-resident reads, at the same offsets."""
    torch = _torch()
    if out is None:
        out = torch.empty_like(reads)
    rc = _lib().grim_reverse_complement(
        _dptr(reads, "reads", 1) if reads.numel() else 0, _dptr(offsets, "offsets", 8),
        _dptr(lens, "lens", 4), int(lens.numel()), _dptr(out, "out", 1) if out.numel() else 0,
        _stream_ptr(stream))
    if rc != GRIM_OK:
        raise GrimError(rc, "grim_reverse_complement")
    return out


def both_strands(reads, offsets, lens, e):
    """A batch of 2n reads for filtering both strands: reads 0..n-1 as given,
    read n+i the reverse complement of read i (same length and budget)."""
    torch = _torch()
    rc = grim_reverse_complement(reads, offsets, lens)
    nb = int(reads.numel())
    return dict(reads=torch.cat([reads, rc]), offsets=torch.cat([offsets, offsets + nb]),
                lens=torch.cat([lens, lens]), e=torch.cat([e, e]))


def grim_filter_host(index: GrimIndex, reads, offsets, lens, e, cand=None, cand_off=None,
                     cap: int | None = None, out=None, stream=None):
    """grim_filter_host on host arrays; returns numpy (read, bin, count).

    ``out`` may be a preallocated host (read, bin, count) triple (pinned
    memory makes the copies asynchronous)."""
    n_reads = len(lens)
    n_cand = len(cand) if cand is not None else 0
    if out is not None:
        cap = len(out[0])
        o_r, o_b, o_c = out
    else:
        if cap is None:
            cap = 4 * n_reads + 1024
        o_r = np.empty(cap, np.uint32)
        o_b = np.empty(cap, np.uint32)
        o_c = np.empty(cap, np.uint8)
    pr, kr = _hptr(reads, "reads", np.uint8)
    po, ko = _hptr(offsets, "offsets", np.uint64)
    pl, kl = _hptr(lens, "lens", np.uint32)
    pe, ke = _hptr(e, "e", np.uint16)
    pc, kc = _hptr(cand, "cand", np.int32)
    pco, kco = _hptr(cand_off, "cand_off", np.uint64)
    pr_o, _ = _hptr(o_r, "out_read", np.uint32)
    pb_o, _ = _hptr(o_b, "out_bin", np.uint32)
    pc_o, _ = _hptr(o_c, "out_count", np.uint8)
    n_out = C.c_uint64(0)
    rc = _lib().grim_filter_host(index.handle, pr, po, pl, n_reads, pe, pc or None, pco or None,
                                 n_cand, pr_o, pb_o, pc_o, cap, C.byref(n_out), _stream_ptr(stream))
    if rc != GRIM_OK:
        err = GrimError(rc, "grim_filter_host")
        err.n_out = int(n_out.value)
        raise err
    n = int(n_out.value)
    return o_r[:n], o_b[:n], o_c[:n]


def grim_noalloc_scratch_bytes() -> int:
    """Bytes of the fixed device scratch array grim_filter_noalloc uses (the
    library's own figure, so callers size batches against the real limit)."""
    return int(_lib().grim_noalloc_scratch_bytes())


def grim_filter_noalloc(index: GrimIndex, reads, offsets, lens, e, out, cand=None, cand_off=None,
                        stream=None):
    """grim_filter_noalloc on CUDA tensors: the filter without any device
    allocation, for callers that cannot allocate (a process whose memory
    manager owns the whole GPU, or a serving loop that keeps cudaMalloc off
    its request path).  Scratch comes from one fixed array inside the library
    (``grim_noalloc_scratch_bytes()`` bytes), shared by all calls: calls must not
    overlap on the GPU.  ``out`` is the caller's (read, bin, count) triple of
    CUDA tensors; returns views of its first n_out records.  Raises
    GrimError(GRIM_E_WORKSPACE) when the call needs more scratch than the
    array holds (``grim_noalloc_scratch_bytes()``)."""
    n_reads = int(lens.numel())
    n_cand = int(cand.numel()) if cand is not None else 0
    cap = _check_out(out, "grim_filter_noalloc")
    n_out = C.c_uint64(0)
    rc = _lib().grim_filter_noalloc(
        index.handle, _dptr(reads, "reads", 1) if reads.numel() else 0, _dptr(offsets, "offsets", 8),
        _dptr(lens, "lens", 4), n_reads, _dptr(e, "e", 2), _dptr(cand, "cand", 4),
        _dptr(cand_off, "cand_off", 8), n_cand, _dptr(out[0], "out_read", 4),
        _dptr(out[1], "out_bin", 4), _dptr(out[2], "out_count", 1), cap, C.byref(n_out),
        _stream_ptr(stream))
    if rc != GRIM_OK:
        err = GrimError(rc, "grim_filter_noalloc")
        err.n_out = int(n_out.value)
        raise err
    n = int(n_out.value)
    return out[0][:n], out[1][:n], out[2][:n]


# ---------------------------------------------------------------------------
# graph-captured plans
# ---------------------------------------------------------------------------

class GrimPlan:
    """Owns a grim_plan handle (and keeps its index alive)."""

    def __init__(self, handle: int, index: GrimIndex, desc: _PlanDesc):
        self._h = handle
        self.index = index
        self.max_reads = int(desc.max_reads)
        self.max_bases = int(desc.max_bases)
        self.max_cand = int(desc.max_cand)
        self.cap = int(desc.cap)
        self.candidates = bool(desc.flags & GRIM_PLAN_CANDIDATES)
        self.host_io = bool(desc.flags & GRIM_PLAN_HOST_IO)
        self.buffers = grim_plan_buffers_get(self)

    @property
    def handle(self) -> int:
        if not self._h:
            raise ValueError("plan already freed")
        return self._h

    def close(self) -> None:
        if self._h:
            _lib().grim_plan_free(self._h)
            self._h = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def stage(self, reads, offsets, lens, e, cand=None, cand_off=None):
        """Copy one batch into the plan's buffers: CUDA or pinned CPU tensors
        on the current stream, or host arrays for a host-memory plan."""
        b = self.buffers
        n = len(lens)
        nb = len(reads)
        if n > self.max_reads or nb > self.max_bases:
            raise ValueError("batch larger than the plan")
        if self.host_io:
            for name, x in (("reads", reads), ("offsets", offsets), ("lens", lens), ("e", e)):
                a = np.asarray(x.cpu() if hasattr(x, "cpu") else x).reshape(-1)
                b[name][:len(a)] = a.view(b[name].dtype)
            if self.candidates:
                c = np.asarray(cand).reshape(-1)
                if len(c) > self.max_cand:
                    raise ValueError("more candidates than the plan holds")
                b["cand"][:len(c)] = c.view(np.int32)
                b["cand_off"][:n + 1] = np.asarray(cand_off).reshape(-1).view(np.uint64)
                return n, len(c)
            return n, 0
        b["reads"][:nb].copy_(reads.view(b["reads"].dtype), non_blocking=True)
        b["offsets"][:n].copy_(offsets.view(b["offsets"].dtype), non_blocking=True)
        b["lens"][:n].copy_(lens.view(b["lens"].dtype), non_blocking=True)
        b["e"][:n].copy_(e.view(b["e"].dtype), non_blocking=True)
        if self.candidates:
            nc = int(cand.numel())
            if nc > self.max_cand:
                raise ValueError("more candidates than the plan holds")
            b["cand"][:nc].copy_(cand.view(b["cand"].dtype), non_blocking=True)
            b["cand_off"][:n + 1].copy_(cand_off.view(b["cand_off"].dtype), non_blocking=True)
            return n, nc
        return n, 0

    def run(self, reads, offsets, lens, e, cand=None, cand_off=None, stream=None):
        """stage + launch + wait; returns (read, bin, count) views of the
        plan's output buffers (valid until the plan's next launch)."""
        n, nc = self.stage(reads, offsets, lens, e, cand, cand_off)
        grim_plan_launch(self, n, nc, stream)
        k = grim_plan_wait(self)
        b = self.buffers
        out = b["out_read"][:k], b["out_bin"][:k], b["out_count"][:k]
        return tuple(x.copy() for x in out) if self.host_io else out


def grim_plan_create(index: GrimIndex, max_reads: int, max_bases: int, max_e: int, cap: int,
                     max_cand: int = 0, candidates: bool = False, cand_unroll: int = 0,
                     host_io: bool = False) -> GrimPlan:
    d = _PlanDesc(max_reads, max_e, max_bases, max_cand, cap,
                  (GRIM_PLAN_CANDIDATES if candidates else 0) | (GRIM_PLAN_HOST_IO if host_io else 0),
                  cand_unroll)
    h = C.c_void_p()
    rc = _lib().grim_plan_create(index.handle, C.byref(d), C.byref(h))
    if rc != GRIM_OK:
        raise GrimError(rc, "grim_plan_create")
    return GrimPlan(h.value, index, d)


#: element types of a host-memory plan's buffers (the C types of grim.h)
_HOST_TYPES = {"reads": np.uint8, "offsets": np.uint64, "lens": np.uint32, "e": np.uint16,
               "cand": np.int32, "cand_off": np.uint64, "out_read": np.uint32,
               "out_bin": np.uint32, "out_count": np.uint8}


def grim_plan_buffers_get(plan: GrimPlan) -> dict:
    """The plan's buffers as zero-copy CUDA tensors (numpy arrays over the
    mapped host memory of a host-memory plan)."""
    torch = _torch()
    b = _PlanBuffers()
    rc = _lib().grim_plan_buffers_get(plan.handle, C.byref(b))
    if rc != GRIM_OK:
        raise GrimError(rc, "grim_plan_buffers_get")
    spec = {"reads": (plan.max_bases, "|u1"), "offsets": (plan.max_reads, "<i8"),
            "lens": (plan.max_reads, "<i4"), "e": (plan.max_reads, "<i2"),
            "cand": (plan.max_cand, "<i4"), "cand_off": (plan.max_reads + 1, "<i8"),
            "out_read": (plan.cap, "<i4"), "out_bin": (plan.cap, "<i4"),
            "out_count": (plan.cap, "|u1")}
    out = {}
    for name, (n, ts) in spec.items():
        ptr = getattr(b, name)
        if ptr and n:
            if plan.host_io:
                dt = np.dtype(_HOST_TYPES[name])
                raw = (C.c_char * (n * dt.itemsize)).from_address(ptr)
                out[name] = np.frombuffer(raw, dtype=dt)
            else:
                out[name] = torch.as_tensor(_CudaArray(ptr, (n,), ts, plan), device="cuda")
    return out


def grim_plan_launch(plan: GrimPlan, n_reads: int, n_cand: int = 0, stream=None) -> None:
    rc = _lib().grim_plan_launch(plan.handle, n_reads, n_cand, _stream_ptr(stream))
    if rc != GRIM_OK:
        raise GrimError(rc, "grim_plan_launch")


def grim_plan_query(plan: GrimPlan) -> bool:
    """True when the plan's last launch has finished."""
    rc = _lib().grim_plan_query(plan.handle)
    if rc == GRIM_E_NOT_READY:
        return False
    if rc != GRIM_OK:
        raise GrimError(rc, "grim_plan_query")
    return True


def grim_plan_wait(plan: GrimPlan) -> int:
    """Wait for the last launch; returns the number of passing records."""
    n_out = C.c_uint64(0)
    rc = _lib().grim_plan_wait(plan.handle, C.byref(n_out))
    if rc != GRIM_OK:
        err = GrimError(rc, "grim_plan_wait")
        err.n_out = int(n_out.value)
        raise err
    return int(n_out.value)


def grim_plan_device_bytes(plan: GrimPlan) -> int:
    return int(_lib().grim_plan_device_bytes(plan.handle))


def grim_plan_free(plan: GrimPlan) -> None:
    plan.close()


# ---------------------------------------------------------------------------
# serving: continuous batching over a resident index
# ---------------------------------------------------------------------------

@dataclass
class RequestInfo:
    status: int
    n_reads: int
    n_out: int
    batch: int
    batch_requests: int
    batch_reads: int
    t_submit_ns: int
    t_launch_ns: int
    t_done_ns: int

    @property
    def latency_s(self) -> float:
        return (self.t_done_ns - self.t_submit_ns) * 1e-9


class GrimServer:
    """Owns a grim_server handle (and keeps its index alive)."""

    def __init__(self, handle: int, index: GrimIndex, desc: _ServerDesc):
        self._h = handle
        self.index = index
        self.candidates = bool(desc.flags & GRIM_PLAN_CANDIDATES)
        self.cap = int(desc.cap)

    @property
    def handle(self) -> int:
        if not self._h:
            raise ValueError("server already freed")
        return self._h

    def close(self) -> None:
        if self._h:
            _lib().grim_server_free(self._h)
            self._h = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def submit(self, reads, offsets, lens, e, cand=None, cand_off=None) -> int:
        return grim_server_submit(self, reads, offsets, lens, e, cand, cand_off)

    def result(self, ticket: int, timeout_s: float | None = None):
        """Wait for a request and take its pass list: ((read, bin, count), RequestInfo)."""
        grim_server_wait(self, ticket, timeout_s)
        return grim_server_take(self, ticket)

    def cancel(self, ticket: int) -> bool:
        return grim_server_cancel(self, ticket)

    def stats(self) -> dict:
        return grim_server_stats_get(self)


def grim_server_create(index: GrimIndex, slots: int, max_reads: int, max_bases: int, max_e: int,
                       cap: int, max_cand: int = 0, candidates: bool = False,
                       mem_budget: int = 0, max_queued_reads: int = 0,
                       cand_unroll: int = 0, max_chunk_reads: int = 0) -> GrimServer:
    """``max_chunk_reads``: cut requests into chunks of at most this many
    consecutive reads (0: run each request whole)."""
    d = _ServerDesc(slots, max_reads, max_bases, max_cand, cap, max_e,
                    GRIM_PLAN_CANDIDATES if candidates else 0, mem_budget, max_queued_reads,
                    cand_unroll, max_chunk_reads)
    h = C.c_void_p()
    rc = _lib().grim_server_create(index.handle, C.byref(d), C.byref(h))
    if rc != GRIM_OK:
        raise GrimError(rc, "grim_server_create")
    return GrimServer(h.value, index, d)


def grim_server_submit(server: GrimServer, reads, offsets, lens, e, cand=None,
                       cand_off=None) -> int:
    """Queue one request (host arrays, copied before return); returns its ticket."""
    pr, kr = _hptr(reads, "reads", np.uint8)
    po, ko = _hptr(offsets, "offsets", np.uint64)
    pl, kl = _hptr(lens, "lens", np.uint32)
    pe, ke = _hptr(e, "e", np.uint16)
    pc, kc = _hptr(cand, "cand", np.int32)
    pco, kco = _hptr(cand_off, "cand_off", np.uint64)
    t = C.c_uint64(0)
    rc = _lib().grim_server_submit(server.handle, pr, po, pl, len(lens), pe, pc or None,
                                   pco or None, C.byref(t))
    if rc != GRIM_OK:
        raise GrimError(rc, "grim_server_submit")
    return int(t.value)


def grim_server_wait(server: GrimServer, ticket: int, timeout_s: float | None = None) -> bool:
    """True once the request has completed; False on timeout."""
    us = -1 if timeout_s is None else int(timeout_s * 1e6)
    rc = _lib().grim_server_wait(server.handle, ticket, us)
    if rc == GRIM_E_NOT_READY:
        return False
    if rc != GRIM_OK:
        raise GrimError(rc, "grim_server_wait")
    return True


def grim_server_take(server: GrimServer, ticket: int):
    """Take a completed request's pass list: ((read, bin, count), RequestInfo)."""
    info = _RequestInfo()
    cap = 0
    o_r = o_b = o_c = None
    while True:
        rc = _lib().grim_server_take(
            server.handle, ticket, o_r.ctypes.data if o_r is not None else None,
            o_b.ctypes.data if o_b is not None else None,
            o_c.ctypes.data if o_c is not None else None, cap, C.byref(info))
        if rc != GRIM_E_OVERFLOW or info.status != GRIM_OK:
            break
        cap = int(info.n_out)  # the request is kept: take it again with room for it
        o_r = np.empty(cap, np.uint32)
        o_b = np.empty(cap, np.uint32)
        o_c = np.empty(cap, np.uint8)
    ri = RequestInfo(*(getattr(info, f) for f, _ in _RequestInfo._fields_))
    if rc != GRIM_OK:
        err = GrimError(rc, "grim_server_take")
        err.n_out = int(info.n_out)
        err.info = ri
        raise err
    n = int(info.n_out)
    if o_r is None:
        o_r, o_b, o_c = np.empty(0, np.uint32), np.empty(0, np.uint32), np.empty(0, np.uint8)
    return (o_r[:n], o_b[:n], o_c[:n]), ri


def grim_server_cancel(server: GrimServer, ticket: int) -> bool:
    """Cancel a queued request; False if it is already running (it then
    completes normally)."""
    rc = _lib().grim_server_cancel(server.handle, ticket)
    if rc == GRIM_E_NOT_READY:
        return False
    if rc != GRIM_OK:
        raise GrimError(rc, "grim_server_cancel")
    return True


def grim_server_stats_get(server: GrimServer) -> dict:
    st = _ServerStats()
    rc = _lib().grim_server_stats_get(server.handle, C.byref(st))
    if rc != GRIM_OK:
        raise GrimError(rc, "grim_server_stats_get")
    return {f: int(getattr(st, f)) for f, _ in _ServerStats._fields_ if f != "reserved"}


def grim_server_free(server: GrimServer) -> None:
    server.close()
