"""Thin Python binding of librr's C ABI (include/rr.h).

Functions carry the C names and only marshal arguments: torch CUDA tensors
become device pointers, the current torch stream becomes the cudaStream_t.
Every step of the pipeline runs in librr's kernels.  There is no fallback:
if librr.so is missing or fails to load, every call raises.

Storage dtypes: uint32 buffers are torch.int32 tensors and uint64 keys are
torch.int64 tensors (same bits); use ``.view(numpy.uint32/uint64)`` on the
host side.  Rays are float32 [N,4] tensors (o_tmin, d_tmax), hits float32 [N,4]
(t, u, v, triangle id bits).
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from dataclasses import dataclass

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
# RR_LIBRARY=checked selects the bounds-checked build (librr_checked.so), where
# every kernel index is checked against its buffer (RR_DEVERR_BAD_INDEX).
LIB_PATH = os.path.join(_HERE, "librr_checked.so" if os.environ.get("RR_LIBRARY") == "checked" else "librr.so")
_lock = threading.Lock()
_lib = None

RR_KEY_AILA, RR_KEY_AILA_COMPACT, RR_KEY_TWO_POINT = 0, 1, 2
RR_KEY_ORIGIN, RR_KEY_REIS, RR_KEY_COSTA, RR_KEY_OCTAHEDRON = 3, 4, 5, 6
RR_T_FIXED, RR_T_ADAPTIVE, RR_T_GIVEN = 0, 1, 2
RR_DEVERR_LOOKBACK_TIMEOUT = 0x1
RR_DEVERR_TRACE_STACK = 0x2
RR_DEVERR_BAD_INDEX = 0x4
RR_DEVERR_COPY_TIMEOUT = 0x8
RR_TRACE_ANY_HIT = 0x1
RR_UPLOAD_ADAPTIVE, RR_UPLOAD_ENGINES, RR_UPLOAD_KERNEL = 0, 1, 2
MISS = 0xFFFFFFFF
TABLE_CELLS = 1 << 20

STATUS = {0: "RR_OK", 1: "RR_ERR_INVALID_ARG", 2: "RR_ERR_CUDA", 3: "RR_ERR_OOM",
          4: "RR_ERR_TIMEOUT", 5: "RR_ERR_STACK", 6: "RR_ERR_UNSUPPORTED", 7: "RR_ERR_TOO_LARGE",
          8: "RR_ERR_DEVICE"}
RR_SORT_NOALLOC_MAX_N = 1 << 20

# every symbol include/rr.h declares
EXPORTS = [
    "rr_compute_keys", "rr_sort_workspace_size", "rr_sort", "rr_permute", "rr_build_bvh",
    "rr_bvh_destroy", "rr_bvh_get_info", "rr_trace", "rr_trace_accumulate", "rr_length_table_create",
    "rr_length_table_reset", "rr_length_table_accumulate", "rr_length_table_read",
    "rr_length_table_write", "rr_length_table_destroy", "rr_pipeline_create",
    "rr_pipeline_destroy", "rr_pipeline_run", "rr_pipeline_run_host", "rr_pipeline_submit_host",
    "rr_pipeline_wait", "rr_device_error",
    "rr_status_string", "rr_last_error_message", "rr_kernel_launch_count", "rr_sort_noalloc",
    "rr_coherence_capsule", "rr_trace_ex", "rr_sort_segments", "rr_batch_create", "rr_batch_destroy",
    "rr_batch_info", "rr_batch_run", "rr_batch_run_loop", "rr_batch_tune", "rr_server_create",
    "rr_server_add_scene", "rr_server_submit", "rr_server_wait", "rr_server_stats", "rr_server_destroy",
    "rr_selftest_lookback_timeout", "rr_stream_error", "rr_bvh_aabb", "rr_fault_inject", "rr_key_sort",
    "rr_bvh_serialize", "rr_bvh_deserialize", "rr_batch_tune_cached",
]


class RRError(RuntimeError):
    def __init__(self, status: int, what: str, msg: str):
        super().__init__("%s: %s (%s)" % (what, STATUS.get(status, status), msg))
        self.status = status


class KeyParams(C.Structure):
    _fields_ = [("layout", C.c_uint32), ("bits", C.c_uint32), ("t_source", C.c_uint32),
                ("ratio", C.c_float), ("aabb_lo", C.c_float * 3), ("aabb_hi", C.c_float * 3),
                ("t_given", C.c_void_p), ("table", C.c_void_p)]


class Wavefront(C.Structure):
    _fields_ = [("bvh", C.c_void_p), ("table", C.c_void_p), ("aabb_lo", C.c_float * 3),
                ("aabb_hi", C.c_float * 3), ("offset", C.c_uint32), ("count", C.c_uint32)]


class BatchConfig(C.Structure):
    _fields_ = [("key_bits", C.c_uint32), ("radix_bits", C.c_uint32), ("trace_block", C.c_uint32),
                ("layout", C.c_int32)]

    def as_tuple(self):
        return (int(self.key_bits), int(self.radix_bits), int(self.trace_block), int(self.layout))


class ServerConfig(C.Structure):
    _fields_ = [("budget_bytes", C.c_uint64), ("slots", C.c_uint32), ("max_batch_rays", C.c_uint32),
                ("layout", C.c_uint32), ("t_source", C.c_uint32), ("ratio", C.c_float),
                ("key_bits", C.c_uint32), ("radix_bits", C.c_uint32), ("trace_block", C.c_uint32),
                ("reserve_bytes", C.c_uint64), ("upload", C.c_uint32)]


class RequestTimes(C.Structure):
    _fields_ = [("submit_ns", C.c_uint64), ("start_ns", C.c_uint64), ("done_ns", C.c_uint64),
                ("batch_requests", C.c_uint32), ("device_flags", C.c_uint32), ("enqueued_ns", C.c_uint64),
                ("copy_in_ms", C.c_float), ("kernels_ms", C.c_float), ("copy_out_ms", C.c_float),
                ("device_ms", C.c_float), ("kernel_copies", C.c_uint32)]


class ServerStats(C.Structure):
    _fields_ = [("batches", C.c_uint64), ("max_batch_requests", C.c_uint64),
                ("peak_reserved_bytes", C.c_uint64), ("reserved_bytes", C.c_uint64), ("waiting", C.c_uint64),
                ("engine_slowdowns", C.c_uint64), ("kernel_copy_groups", C.c_uint64)]


class BvhInfo(C.Structure):
    _fields_ = [("n_tris", C.c_uint32), ("n_nodes", C.c_uint32), ("n_leaves", C.c_uint32),
                ("depth", C.c_uint32), ("node_bytes", C.c_uint64), ("tri_bytes", C.c_uint64),
                ("aabb_lo", C.c_float * 3), ("aabb_hi", C.c_float * 3),
                ("build_seconds", C.c_double)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError("librr.so is not built (%s); run __graft_entry__.build() or "
                                   "python paper_2506_11273_gb300/build.py" % LIB_PATH)
            L = C.CDLL(LIB_PATH)
            vp, u32, i32 = C.c_void_p, C.c_uint32, C.c_int
            L.rr_compute_keys.argtypes = [vp, vp, u32, C.POINTER(KeyParams), vp, vp]
            L.rr_sort_workspace_size.argtypes = [u32, u32, u32, C.POINTER(C.c_size_t)]
            L.rr_sort.argtypes = [vp, vp, vp, u32, u32, u32, vp, C.c_size_t, vp]
            L.rr_key_sort.argtypes = [vp, vp, u32, C.POINTER(KeyParams), vp, vp, u32, vp, C.c_size_t, vp]
            L.rr_sort_noalloc.argtypes = [vp, vp, vp, u32, u32, u32, vp]
            L.rr_permute.argtypes = [vp, vp, vp, vp, u32, vp, vp, vp, vp]
            L.rr_build_bvh.argtypes = [vp, u32, C.POINTER(vp)]
            L.rr_bvh_serialize.argtypes = [vp, vp, C.POINTER(C.c_size_t)]
            L.rr_bvh_deserialize.argtypes = [vp, C.c_size_t, C.POINTER(vp)]
            L.rr_bvh_destroy.argtypes = [vp]
            L.rr_bvh_get_info.argtypes = [vp, C.POINTER(BvhInfo)]
            L.rr_trace.argtypes = [vp, vp, vp, u32, vp, vp]
            L.rr_trace_accumulate.argtypes = [vp, vp, vp, u32, vp, vp, vp]
            L.rr_length_table_create.argtypes = [C.POINTER(C.c_float), C.POINTER(C.c_float),
                                                 C.POINTER(vp), vp]
            L.rr_length_table_reset.argtypes = [vp, vp]
            L.rr_length_table_accumulate.argtypes = [vp, vp, vp, vp, u32, vp]
            L.rr_length_table_read.argtypes = [vp, vp, vp]
            L.rr_length_table_write.argtypes = [vp, vp, vp]
            L.rr_length_table_destroy.argtypes = [vp]
            L.rr_pipeline_create.argtypes = [vp, u32, C.POINTER(KeyParams), u32, C.POINTER(vp)]
            L.rr_pipeline_destroy.argtypes = [vp]
            L.rr_pipeline_run.argtypes = [vp, vp, vp, vp, u32, vp, vp, vp]
            L.rr_pipeline_run_host.argtypes = [vp, vp, vp, vp, u32, vp, vp, vp]
            L.rr_pipeline_submit_host.argtypes = [vp, vp, vp, vp, u32, vp, vp, vp, C.POINTER(C.c_uint64)]
            L.rr_pipeline_wait.argtypes = [vp, C.c_uint64]
            L.rr_sort_segments.argtypes = [vp, vp, vp, u32, u32, u32, vp]
            L.rr_trace_ex.argtypes = [vp, vp, vp, vp, u32, vp, u32, vp, vp]
            L.rr_batch_create.argtypes = [C.POINTER(Wavefront), u32, u32, u32, C.c_float, C.POINTER(vp)]
            L.rr_batch_destroy.argtypes = [vp]
            L.rr_batch_info.argtypes = [vp, C.POINTER(u32), C.POINTER(u32), C.POINTER(u32)]
            L.rr_batch_run.argtypes = [vp, vp, vp, vp, vp, C.POINTER(BatchConfig), vp]
            L.rr_batch_run_loop.argtypes = [vp, vp, vp, vp, vp, C.POINTER(BatchConfig), vp]
            L.rr_batch_tune.argtypes = [vp, vp, vp, vp, C.POINTER(BatchConfig), C.POINTER(C.c_float), vp]
            L.rr_batch_tune_cached.argtypes = [vp, vp, vp, vp, C.c_char_p, C.POINTER(BatchConfig),
                                               C.POINTER(C.c_float), C.POINTER(C.c_uint32), vp]
            L.rr_server_create.argtypes = [C.POINTER(ServerConfig), C.POINTER(vp)]
            L.rr_server_add_scene.argtypes = [vp, vp, vp, C.POINTER(C.c_float), C.POINTER(C.c_float),
                                              C.POINTER(u32)]
            L.rr_server_submit.argtypes = [vp, u32, vp, vp, u32, vp, C.POINTER(C.c_uint64)]
            L.rr_server_wait.argtypes = [vp, C.c_uint64, C.c_double, C.POINTER(RequestTimes)]
            L.rr_server_stats.argtypes = [vp, C.POINTER(ServerStats)]
            L.rr_server_destroy.argtypes = [vp]
            L.rr_selftest_lookback_timeout.argtypes = [vp]
            L.rr_coherence_capsule.argtypes = [vp, vp, vp, u32, u32, C.c_float, vp, vp]
            L.rr_device_error.argtypes = [C.POINTER(C.c_uint32)]
            L.rr_stream_error.argtypes = [vp, vp]
            L.rr_fault_inject.argtypes = [C.c_char_p]
            L.rr_bvh_aabb.argtypes = [vp, C.POINTER(C.c_float), C.POINTER(C.c_float)]
            L.rr_status_string.argtypes = [i32]
            L.rr_status_string.restype = C.c_char_p
            L.rr_last_error_message.argtypes = []
            L.rr_last_error_message.restype = C.c_char_p
            L.rr_kernel_launch_count.argtypes = []
            L.rr_kernel_launch_count.restype = C.c_uint64
            _lib = L
    return _lib


def _check(status: int, what: str):
    if status != 0:
        msg = lib().rr_last_error_message().decode(errors="replace")
        raise RRError(status, what, msg)


def _ptr(t) -> int | None:
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return t.data_ptr()


def _hptr(t) -> int | None:
    """Host pointer of a numpy array or a CPU (ideally pinned) torch tensor."""
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        if not t.flags["C_CONTIGUOUS"]:
            raise ValueError("expected a contiguous array")
        return t.ctypes.data
    if t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CPU tensor")
    return t.data_ptr()


def _stream(stream) -> int | None:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


# ---------------------------------------------------------------- keys

def key_params(layout: int, bits: int, aabb_lo, aabb_hi, t_source: int = RR_T_FIXED,
               ratio: float = 0.25, t_given=None, table: "LengthTable | None" = None) -> KeyParams:
    p = KeyParams()
    p.layout, p.bits, p.t_source, p.ratio = layout, bits, t_source, float(np.float32(ratio))
    for c in range(3):
        p.aabb_lo[c] = float(np.float32(aabb_lo[c]))
        p.aabb_hi[c] = float(np.float32(aabb_hi[c]))
    p.t_given = _ptr(t_given)
    p.table = table.handle if table is not None else None
    p._keep = (t_given, table)  # keep referenced objects alive with the struct
    return p


def rr_compute_keys(o_tmin, d_tmax, params: KeyParams, keys_out, n: int | None = None, stream=None):
    n = o_tmin.shape[0] if n is None else n
    _check(lib().rr_compute_keys(_ptr(o_tmin), _ptr(d_tmax), n, C.byref(params), _ptr(keys_out),
                                 _stream(stream)), "rr_compute_keys")


# ---------------------------------------------------------------- sort

def rr_sort_workspace_size(n: int, bits: int, radix_bits: int = 8) -> int:
    b = C.c_size_t()
    _check(lib().rr_sort_workspace_size(n, bits, radix_bits, C.byref(b)), "rr_sort_workspace_size")
    return int(b.value)


def rr_sort(keys_in, keys_out, perm_out, n: int, bits: int, radix_bits: int, workspace,
            stream=None):
    nbytes = workspace.numel() * workspace.element_size()
    _check(lib().rr_sort(_ptr(keys_in), _ptr(keys_out), _ptr(perm_out), n, bits, radix_bits,
                         _ptr(workspace), nbytes, _stream(stream)), "rr_sort")


def rr_key_sort(o_tmin, d_tmax, params: KeyParams, keys_out, perm_out, radix_bits: int, workspace,
                n: int | None = None, stream=None):
    """rr_compute_keys followed by rr_sort of those keys, the sort's digit
    counting done by the key kernel."""
    n = o_tmin.shape[0] if n is None else n
    nbytes = workspace.numel() * workspace.element_size()
    _check(lib().rr_key_sort(_ptr(o_tmin), _ptr(d_tmax), n, C.byref(params), _ptr(keys_out), _ptr(perm_out),
                             radix_bits, _ptr(workspace), nbytes, _stream(stream)), "rr_key_sort")


def rr_sort_segments(keys_in, keys_out, perm_out, n: int, bits: int, segment: int, stream=None):
    """Stable sort inside each run of `segment` consecutive keys (local sort)."""
    _check(lib().rr_sort_segments(_ptr(keys_in), _ptr(keys_out), _ptr(perm_out), n, bits, segment,
                                  _stream(stream)), "rr_sort_segments")


def rr_sort_noalloc(keys_in, keys_out, perm_out, n: int, bits: int, radix_bits: int, stream=None):
    """rr_sort without a workspace argument, for callers that cannot allocate device
    memory (n <= RR_SORT_NOALLOC_MAX_N).  Errors come back as the status only."""
    st = lib().rr_sort_noalloc(_ptr(keys_in), _ptr(keys_out), _ptr(perm_out), n, bits, radix_bits,
                               _stream(stream))
    if st != 0:
        raise RRError(st, "rr_sort_noalloc", rr_status_string(st))


def sort_workspace(n: int, bits: int, radix_bits: int = 8, device="cuda") -> torch.Tensor:
    size = rr_sort_workspace_size(n, bits, radix_bits)
    # torch's caching allocator returns 512-byte aligned blocks
    return torch.empty(max(size, 256), dtype=torch.uint8, device=device)


# ---------------------------------------------------------------- reorder

def rr_permute(o_tmin_in, d_tmax_in, payload_in, perm, o_tmin_out, d_tmax_out, payload_out,
               n: int | None = None, stream=None):
    n = perm.shape[0] if n is None else n
    _check(lib().rr_permute(_ptr(o_tmin_in), _ptr(d_tmax_in), _ptr(payload_in), _ptr(perm), n,
                            _ptr(o_tmin_out), _ptr(d_tmax_out), _ptr(payload_out),
                            _stream(stream)), "rr_permute")


# ---------------------------------------------------------------- BVH and trace

class BVH:
    """Owner of an rr_bvh handle built from a host triangle soup [T,9] float32."""

    def __init__(self, tris: np.ndarray | None = None, *, serialized: bytes | None = None):
        h = C.c_void_p()
        if serialized is not None:
            buf = C.create_string_buffer(bytes(serialized), len(serialized))
            _check(lib().rr_bvh_deserialize(buf, len(serialized), C.byref(h)), "rr_bvh_deserialize")
            self.handle = h.value
            self.n_tris = self.info().n_tris
            return
        tris = np.ascontiguousarray(tris, dtype=np.float32).reshape(-1, 9)
        self.n_tris = tris.shape[0]
        _check(lib().rr_build_bvh(tris.ctypes.data if self.n_tris else None, self.n_tris,
                                  C.byref(h)), "rr_build_bvh")
        self.handle = h.value

    def serialize(self) -> bytes:
        """The BVH in rr_bvh_serialize's format (BVH(serialized=...) reloads it)."""
        need = C.c_size_t()
        _check(lib().rr_bvh_serialize(self.handle, None, C.byref(need)), "rr_bvh_serialize")
        buf = C.create_string_buffer(need.value)
        cap = C.c_size_t(need.value)
        _check(lib().rr_bvh_serialize(self.handle, buf, C.byref(cap)), "rr_bvh_serialize")
        return buf.raw[: cap.value]

    def info(self) -> BvhInfo:
        i = BvhInfo()
        _check(lib().rr_bvh_get_info(self.handle, C.byref(i)), "rr_bvh_get_info")
        return i

    def aabb(self):
        i = self.info()
        return (np.array(list(i.aabb_lo), np.float32), np.array(list(i.aabb_hi), np.float32))

    def close(self):
        if getattr(self, "handle", None):
            lib().rr_bvh_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def rr_build_bvh(tris: np.ndarray) -> BVH:
    return BVH(tris)


def rr_trace(bvh: BVH, o_tmin, d_tmax, hits_out, n: int | None = None, stream=None):
    n = o_tmin.shape[0] if n is None else n
    _check(lib().rr_trace(bvh.handle, _ptr(o_tmin), _ptr(d_tmax), n, _ptr(hits_out),
                          _stream(stream)), "rr_trace")


def rr_trace_accumulate(bvh: BVH, o_tmin, d_tmax, hits_out, table: "LengthTable", n: int | None = None,
                        stream=None):
    n = o_tmin.shape[0] if n is None else n
    _check(lib().rr_trace_accumulate(bvh.handle, _ptr(o_tmin), _ptr(d_tmax), n, _ptr(hits_out),
                                     table.handle, _stream(stream)), "rr_trace_accumulate")


def rr_trace_ex(bvh: BVH, o_tmin, d_tmax, hits_out, order=None, flags: int = 0, table: "LengthTable" = None,
                n: int | None = None, stream=None):
    """Trace with an optional index buffer (indirect access) and any-hit flag."""
    n = o_tmin.shape[0] if n is None else n
    _check(lib().rr_trace_ex(bvh.handle, _ptr(o_tmin), _ptr(d_tmax), _ptr(order) if order is not None else None,
                             n, _ptr(hits_out), flags, table.handle if table is not None else None,
                             _stream(stream)), "rr_trace_ex")


# ---------------------------------------------------------------- ray-length table

class LengthTable:
    """Owner of an rr_length_table (2^20 cells) for one scene box."""

    def __init__(self, aabb_lo, aabb_hi, stream=None):
        lo = (C.c_float * 3)(*[float(np.float32(x)) for x in aabb_lo])
        hi = (C.c_float * 3)(*[float(np.float32(x)) for x in aabb_hi])
        h = C.c_void_p()
        _check(lib().rr_length_table_create(lo, hi, C.byref(h), _stream(stream)),
               "rr_length_table_create")
        self.handle = h.value

    def reset(self, stream=None):
        _check(lib().rr_length_table_reset(self.handle, _stream(stream)), "rr_length_table_reset")

    def accumulate(self, o_tmin, d_tmax, hits, n: int | None = None, stream=None):
        rr_length_table_accumulate(self, o_tmin, d_tmax, hits, n, stream)

    def read(self):
        s = np.zeros(TABLE_CELLS, np.uint64)
        c = np.zeros(TABLE_CELLS, np.uint32)
        _check(lib().rr_length_table_read(self.handle, s.ctypes.data, c.ctypes.data),
               "rr_length_table_read")
        return s, c

    def write(self, s: np.ndarray, c: np.ndarray):
        s = np.ascontiguousarray(s, np.uint64)
        c = np.ascontiguousarray(c, np.uint32)
        _check(lib().rr_length_table_write(self.handle, s.ctypes.data, c.ctypes.data),
               "rr_length_table_write")

    def close(self):
        if getattr(self, "handle", None):
            lib().rr_length_table_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def rr_length_table_accumulate(table: LengthTable, o_tmin, d_tmax, hits, n: int | None = None,
                               stream=None):
    n = o_tmin.shape[0] if n is None else n
    _check(lib().rr_length_table_accumulate(table.handle, _ptr(o_tmin), _ptr(d_tmax), _ptr(hits), n,
                                            _stream(stream)), "rr_length_table_accumulate")


# ---------------------------------------------------------------- one bounce

class Pipeline:
    """Owner of an rr_pipeline: keys -> sort -> permute -> trace (-> table update)."""

    def __init__(self, bvh: BVH, max_n: int, params: KeyParams, radix_bits: int = 8):
        h = C.c_void_p()
        _check(lib().rr_pipeline_create(bvh.handle, max_n, C.byref(params), radix_bits, C.byref(h)),
               "rr_pipeline_create")
        self.handle = h.value
        self._keep = (bvh, params)

    def run(self, o_tmin, d_tmax, payload_in, hits_out, payload_out, n: int | None = None,
            stream=None):
        n = o_tmin.shape[0] if n is None else n
        _check(lib().rr_pipeline_run(self.handle, _ptr(o_tmin), _ptr(d_tmax), _ptr(payload_in), n,
                                     _ptr(hits_out), _ptr(payload_out), _stream(stream)),
               "rr_pipeline_run")

    def run_host(self, o_tmin, d_tmax, payload_in, hits_out, payload_out, n: int | None = None,
                 stream=None):
        n = o_tmin.shape[0] if n is None else n
        _check(lib().rr_pipeline_run_host(self.handle, _hptr(o_tmin), _hptr(d_tmax),
                                          _hptr(payload_in), n, _hptr(hits_out), _hptr(payload_out),
                                          _stream(stream)), "rr_pipeline_run_host")

    def submit_host(self, o_tmin, d_tmax, payload_in, hits_out, payload_out, n: int | None = None,
                    stream=None) -> int:
        """Enqueues one bounce on host buffers and returns its ticket; the
        buffers belong to the submission until wait(ticket) returns."""
        n = o_tmin.shape[0] if n is None else n
        t = C.c_uint64(0)
        _check(lib().rr_pipeline_submit_host(self.handle, _hptr(o_tmin), _hptr(d_tmax), _hptr(payload_in), n,
                                             _hptr(hits_out), _hptr(payload_out), _stream(stream), C.byref(t)),
               "rr_pipeline_submit_host")
        return t.value

    def wait(self, ticket: int):
        _check(lib().rr_pipeline_wait(self.handle, ticket), "rr_pipeline_wait")

    def close(self):
        if getattr(self, "handle", None):
            lib().rr_pipeline_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- batched execution

class Batch:
    """Owner of an rr_batch: wavefronts over resident scenes, run as one graph.

    fronts: list of (bvh: BVH, table: LengthTable | None, aabb_lo, aabb_hi, count);
    offsets follow from the counts (contiguous, in order)."""

    def __init__(self, fronts, layout: int, t_source: int = RR_T_FIXED, ratio: float = 0.25):
        arr = (Wavefront * len(fronts))()
        off = 0
        self._keep = []
        for k, (bvh, table, lo, hi, count) in enumerate(fronts):
            w = arr[k]
            w.bvh = bvh.handle
            w.table = table.handle if table is not None else None
            for c in range(3):
                w.aabb_lo[c] = float(lo[c])
                w.aabb_hi[c] = float(hi[c])
            w.offset = off
            w.count = int(count)
            off += int(count)
            self._keep.append((bvh, table))
        self.n = off
        self.offsets = [w.offset for w in arr] + [off]
        h = C.c_void_p()
        _check(lib().rr_batch_create(arr, len(fronts), layout, t_source, float(np.float32(ratio)), C.byref(h)),
               "rr_batch_create")
        self.handle = h

    def info(self):
        n, sb, g = C.c_uint32(), C.c_uint32(), C.c_uint32()
        _check(lib().rr_batch_info(self.handle, C.byref(n), C.byref(sb), C.byref(g)), "rr_batch_info")
        return dict(n_rays=n.value, seg_bits=sb.value, graphs=g.value)

    @staticmethod
    def config(key_bits: int, radix_bits: int = 8, trace_block: int = 256, layout: int = -1) -> BatchConfig:
        return BatchConfig(key_bits, radix_bits, trace_block, layout)

    def run(self, o_tmin, d_tmax, hits_out, cfg: BatchConfig, perm_out=None, stream=None):
        _check(lib().rr_batch_run(self.handle, _ptr(o_tmin), _ptr(d_tmax), _ptr(hits_out), _ptr(perm_out),
                                  C.byref(cfg), _stream(stream)), "rr_batch_run")

    def run_loop(self, o_tmin, d_tmax, hits_out, cfg: BatchConfig, perm_out=None, stream=None):
        _check(lib().rr_batch_run_loop(self.handle, _ptr(o_tmin), _ptr(d_tmax), _ptr(hits_out),
                                       _ptr(perm_out), C.byref(cfg), _stream(stream)), "rr_batch_run_loop")

    def tune(self, o_tmin, d_tmax, hits_out, stream=None):
        best = BatchConfig()
        ms = C.c_float()
        _check(lib().rr_batch_tune(self.handle, _ptr(o_tmin), _ptr(d_tmax), _ptr(hits_out), C.byref(best),
                                   C.byref(ms), _stream(stream)), "rr_batch_tune")
        return best, float(ms.value)

    def tune_cached(self, o_tmin, d_tmax, hits_out, cache_path: str, stream=None):
        """rr_batch_tune_cached: (config, ms, from_cache)."""
        best = BatchConfig()
        ms = C.c_float()
        hit = C.c_uint32()
        _check(lib().rr_batch_tune_cached(self.handle, _ptr(o_tmin), _ptr(d_tmax), _ptr(hits_out),
                                          os.fsencode(cache_path), C.byref(best), C.byref(ms), C.byref(hit),
                                          _stream(stream)), "rr_batch_tune_cached")
        return best, float(ms.value), bool(hit.value)

    def close(self):
        if getattr(self, "handle", None):
            lib().rr_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- serving

class Server:
    """Owner of an rr_server: resident scenes, continuous batching of requests.

    Host buffers passed to submit (numpy arrays or pinned CPU tensors) must stay
    alive and untouched until wait() returns for the ticket."""

    def __init__(self, budget_bytes: int, slots: int = 4, max_batch_rays: int = 1 << 24,
                 layout: int = RR_KEY_TWO_POINT, t_source: int = RR_T_FIXED, ratio: float = 0.25,
                 key_bits: int = 24, radix_bits: int = 8, trace_block: int = 128, reserve_bytes: int = 0,
                 upload: int = 0):
        cfg = ServerConfig(int(budget_bytes), slots, max_batch_rays, layout, t_source, float(np.float32(ratio)),
                           key_bits, radix_bits, trace_block, int(reserve_bytes), int(upload))
        h = C.c_void_p()
        _check(lib().rr_server_create(C.byref(cfg), C.byref(h)), "rr_server_create")
        self.handle = h
        self._keep = []
        self._held = {}

    def add_scene(self, bvh: "BVH", aabb_lo, aabb_hi, table: "LengthTable" = None) -> int:
        lo = (C.c_float * 3)(*[float(x) for x in aabb_lo])
        hi = (C.c_float * 3)(*[float(x) for x in aabb_hi])
        sid = C.c_uint32()
        _check(lib().rr_server_add_scene(self.handle, bvh.handle, table.handle if table is not None else None,
                                         lo, hi, C.byref(sid)), "rr_server_add_scene")
        self._keep.append((bvh, table))
        return sid.value

    @staticmethod
    def _host_ptr(a):
        if isinstance(a, np.ndarray):
            if not a.flags.c_contiguous:
                raise ValueError("expected a contiguous array")
            return a.ctypes.data
        if a.is_cuda or not a.is_contiguous():
            raise ValueError("expected a contiguous host tensor")
        return a.data_ptr()

    def submit(self, scene: int, o_tmin, d_tmax, hits_out, n: int | None = None) -> int:
        n = int(o_tmin.shape[0]) if n is None else n
        t = C.c_uint64()
        _check(lib().rr_server_submit(self.handle, scene, self._host_ptr(o_tmin), self._host_ptr(d_tmax), n,
                                      self._host_ptr(hits_out), C.byref(t)), "rr_server_submit")
        self._held[t.value] = (o_tmin, d_tmax, hits_out)
        return t.value

    def wait(self, ticket: int, timeout_s: float = 120.0) -> dict:
        tm = RequestTimes()
        _check(lib().rr_server_wait(self.handle, ticket, timeout_s, C.byref(tm)), "rr_server_wait")
        self._held.pop(ticket, None)
        return {k: getattr(tm, k) for k, _ in RequestTimes._fields_}

    def stats(self) -> dict:
        st = ServerStats()
        _check(lib().rr_server_stats(self.handle, C.byref(st)), "rr_server_stats")
        return {k: int(getattr(st, k)) for k, _ in ServerStats._fields_}

    def close(self):
        if getattr(self, "handle", None):
            lib().rr_server_destroy(self.handle)
            self.handle = None
            self._held.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- coherence measure

def rr_coherence_capsule(o_tmin, d_tmax, hits, E: float, subset: int = 64, areas_out=None,
                         n: int | None = None, stream=None):
    """Capsule area of every run of `subset` consecutive rays (Section 4.3)."""
    n = o_tmin.shape[0] if n is None else n
    groups = 1 if n < subset else n // subset
    if areas_out is None:
        areas_out = torch.empty(groups, dtype=torch.float32, device=o_tmin.device)
    _check(lib().rr_coherence_capsule(_ptr(o_tmin), _ptr(d_tmax), _ptr(hits), n, subset,
                                      float(np.float32(E)), _ptr(areas_out), _stream(stream)),
           "rr_coherence_capsule")
    return areas_out


# ---------------------------------------------------------------- diagnostics

def rr_selftest_lookback_timeout(stream=None):
    """Runs the look-back wait out on purpose (bounded); see include/rr.h."""
    _check(lib().rr_selftest_lookback_timeout(_stream(stream)), "rr_selftest_lookback_timeout")


def rr_device_error() -> int:
    v = C.c_uint32()
    _check(lib().rr_device_error(C.byref(v)), "rr_device_error")
    return int(v.value)


def rr_stream_error(flags_out, stream=None):
    """Enqueues on `stream` the read-and-clear of its error word into flags_out
    (a CUDA int32 tensor of one element, or a pinned CPU one); read it after
    the stream has synchronised."""
    if flags_out.dtype != torch.int32 or flags_out.numel() < 1:
        raise ValueError("flags_out must hold one int32")
    _check(lib().rr_stream_error(_stream(stream), flags_out.data_ptr()), "rr_stream_error")


def rr_fault_inject(spec: str | None):
    """Host-side fault injection: "alloc@N", "launch@N", "timeout@N", or None
    to clear (see include/rr.h)."""
    _check(lib().rr_fault_inject(spec.encode() if spec else None), "rr_fault_inject")


def rr_bvh_aabb(bvh: "BVH"):
    lo, hi = (C.c_float * 3)(), (C.c_float * 3)()
    _check(lib().rr_bvh_aabb(bvh.handle, lo, hi), "rr_bvh_aabb")
    return np.array(lo[:], np.float32), np.array(hi[:], np.float32)


def rr_kernel_launch_count() -> int:
    return int(lib().rr_kernel_launch_count())


def rr_status_string(s: int) -> str:
    return lib().rr_status_string(s).decode()


# ---------------------------------------------------------------- helpers for callers

def to_device_rays(rays, device="cuda"):
    """numpy Rays -> (o_tmin, d_tmax, payload) CUDA tensors (payload as int32 bits)."""
    o = torch.from_numpy(np.ascontiguousarray(rays.o_tmin)).to(device)
    d = torch.from_numpy(np.ascontiguousarray(rays.d_tmax)).to(device)
    p = torch.from_numpy(np.ascontiguousarray(rays.payload).view(np.int32)).to(device)
    return o, d, p


def key_dtype(bits: int):
    return torch.int64 if bits > 32 else torch.int32


def keys_to_numpy(t: torch.Tensor) -> np.ndarray:
    a = t.cpu().numpy()
    return a.view(np.uint64) if a.dtype == np.int64 else a.view(np.uint32).astype(np.uint64)


def u32_to_numpy(t: torch.Tensor) -> np.ndarray:
    return t.cpu().numpy().view(np.uint32)
