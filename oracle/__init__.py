"""Python view of the CPU oracle (``oracle.c``).

TEST INFRASTRUCTURE: only the test suite, ``__graft_entry__.smoke()`` and the
bench's CPU-baseline leg import this package.  The product path never does.

The C library is compiled on first use (``gcc -O2 -std=c11 -ffp-contract=off``)
next to its source; ``build()`` compiles it explicitly.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

AILA, AILA_COMPACT, TWO_POINT, ORIGIN, REIS, COSTA, OCTAHEDRON = 0, 1, 2, 3, 4, 5, 6
T_FIXED, T_ADAPTIVE, T_GIVEN = 0, 1, 2
MISS = 0xFFFFFFFF
TABLE_CELLS = 1 << 20

_f32p = np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
_u32p = np.ctypeslib.ndpointer(np.uint32, flags="C_CONTIGUOUS")
_u64p = np.ctypeslib.ndpointer(np.uint64, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile liboracle.so if it is missing or older than oracle.c."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            L.or_quantise_unit.restype = C.c_uint32
            L.or_quantise_unit.argtypes = [C.c_float]
            L.or_largest_extent.restype = C.c_float
            L.or_largest_extent.argtypes = [_f32p, _f32p]
            L.or_quantise_point.argtypes = [_f32p, _f32p, _f32p, _u32p]
            L.or_quantise_direction.argtypes = [_f32p, _u32p]
            L.or_interleave.restype = C.c_uint64
            L.or_interleave.argtypes = [C.c_int, _u32p, C.c_uint32]
            L.or_table_cell.restype = C.c_uint32
            L.or_table_cell.argtypes = [_f32p, _f32p, _f32p, _f32p]
            L.or_table_init.argtypes = [_u64p, _u32p]
            L.or_fixed_length.restype = C.c_uint32
            L.or_fixed_length.argtypes = [C.c_float, _f32p, C.c_float]
            L.or_table_accumulate.argtypes = [_u64p, _u32p, _f32p, _f32p, C.c_float, _f32p,
                                              _f32p, _f32p, C.c_uint32]
            L.or_table_estimate.restype = C.c_float
            L.or_table_estimate.argtypes = [_u64p, _u32p, C.c_uint32, C.c_float]
            L.or_key.restype = C.c_uint64
            L.or_key.argtypes = [C.c_int, C.c_uint32, _f32p, _f32p, C.c_float, _f32p, _f32p]
            L.or_compute_keys.argtypes = [C.c_int, C.c_uint32, C.c_int, C.c_float, _f32p, _f32p,
                                          C.c_void_p, C.c_void_p, C.c_void_p, C.c_float, _f32p,
                                          _f32p, C.c_uint32, _u64p]
            L.or_morton3_prefix.restype = C.c_uint64
            L.or_morton3_prefix.argtypes = [C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32]
            L.or_octahedral.argtypes = [_f32p, C.POINTER(C.c_float), C.POINTER(C.c_float)]
            L.or_interleave_od.restype = C.c_uint64
            L.or_interleave_od.argtypes = [C.c_int, _u32p, C.c_uint32]
            L.or_key_od.restype = C.c_uint64
            L.or_key_od.argtypes = [C.c_int, C.c_uint32, _f32p, _f32p, _f32p, _f32p]
            L.or_capsule_areas.restype = C.c_uint32
            L.or_capsule_areas.argtypes = [_f32p, _f32p, _f32p, C.c_uint32, C.c_uint32, C.c_float, _f64p]
            L.or_stable_sort.restype = C.c_int
            L.or_stable_sort.argtypes = [_u64p, C.c_uint32, _u32p, _u64p]
            L.or_segment_sort.restype = C.c_int
            L.or_segment_sort.argtypes = [_u64p, C.c_uint32, C.c_uint32, _u32p]
            L.or_permute.argtypes = [_f32p, _f32p, _u32p, _u32p, C.c_uint32, _f32p, _f32p, _u32p]
            L.or_ray_triangle.restype = C.c_int
            L.or_ray_triangle.argtypes = [_f64p, _f64p, _f32p, C.POINTER(C.c_double),
                                          C.POINTER(C.c_double), C.POINTER(C.c_double)]
            L.or_ray_triangle_uv.restype = C.c_int
            L.or_ray_triangle_uv.argtypes = [_f64p, _f64p, _f32p, C.POINTER(C.c_double),
                                             C.POINTER(C.c_double), C.POINTER(C.c_double)]
            L.or_trace_brute.argtypes = [_f32p, C.c_uint32, _f32p, _f32p, C.c_uint32, _f32p,
                                         C.c_void_p]
            L.or_bvh_build.restype = C.c_void_p
            L.or_bvh_build.argtypes = [_f32p, C.c_uint32]
            L.or_bvh_free.argtypes = [C.c_void_p]
            L.or_trace_bvh.argtypes = [C.c_void_p, _f32p, _f32p, C.c_uint32, _f32p, C.c_void_p]
            L.or_bvh_depth.restype = C.c_uint32
            L.or_bvh_depth.argtypes = [C.c_void_p]
            _lib = L
    return _lib


def _f32(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float32)
    if shape is not None:
        a = a.reshape(shape)
    return a


# ---------------------------------------------------------------- quantisation

def quantise_unit(x) -> int:
    return int(lib().or_quantise_unit(float(np.float32(x))))


def largest_extent(lo, hi) -> np.float32:
    return np.float32(lib().or_largest_extent(_f32(lo, 3), _f32(hi, 3)))


def quantise_point(p, lo, hi) -> np.ndarray:
    q = np.zeros(3, np.uint32)
    lib().or_quantise_point(_f32(p, 3), _f32(lo, 3), _f32(hi, 3), q)
    return q


def quantise_direction(d) -> np.ndarray:
    q = np.zeros(3, np.uint32)
    lib().or_quantise_direction(_f32(d, 3), q)
    return q


def interleave(layout: int, comp, bits: int) -> int:
    return int(lib().or_interleave(layout, np.ascontiguousarray(comp, dtype=np.uint32), bits))


def key(layout: int, bits: int, o, d, t_est, lo, hi) -> int:
    return int(lib().or_key(layout, bits, _f32(o, 3), _f32(d, 3), float(np.float32(t_est)),
                            _f32(lo, 3), _f32(hi, 3)))


def morton3_prefix(c0, c1, c2, bits) -> int:
    return int(lib().or_morton3_prefix(int(c0), int(c1), int(c2), bits))


def octahedral(d):
    u, v = C.c_float(), C.c_float()
    lib().or_octahedral(_f32(d, 3), C.byref(u), C.byref(v))
    return np.float32(u.value), np.float32(v.value)


def interleave_od(layout: int, comp, bits: int) -> int:
    c = np.zeros(6, np.uint32)
    c[:len(comp)] = comp
    return int(lib().or_interleave_od(layout, c, bits))


def key_od(layout: int, bits: int, o, d, lo, hi) -> int:
    return int(lib().or_key_od(layout, bits, _f32(o, 3), _f32(d, 3), _f32(lo, 3), _f32(hi, 3)))


# ---------------------------------------------------------------- length table

class LengthTable:
    """2^20 cells of (u64 fixed-point length sum, u32 count); starts with one
    dummy ray of length 0.25*E per cell (Section 3.1.6)."""

    def __init__(self, E: float):
        self.E = np.float32(E)
        self.sum = np.zeros(TABLE_CELLS, np.uint64)
        self.cnt = np.zeros(TABLE_CELLS, np.uint32)
        lib().or_table_init(self.sum, self.cnt)

    def accumulate(self, lo, hi, o_tmin, d_tmax, hits):
        n = o_tmin.shape[0]
        lib().or_table_accumulate(self.sum, self.cnt, _f32(lo, 3), _f32(hi, 3), float(self.E),
                                  _f32(o_tmin), _f32(d_tmax), _f32(hits), n)

    def estimate(self, cell: int) -> np.float32:
        return np.float32(lib().or_table_estimate(self.sum, self.cnt, cell, float(self.E)))


def table_cell(o, d, lo, hi) -> int:
    return int(lib().or_table_cell(_f32(o, 3), _f32(d, 3), _f32(lo, 3), _f32(hi, 3)))


def fixed_length(t, d, E) -> int:
    return int(lib().or_fixed_length(float(np.float32(t)), _f32(d, 3), float(np.float32(E))))


# ---------------------------------------------------------------- keys

def compute_keys(layout: int, bits: int, o_tmin, d_tmax, lo, hi, tsrc: int = T_FIXED,
                 ratio: float = 0.25, t_given=None, table: LengthTable | None = None) -> np.ndarray:
    o_tmin = _f32(o_tmin)
    d_tmax = _f32(d_tmax)
    n = o_tmin.shape[0]
    keys = np.zeros(n, np.uint64)
    tg = None
    if t_given is not None:
        tg = _f32(t_given)
    ts = table.sum if table is not None else None
    tc = table.cnt if table is not None else None
    lib().or_compute_keys(layout, bits, tsrc, float(np.float32(ratio)), _f32(lo, 3), _f32(hi, 3),
                          None if tg is None else tg.ctypes.data,
                          None if ts is None else ts.ctypes.data,
                          None if tc is None else tc.ctypes.data,
                          float(table.E) if table is not None else 0.0,
                          o_tmin, d_tmax, n, keys)
    return keys


# ---------------------------------------------------------------- sort and reorder

def stable_sort(keys):
    keys = np.ascontiguousarray(keys, dtype=np.uint64)
    n = keys.shape[0]
    perm = np.zeros(n, np.uint32)
    sk = np.zeros(n, np.uint64)
    if lib().or_stable_sort(keys, n, perm, sk) != 0:
        raise MemoryError("oracle sort")
    return perm, sk


def segment_sort(keys, segment: int):
    """Stable sort inside each run of `segment` consecutive keys (Section 3.2)."""
    keys = np.ascontiguousarray(keys, dtype=np.uint64)
    perm = np.zeros(keys.shape[0], np.uint32)
    if lib().or_segment_sort(keys, keys.shape[0], segment, perm) != 0:
        raise ValueError("oracle segment sort")
    return perm


def permute(o_tmin, d_tmax, payload, perm):
    n = perm.shape[0]
    o = np.zeros((n, 4), np.float32)
    d = np.zeros((n, 4), np.float32)
    p = np.zeros(n, np.uint32)
    lib().or_permute(_f32(o_tmin), _f32(d_tmax), np.ascontiguousarray(payload, np.uint32),
                     np.ascontiguousarray(perm, np.uint32), n, o, d, p)
    return o, d, p


# ---------------------------------------------------------------- trace

def ray_triangle(o, d, tri):
    t, u, v = C.c_double(), C.c_double(), C.c_double()
    ok = lib().or_ray_triangle(np.ascontiguousarray(o, np.float64), np.ascontiguousarray(d, np.float64),
                               _f32(tri, 9), C.byref(t), C.byref(u), C.byref(v))
    return (bool(ok), t.value, u.value, v.value)


def ray_plane_barycentrics(o, d, tri):
    """(ok, t, u, v) of the ray's meeting point with the triangle's plane (no inside test)."""
    t, u, v = C.c_double(), C.c_double(), C.c_double()
    ok = lib().or_ray_triangle_uv(np.ascontiguousarray(o, np.float64),
                                  np.ascontiguousarray(d, np.float64), _f32(tri, 9), C.byref(t),
                                  C.byref(u), C.byref(v))
    return (bool(ok), t.value, u.value, v.value)


def trace_brute(tris, o_tmin, d_tmax):
    """hits [N,4] float32 (t,u,v,tri bits) and info [N,2] float64 (t, barycentric margin)."""
    tris = _f32(tris).reshape(-1, 9)
    o_tmin = _f32(o_tmin).reshape(-1, 4)
    d_tmax = _f32(d_tmax).reshape(-1, 4)
    n = o_tmin.shape[0]
    hits = np.zeros((n, 4), np.float32)
    info = np.zeros((n, 2), np.float64)
    lib().or_trace_brute(tris, tris.shape[0], o_tmin, _f32(d_tmax), n, hits, info.ctypes.data)
    return hits, info


class BVH:
    """Oracle-owned binary BVH; its answers equal ``trace_brute`` (pinned in the tests)."""

    def __init__(self, tris):
        self.tris = _f32(tris).reshape(-1, 9)
        self.h = lib().or_bvh_build(self.tris, self.tris.shape[0])
        if not self.h:
            raise MemoryError("oracle bvh")

    def depth(self) -> int:
        return int(lib().or_bvh_depth(self.h))

    def trace(self, o_tmin, d_tmax):
        o_tmin = _f32(o_tmin).reshape(-1, 4)
        d_tmax = _f32(d_tmax).reshape(-1, 4)
        n = o_tmin.shape[0]
        hits = np.zeros((n, 4), np.float32)
        info = np.zeros((n, 2), np.float64)
        lib().or_trace_bvh(self.h, o_tmin, _f32(d_tmax), n, hits, info.ctypes.data)
        return hits, info

    def __del__(self):
        if getattr(self, "h", None):
            lib().or_bvh_free(self.h)
            self.h = None


def capsule_areas(o_tmin, d_tmax, hits, E, subset: int = 64) -> np.ndarray:
    """Capsule surface area of each consecutive subset of rays (Section 4.3)."""
    o_tmin = _f32(o_tmin).reshape(-1, 4)
    n = o_tmin.shape[0]
    out = np.zeros(max(1, n // max(subset, 1) + 1), np.float64)
    k = lib().or_capsule_areas(o_tmin, _f32(d_tmax).reshape(-1, 4), _f32(hits).reshape(-1, 4), n, subset,
                               float(np.float32(E)), out)
    return out[:k]


def hit_tri(hits) -> np.ndarray:
    return np.ascontiguousarray(hits[:, 3]).view(np.uint32)
