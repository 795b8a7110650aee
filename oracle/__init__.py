"""CPU oracle for IG raycasting -- TEST INFRASTRUCTURE, NOT PRODUCT CODE.

Thin ctypes wrapper over ``nbt_oracle.c`` (built by :func:`oracle.build.build`).
Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's CPU
baseline use this package; the CUDA library never imports it, and it never
imports the library.  See ``nbt_oracle.c`` for what each function computes
and which passage of the paper it follows.
"""

from __future__ import annotations

import contextlib
import ctypes as C
import os

import numpy as np

from .build import LIB_PATH, build

METRICS = {"count": 0, "eq2": 1, "entropy": 2}
REDUCE = {"sum": 0, "mean": 1}
GRID = {"corners": 0, "centers": 1}
RANGE = {"planar": 0, "spherical": 1}
WALKS = {"f32": 0, "f64": 1, "brute": 2}
ENC = {"u8": 0, "u2": 0, "f32": 1}


class OrcMap(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("encoding", C.c_int32),
                ("voxel_size", C.c_float), ("origin", C.c_float * 3), ("data", C.c_void_p)]


class OrcCamera(C.Structure):
    _fields_ = [("width", C.c_int32), ("height", C.c_int32), ("fov_h", C.c_float), ("fov_v", C.c_float),
                ("max_range", C.c_float), ("grid_mode", C.c_int32), ("range_mode", C.c_int32)]


class OrcParams(C.Structure):
    _fields_ = [("metric", C.c_int32), ("occ_threshold", C.c_float), ("free_threshold", C.c_float),
                ("include_hit", C.c_int32), ("reduce", C.c_int32)]


class OrcCamConsts(C.Structure):
    _fields_ = [("x0", C.c_float), ("xstep", C.c_float), ("y0", C.c_float), ("ystep", C.c_float),
                ("zc", C.c_float), ("spherical", C.c_int32)]


_lib = None


def lib():
    """Load (building first if needed) the oracle shared library."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            build()
        _lib = _bind(C.CDLL(LIB_PATH))
    return _lib


@contextlib.contextmanager
def using_library(path: str):
    """Run the wrappers against another build of ``nbt_oracle.c`` (the tests' planted-mistake builds)."""
    global _lib
    saved = _lib
    _lib = _bind(C.CDLL(path))
    try:
        yield
    finally:
        _lib = saved


def _bind(L):
    """Argument and result types of the oracle's entry points."""
    P = C.POINTER
    f32p, f64p, i64p, i32p = P(C.c_float), P(C.c_double), P(C.c_int64), P(C.c_int32)
    L.orc_camera_consts.argtypes = [P(OrcCamera), P(OrcCamConsts)]
    L.orc_view_rays.argtypes = [P(OrcMap), P(OrcCamera), f32p, f32p, f32p]
    L.orc_trace.argtypes = [i32p, f32p, f32p, C.c_int, i64p, C.c_int64]
    L.orc_trace.restype = C.c_int64
    L.orc_trace_occluded.argtypes = [P(OrcMap), f32p, f32p, P(OrcParams), C.c_int, i64p, C.c_int64]
    L.orc_trace_occluded.restype = C.c_int64
    L.orc_segments_ig.argtypes = [P(OrcMap), f32p, f32p, C.c_int64, P(OrcParams), C.c_int, f64p, i64p]
    L.orc_views_ig.argtypes = [P(OrcMap), f32p, C.c_int64, P(OrcCamera), P(OrcParams), C.c_int, C.c_int,
                               f64p, i64p]
    L.orc_views_ig.restype = C.c_int
    L.orc_traj_ig.argtypes = [P(OrcMap), f32p, i32p, C.c_int32, P(OrcCamera), P(OrcParams), C.c_int, C.c_int,
                              f64p, i64p]
    L.orc_traj_ig.restype = C.c_int
    L.orc_min_tie_gap.argtypes = [i32p, f32p, f32p]
    L.orc_min_tie_gap.restype = C.c_double
    L.orc_entropy.argtypes = [C.c_double]
    L.orc_entropy.restype = C.c_double
    L.orc_voxel_gain.argtypes = [P(OrcMap), C.c_int64, P(OrcParams), f64p, P(C.c_int)]
    return L


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(C.POINTER(ctype))


class Map:
    """A dense grid (nz, ny, nx) plus geometry; keeps the array alive."""

    def __init__(self, grid: np.ndarray, voxel_size: float = 0.01, origin=(0.0, 0.0, 0.0)):
        if grid.dtype == np.uint8:
            enc = 0
        elif grid.dtype == np.float32:
            enc = 1
        else:
            raise TypeError("oracle maps are uint8 states or float32 probabilities")
        self.grid = np.ascontiguousarray(grid)
        nz, ny, nx = self.grid.shape
        self.s = OrcMap(nx, ny, nz, enc, float(voxel_size), (C.c_float * 3)(*origin),
                        self.grid.ctypes.data_as(C.c_void_p))

    @property
    def dims(self) -> np.ndarray:
        return np.array([self.s.nx, self.s.ny, self.s.nz], dtype=np.int32)


def camera(width: int, height: int, fov_h: float, fov_v: float, max_range: float,
           grid_mode: str = "corners", range_mode: str = "planar") -> OrcCamera:
    return OrcCamera(int(width), int(height), float(fov_h), float(fov_v), float(max_range), GRID[grid_mode],
                     RANGE[range_mode])


def camera_of(cam) -> OrcCamera:
    """Oracle camera from a ``workload.configs.Camera``."""
    return camera(cam.width, cam.height, cam.fov_h, cam.fov_v, cam.max_range, cam.grid_mode, cam.range_mode)


def params(metric: str = "count", occ_threshold: float = 0.7, free_threshold: float = 0.3,
           include_hit: bool = True, reduce: str = "sum") -> OrcParams:
    return OrcParams(METRICS[metric], float(occ_threshold), float(free_threshold), int(bool(include_hit)),
                     REDUCE[reduce])


def camera_consts(cam: OrcCamera) -> OrcCamConsts:
    cc = OrcCamConsts()
    lib().orc_camera_consts(C.byref(cam), C.byref(cc))
    return cc


def view_rays(m: Map, cam: OrcCamera, pose: np.ndarray):
    """FP32 segments (o, d) of every ray of one perspective, ray k = j*W + i."""
    n = cam.width * cam.height
    o = np.zeros((n, 3), np.float32)
    d = np.zeros((n, 3), np.float32)
    p = np.ascontiguousarray(pose, dtype=np.float32)
    lib().orc_view_rays(C.byref(m.s), C.byref(cam), _ptr(p, C.c_float), _ptr(o, C.c_float), _ptr(d, C.c_float))
    return o, d


def trace(dims, o, d, walk: str = "f32", cap: int | None = None) -> np.ndarray:
    """Linear voxel indices of the whole segment (no occlusion)."""
    dims = np.ascontiguousarray(dims, dtype=np.int32)
    o = np.ascontiguousarray(o, dtype=np.float32)
    d = np.ascontiguousarray(d, dtype=np.float32)
    cap = int(dims.sum()) + 3 if cap is None else cap
    out = np.zeros(cap, np.int64)
    n = lib().orc_trace(_ptr(dims, C.c_int32), _ptr(o, C.c_float), _ptr(d, C.c_float), WALKS[walk],
                        _ptr(out, C.c_int64), cap)
    return out[:min(n, cap)].copy()


def trace_occluded(m: Map, o, d, prm: OrcParams, walk: str = "f32") -> np.ndarray:
    """Linear voxel indices up to and including the first occupied voxel."""
    o = np.ascontiguousarray(o, dtype=np.float32)
    d = np.ascontiguousarray(d, dtype=np.float32)
    cap = int(m.dims.sum()) + 3
    out = np.zeros(cap, np.int64)
    n = lib().orc_trace_occluded(C.byref(m.s), _ptr(o, C.c_float), _ptr(d, C.c_float), C.byref(prm), WALKS[walk],
                                 _ptr(out, C.c_int64), cap)
    return out[:min(n, cap)].copy()


def segments_ig(m: Map, o: np.ndarray, d: np.ndarray, prm: OrcParams, walk: str = "f32"):
    """Per-segment IG (FP64) and voxel steps."""
    o = np.ascontiguousarray(o, dtype=np.float32).reshape(-1, 3)
    d = np.ascontiguousarray(d, dtype=np.float32).reshape(-1, 3)
    n = len(o)
    ig = np.zeros(n, np.float64)
    st = np.zeros(n, np.int64)
    lib().orc_segments_ig(C.byref(m.s), _ptr(o, C.c_float), _ptr(d, C.c_float), n, C.byref(prm), WALKS[walk],
                          _ptr(ig, C.c_double), _ptr(st, C.c_int64))
    return ig, st


def views_ig(m: Map, poses: np.ndarray, cam: OrcCamera, prm: OrcParams, walk: str = "f32", threads: int = 1):
    """Per-perspective IG (FP64; sum or mean over rays) and voxel steps."""
    poses = np.ascontiguousarray(poses, dtype=np.float32).reshape(-1, 7)
    n = len(poses)
    ig = np.zeros(n, np.float64)
    st = np.zeros(n, np.int64)
    if n:
        rc = lib().orc_views_ig(C.byref(m.s), _ptr(poses, C.c_float), n, C.byref(cam), C.byref(prm), WALKS[walk],
                                int(threads), _ptr(ig, C.c_double), _ptr(st, C.c_int64))
        if rc != 0:
            raise RuntimeError("oracle views_ig failed")
    return ig, st


def traj_ig(m: Map, poses: np.ndarray, offsets: np.ndarray, cam: OrcCamera, prm: OrcParams, walk: str = "f32",
            threads: int = 1):
    """Per-trajectory IG (sum of perspective IGs over the CSR ranges) and steps."""
    poses = np.ascontiguousarray(poses, dtype=np.float32).reshape(-1, 7)
    offsets = np.ascontiguousarray(offsets, dtype=np.int32)
    nt = len(offsets) - 1
    ig = np.zeros(max(nt, 0), np.float64)
    st = np.zeros(max(nt, 0), np.int64)
    if nt > 0:
        rc = lib().orc_traj_ig(C.byref(m.s), _ptr(poses, C.c_float), _ptr(offsets, C.c_int32), nt, C.byref(cam),
                               C.byref(prm), WALKS[walk], int(threads), _ptr(ig, C.c_double), _ptr(st, C.c_int64))
        if rc != 0:
            raise RuntimeError("oracle traj_ig failed")
    return ig, st


def min_tie_gap(dims, o, d) -> float:
    dims = np.ascontiguousarray(dims, dtype=np.int32)
    o = np.ascontiguousarray(o, dtype=np.float32)
    d = np.ascontiguousarray(d, dtype=np.float32)
    return float(lib().orc_min_tie_gap(_ptr(dims, C.c_int32), _ptr(o, C.c_float), _ptr(d, C.c_float)))


def entropy(p: float) -> float:
    return float(lib().orc_entropy(float(p)))


def voxel_gain(m: Map, idx: int, prm: OrcParams):
    g = C.c_double()
    occ = C.c_int()
    lib().orc_voxel_gain(C.byref(m.s), int(idx), C.byref(prm), C.byref(g), C.byref(occ))
    return g.value, bool(occ.value)
