"""ctypes declarations of the C ABI in include/nbt.h (argument marshalling only)."""

from __future__ import annotations

import ctypes as C
import os

from .build import LIB_PATH

NBT_OK = 0
STATUS = {0: "NBT_OK", -1: "NBT_EINVAL", -2: "NBT_ENOMEM", -3: "NBT_ECUDA", -4: "NBT_ETIMEOUT",
          -5: "NBT_EUNSUPPORTED", -6: "NBT_EWORKSPACE", -7: "NBT_ESCRATCH"}
ENCODINGS = {"u8": 0, "f32": 1, "u2": 2}
METRICS = {"count": 0, "eq2": 1, "entropy": 2}
REDUCE = {"sum": 0, "mean": 1}
GRID = {"corners": 0, "centers": 1}
RANGE = {"planar": 0, "spherical": 1}


class NbtError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)}")


class LibraryMissing(ImportError):
    pass


class MapDesc(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("voxel_size", C.c_float),
                ("origin", C.c_float * 3), ("encoding", C.c_int32), ("brick", C.c_int32)]


class Camera(C.Structure):
    _fields_ = [("width", C.c_int32), ("height", C.c_int32), ("fov_h", C.c_float), ("fov_v", C.c_float),
                ("max_range", C.c_float), ("grid_mode", C.c_int32), ("range_mode", C.c_int32)]


class Tuning(C.Structure):
    _fields_ = [("packet_w", C.c_int32), ("brick", C.c_int32), ("skip", C.c_int32)]


class IgParams(C.Structure):
    _fields_ = [("metric", C.c_int32), ("occ_threshold", C.c_float), ("free_threshold", C.c_float),
                ("include_hit", C.c_int32), ("reduce", C.c_int32)]


class InsertParams(C.Structure):
    _fields_ = [("prob_hit", C.c_float), ("prob_miss", C.c_float), ("clamp_min", C.c_float), ("clamp_max", C.c_float),
                ("max_range", C.c_float)]


class CostParams(C.Structure):
    _fields_ = [("power", C.c_float), ("w_info", C.c_float), ("eps", C.c_float)]


# Every symbol include/nbt.h declares, with (restype, argtypes).
_vp, _i32, _i64, _f = C.c_void_p, C.c_int32, C.c_int64, C.c_float
P = C.POINTER
SIGNATURES = {
    "nbt_status_string": (C.c_char_p, [C.c_int]),
    "nbt_get_version": (C.c_int, [P(C.c_int32)]),
    "nbt_map_create": (C.c_int, [P(MapDesc), P(_vp)]),
    "nbt_map_destroy": (C.c_int, [_vp]),
    "nbt_map_upload": (C.c_int, [_vp, _vp, _i64, _i32, _vp]),
    "nbt_map_info": (C.c_int, [_vp, P(MapDesc), P(C.c_int64)]),
    "nbt_map_download": (C.c_int, [_vp, _vp, _i64, _vp]),
    "nbt_map_insert_points": (C.c_int, [_vp, _vp, _i64, P(_f), P(InsertParams), _vp, _vp]),
    "nbt_workspace_size": (C.c_int, [_i64, P(Camera), P(C.c_int64)]),
    "nbt_camera_from_grid_scale": (C.c_int, [_f, _f, _f, _f, _f, P(Camera)]),
    "nbt_views_ig": (C.c_int, [_vp, _vp, _i64, P(Camera), P(IgParams), _vp, _vp, _vp, _i64, _vp]),
    "nbt_traj_ig": (C.c_int, [_vp, _vp, _i64, _vp, _i32, P(Camera), P(IgParams), _vp, _vp, _vp, _i64, _vp]),
    "nbt_trace_segments": (C.c_int, [_vp, _vp, _vp, _i32, P(IgParams), _vp, _i32, _vp, _vp]),
    "nbt_view_segments": (C.c_int, [_vp, _vp, _i64, P(Camera), _vp, _vp, _vp]),
    "nbt_views_ig_noalloc": (C.c_int, [_vp, _vp, _i64, P(Camera), P(IgParams), _vp, _vp, _vp]),
    "nbt_map_set_tuning": (C.c_int, [_vp, P(Tuning)]),
    "nbt_plan_create_traj": (C.c_int, [_vp, _vp, _i64, _vp, _i32, P(Camera), P(IgParams), _vp, _vp, _vp, _i64,
                                       P(_vp)]),
    "nbt_plan_launch": (C.c_int, [_vp, _vp]),
    "nbt_plan_destroy": (C.c_int, [_vp]),
    "nbt_tc_gemm": (C.c_int, [_vp, _vp, _vp, _i32, _i32, _i32, _vp]),
    "nbt_tc_error": (C.c_int, [P(C.c_int32)]),
    "nbt_surrogate_param_count": (C.c_int, [P(C.c_int64)]),
    "nbt_segment_topk": (C.c_int, [_vp, _i64, _i32, _i32, _vp, _vp, _vp, _vp]),
    "nbt_segment_argmax": (C.c_int, [_vp, _vp, _i64, _i32, _vp, _vp, _vp]),
    "nbt_surrogate_create": (C.c_int, [_i32, P(_vp)]),
    "nbt_surrogate_destroy": (C.c_int, [_vp]),
    "nbt_surrogate_set_params": (C.c_int, [_vp, _vp, _i64]),
    "nbt_surrogate_get_params": (C.c_int, [_vp, _vp, _i64]),
    "nbt_surrogate_crops": (C.c_int, [_vp, _vp, _i64, P(Camera), P(IgParams), _vp, _vp, _vp]),
    "nbt_surrogate_forward": (C.c_int, [_vp, _vp, _vp, _i64, _vp, _vp]),
    "nbt_surrogate_backward": (C.c_int, [_vp, _vp, _vp, _vp, _i32, _vp, _vp, _vp]),
    "nbt_surrogate_train_step": (C.c_int, [_vp, _vp, _vp, _vp, _i32, C.c_float, _vp, _vp]),
    "nbt_surrogate_set_target_scale": (C.c_int, [_vp, _f]),
    "nbt_surrogate_get_adam": (C.c_int, [_vp, _vp, _vp, _i64, P(C.c_int64)]),
    "nbt_surrogate_set_adam": (C.c_int, [_vp, _vp, _vp, _i64, _i64]),
    "nbt_tc_set_wait_limit": (C.c_int, [C.c_uint64]),
    "nbt_tc_wait_probe": (C.c_int, [_vp]),
    "nbt_pruned_workspace_size": (C.c_int, [_vp, _i64, _i32, _i32, P(Camera), P(C.c_int64)]),
    "nbt_plan_pruned": (C.c_int, [_vp, _vp, _vp, _i64, _i32, _i32, P(Camera), P(IgParams), _vp, _vp, _vp, _vp, _i64,
                                  _vp]),
    "nbt_map_get_tuning": (C.c_int, [_vp, P(Tuning)]),
    "nbt_id_buffer_create": (C.c_int, [_i32, _i32, P(_vp)]),
    "nbt_id_buffer_destroy": (C.c_int, [_vp]),
    "nbt_id_buffer_push": (C.c_int, [_vp, _vp, _vp, _i32, _vp]),
    "nbt_id_buffer_clear": (C.c_int, [_vp]),
    "nbt_id_buffer_count": (C.c_int, [_vp, P(C.c_int32)]),
    "nbt_idw_gain": (C.c_int, [_vp, _vp, _i64, _f, _vp, _vp]),
    "nbt_ig_cost": (C.c_int, [_vp, _vp, _i64, _vp, _i32, P(_f), _f, _f, P(CostParams), _vp, _vp, _vp, _vp, _vp]),
}

_lib = None


def lib():
    """The loaded libnbt.so; raises LibraryMissing if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise LibraryMissing(f"{LIB_PATH} is missing: build it with paper_2503_22588_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def check(status: int, where: str) -> None:
    if status != NBT_OK:
        raise NbtError(status, where)
