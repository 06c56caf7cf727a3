"""ctypes declarations of the C ABI in ``include/sbr.h`` (argument marshalling only).

The shared library is built in-tree (``build.py``).  There is no fallback: if the
library is missing or fails to load, importing this module raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

MAX_ORDER = 8

_c = ctypes
_vp = _c.c_void_p
_i32 = _c.c_int32
_i64 = _c.c_int64
_f32 = _c.c_float
_f64 = _c.c_double
_pf = _c.POINTER(_c.c_float)
_pd = _c.POINTER(_c.c_double)
_pi32 = _c.POINTER(_c.c_int32)
_pi64 = _c.POINTER(_c.c_int64)

ALLOC_FN = _c.CFUNCTYPE(_vp, _c.c_size_t, _vp, _vp)
FREE_FN = _c.CFUNCTYPE(None, _vp, _c.c_size_t, _vp, _vp)


class SceneInfo(_c.Structure):
    _fields_ = [("num_triangles", _i64), ("num_faces", _i32), ("bvh_nodes", _i32), ("bvh_depth", _i32),
                ("max_leaf", _i32), ("device_bytes", _i64), ("bbox_lo", _f32 * 3), ("bbox_hi", _f32 * 3),
                ("num_wedges", _i32)]


class LaunchParams(_c.Structure):
    _fields_ = [("n_div", _i32), ("max_order", _i32), ("rx_angle_scale", _f32), ("flags", _i32),
                ("dump_stride", _i32), ("dump_faces", _vp), ("dump_cap", _i64), ("grid_blocks", _i32),
                ("block_threads", _i32), ("refill_min", _i32), ("launcher", _i32), ("ray_begin", _i64),
                ("ray_end", _i64)]


class LaunchStats(_c.Structure):
    _fields_ = [("rays", _i64), ("segments", _i64), ("node_visits", _i64), ("tri_tests", _i64), ("rx_tests", _i64),
                ("records", _i64), ("paths", _i64), ("collisions", _i64), ("ntx", _i32), ("nrx", _i32),
                ("n_div", _i32), ("max_order", _i32), ("ms_raygen", _f32), ("ms_trace", _f32), ("ms_dedup", _f32),
                ("trace_grid", _i32), ("trace_block", _i32), ("ms_diffract", _f32), ("wedge_tests", _i64),
                ("diffraction_records", _i64), ("diffraction_candidates", _i64), ("candidate_cap", _i64),
                ("check_flags", _i64)]


class RefineParams(_c.Structure):
    _fields_ = [("max_iters", _i32), ("subrays", _i32), ("target_err_rad", _f64), ("fp64_below_rad", _f64),
                ("freq_hz", _f64), ("ptx_dbm", _f64), ("choice_log", _vp)]


class BatchConfig(_c.Structure):
    _fields_ = [("block_threads", _i32), ("blocks_per_sm", _i32), ("lanes_per_path", _i32)]


LAUNCH_SYNC = 1
LAUNCH_TIMING = 2
LAUNCH_DIFFRACTION = 4
LAUNCH_RAY_RANGE = 8
LAUNCH_RECORDS_ONLY = 16
LAUNCH_ID_ORDER = 32
PATH_REFINED, PATH_FP64, PATH_TRACE_FAIL, PATH_DIFFRACTED, PATH_STALLED = 1, 2, 4, 8, 16

PATH_DTYPE = np.dtype([("tx", "<i4"), ("rx", "<i4"), ("ray", "<i4"), ("order", "<i4"), ("faces", "<i4", (MAX_ORDER,)),
                       ("rough_err", "<f4"), ("rough_dray", "<f4"), ("iters", "<i4"), ("valid", "<i4"),
                       ("dir", "<f8", (3,)), ("err", "<f8"), ("delay", "<f8"), ("aod", "<f4", (2,)),
                       ("aoa", "<f4", (2,)), ("power_dbm", "<f4"), ("flags", "<i4")])
assert PATH_DTYPE.itemsize == 128

RECORD_DTYPE = np.dtype([("tx", "<i4"), ("rx", "<i4"), ("ray", "<i4"), ("order", "<i4"),
                         ("faces", "<i4", (MAX_ORDER,)), ("err", "<f4"), ("dray", "<f4"), ("slot", "<i4"),
                         ("pad", "<i4")])
assert RECORD_DTYPE.itemsize == 64

STATUS = {0: "SBR_OK", 1: "SBR_EINVAL", 2: "SBR_ENOMEM", 3: "SBR_ECUDA", 4: "SBR_ETIMEOUT", 5: "SBR_EOVERFLOW",
          6: "SBR_EDEGENERATE", 7: "SBR_ECOLLISION", 8: "SBR_ECHECK"}
CHECK_BITS = {1: "trace stack", 2: "occlusion stack", 4: "receiver stack", 8: "face id", 16: "binary-BVH stack"}

# name -> (restype, argtypes); every entry point of include/sbr.h
SIGNATURES = {
    "sbr_ctx_create": (_i32, [_c.c_int, _vp, ALLOC_FN, FREE_FN, _vp, _c.POINTER(_vp)]),
    "sbr_ctx_destroy": (_i32, [_vp]),
    "sbr_ctx_set_stream": (_i32, [_vp, _vp]),
    "sbr_last_error": (_c.c_char_p, [_vp]),
    "sbr_status_string": (_c.c_char_p, [_i32]),
    "sbr_abi_version": (_i32, []),
    "sbr_ctx_num_sms": (_i32, [_vp]),
    "sbr_num_rays": (_i64, [_i32]),
    "sbr_theta_launch": (_f64, [_i32]),
    "sbr_subray_pattern": (_i32, [_i32, _pd, _pd, _pd]),
    "sbr_raygen": (_i32, [_vp, _i32, _vp, _i64]),
    "sbr_raygen_equidistant": (_i32, [_vp, _i32, _i32, _vp, _i64]),
    "sbr_num_rays_launcher": (_i64, [_i32, _i32]),
    "sbr_scene_upload": (_i32, [_vp, _pf, _i64, _pi32, _pi32, _i64, _pf, _i32, _c.POINTER(_vp)]),
    "sbr_scene_destroy": (_i32, [_vp, _vp]),
    "sbr_face_outline_corners": (_i32, [_pf, _i64, _pi32, _pi32, _i64, _i32, _pi32]),
    "sbr_scene_get_info": (_i32, [_vp, _c.POINTER(SceneInfo)]),
    "sbr_scene_wedges": (_i32, [_vp, _vp, _vp, _i64, _c.POINTER(_i64)]),
    "sbr_rx_upload": (_i32, [_vp, _vp, _i32, _c.POINTER(_vp)]),
    "sbr_rx_destroy": (_i32, [_vp, _vp]),
    "sbr_paths_create": (_i32, [_vp, _i64, _i64, _c.POINTER(_vp)]),
    "sbr_paths_destroy": (_i32, [_vp, _vp]),
    "sbr_launch": (_i32, [_vp, _vp, _vp, _i32, _vp, _c.POINTER(LaunchParams), _vp]),
    "sbr_launch_get_stats": (_i32, [_vp, _vp, _c.POINTER(LaunchStats)]),
    "sbr_refine": (_i32, [_vp, _vp, _vp, _c.POINTER(RefineParams)]),
    "sbr_refine_pair": (_i32, [_vp, _vp, _vp, _i32, _i32, _c.POINTER(RefineParams)]),
    "sbr_batch_refine": (_i32, [_vp, _vp, _vp, _c.POINTER(RefineParams), _c.POINTER(BatchConfig)]),
    "sbr_paths_count": (_i32, [_vp, _vp, _pi64]),
    "sbr_query": (_i32, [_vp, _vp, _vp, _i64, _pi64]),
    "sbr_paths_import": (_i32, [_vp, _vp, _vp, _i64, _vp, _i32, _vp, _i32]),
    "sbr_unfold_fwd": (_i32, [_vp, _vp, _i64, _vp, _vp, _vp, _vp, _vp, _vp]),
    "sbr_unfold_bwd": (_i32, [_vp, _vp, _i64, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "sbr_dedup_noalloc": (_i32, [_vp, _vp, _vp, _i64, _vp]),
    "sbr_records_read": (_i32, [_vp, _vp, _vp, _i64, _pi64]),
    "sbr_records_dedup": (_i32, [_vp, _vp, _vp, _i64, _i32, _i32]),
    "sbr_paths_nonfinite": (_i32, [_vp, _vp, _pi64]),
}

_libs = {}


def library_path(checked: bool = False) -> str:
    return _build.SO_CHECKED if checked else _build.SO


def load(build_if_missing: bool = True, checked: bool = False):
    """Load libsbr.so, or with checked=True the bounds-checked variant libsbr_checked.so
    (building first if missing or stale and nvcc exists)."""
    if checked in _libs:
        return _libs[checked]
    path = library_path(checked)
    if build_if_missing:
        try:
            _build.build()
        except RuntimeError:
            if not os.path.exists(path):
                raise
    if not os.path.exists(path):
        raise ImportError(f"CUDA library not built: {path} (run __graft_entry__.build())")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _libs[checked] = lib
    return lib
