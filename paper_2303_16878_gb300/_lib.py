"""ctypes declarations of the C ABI in include/pba.h (argument marshalling only).

The library is paper_2303_16878_gb300/_build/libpba.so, built from csrc/ for
sm_103a.  Loading fails loudly when it is missing and cannot be built: there
is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

PBA_OK = 0
PBA_EINVAL = -1
PBA_ENOMEM = -2
PBA_ECUDA = -3
PBA_ENOTPD = -4
PBA_ENOTREADY = -6
PBA_ETOOBIG = -7
PBA_NOALLOC_MAX_PAIRS = 4096
PBA_NOALLOC_PAIR_STRIDE = 160

PBA_PINHOLE = 0
PBA_SPHERICAL = 1
PBA_PATH_BATCHED = 0
PBA_PATH_PLAIN = 1
PBA_TEXEL_F32 = 0
PBA_TEXEL_F16 = 1
PBA_SOLVE_CHOLESKY_F64 = 0
PBA_SOLVE_MIXED = 1
PBA_SOLVE_MIXED_STEPS = 2
PBA_SOLVE_SPARSE = 3

ERROR_NAMES = {PBA_EINVAL: "PBA_EINVAL", PBA_ENOMEM: "PBA_ENOMEM", PBA_ECUDA: "PBA_ECUDA",
               PBA_ENOTPD: "PBA_ENOTPD", PBA_ENOTREADY: "PBA_ENOTREADY",
               PBA_ETOOBIG: "PBA_ETOOBIG"}

# every exported symbol of include/pba.h
EXPORTS = ["pba_create", "pba_destroy", "pba_last_error", "pba_set_stream", "pba_upload_frames",
           "pba_frame_points", "pba_set_poses", "pba_get_poses", "pba_set_pairs", "pba_linearize",
           "pba_get_system", "pba_get_pair_system", "pba_set_mask_export", "pba_get_mask", "pba_solve_step",
           "pba_set_lambda", "pba_iterate", "pba_iterate_frames", "pba_iterate_async", "pba_get_stats",
           "pba_iteration_launches",
           "pba_iterate_timed", "pba_linearize_pairs_noalloc", "pba_autotune", "pba_get_tuning", "pba_build_pairs",
           "pba_set_extrinsic", "pba_cost_gradient", "pba_tangent_gradient", "pba_estimate_normals", "pba_get_channels",
           "pba_build_pyramid", "pba_pyramid_level", "pba_optimize", "pba_set_variables",
           "pba_set_variants", "pba_set_tuning", "pba_refine_extrinsic",
           "pba_get_extrinsic", "pba_set_offset_free"]
PBA_N_VARIANTS = 8
PBA_MAX_LEVELS = 8
PBA_NORMALS_MAX_RADIUS = 32
PBA_N_PHASES = 5
PHASE_NAMES = ["solve", "update", "linearize", "reduce_assemble", "accept"]


class PbaSensor(ctypes.Structure):
    _fields_ = [("model", ctypes.c_int32), ("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("fx", ctypes.c_double), ("fy", ctypes.c_double),
                ("cx", ctypes.c_double), ("cy", ctypes.c_double), ("extrinsic", ctypes.c_double * 12)]


class PbaConfig(ctypes.Structure):
    _fields_ = [("n_frames", ctypes.c_int32), ("n_sensors", ctypes.c_int32),
                ("sensors", ctypes.POINTER(PbaSensor)), ("frame_sensor", ctypes.POINTER(ctypes.c_int32)),
                ("w_int", ctypes.c_double), ("w_depth", ctypes.c_double), ("w_normal", ctypes.c_double),
                ("huber_delta", ctypes.c_double), ("occ_abs", ctypes.c_double), ("occ_rel", ctypes.c_double),
                ("z_min", ctypes.c_double), ("range_min", ctypes.c_double), ("range_max", ctypes.c_double),
                ("grad_mode", ctypes.c_int32), ("texel_precision", ctypes.c_int32), ("path", ctypes.c_int32),
                ("solver", ctypes.c_int32)]


class PbaIterStats(ctypes.Structure):
    _fields_ = [("cost", ctypes.c_double), ("new_cost", ctypes.c_double), ("lambda_used", ctypes.c_double),
                ("lambda_next", ctypes.c_double), ("n_valid", ctypes.c_int64), ("accepted", ctypes.c_int32),
                ("status", ctypes.c_int32), ("n_nonfinite", ctypes.c_int64), ("nonfinite_pairs", ctypes.c_int64)]


class PbaTuning(ctypes.Structure):
    _fields_ = [("variant_full", ctypes.c_int32), ("variant_cost", ctypes.c_int32), ("chunk", ctypes.c_int32),
                ("chunk_tail", ctypes.c_int32), ("from_cache", ctypes.c_int32), ("tile_err", ctypes.c_int32),
                ("ms_full", ctypes.c_float), ("ms_cost", ctypes.c_float), ("reduction", ctypes.c_int32)]


class PbaLevelStats(ctypes.Structure):
    _fields_ = [("level", ctypes.c_int32), ("iterations", ctypes.c_int32), ("accepted", ctypes.c_int32),
                ("status", ctypes.c_int32), ("cost_first", ctypes.c_double), ("cost_last", ctypes.c_double)]


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """The loaded libpba with argument types declared."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not os.path.exists(path) or not _build.up_to_date():
            if not build_if_missing:
                raise ImportError(f"libpba not built ({path}); run __graft_entry__.build()")
            _build.build()
        lib = ctypes.CDLL(path)
        P = ctypes.POINTER
        vp, i32, i64, d = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        sig = {
            "pba_create": ([P(PbaConfig), vp, P(vp)], ctypes.c_int),
            "pba_destroy": ([vp], None),
            "pba_last_error": ([vp], ctypes.c_char_p),
            "pba_set_stream": ([vp, vp], ctypes.c_int),
            "pba_upload_frames": ([vp, ctypes.c_int, ctypes.c_int, vp, ctypes.c_int], ctypes.c_int),
            "pba_frame_points": ([vp, ctypes.c_int, P(i32)], ctypes.c_int),
            "pba_set_poses": ([vp, vp, ctypes.c_int], ctypes.c_int),
            "pba_get_poses": ([vp, vp], ctypes.c_int),
            "pba_set_pairs": ([vp, vp, ctypes.c_int], ctypes.c_int),
            "pba_linearize": ([vp, P(d), P(i64)], ctypes.c_int),
            "pba_get_system": ([vp, vp, vp], ctypes.c_int),
            "pba_get_pair_system": ([vp, vp, vp, vp, vp], ctypes.c_int),
            "pba_set_mask_export": ([vp, ctypes.c_int], ctypes.c_int),
            "pba_get_mask": ([vp, ctypes.c_int, vp, ctypes.c_int], ctypes.c_int),
            "pba_solve_step": ([vp, d, P(PbaIterStats)], ctypes.c_int),
            "pba_set_lambda": ([vp, d], ctypes.c_int),
            "pba_iterate": ([vp, P(PbaIterStats)], ctypes.c_int),
            "pba_iterate_async": ([vp, ctypes.c_int], ctypes.c_int),
            "pba_get_stats": ([vp, P(PbaIterStats)], ctypes.c_int),
            "pba_iteration_launches": ([vp, P(i32)], ctypes.c_int),
            "pba_iterate_timed": ([vp, P(ctypes.c_float), ctypes.c_int, P(PbaIterStats)], ctypes.c_int),
            "pba_autotune": ([vp, ctypes.c_int, P(i32), P(i32)], ctypes.c_int),
            "pba_get_tuning": ([vp, P(PbaTuning)], ctypes.c_int),
            "pba_build_pairs": ([vp, d, d, d, ctypes.c_int, vp, vp, ctypes.c_int, P(i32)], ctypes.c_int),
            "pba_set_extrinsic": ([vp, ctypes.c_int, vp], ctypes.c_int),
            "pba_estimate_normals": ([vp, ctypes.c_int, ctypes.c_int, ctypes.c_float, ctypes.c_int], ctypes.c_int),
            "pba_get_channels": ([vp, ctypes.c_int, ctypes.c_int, vp, ctypes.c_int], ctypes.c_int),
            "pba_build_pyramid": ([vp, ctypes.c_int], ctypes.c_int),
            "pba_set_variables": ([vp, P(ctypes.c_int32), ctypes.c_int], ctypes.c_int),
            "pba_set_variants": ([vp, ctypes.c_int, ctypes.c_int], ctypes.c_int),
            "pba_set_tuning": ([vp, P(PbaTuning)], ctypes.c_int),
            "pba_iterate_frames": ([vp, vp, vp, P(PbaIterStats)], ctypes.c_int),
            "pba_get_extrinsic": ([vp, ctypes.c_int, vp], ctypes.c_int),
            "pba_set_offset_free": ([vp, ctypes.c_int, ctypes.c_int], ctypes.c_int),
            "pba_refine_extrinsic": ([vp, ctypes.c_int, ctypes.c_int, ctypes.c_double, P(ctypes.c_double),
                                      P(ctypes.c_double), P(ctypes.c_int32)], ctypes.c_int),
            "pba_pyramid_level": ([vp, ctypes.c_int, P(vp)], ctypes.c_int),
            "pba_optimize": ([vp, ctypes.c_int, P(ctypes.c_int32), ctypes.c_double, P(PbaLevelStats)], ctypes.c_int),
            "pba_cost_gradient": ([vp, P(d), P(i64), vp, vp, vp], ctypes.c_int),
            "pba_tangent_gradient": ([vp, vp, vp, ctypes.c_int, vp], ctypes.c_int),
            "pba_linearize_pairs_noalloc": ([P(PbaSensor), P(PbaConfig), vp, ctypes.c_int, vp, vp, ctypes.c_int, vp,
                                             vp], ctypes.c_int),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
        return lib


class PbaError(RuntimeError):
    def __init__(self, code: int, message: str):
        super().__init__(f"{ERROR_NAMES.get(code, code)}: {message}")
        self.code = code
