"""ctypes view of the C ABI declared in ``include/swift.h``.

Loads the in-tree ``libswift_gb300.so``.  There is no fallback: if the library
is missing or fails to load, importing this module raises.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libswift_gb300.so")

# status codes
SWIFT_OK = 0
SWIFT_ERR_INVALID_ARG = 1
SWIFT_ERR_UNSUPPORTED = 2
SWIFT_ERR_CUDA = 3
SWIFT_ERR_OOM = 4
SWIFT_ERR_TIMEOUT = 5
SWIFT_ERR_CAPACITY = 6

APOD = {"none": 0, "hann": 1, "tukey": 2}
DTYPE = {"u8": 0, "f32": 1}
PRECISION = {"fp32": 0, "bf16x2": 1, "fp16x2": 2}
SCHEDULE = {"default": 0, "fused": 1, "stream": 2, "persistent": 3}

WIN_OK, WIN_OUT_OF_BOUNDS, WIN_FLAT, WIN_NONFINITE, WIN_TIMEOUT = 0, 1, 2, 3, 4

# every symbol include/swift.h declares
EXPORTS = (
    "swift_plan_create",
    "swift_plan_destroy",
    "swift_match_batch",
    "swift_match_batch_noalloc",
    "swift_match_backward",
    "swift_plan_set_whitening",
    "swift_plan_set_schedule",
    "swift_plan_autotune",
    "swift_plan_capture",
    "swift_plan_replay",
    "swift_plan_set_timing",
    "swift_plan_set_test_stall",
    "swift_plan_set_test_hold",
    "swift_plan_set_skew",
    "swift_plan_set_lanes",
    "swift_plan_get_lanes",
    "swift_plan_set_row_tma",
    "swift_plan_get_row_tma",
    "swift_plan_set_test_stale_status",
    "swift_window_check",
    "swift_plan_timings",
    "swift_status_string",
    "swift_version",
    "swift_correspondences",
    "swift_fit_affine",
    "swift_fit_affine_update",
    "swift_mesh_fit",
    "swift_render_prepare",
    "swift_render",
    "swift_downsample",
    "swift_zmodel",
)

FIT_OK, FIT_FALLBACK, FIT_DEGENERATE = 0, 1, 2


class SwiftLevel(C.Structure):
    _fields_ = [("n", C.c_int32), ("whiten_exponent", C.c_float), ("apod", C.c_int32),
                ("tukey_alpha", C.c_float), ("snr_exclusion_radius", C.c_float)]


class SwiftImage(C.Structure):
    _fields_ = [("data", C.c_void_p), ("pitch", C.c_int64), ("stride", C.c_int64),
                ("height", C.c_int32), ("width", C.c_int32), ("count", C.c_int32)]


class SwiftBatch(C.Structure):
    _fields_ = [("ref", C.POINTER(SwiftImage)), ("mov", C.POINTER(SwiftImage)),
                ("ref_origin", C.c_void_p), ("mov_origin", C.c_void_p), ("level", C.c_void_p),
                ("n_windows", C.c_int64), ("patch_mode", C.c_int32), ("affine", C.c_void_p),
                ("level_offsets", C.POINTER(C.c_int64))]


class SwiftResult(C.Structure):
    _fields_ = [("dy", C.c_int32), ("dx", C.c_int32), ("sy", C.c_float), ("sx", C.c_float),
                ("snr", C.c_float), ("peak", C.c_float), ("status", C.c_int32),
                ("reserved", C.c_int32)]


assert C.sizeof(SwiftResult) == 32


class SwiftMesh(C.Structure):
    _fields_ = [("origin_y", C.c_int32), ("origin_x", C.c_int32), ("cell", C.c_int32),
                ("ny", C.c_int32), ("nx", C.c_int32)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"{LIB_PATH} is missing: build it first (python -c 'import __graft_entry__ as g; g.build()')")
    lib = C.CDLL(LIB_PATH)
    lib.swift_plan_create.argtypes = [C.POINTER(SwiftLevel), C.c_int32, C.c_int, C.c_int, C.c_int64,
                                      C.POINTER(C.c_void_p)]
    lib.swift_plan_create.restype = C.c_int
    lib.swift_plan_destroy.argtypes = [C.c_void_p]
    lib.swift_plan_destroy.restype = C.c_int
    lib.swift_match_batch.argtypes = [C.c_void_p, C.POINTER(SwiftBatch), C.c_void_p, C.c_void_p]
    lib.swift_match_batch.restype = C.c_int
    lib.swift_match_batch_noalloc.argtypes = [C.POINTER(SwiftLevel), C.c_int, C.POINTER(SwiftBatch), C.c_void_p,
                                              C.c_void_p]
    lib.swift_match_batch_noalloc.restype = C.c_int
    lib.swift_match_backward.argtypes = [C.c_void_p, C.POINTER(SwiftBatch), C.c_void_p, C.c_void_p, C.c_void_p,
                                         C.c_void_p, C.c_void_p]
    lib.swift_match_backward.restype = C.c_int
    lib.swift_plan_set_whitening.argtypes = [C.c_void_p, C.c_int32, C.c_float]
    lib.swift_plan_set_whitening.restype = C.c_int
    lib.swift_plan_set_schedule.argtypes = [C.c_void_p, C.c_int32, C.c_int32]
    lib.swift_plan_set_schedule.restype = C.c_int
    lib.swift_plan_autotune.argtypes = [C.c_void_p, C.POINTER(SwiftBatch), C.c_void_p, C.c_void_p,
                                        C.POINTER(C.c_int32)]
    lib.swift_plan_autotune.restype = C.c_int
    lib.swift_plan_capture.argtypes = [C.c_void_p, C.POINTER(SwiftBatch), C.c_void_p, C.c_void_p]
    lib.swift_plan_capture.restype = C.c_int
    lib.swift_plan_replay.argtypes = [C.c_void_p, C.c_void_p]
    lib.swift_plan_replay.restype = C.c_int
    lib.swift_plan_set_timing.argtypes = [C.c_void_p, C.c_int32]
    lib.swift_plan_set_timing.restype = C.c_int
    lib.swift_plan_set_test_stall.argtypes = [C.c_void_p, C.c_int32]
    lib.swift_plan_set_test_stall.restype = C.c_int
    lib.swift_plan_set_test_hold.argtypes = [C.c_void_p, C.c_int64]
    lib.swift_plan_set_test_hold.restype = C.c_int
    lib.swift_plan_set_skew.argtypes = [C.c_void_p, C.c_int32]
    lib.swift_plan_set_skew.restype = C.c_int
    lib.swift_plan_set_lanes.argtypes = [C.c_void_p, C.c_int32]
    lib.swift_plan_set_lanes.restype = C.c_int
    lib.swift_plan_get_lanes.argtypes = [C.c_void_p, C.POINTER(C.c_int32)]
    lib.swift_plan_get_lanes.restype = C.c_int
    lib.swift_plan_set_row_tma.argtypes = [C.c_void_p, C.c_int32]
    lib.swift_plan_set_row_tma.restype = C.c_int
    lib.swift_plan_get_row_tma.argtypes = [C.c_void_p, C.POINTER(C.c_int32)]
    lib.swift_plan_get_row_tma.restype = C.c_int
    lib.swift_plan_set_test_stale_status.argtypes = [C.c_void_p, C.c_int32]
    lib.swift_plan_set_test_stale_status.restype = C.c_int
    lib.swift_window_check.argtypes = [C.c_int32, C.c_int32, C.c_int32, C.POINTER(C.c_int32),
                                       C.POINTER(C.c_int32), C.c_int32, C.c_int32, C.c_int32, C.c_int32]
    lib.swift_window_check.restype = C.c_int32
    lib.swift_plan_timings.argtypes = [C.c_void_p, C.POINTER(C.c_float), C.POINTER(C.c_int32)]
    lib.swift_plan_timings.restype = C.c_int
    lib.swift_status_string.argtypes = [C.c_int]
    lib.swift_status_string.restype = C.c_char_p
    lib.swift_version.argtypes = []
    lib.swift_version.restype = C.c_char_p
    lib.swift_correspondences.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_int32, C.c_float,
                                          C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    lib.swift_correspondences.restype = C.c_int
    lib.swift_fit_affine.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p,
                                     C.c_void_p, C.c_void_p]
    lib.swift_fit_affine.restype = C.c_int
    lib.swift_fit_affine_update.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p,
                                     C.c_void_p, C.c_void_p]
    lib.swift_fit_affine_update.restype = C.c_int
    lib.swift_mesh_fit.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.POINTER(SwiftMesh), C.c_int32,
                                   C.c_void_p, C.c_void_p, C.c_void_p]
    lib.swift_mesh_fit.restype = C.c_int
    lib.swift_render_prepare.argtypes = [C.c_void_p, C.POINTER(SwiftMesh), C.c_void_p, C.c_void_p]
    lib.swift_render_prepare.restype = C.c_int
    lib.swift_render.argtypes = [C.POINTER(SwiftImage), C.c_int, C.c_void_p, C.POINTER(SwiftMesh), C.c_void_p,
                                 C.c_int, C.c_int32, C.c_int32, C.c_int64, C.c_float, C.c_void_p]
    lib.swift_render.restype = C.c_int
    lib.swift_downsample.argtypes = [C.POINTER(SwiftImage), C.c_int, C.c_int32, C.c_void_p, C.c_int64, C.c_void_p]
    lib.swift_downsample.restype = C.c_int
    lib.swift_zmodel.argtypes = [C.c_void_p, C.c_int64, C.c_int32, C.c_int32, C.c_int32, C.c_int64, C.c_int32,
                                 C.c_void_p, C.c_void_p, C.c_int, C.c_int64, C.c_int64, C.c_void_p]
    lib.swift_zmodel.restype = C.c_int
    return lib


lib = _load()


class SwiftError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {lib.swift_status_string(code).decode()}")


def check(code: int, where: str):
    if code != SWIFT_OK:
        raise SwiftError(code, where)
