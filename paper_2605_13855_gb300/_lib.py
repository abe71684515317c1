"""ctypes declarations of the C ABI in include/sparseoit.h (argument marshalling only).

The library is loaded from the package directory; loading fails loudly when
it is missing (there is no fallback implementation).
"""
from __future__ import annotations

import ctypes
import os
import threading

PKG_DIR = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG_DIR, "libsparseoit.so")

OK = 0
ERR_INVALID_ARG = -1
ERR_OOM = -2
ERR_CUDA = -3
ERR_STATE = -4
ERR_CAPACITY = -5
ERR_TIMEOUT = -6
F32 = 0
BF16 = 1
COMMIT_INCREMENTAL = 0
COMMIT_RECOMPUTE = 1
ROWS_BY_SPLAT = 0
ROWS_ACTIVE = 1
MAX_BATCH_VIEWS = 32

ERROR_NAMES = {ERR_INVALID_ARG: "INVALID_ARG", ERR_OOM: "OOM", ERR_CUDA: "CUDA", ERR_STATE: "STATE",
               ERR_CAPACITY: "CAPACITY", ERR_TIMEOUT: "TIMEOUT"}

# Every entry point declared in include/sparseoit.h.
EXPORTED = (
    "sparseoit_create", "sparseoit_destroy", "sparseoit_set_active", "sparseoit_set_active_async",
    "sparseoit_get_active",
    "sparseoit_commit_frozen", "sparseoit_get_frozen", "sparseoit_set_frozen", "sparseoit_forward",
    "sparseoit_backward",
    "sparseoit_reserve_pairs", "sparseoit_status", "sparseoit_last_counts", "sparseoit_set_counting",
    "sparseoit_set_profiling", "sparseoit_get_profile", "sparseoit_last_error", "sparseoit_version",
    "sparseoit_compact_active_static", "sparseoit_autotune", "sparseoit_fps_views", "sparseoit_activeness",
    "sparseoit_update_active_set", "sparseoit_adam_step", "sparseoit_loss_l1_dssim", "sparseoit_gather_active",
    "sparseoit_scatter_active", "sparseoit_inject_scan_stall",
)
STATIC_MAX_SPLATS = 16 * 1024 * 1024


class Rows(ctypes.Structure):
    _fields_ = [("means", ctypes.c_void_p), ("quats", ctypes.c_void_p), ("log_scales", ctypes.c_void_p),
                ("opacity_logits", ctypes.c_void_p), ("sh_color", ctypes.c_void_p), ("sh_weight", ctypes.c_void_p),
                ("sigma", ctypes.c_void_p)]


class Adam(ctypes.Structure):
    _fields_ = [("lr", ctypes.c_float * 8), ("beta1", ctypes.c_float), ("beta2", ctypes.c_float),
                ("eps", ctypes.c_float), ("step", ctypes.c_int32), ("rows", ctypes.c_int32)]


class Camera(ctypes.Structure):
    _fields_ = [("R", ctypes.c_float * 9), ("t", ctypes.c_float * 3), ("fx", ctypes.c_float),
                ("fy", ctypes.c_float), ("cx", ctypes.c_float), ("cy", ctypes.c_float),
                ("width", ctypes.c_int32), ("height", ctypes.c_int32)]


class Splats(ctypes.Structure):
    _fields_ = [("means", ctypes.c_void_p), ("quats", ctypes.c_void_p), ("log_scales", ctypes.c_void_p),
                ("opacity_logits", ctypes.c_void_p), ("sh_color", ctypes.c_void_p), ("sh_weight", ctypes.c_void_p),
                ("sh_dtype", ctypes.c_int32), ("sigma", ctypes.c_float), ("bg", ctypes.c_float * 3),
                ("n", ctypes.c_int64), ("rows", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class Grads(ctypes.Structure):
    _fields_ = [("means", ctypes.c_void_p), ("quats", ctypes.c_void_p), ("log_scales", ctypes.c_void_p),
                ("opacity_logits", ctypes.c_void_p), ("sh_color", ctypes.c_void_p), ("sh_weight", ctypes.c_void_p),
                ("sigma", ctypes.c_void_p), ("rows_by_splat", ctypes.c_int32), ("accumulate", ctypes.c_int32)]


class KernelTime(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int64), ("total_ms", ctypes.c_double)]


class Tuning(ctypes.Structure):
    _fields_ = [("fwd_pixels_per_thread", ctypes.c_int32), ("n_candidates", ctypes.c_int32),
                ("candidates", ctypes.c_int32 * 4), ("ms", ctypes.c_float * 4),
                ("fwd_persistent", ctypes.c_int32), ("fwd_persistent_ms", ctypes.c_float),
                ("bwd_walk", ctypes.c_int32), ("bwd_persistent", ctypes.c_int32), ("bwd_ms", ctypes.c_float * 4)]


class Config(ctypes.Structure):
    _fields_ = [("max_pairs", ctypes.c_int64), ("fwd_pixels_per_thread", ctypes.c_int32),
                ("proj_lanes_per_splat", ctypes.c_int32), ("bwd_walk", ctypes.c_int32),
                ("raster_tile_order", ctypes.c_int32), ("bwd_parallel", ctypes.c_int32),
                ("raster_persistent", ctypes.c_int32)]


_lock = threading.Lock()
_lib = None


def load(path: str = LIB_PATH):
    """Load libsparseoit.so and declare its signatures (raises if missing)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"libsparseoit.so not built at {path}; run __graft_entry__.build() "
                               "(or python -m paper_2605_13855_gb300.build)")
        lib = ctypes.CDLL(path)
        vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
        P = ctypes.POINTER
        sig = {
            "sparseoit_create": ([P(vp), i64, i32, P(i32), P(i32), P(Config)], ctypes.c_int),
            "sparseoit_destroy": ([vp], ctypes.c_int),
            "sparseoit_set_active": ([vp, vp, i64, vp], ctypes.c_int),
            "sparseoit_set_active_async": ([vp, vp, i64, vp], ctypes.c_int),
            "sparseoit_get_active": ([vp, P(vp), P(i64)], ctypes.c_int),
            "sparseoit_commit_frozen": ([vp, P(Splats), P(Camera), i32, i32, vp], ctypes.c_int),
            "sparseoit_get_frozen": ([vp, i32, P(vp)], ctypes.c_int),
            "sparseoit_set_frozen": ([vp, i32, vp, vp], ctypes.c_int),
            "sparseoit_forward": ([vp, P(Splats), P(Camera), P(i32), i32, P(vp), P(vp), vp, vp], ctypes.c_int),
            "sparseoit_backward": ([vp, P(Splats), P(vp), P(Grads), vp], ctypes.c_int),
            "sparseoit_reserve_pairs": ([vp, i64], ctypes.c_int),
            "sparseoit_status": ([vp, vp], ctypes.c_int),
            "sparseoit_inject_scan_stall": ([vp, ctypes.c_int32], ctypes.c_int),
            "sparseoit_last_counts": ([vp, vp, P(i64), P(i64)], ctypes.c_int),
            "sparseoit_set_counting": ([vp, i32], ctypes.c_int),
            "sparseoit_set_profiling": ([vp, i32], ctypes.c_int),
            "sparseoit_get_profile": ([vp, i32, P(KernelTime), P(i32)], ctypes.c_int),
            "sparseoit_last_error": ([vp], ctypes.c_char_p),
            "sparseoit_version": ([], ctypes.c_int),
            "sparseoit_compact_active_static": ([vp, i64, vp, vp, vp], ctypes.c_int),
            "sparseoit_autotune": ([vp, P(Splats), P(Camera), P(i32), i32, P(vp), P(vp), vp, i32, P(Tuning), vp],
                                   ctypes.c_int),
            "sparseoit_fps_views": ([P(Camera), i32, i32, i32, P(i32)], ctypes.c_int),
            "sparseoit_update_active_set": ([vp, P(Splats), P(Camera), i32, P(vp), i32, i32, P(ctypes.c_float),
                                             P(Grads), vp, P(i32), vp], ctypes.c_int),
            "sparseoit_loss_l1_dssim": ([vp, P(vp), ctypes.c_float, vp, P(vp), P(ctypes.c_float), vp], ctypes.c_int),
            "sparseoit_gather_active": ([vp, P(Rows), P(Rows), i32, vp], ctypes.c_int),
            "sparseoit_scatter_active": ([vp, P(Rows), P(Rows), i32, vp], ctypes.c_int),
            "sparseoit_adam_step": ([vp, P(Grads), P(Rows), P(Rows), P(Rows), P(Adam), vp], ctypes.c_int),
            "sparseoit_activeness": ([P(Grads), i64, P(ctypes.c_float), vp, vp, vp], ctypes.c_int),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
        return lib


class SparseOITError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"sparseoit error {ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code
