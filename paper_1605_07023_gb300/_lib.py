"""ctypes loader for libgb300gridder.so (the C ABI in include/gridder.h).

There is no fallback. If the library is missing or cannot load, every entry
point raises RuntimeError.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgb300gridder.so")

GRID_OK = 0
GRID_ERR_INVALID = -1
GRID_ERR_UNSUPPORTED = -2
GRID_ERR_NOMEM = -3
GRID_ERR_CUDA = -4

PREC = {"f32": 0, "bf16": 1, "f16": 2}
SCHED = {"chunked": 0, "patch": 1, "tile": 2, "lazy": 3, "sorted": 4}

EXPORTS = ("grid_plan_desc_init", "grid_plan_create", "grid_plan_create_ex", "grid_plan_destroy", "grid_plan_describe",
           "grid", "degrid", "degrid_weighted", "grid_make_kernel_table", "grid_compute_indices", "grid_plan_skipped", "grid_plan_status", "grid_plan_gridder",
           "grid_last_error", "grid_device_info", "grid_tap_form", "grid_batch_create", "grid_batch_set", "grid_batch_execute",
           "grid_batch_skipped", "grid_batch_describe", "grid_batch_destroy", "grid_batch_last_error",
           "grid_patch_static", "grid_patch_static_last_error", "grid_compress", "degrid_expand", "grid_degrid_host", "grid_batch_create_ex",
           "grid_degrid_host_steps", "grid_measure_fma_peak")


class GridHostStep(ctypes.Structure):
    _fields_ = [("uv_host", ctypes.c_void_p), ("vis_host", ctypes.c_void_p), ("weights_host", ctypes.c_void_p),
                ("vis_out_host", ctypes.c_void_p), ("grid_host", ctypes.c_void_p)]


class GridBatchItem(ctypes.Structure):
    _fields_ = [("n_vis", ctypes.c_int64), ("uv", ctypes.c_void_p), ("vis", ctypes.c_void_p),
                ("weights", ctypes.c_void_p), ("kernel_table", ctypes.c_void_p), ("grid", ctypes.c_void_p),
                ("S", ctypes.c_int)]


class GridPlanDesc(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int) for n in ("G", "S", "oversample", "npol", "Bu", "Bv", "vis_per_chunk", "threads",
                                             "precision", "schedule", "patch", "bin_u", "bin_v", "tile_group")]


class GridderError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"gridder error {code}: {msg}")
        self.code = code


_lib = None


def load(path: str | None = None) -> ctypes.CDLL:
    """Load the library (once) and declare the C signatures."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"CUDA library not built: {p} is missing. Run __graft_entry__.build() "
                           "(or python paper_1605_07023_gb300/build.py) first.")
    lib = ctypes.CDLL(p)
    i32, i64, vp = ctypes.c_int, ctypes.c_int64, ctypes.c_void_p
    pdesc = ctypes.POINTER(GridPlanDesc)
    lib.grid_plan_desc_init.argtypes = [pdesc, i32, i32, i32, i32, i32]
    lib.grid_plan_desc_init.restype = None
    lib.grid_plan_create.argtypes = [ctypes.POINTER(vp), i32, i32, i32, i32, i32]
    lib.grid_plan_create.restype = i32
    lib.grid_plan_create_ex.argtypes = [ctypes.POINTER(vp), pdesc]
    lib.grid_plan_create_ex.restype = i32
    lib.grid_plan_destroy.argtypes = [vp]
    lib.grid_plan_destroy.restype = None
    lib.grid_plan_describe.argtypes = [vp, pdesc, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32)]
    lib.grid_plan_describe.restype = i32
    lib.grid.argtypes = [vp, i64, vp, vp, vp, vp, vp, vp]
    lib.grid.restype = i32
    lib.degrid.argtypes = [vp, i64, vp, vp, vp, vp, vp]
    lib.degrid.restype = i32
    lib.degrid_weighted.argtypes = [vp, i64, vp, vp, vp, vp, vp, vp]
    lib.degrid_weighted.restype = i32
    lib.grid_make_kernel_table.argtypes = [i32, i32, ctypes.c_double, i32, vp, vp]
    lib.grid_make_kernel_table.restype = i32
    lib.grid_compute_indices.argtypes = [vp, i64, vp, vp, vp, vp]
    lib.grid_compute_indices.restype = i32
    lib.grid_plan_skipped.argtypes = [vp, ctypes.POINTER(i64), i32]
    lib.grid_plan_skipped.restype = i32
    lib.grid_plan_status.argtypes = [vp, ctypes.POINTER(ctypes.c_uint), i32]
    lib.grid_plan_status.restype = i32
    lib.grid_plan_gridder.argtypes = [vp]
    lib.grid_plan_gridder.restype = ctypes.c_char_p
    lib.grid_compress.argtypes = [vp, i64, vp, vp, vp, vp, vp, vp, vp, vp]
    lib.grid_compress.restype = i32
    lib.degrid_expand.argtypes = [vp, i64, vp, i64, vp, vp, vp, vp]
    lib.degrid_expand.restype = i32
    lib.grid_degrid_host.argtypes = [vp, vp, i64, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, i64, vp]
    lib.grid_degrid_host.restype = i32
    lib.grid_degrid_host_steps.argtypes = [vp, vp, i32, ctypes.POINTER(GridHostStep), i64, ctypes.POINTER(vp),
                                           ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp), vp, vp, i64, vp]
    lib.grid_degrid_host_steps.restype = i32
    lib.grid_last_error.argtypes = []
    lib.grid_last_error.restype = ctypes.c_char_p
    lib.grid_device_info.argtypes = [ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32)]
    lib.grid_device_info.restype = i32
    lib.grid_measure_fma_peak.argtypes = [i32, ctypes.POINTER(ctypes.c_double), vp]
    lib.grid_measure_fma_peak.restype = i32
    lib.grid_tap_form.argtypes = [i32, i32, i32, ctypes.POINTER(i32), ctypes.POINTER(i32)]
    lib.grid_tap_form.restype = i32
    lib.grid_batch_create.argtypes = [ctypes.POINTER(vp), i32, i32, i32, i32, i32, i32, i32, i32, i32]
    lib.grid_batch_create.restype = i32
    lib.grid_batch_create_ex.argtypes = [ctypes.POINTER(vp), i32, i32, i32, i32, i32, i32, i32, i32, i32, i32, i32, i32]
    lib.grid_batch_create_ex.restype = i32
    lib.grid_batch_set.argtypes = [vp, i32, ctypes.POINTER(GridBatchItem)]
    lib.grid_batch_set.restype = i32
    lib.grid_batch_execute.argtypes = [vp, vp]
    lib.grid_batch_execute.restype = i32
    lib.grid_batch_skipped.argtypes = [vp, ctypes.POINTER(i64), i32]
    lib.grid_batch_skipped.restype = i32
    lib.grid_batch_describe.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32)]
    lib.grid_batch_describe.restype = i32
    lib.grid_batch_destroy.argtypes = [vp]
    lib.grid_batch_destroy.restype = None
    lib.grid_batch_last_error.argtypes = []
    lib.grid_batch_last_error.restype = ctypes.c_char_p
    _lib = lib
    return lib


def check(rc: int, batch: bool = False) -> None:
    if rc != GRID_OK:
        lib = load()
        msg = (lib.grid_batch_last_error() if batch else lib.grid_last_error()).decode(errors="replace")
        raise GridderError(rc, msg)
