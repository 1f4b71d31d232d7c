"""FP64 CPU oracle for convolutional gridding and degridding.

TEST INFRASTRUCTURE ONLY. This package is the correctness oracle. Only
``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may
import it. The CUDA product path neither imports it nor shares code with it.

Each function wraps one C routine in ``oracle.c`` (plain FP64, built with
``-ffp-contract=off``). The C file states which passage of Merry 2016 each
routine follows and how the paper's silent points are read.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` into ``liboracle.so`` next to it (gcc, -O2, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
             _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        i64, i32, dbl = ctypes.c_int64, ctypes.c_int, ctypes.c_double
        vp = ctypes.c_void_p
        lib.oracle_fine_position.argtypes = [dbl, i32, ctypes.POINTER(ctypes.c_int64)]
        lib.oracle_fine_position.restype = i32
        lib.oracle_indices.argtypes = [i32, i32, i32, i64, vp, vp, vp]
        lib.oracle_indices.restype = i64
        lib.oracle_bessel_i0.argtypes = [dbl]
        lib.oracle_bessel_i0.restype = dbl
        lib.oracle_kb_table.argtypes = [i32, i32, dbl, vp]
        lib.oracle_kb_table.restype = i32
        lib.oracle_grid.argtypes = [i32, i32, i32, i32, i64, vp, vp, vp, vp, vp]
        lib.oracle_grid.restype = i64
        lib.oracle_degrid.argtypes = [i32, i32, i32, i32, i64, vp, vp, vp, vp]
        lib.oracle_degrid.restype = i64
        lib.oracle_compress.argtypes = [i32, i32, i64, vp, vp, vp, vp, vp, vp]
        lib.oracle_compress.restype = i64
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def fine_position(u: float, oversample: int) -> int:
    """f = floor(u*O + 1/2), exact. Raises ValueError for non-finite or out-of-range u."""
    f = ctypes.c_int64()
    if _load().oracle_fine_position(float(u), int(oversample), ctypes.byref(f)) != 0:
        raise ValueError("invalid coordinate")
    return f.value


def indices(G: int, S: int, oversample: int, uv: np.ndarray):
    """Absolute centre cells and table rows.

    Returns ``(cell [n,2] int32, sub [n,2] int32, n_skipped)``. A skipped
    visibility has cell = sub = -1.
    """
    uv = np.ascontiguousarray(uv, dtype=np.float64).reshape(-1, 2)
    n = uv.shape[0]
    cell = np.empty((n, 2), np.int32)
    sub = np.empty((n, 2), np.int32)
    r = _load().oracle_indices(G, S, oversample, n, _ptr(uv), _ptr(cell), _ptr(sub))
    if r < 0:
        raise ValueError("bad arguments")
    return cell, sub, int(r)


def bessel_i0(x: float) -> float:
    """I0(x) from its power series, in FP64."""
    return _load().oracle_bessel_i0(float(x))


def kb_table(S: int, oversample: int, beta: float) -> np.ndarray:
    """Oversampled Kaiser-Bessel table, ``[O][S]`` float64."""
    t = np.empty((oversample, S), np.float64)
    if _load().oracle_kb_table(S, oversample, float(beta), _ptr(t)) != 0:
        raise ValueError("bad arguments")
    return t


def grid(G: int, S: int, oversample: int, uv, vis, weights, table, out=None):
    """Grid visibilities onto ``[P][G][G]`` complex128 (accumulates into ``out`` if given).

    ``vis`` is [n][P] complex. ``weights`` is [n] real, or None for unit weights.
    ``table`` is [O][S] real. All of them are upcast to FP64 exactly.
    Returns ``(grid, n_skipped)``.
    """
    uv = np.ascontiguousarray(uv, dtype=np.float64).reshape(-1, 2)
    n = uv.shape[0]
    vis = np.ascontiguousarray(vis, dtype=np.complex128).reshape(n, -1)
    P = vis.shape[1]
    table = np.ascontiguousarray(table, dtype=np.float64).reshape(oversample, S)
    w = None if weights is None else np.ascontiguousarray(weights, dtype=np.float64).reshape(n)
    if out is None:
        out = np.zeros((P, G, G), np.complex128)
    assert out.dtype == np.complex128 and out.shape == (P, G, G) and out.flags.c_contiguous
    r = _load().oracle_grid(G, S, oversample, P, n, _ptr(uv), _ptr(vis),
                            None if w is None else _ptr(w), _ptr(table), _ptr(out))
    if r < 0:
        raise ValueError("bad arguments")
    return out, int(r)


def degrid(G: int, S: int, oversample: int, uv, grid_in, table):
    """Degrid ``[P][G][G]`` complex onto the visibilities. Returns ``(vis [n][P] complex128, n_skipped)``."""
    uv = np.ascontiguousarray(uv, dtype=np.float64).reshape(-1, 2)
    n = uv.shape[0]
    g = np.ascontiguousarray(grid_in, dtype=np.complex128)
    P = g.shape[0]
    assert g.shape == (P, G, G)
    table = np.ascontiguousarray(table, dtype=np.float64).reshape(oversample, S)
    vis = np.empty((n, P), np.complex128)
    r = _load().oracle_degrid(G, S, oversample, P, n, _ptr(uv), _ptr(g), _ptr(table), _ptr(vis))
    if r < 0:
        raise ValueError("bad arguments")
    return vis, int(r)


def compress(oversample: int, uv, vis, weights=None):
    """Merge runs of adjacent visibilities that share a fine position (compression, Sec. 2.2).

    Returns ``(uv_out [m][2] float64, vis_out [m][P] complex128, run_of [n] int64)``. ``vis_out`` holds
    the weighted sums; grid it with unit weights. ``run_of[k]`` is the merged record of visibility k.
    """
    uv = np.ascontiguousarray(uv, dtype=np.float64).reshape(-1, 2)
    n = uv.shape[0]
    vis = np.ascontiguousarray(vis, dtype=np.complex128)
    vis = vis if vis.ndim == 2 else vis.reshape(n, -1)
    P = vis.shape[1]
    w = None if weights is None else np.ascontiguousarray(weights, dtype=np.float64).reshape(n)
    uv_out = np.empty((n, 2), np.float64)
    vis_out = np.empty((n, P), np.complex128)
    run_of = np.empty(n, np.int64)
    m = _load().oracle_compress(oversample, P, n, _ptr(uv), _ptr(vis), None if w is None else _ptr(w),
                                _ptr(uv_out), _ptr(vis_out), _ptr(run_of))
    if m < 0:
        raise ValueError("bad arguments")
    return uv_out[:m].copy(), vis_out[:m].copy(), run_of
