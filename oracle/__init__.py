"""CPU oracle for the sliding-window inter-channel Pearson correlation.

TEST INFRASTRUCTURE ONLY.  This package is the slow, plain reference that the
CUDA path is checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline leg may import it; the product package never does,
and the two share no code.

It wraps ``swcorr_oracle.c`` (plain C, double precision, two-pass classical
Pearson per window, Eq. 1 of Poyda & Zhizhin, arXiv:1807.06507; clipped
windows; NaN for constant windows as the paper's equality check prescribes).
The shared library is built with gcc on first use (or by ``build()``) into
``oracle/_build/``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "swcorr_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libswcorr_oracle.so")
_lock = threading.Lock()
_lib = None

U16, F32 = 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no fast-math).  Returns the .so path."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread",
           "-fno-fast-math", "-ffp-contract=off", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _configure(lib):
    """Declare the C entry points' signatures on a loaded oracle library."""
    i64p = ctypes.POINTER(ctypes.c_int64)
    i32p = ctypes.POINTER(ctypes.c_int32)
    dp = ctypes.POINTER(ctypes.c_double)
    lib.swo_corr.argtypes = [ctypes.c_int, i64p, i32p, i32p, ctypes.c_int,
                             ctypes.c_void_p, ctypes.c_void_p, i64p, ctypes.c_int64,
                             dp, dp, dp, ctypes.c_int]
    lib.swo_corr.restype = ctypes.c_int
    lib.swo_corr_border.argtypes = [ctypes.c_int, i64p, i32p, i32p, ctypes.c_int,
                                    ctypes.c_void_p, ctypes.c_void_p, i64p, ctypes.c_int64,
                                    dp, dp, dp, ctypes.c_int, ctypes.c_int]
    lib.swo_corr_border.restype = ctypes.c_int
    lib.swo_sums_u16.argtypes = [ctypes.c_int, i64p, i32p, i32p,
                                 ctypes.c_void_p, ctypes.c_void_p, i64p, ctypes.c_int64,
                                 i64p, ctypes.c_int]
    lib.swo_sums_u16.restype = ctypes.c_int
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _configure(ctypes.CDLL(build()))
    return _lib


def _swap_library(path_or_lib):
    """Tests only (planted-mistake checks): make later calls use another
    build of the oracle -- a path to a shared library, a handle returned
    earlier, or None for the regular build.  Returns the previous handle."""
    global _lib
    lib = path_or_lib
    if isinstance(path_or_lib, (str, os.PathLike)):
        lib = _configure(ctypes.CDLL(os.fspath(path_or_lib)))
    with _lock:
        prev, _lib = _lib, lib
    return prev


def _ptr(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct)) if a is not None else None


def _args(x, y, k, stride):
    x = np.ascontiguousarray(x)
    y = np.ascontiguousarray(y)
    if x.shape != y.shape:
        raise ValueError("x and y must have the same shape")
    if x.dtype != y.dtype:
        raise ValueError("x and y must have the same dtype")
    if x.dtype == np.uint16:
        dt = U16
    elif x.dtype == np.float32:
        dt = F32
    else:
        raise TypeError("oracle takes uint16 or float32 grids")
    nd = x.ndim
    k = np.broadcast_to(np.asarray(k, dtype=np.int32), (nd,)).copy()
    stride = np.broadcast_to(np.asarray(1 if stride is None else stride, dtype=np.int32),
                             (nd,)).copy()
    shape = np.asarray(x.shape, dtype=np.int64)
    oshape = tuple(int(-(-n // s)) for n, s in zip(x.shape, stride))
    return x, y, dt, shape, k, stride, oshape


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


BORDERS = {"clip": 0, "paper": 1}


def corr(x, y, k, stride=None, idx=None, threads=None, relvar=False, border="clip"):
    """Pearson c per output window (float64), NaN for constant windows.

    x, y: same-shape uint16 or float32 arrays (1 to 8 dims, C order).
    k, stride: per-dimension window size and step (scalars broadcast).
    idx: optional flat output indices (C order over the output grid); when
    given, the result is 1-D with one entry per index.  Otherwise it has the
    output grid's shape, ceil(N_d / stride_d) per dimension.
    relvar=True also returns (relvar_x, relvar_y).
    border: "clip" (windows clipped to the grid, n = in-grid cells) or
    "paper" (Section 3's convention: -2 for a window past an edge or holding
    a value <= -999 in x or y; the relative variances are 0 there).
    """
    x, y, dt, shape, k, stride, oshape = _args(x, y, k, stride)
    bmode = BORDERS[border]
    if idx is not None:
        idx = np.ascontiguousarray(idx, dtype=np.int64).ravel()
        n = idx.size
    else:
        n = int(np.prod(oshape))
    c = np.empty(n, dtype=np.float64)
    rx = np.empty(n, dtype=np.float64) if relvar else None
    ry = np.empty(n, dtype=np.float64) if relvar else None
    rc = _load().swo_corr_border(x.ndim, _ptr(shape, ctypes.c_int64), _ptr(k, ctypes.c_int32),
                                 _ptr(stride, ctypes.c_int32), dt, x.ctypes.data, y.ctypes.data,
                                 _ptr(idx, ctypes.c_int64), n, _ptr(c, ctypes.c_double),
                                 _ptr(rx, ctypes.c_double), _ptr(ry, ctypes.c_double), bmode,
                                 int(threads or default_threads()))
    if rc != 0:
        raise ValueError(f"oracle rejected the arguments (code {rc})")
    if idx is None:
        c = c.reshape(oshape)
        if relvar:
            rx, ry = rx.reshape(oshape), ry.reshape(oshape)
    return (c, rx, ry) if relvar else c


def sums_u16(x, y, k, stride=None, idx=None, threads=None):
    """Exact int64 window sums for uint16 grids, shape (..., 5).

    The last axis holds sum x, sum y, sum x^2, sum y^2, sum xy over each
    clipped window (steps 1-3 of the optimized algorithm, by brute force).
    """
    x, y, dt, shape, k, stride, oshape = _args(x, y, k, stride)
    if dt != U16:
        raise TypeError("sums_u16 takes uint16 grids")
    if idx is not None:
        idx = np.ascontiguousarray(idx, dtype=np.int64).ravel()
        n = idx.size
    else:
        n = int(np.prod(oshape))
    s = np.empty((n, 5), dtype=np.int64)
    rc = _load().swo_sums_u16(x.ndim, _ptr(shape, ctypes.c_int64), _ptr(k, ctypes.c_int32),
                              _ptr(stride, ctypes.c_int32), x.ctypes.data, y.ctypes.data,
                              _ptr(idx, ctypes.c_int64), n, _ptr(s, ctypes.c_int64),
                              int(threads or default_threads()))
    if rc != 0:
        raise ValueError(f"oracle rejected the arguments (code {rc})")
    return s if idx is not None else s.reshape(oshape + (5,))


def window_bounds(centre: int, k: int, n: int):
    """Clipped window [lo, hi] (inclusive) along one dimension."""
    lo = centre - (k - 1) // 2
    hi = centre + k // 2
    return max(lo, 0), min(hi, n - 1)
