"""ctypes binding of libswcorr.so (the C ABI in include/swcorr.h).

Argument marshalling only: every step of the computation runs in the CUDA
kernels of the shared library.  PyTorch supplies device memory and streams.
If the library has not been built, every call raises: there is no CPU path.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libswcorr.so")

OK, ERR_INVALID_ARG, ERR_UNSUPPORTED, ERR_ALIGNMENT, ERR_CUDA, ERR_OOM, ERR_TIMEOUT, ERR_NO_DEVICE = range(8)
U16, F32 = 1, 2
BORDER_CLIP, BORDER_PAPER = 0, 1
BORDERS = {"clip": BORDER_CLIP, "paper": BORDER_PAPER}
FLAG_EMIT_SUMS = 1
FLAG_TEST_STALL = 2
FLAG_SAT = 4
FLAG_UNFUSED = 8

EXPORTS = ("swcorr_plan_create", "swcorr_plan_create_tuned", "swcorr_plan_tune", "swcorr_set_tune_file",
           "swcorr_tune_lookup", "swcorr_run", "swcorr_run_host", "swcorr_plan_batched", "swcorr_plan_batched_tuned",
           "swcorr_run_batched", "swcorr_plan_status", "swcorr_plan_fallbacks", "swcorr_plan_outputs",
           "swcorr_plan_destroy", "swcorr_status_string", "swcorr_last_error", "swcorr_version",
           "swcorr_run2d_u16_noalloc", "swcorr_noalloc_status")

# Tune cache shipped with the package (written by autotune.py); used unless
# SWCORR_TUNE_FILE names another file.
DEFAULT_TUNE_FILE = os.path.join(_HERE, "tune_cache.json")
TUNE_FIELDS = ("prefetch", "tile_rows", "ctas_per_sm")


class SwcorrError(RuntimeError):
    def __init__(self, status: int, detail: str):
        super().__init__(f"swcorr status {status}: {detail}")
        self.status = status
        self.detail = detail


class SceneStruct(ctypes.Structure):
    _fields_ = [("shape", ctypes.c_int64 * 2), ("k", ctypes.c_int32 * 2), ("x", ctypes.c_void_p),
                ("y", ctypes.c_void_p), ("in_pitch", ctypes.c_int64), ("c", ctypes.c_void_p),
                ("out_pitch", ctypes.c_int64)]


class TuneStruct(ctypes.Structure):
    _fields_ = [("prefetch", ctypes.c_int32), ("tile_rows", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 5)]


def _tune_struct(tune):
    if tune is None:
        return None
    t = TuneStruct()
    for k, v in dict(tune).items():
        if k not in TUNE_FIELDS:
            raise KeyError(f"unknown tune field {k!r}")
        setattr(t, k, int(v))
    return t


def _tune_dict(t):
    return {k: int(getattr(t, k)) for k in TUNE_FIELDS}


_lock = threading.Lock()
_lib = None


def load(path: str | None = None):
    """Load libswcorr.so; raises if it is missing (build it with build.build())."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"libswcorr.so is not built ({p}); run paper_1807_06507_gb300.build.build()")
        lib = ctypes.CDLL(p)
        i64p = ctypes.POINTER(ctypes.c_int64)
        i32p = ctypes.POINTER(ctypes.c_int32)
        vp = ctypes.c_void_p
        lib.swcorr_plan_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, i64p, i32p, i32p, ctypes.c_int,
                                           ctypes.c_int, ctypes.c_uint32]
        tp = ctypes.POINTER(TuneStruct)
        lib.swcorr_plan_create_tuned.argtypes = [ctypes.POINTER(vp), ctypes.c_int, i64p, i32p, i32p, ctypes.c_int,
                                                 ctypes.c_int, ctypes.c_uint32, tp]
        lib.swcorr_plan_tune.argtypes = [vp, tp]
        lib.swcorr_set_tune_file.argtypes = [ctypes.c_char_p]
        lib.swcorr_tune_lookup.argtypes = [ctypes.c_char_p, ctypes.c_int, ctypes.c_int, i32p, ctypes.c_int, tp]
        lib.swcorr_tune_lookup.restype = ctypes.c_int
        lib.swcorr_plan_batched_tuned.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(SceneStruct), ctypes.c_int,
                                                  ctypes.c_int, ctypes.c_uint32, tp]
        lib.swcorr_run.argtypes = [vp, vp, vp, i64p, vp, i64p, vp, vp]
        lib.swcorr_run_host.argtypes = [vp, vp, vp, vp, vp]
        lib.swcorr_plan_batched.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(SceneStruct), ctypes.c_int,
                                            ctypes.c_int, ctypes.c_uint32]
        lib.swcorr_run_batched.argtypes = [vp, vp]
        lib.swcorr_plan_status.argtypes = [vp]
        lib.swcorr_plan_fallbacks.argtypes = [vp]
        lib.swcorr_plan_fallbacks.restype = ctypes.c_int64
        lib.swcorr_plan_outputs.argtypes = [vp]
        lib.swcorr_plan_outputs.restype = ctypes.c_int64
        lib.swcorr_plan_destroy.argtypes = [vp]
        lib.swcorr_plan_destroy.restype = None
        lib.swcorr_run2d_u16_noalloc.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, vp,
                                                 vp, ctypes.c_int64, vp, ctypes.c_int64, vp]
        lib.swcorr_run2d_u16_noalloc.restype = ctypes.c_int
        lib.swcorr_noalloc_status.argtypes = [vp, i64p]
        lib.swcorr_noalloc_status.restype = ctypes.c_int
        lib.swcorr_status_string.argtypes = [ctypes.c_int]
        lib.swcorr_status_string.restype = ctypes.c_char_p
        lib.swcorr_last_error.restype = ctypes.c_char_p
        lib.swcorr_version.restype = ctypes.c_char_p
        for name in ("swcorr_plan_create", "swcorr_plan_create_tuned", "swcorr_plan_tune", "swcorr_set_tune_file",
                     "swcorr_run", "swcorr_run_host", "swcorr_plan_batched", "swcorr_plan_batched_tuned",
                     "swcorr_run_batched", "swcorr_plan_status"):
            getattr(lib, name).restype = ctypes.c_int
        if not os.environ.get("SWCORR_TUNE_FILE") and os.path.exists(DEFAULT_TUNE_FILE):
            lib.swcorr_set_tune_file(DEFAULT_TUNE_FILE.encode())
        _lib = lib
        return lib


def _check(st: int):
    if st != OK:
        lib = load()
        raise SwcorrError(st, lib.swcorr_last_error().decode())


def _arr(vals, ct):
    a = (ct * len(vals))(*vals)
    return ctypes.cast(a, ctypes.POINTER(ct)), a


def _dtype_code(dtype) -> int:
    s = str(dtype)
    if s in ("u16", "uint16", "torch.uint16") or dtype is np.uint16:
        return U16
    if s in ("f32", "float32", "torch.float32") or dtype is np.float32:
        return F32
    raise TypeError(f"unsupported dtype {dtype}")


def _stream_ptr(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def set_tune_file(path):
    """(Re)load the tune cache from `path` (None: no cache)."""
    _check(load().swcorr_set_tune_file(path.encode() if path else None))


def tune_lookup(ndim, k, dtype, device=None, batched=False):
    """The cached launch parameters for (device, ndim, k, dtype), or None."""
    t = TuneStruct()
    kk, _a = _arr([int(v) for v in np.broadcast_to(np.asarray(k), (ndim,))], ctypes.c_int32)
    found = load().swcorr_tune_lookup(device.encode() if device else None, 1 if batched else 0, ndim, kk,
                                      _dtype_code(dtype), ctypes.byref(t))
    return _tune_dict(t) if found else None


class Plan:
    """A plan for one grid shape (swcorr_plan_create / swcorr_run).

    tune: None (the tune cache or built-in defaults) or a dict with any of
    prefetch, tile_rows, ctas_per_sm (swcorr_plan_create_tuned).
    border: "clip" or "paper" (SWCORR_BORDER_PAPER)."""

    def __init__(self, shape, k, stride=None, dtype="u16", flags=0, tune=None, border="clip"):
        lib = load()
        self.shape = tuple(int(v) for v in shape)
        nd = len(self.shape)
        self.k = tuple(int(v) for v in np.broadcast_to(np.asarray(k), (nd,)))
        self.stride = tuple(int(v) for v in np.broadcast_to(np.asarray(1 if stride is None else stride), (nd,)))
        self.dtype = _dtype_code(dtype)
        self.flags = int(flags)
        self.oshape = tuple(-(-n // s) for n, s in zip(self.shape, self.stride))
        h = ctypes.c_void_p()
        shp, _a = _arr(self.shape, ctypes.c_int64)
        kk, _b = _arr(self.k, ctypes.c_int32)
        ss, _c = _arr(self.stride, ctypes.c_int32)
        t = _tune_struct(tune)
        self.border = BORDERS[border]
        _check(lib.swcorr_plan_create_tuned(ctypes.byref(h), nd, shp, kk, ss, self.dtype, self.border, self.flags,
                                            ctypes.byref(t) if t is not None else None))
        self._h = h

    @property
    def handle(self):
        return self._h

    def run(self, x, y, c=None, sums=None, stream=None, in_pitch=None, out_pitch=None):
        """x, y: CUDA tensors of the plan's shape/dtype (rows may be padded:
        pass in_pitch in elements).  Returns c (float32 CUDA tensor)."""
        import torch
        if c is None:
            c = torch.empty(self.oshape, dtype=torch.float32, device=x.device)
        ip = op = None
        keep = []
        if in_pitch is not None:
            ip, a = _arr([int(v) for v in in_pitch], ctypes.c_int64)
            keep.append(a)
        elif not x.is_contiguous():
            ip, a = _arr([int(v) for v in x.stride()], ctypes.c_int64)
            keep.append(a)
        if out_pitch is not None:
            op, b = _arr([int(v) for v in out_pitch], ctypes.c_int64)
            keep.append(b)
        elif not c.is_contiguous():
            op, b = _arr([int(v) for v in c.stride()], ctypes.c_int64)
            keep.append(b)
        sp = ctypes.c_void_p(sums.data_ptr()) if sums is not None else None
        _check(load().swcorr_run(self._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()), ip,
                                 ctypes.c_void_p(c.data_ptr()), op, sp, _stream_ptr(stream)))
        return c

    def run_host(self, x: np.ndarray, y: np.ndarray, c: np.ndarray | None = None, stream=None) -> np.ndarray:
        """Host buffers in, host result out (copies inside the call)."""
        x = np.ascontiguousarray(x)
        y = np.ascontiguousarray(y)
        if c is None:
            c = np.empty(self.oshape, dtype=np.float32)
        _check(load().swcorr_run_host(self._h, ctypes.c_void_p(x.ctypes.data), ctypes.c_void_p(y.ctypes.data),
                                      ctypes.c_void_p(c.ctypes.data), _stream_ptr(stream)))
        return c

    def tune(self) -> dict:
        """Launch parameters the plan uses."""
        t = TuneStruct()
        _check(load().swcorr_plan_tune(self._h, ctypes.byref(t)))
        return _tune_dict(t)

    def status(self) -> int:
        return load().swcorr_plan_status(self._h)

    def check_status(self):
        _check(self.status())

    def fallbacks(self) -> int:
        return int(load().swcorr_plan_fallbacks(self._h))

    def outputs(self) -> int:
        return int(load().swcorr_plan_outputs(self._h))

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().swcorr_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BatchedPlan:
    """One persistent launch over many 2-D scenes of one dtype, uint16 or
    float32 (swcorr_plan_batched)."""

    def __init__(self, scenes, flags=0, tune=None):
        """scenes: list of (x, y, c, (kh, kw)) with CUDA tensors (all uint16,
        carried as int16, or all float32); x/y rows may be padded (strided
        views with unit last stride).  tune: as for Plan."""
        lib = load()
        dts = {str(t.dtype) for sc in scenes for t in sc[:2]}
        if len(dts) != 1:
            raise ValueError(f"a batched plan takes scenes of one dtype, got {sorted(dts)}")
        dt = F32 if dts == {"torch.float32"} else U16
        arr = (SceneStruct * len(scenes))()
        self._keep = []
        for i, (x, y, c, k) in enumerate(scenes):
            kh, kw = (k, k) if np.isscalar(k) else k
            s = arr[i]
            s.shape[0], s.shape[1] = int(x.shape[0]), int(x.shape[1])
            s.k[0], s.k[1] = int(kh), int(kw)
            s.x, s.y, s.c = x.data_ptr(), y.data_ptr(), c.data_ptr()
            s.in_pitch = int(x.stride(0))
            s.out_pitch = int(c.stride(0))
            self._keep.append((x, y, c))
        h = ctypes.c_void_p()
        t = _tune_struct(tune)
        _check(lib.swcorr_plan_batched_tuned(ctypes.byref(h), arr, len(scenes), dt, int(flags),
                                             ctypes.byref(t) if t is not None else None))
        self._h = h

    def run(self, stream=None):
        _check(load().swcorr_run_batched(self._h, _stream_ptr(stream)))

    def tune(self) -> dict:
        t = TuneStruct()
        _check(load().swcorr_plan_tune(self._h, ctypes.byref(t)))
        return _tune_dict(t)

    def check_status(self):
        _check(load().swcorr_plan_status(self._h))

    def fallbacks(self) -> int:
        return int(load().swcorr_plan_fallbacks(self._h))

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().swcorr_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def corr(x, y, k, stride=None, stream=None):
    """One-shot convenience: Pearson c of every window of CUDA tensors x, y."""
    p = Plan(tuple(x.shape), k, stride, dtype=str(x.dtype).replace("torch.", ""))
    try:
        return p.run(x, y, stream=stream)
    finally:
        p.close()


def version() -> str:
    return load().swcorr_version().decode()
