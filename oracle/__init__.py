"""CPU oracle for the downscaler filter stage -- TEST INFRASTRUCTURE ONLY.

The plain FP64 / int64 loop nest in ``ds_oracle.c`` that the CUDA library is
checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / reference leg of ``bench.py`` may import this package.  It
shares no code with ``paper_1103_4881_b300``; it is built by gcc, not nvcc.

Functions follow the paper's Sec. 3 (horizontal then vertical filter over
packets of q pixels giving p outputs) and Sec. 3.A (Array-OL tiler with
origin, paving and fitting); the readings the paper leaves open are listed
in ``ds_oracle.h``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ds_oracle.c")
_LIB = os.path.join(_HERE, "libds_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile ds_oracle.c into libds_oracle.so with gcc (OpenMP, no FP contraction)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "ds_oracle.h"))
    ):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


class _Axes(ctypes.Structure):
    _fields_ = [("ph", ctypes.c_int), ("qh", ctypes.c_int), ("Kh", ctypes.c_int),
                ("pv", ctypes.c_int), ("qv", ctypes.c_int), ("Kv", ctypes.c_int),
                ("boundary", ctypes.c_int), ("taps_h", ctypes.c_void_p), ("taps_v", ctypes.c_void_p)]


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        c_int, c_long, c_void = ctypes.c_int, ctypes.c_long, ctypes.c_void_p
        lib.dso_out_extent.restype = c_long
        lib.dso_out_extent.argtypes = [c_long, c_int, c_int]
        lib.dso_phase_windows.argtypes = [c_int, c_int, c_int, c_void, c_void]
        lib.dso_taps_f64.argtypes = [c_int, c_int, c_int, c_void]
        lib.dso_taps_q14.argtypes = [c_int, c_int, c_int, c_void]
        sig = [c_void, c_void, c_long, c_int, c_int, c_int, c_int, c_int, c_int, c_int]
        lib.dso_filter_f64.argtypes = sig
        lib.dso_filter_u8.argtypes = sig
        lib.dso_max_threads.argtypes = []
        lib.dso_quantize_q14.argtypes = [c_void, c_int, c_int, c_void]
        sig_ex = [c_void, c_void, c_long, c_int, c_int, c_int, ctypes.POINTER(_Axes), c_int]
        lib.dso_filter_ex_f64.argtypes = sig_ex
        lib.dso_filter_ex_u8.argtypes = sig_ex
        _lib = lib
    return _lib


def out_extent(n_in: int, p: int, q: int) -> int:
    """floor(n_in * p / q) (paper Sec. 3: 352 -> 132 at 3/8)."""
    return int(_load().dso_out_extent(n_in, p, q))


def phase_windows(p: int, q: int, K: int):
    """(b, c): window start b_j and centre c_j of each phase j < p."""
    b = np.zeros(p, np.int32)
    c = np.zeros(p, np.float64)
    if _load().dso_phase_windows(p, q, K, b.ctypes.data, c.ctypes.data):
        raise ValueError("bad filter arguments")
    return b, c


def taps_f64(p: int, q: int, K: int) -> np.ndarray:
    """FP64 Lanczos-3 taps, shape (p, K), rows summing to 1."""
    w = np.zeros((p, K), np.float64)
    if _load().dso_taps_f64(p, q, K, w.ctypes.data):
        raise ValueError("bad filter arguments")
    return w


def taps_q14(p: int, q: int, K: int) -> np.ndarray:
    """Q14 taps, shape (p, K), rows summing to 16384."""
    w = np.zeros((p, K), np.int32)
    if _load().dso_taps_q14(p, q, K, w.ctypes.data):
        raise ValueError("bad filter arguments")
    return w


def _as_nhwc(x: np.ndarray):
    """Accept (H,W), (N,H,W) or (N,H,W,C); return the array as (N,H,W,C) and a reshaper."""
    if x.ndim == 2:
        return x[None, :, :, None], lambda y: y[0, :, :, 0]
    if x.ndim == 3:
        return x[:, :, :, None], lambda y: y[:, :, :, 0]
    if x.ndim == 4:
        return x, lambda y: y
    raise ValueError("expected (H,W), (N,H,W) or (N,H,W,C)")


def filter_f64(x: np.ndarray, p: int, q: int, K: int, threads: int = 0) -> np.ndarray:
    """Separable filter (H pass then V pass) in FP64.

    ``x`` of any float dtype is decoded exactly to float64 first; channels
    (last axis of a 4-D input) are filtered independently.
    """
    x4, back = _as_nhwc(np.asarray(x))
    x4 = np.ascontiguousarray(x4, dtype=np.float64)
    n, H, W, C = x4.shape
    OH, OW = out_extent(H, p, q), out_extent(W, p, q)
    y = np.empty((n, OH, OW, C), np.float64)
    if _load().dso_filter_f64(x4.ctypes.data, y.ctypes.data, n, H, W, C, p, q, K, threads):
        raise ValueError("bad filter arguments")
    return back(y)


def filter_u8(x: np.ndarray, p: int, q: int, K: int, threads: int = 0) -> np.ndarray:
    """Separable filter on uint8 with Q14 taps and a uint8 intermediate."""
    x4, back = _as_nhwc(np.asarray(x))
    x4 = np.ascontiguousarray(x4, dtype=np.uint8)
    n, H, W, C = x4.shape
    OH, OW = out_extent(H, p, q), out_extent(W, p, q)
    y = np.empty((n, OH, OW, C), np.uint8)
    if _load().dso_filter_u8(x4.ctypes.data, y.ctypes.data, n, H, W, C, p, q, K, threads):
        raise ValueError("bad filter arguments")
    return back(y)


def quantize_q14(w: np.ndarray) -> np.ndarray:
    """Q14 of a tap table (p, K): round half up, residual on the largest tap."""
    w = np.ascontiguousarray(w, dtype=np.float64)
    p, K = w.shape
    qt = np.zeros((p, K), np.int32)
    if _load().dso_quantize_q14(w.ctypes.data, p, K, qt.ctypes.data):
        raise ValueError("bad tap table")
    return qt


def filter_ex(x: np.ndarray, ratio_h, taps_h: int, ratio_v, taps_v: int, wrap: bool = False,
              weights_h=None, weights_v=None, threads: int = 0) -> np.ndarray:
    """Separable filter with its own ratio, tap count and (optionally) FP64 tap
    table (p, K) per axis, and clamp-to-edge or modular (wrap) tilers.  uint8
    input takes the Q14 integer path, anything else FP64."""
    x4, back = _as_nhwc(np.asarray(x))
    u8 = x4.dtype == np.uint8
    x4 = np.ascontiguousarray(x4, dtype=np.uint8 if u8 else np.float64)
    n, H, W, C = x4.shape
    wh = None if weights_h is None else np.ascontiguousarray(weights_h, dtype=np.float64)
    wv = None if weights_v is None else np.ascontiguousarray(weights_v, dtype=np.float64)
    ax = _Axes(ratio_h[0], ratio_h[1], taps_h, ratio_v[0], ratio_v[1], taps_v, 1 if wrap else 0,
               None if wh is None else wh.ctypes.data, None if wv is None else wv.ctypes.data)
    OH, OW = out_extent(H, ratio_v[0], ratio_v[1]), out_extent(W, ratio_h[0], ratio_h[1])
    y = np.empty((n, OH, OW, C), np.uint8 if u8 else np.float64)
    fn = _load().dso_filter_ex_u8 if u8 else _load().dso_filter_ex_f64
    if fn(x4.ctypes.data, y.ctypes.data, n, H, W, C, ctypes.byref(ax), threads):
        raise ValueError("bad filter arguments")
    return back(y)


def max_threads() -> int:
    return int(_load().dso_max_threads())
