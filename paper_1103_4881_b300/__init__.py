"""Python binding of libds: the B300 (sm_103a) separable decimating FIR filter
stage ("downscaler") of arXiv:1103.4881.

Argument marshalling only: every step of the filter runs in the CUDA kernels
of ``libds.so`` (built in-tree by ``python -m paper_1103_4881_b300.build``).
Function names and arguments follow the C ABI in ``include/ds.h``; device
pointers and CUDA streams are plain integers (``tensor.data_ptr()``,
``torch.cuda.current_stream().cuda_stream``).  A failing call raises
``DsError`` carrying ``ds_last_error()``.  There is no CPU fallback: if the
library is missing, importing the binding's functions raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Iterable, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# the same library built with DS_CHECK_BOUNDS (the kernel checks its own
# indices); load it instead with use_library(CHECK_LIB_PATH), or for the whole
# process by setting DS_CHECK_BOUNDS=1 in the environment before the import
CHECK_LIB_PATH = os.path.join(_HERE, "libds_check.so")
LIB_PATH = CHECK_LIB_PATH if os.environ.get("DS_CHECK_BOUNDS") == "1" else os.path.join(_HERE, "libds.so")

DS_F32, DS_F16, DS_U8, DS_U8_RGB = 0, 1, 2, 3
DS_CLAMP, DS_WRAP = 0, 1
DS_OK, DS_ERR_ARG, DS_ERR_NOMEM, DS_ERR_CUDA, DS_ERR_TIMEOUT, DS_ERR_UNSUPPORTED, DS_ERR_BOUNDS = 0, -1, -2, -3, -4, -5, -6
_STATUS_NAMES = {0: "DS_OK", -1: "DS_ERR_ARG", -2: "DS_ERR_NOMEM", -3: "DS_ERR_CUDA",
                 -4: "DS_ERR_TIMEOUT", -5: "DS_ERR_UNSUPPORTED", -6: "DS_ERR_BOUNDS"}

# exported symbols of libds (the declarations in include/ds.h)
ABI_SYMBOLS = (
    "ds_plan_create", "ds_destroy", "ds_plan_get_params", "ds_plan_out_shape", "ds_plan_frame_bytes",
    "ds_plan_get_taps", "ds_plan_describe", "ds_plan_set_schedule", "ds_plan_get_schedule",
    "ds_run", "ds_run_frames", "ds_batch_run", "ds_plan_workspace_bytes", "ds_run_unfused",
    "ds_stream_check", "ds_debug_check_plan", "ds_graph_create", "ds_graph_launch", "ds_graph_destroy",
    "ds_pipeline_create", "ds_pipeline_run", "ds_pipeline_destroy", "ds_last_error", "ds_version",
    "ds_launch_count", "ds_static_workspace_bytes", "ds_run_unfused_static", "ds_plan_autotune",
    "ds_debug_timeout_probe", "ds_plan_create_ex", "ds_plan_get_axes", "ds_plan_get_axis_taps",
    "ds_bounds_checked", "ds_debug_bounds_probe", "ds_plan_tile_shapes", "ds_plan_set_schedule_ex",
    "ds_plan_get_schedule_ex", "ds_plan_autotune_ex", "ds_server_create", "ds_server_run", "ds_server_destroy",
    "ds_batch_autotune",
)
DS_SERVE_REALTIME, DS_SERVE_COPIES, DS_SERVE_PLAIN = 1, 2, 4


class DsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s: %s" % (_STATUS_NAMES.get(status, str(status)), msg))
        self.status = status


class ds_ratio(ctypes.Structure):
    _fields_ = [("p", ctypes.c_int), ("q", ctypes.c_int)]


class ds_plan_desc(ctypes.Structure):
    _fields_ = [("in_h", ctypes.c_int), ("in_w", ctypes.c_int), ("ratio_h", ds_ratio), ("taps_h", ctypes.c_int),
                ("ratio_v", ds_ratio), ("taps_v", ctypes.c_int), ("dtype", ctypes.c_int), ("boundary", ctypes.c_int),
                ("weights_h", ctypes.c_void_p), ("weights_v", ctypes.c_void_p)]


class ds_schedule(ctypes.Structure):
    _fields_ = [("row_blocks", ctypes.c_int), ("ctas_per_sm", ctypes.c_int), ("shape", ctypes.c_int)]


class ds_tune_result(ctypes.Structure):
    _fields_ = [("best", ds_schedule), ("best_us", ctypes.c_float), ("default_us", ctypes.c_float),
                ("candidates", ctypes.c_int)]


class ds_request(ctypes.Structure):
    _fields_ = [("plan", ctypes.c_void_p), ("in_", ctypes.c_void_p), ("out", ctypes.c_void_p),
                ("arrival_s", ctypes.c_double)]


class ds_serve_stats(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_int), ("batches", ctypes.c_int), ("max_batch", ctypes.c_int),
                ("max_queue", ctypes.c_int), ("launches", ctypes.c_longlong), ("wall_s", ctypes.c_double),
                ("peak_admitted_bytes", ctypes.c_size_t)]


class ds_job(ctypes.Structure):
    _fields_ = [("plan", ctypes.c_void_p), ("in_", ctypes.c_void_p), ("out", ctypes.c_void_p),
                ("n_frames", ctypes.c_int)]


_lib = None


def lib() -> ctypes.CDLL:
    """The loaded libds.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libds.so is not built (%s); run: python -m paper_1103_4881_b300.build" % LIB_PATH)
    L = ctypes.CDLL(LIB_PATH)
    vp, i, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t
    ip = ctypes.POINTER(ctypes.c_int)
    sig = {
        "ds_plan_create": (vp, [i, i, ds_ratio, i, i]),
        "ds_destroy": (None, [vp]),
        "ds_plan_get_params": (i, [vp, ip, ip, ip, ip, ip, ip]),
        "ds_plan_out_shape": (i, [vp, ip, ip, ip]),
        "ds_plan_frame_bytes": (i, [vp, ctypes.POINTER(sz), ctypes.POINTER(sz)]),
        "ds_plan_get_taps": (i, [vp, vp, vp, vp, vp]),
        "ds_plan_describe": (i, [vp, ctypes.c_char_p, sz]),
        "ds_plan_set_schedule": (i, [vp, i, i]),
        "ds_plan_get_schedule": (i, [vp, ip, ip]),
        "ds_run": (i, [vp, vp, vp, vp]),
        "ds_run_frames": (i, [vp, vp, vp, i, vp]),
        "ds_batch_run": (i, [vp, i, vp]),
        "ds_plan_workspace_bytes": (sz, [vp]),
        "ds_run_unfused": (i, [vp, vp, vp, i, vp, sz, vp]),
        "ds_stream_check": (i, [vp]),
        "ds_debug_check_plan": (i, [vp]),
        "ds_graph_create": (vp, [vp, i]),
        "ds_graph_launch": (i, [vp, vp]),
        "ds_graph_destroy": (None, [vp]),
        "ds_pipeline_create": (vp, [vp, i, i]),
        "ds_pipeline_run": (i, [vp, vp, vp, i]),
        "ds_pipeline_destroy": (None, [vp]),
        "ds_last_error": (ctypes.c_char_p, []),
        "ds_version": (ctypes.c_char_p, []),
        "ds_launch_count": (ctypes.c_longlong, []),
        "ds_static_workspace_bytes": (sz, []),
        "ds_plan_autotune": (i, [vp, vp, vp, i, vp, i, ip, ctypes.POINTER(ctypes.c_float)]),
        "ds_run_unfused_static": (i, [vp, vp, vp, i, vp]),
        "ds_debug_timeout_probe": (i, [ctypes.c_longlong, vp]),
        "ds_bounds_checked": (i, []),
        "ds_debug_bounds_probe": (i, [vp]),
        "ds_plan_create_ex": (vp, [ctypes.POINTER(ds_plan_desc)]),
        "ds_plan_get_axes": (i, [vp, ip, ip, ip, ip, ip, ip, ip]),
        "ds_plan_get_axis_taps": (i, [vp, i, vp, vp, vp, vp]),
        "ds_plan_tile_shapes": (i, [vp]),
        "ds_plan_set_schedule_ex": (i, [vp, ctypes.POINTER(ds_schedule)]),
        "ds_plan_get_schedule_ex": (i, [vp, ctypes.POINTER(ds_schedule)]),
        "ds_plan_autotune_ex": (i, [vp, vp, vp, i, vp, i, ctypes.POINTER(ds_tune_result)]),
        "ds_server_create": (vp, [sz, i, i]),
        "ds_server_run": (i, [vp, ctypes.POINTER(ds_request), i, i, ctypes.POINTER(ctypes.c_double),
                              ctypes.POINTER(ds_serve_stats)]),
        "ds_server_destroy": (None, [vp]),
        "ds_batch_autotune": (i, [vp, i, vp, i, ctypes.POINTER(ds_tune_result)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def ds_last_error() -> str:
    return lib().ds_last_error().decode()


def ds_version() -> str:
    return lib().ds_version().decode()


def ds_launch_count() -> int:
    return int(lib().ds_launch_count())


def _check(status: int) -> None:
    if status != DS_OK:
        raise DsError(status, ds_last_error())


def _ptr(x):
    return None if x is None else ctypes.c_void_p(int(x))


# ----------------------------------------------------------------------- plans

def ds_plan_create(in_h: int, in_w: int, ratio: Sequence[int], taps: int, dtype: int) -> int:
    h = lib().ds_plan_create(in_h, in_w, ds_ratio(int(ratio[0]), int(ratio[1])), taps, dtype)
    if not h:
        raise DsError(DS_ERR_ARG, ds_last_error())
    return h


def ds_plan_create_ex(in_h: int, in_w: int, ratio_h: Sequence[int], taps_h: int, ratio_v: Sequence[int],
                      taps_v: int, dtype: int, boundary: int = DS_CLAMP, weights_h=None, weights_v=None) -> int:
    """Plan with a ratio and tap count per axis, a boundary (DS_CLAMP / DS_WRAP)
    and optional FP64 tap tables (p, K) per axis (copied by the library)."""
    wh = None if weights_h is None else np.ascontiguousarray(weights_h, dtype=np.float64)
    wv = None if weights_v is None else np.ascontiguousarray(weights_v, dtype=np.float64)
    d = ds_plan_desc(in_h, in_w, ds_ratio(int(ratio_h[0]), int(ratio_h[1])), taps_h,
                     ds_ratio(int(ratio_v[0]), int(ratio_v[1])), taps_v, dtype, boundary,
                     None if wh is None else wh.ctypes.data, None if wv is None else wv.ctypes.data)
    h = lib().ds_plan_create_ex(ctypes.byref(d))
    if not h:
        raise DsError(DS_ERR_ARG, ds_last_error())
    return h


def ds_plan_get_axes(plan: int):
    """((p_h, q_h, taps_h), (p_v, q_v, taps_v), boundary)"""
    v = [ctypes.c_int() for _ in range(7)]
    _check(lib().ds_plan_get_axes(_ptr(plan), *[ctypes.byref(x) for x in v]))
    return (v[0].value, v[1].value, v[2].value), (v[3].value, v[4].value, v[5].value), v[6].value


def ds_plan_get_axis_taps(plan: int, axis: int):
    """ds_plan_get_taps for axis 0 (horizontal) or 1 (vertical)."""
    (ph, _, Kh), (pv, _, Kv), _ = ds_plan_get_axes(plan)
    p, K = (ph, Kh) if axis == 0 else (pv, Kv)
    f64 = np.zeros((p, K), np.float64)
    f32 = np.zeros((p, K), np.float32)
    q14 = np.zeros((p, K), np.int16)
    b = np.zeros(p, np.int32)
    _check(lib().ds_plan_get_axis_taps(_ptr(plan), axis, f64.ctypes.data, f32.ctypes.data, q14.ctypes.data,
                                       b.ctypes.data))
    return {"fp64": f64, "fp32": f32, "q14": q14, "window_start": b}


def ds_destroy(plan: int) -> None:
    lib().ds_destroy(_ptr(plan))


def ds_plan_get_params(plan: int):
    """(in_h, in_w, p, q, taps, dtype)"""
    v = [ctypes.c_int() for _ in range(6)]
    _check(lib().ds_plan_get_params(_ptr(plan), *[ctypes.byref(x) for x in v]))
    return tuple(x.value for x in v)


def ds_plan_out_shape(plan: int):
    """(out_h, out_w, channels)"""
    v = [ctypes.c_int() for _ in range(3)]
    _check(lib().ds_plan_out_shape(_ptr(plan), *[ctypes.byref(x) for x in v]))
    return tuple(x.value for x in v)


def ds_plan_frame_bytes(plan: int):
    a, b = ctypes.c_size_t(), ctypes.c_size_t()
    _check(lib().ds_plan_frame_bytes(_ptr(plan), ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def ds_plan_get_taps(plan: int):
    """dict with fp64 / fp32 / q14 tap tables of shape (p, K) and window_start (p,)."""
    _, _, p, _, K, _ = ds_plan_get_params(plan)
    f64 = np.zeros((p, K), np.float64)
    f32 = np.zeros((p, K), np.float32)
    q14 = np.zeros((p, K), np.int16)
    b = np.zeros(p, np.int32)
    _check(lib().ds_plan_get_taps(_ptr(plan), f64.ctypes.data, f32.ctypes.data, q14.ctypes.data, b.ctypes.data))
    return {"fp64": f64, "fp32": f32, "q14": q14, "window_start": b}


def ds_plan_describe(plan: int) -> str:
    buf = ctypes.create_string_buffer(1024)
    _check(lib().ds_plan_describe(_ptr(plan), buf, len(buf)))
    return buf.value.decode()


def ds_plan_set_schedule(plan: int, row_blocks: int, ctas_per_sm: int = 0) -> None:
    _check(lib().ds_plan_set_schedule(_ptr(plan), row_blocks, ctas_per_sm))


def ds_plan_get_schedule(plan: int):
    a, b = ctypes.c_int(), ctypes.c_int()
    _check(lib().ds_plan_get_schedule(_ptr(plan), ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def ds_plan_autotune(plan: int, in_ptr: int, out_ptr: int, n_frames: int, stream: int = 0, iters: int = 10):
    """Time the candidate tile bands on the given buffers, keep the fastest;
    returns (row_blocks, us_per_launch)."""
    rb, us = ctypes.c_int(), ctypes.c_float()
    _check(lib().ds_plan_autotune(_ptr(plan), _ptr(in_ptr), _ptr(out_ptr), n_frames, _ptr(stream), iters,
                                  ctypes.byref(rb), ctypes.byref(us)))
    return rb.value, us.value


def ds_plan_tile_shapes(plan: int) -> int:
    return int(lib().ds_plan_tile_shapes(_ptr(plan)))


def ds_plan_set_schedule_ex(plan: int, row_blocks: int = 0, ctas_per_sm: int = 0, shape: int = 0) -> None:
    """row_blocks 0 = the class default (adaptive) band; ctas_per_sm 0 = as many as fit."""
    sc = ds_schedule(row_blocks, ctas_per_sm, shape)
    _check(lib().ds_plan_set_schedule_ex(_ptr(plan), ctypes.byref(sc)))


def ds_plan_get_schedule_ex(plan: int) -> dict:
    sc = ds_schedule()
    _check(lib().ds_plan_get_schedule_ex(_ptr(plan), ctypes.byref(sc)))
    return {"row_blocks": sc.row_blocks, "ctas_per_sm": sc.ctas_per_sm, "shape": sc.shape}


def ds_plan_autotune_ex(plan: int, in_ptr: int, out_ptr: int, n_frames: int, stream: int = 0, iters: int = 10) -> dict:
    """Time tile shapes, bands and CTAs per SM on the given buffers and keep the
    fastest schedule in the plan; returns it with its time and the default's."""
    r = ds_tune_result()
    _check(lib().ds_plan_autotune_ex(_ptr(plan), _ptr(in_ptr), _ptr(out_ptr), n_frames, _ptr(stream), iters,
                                     ctypes.byref(r)))
    return {"row_blocks": r.best.row_blocks, "ctas_per_sm": r.best.ctas_per_sm, "shape": r.best.shape,
            "us_per_launch": r.best_us, "default_us_per_launch": r.default_us, "candidates": r.candidates}


def ds_server_create(mem_budget_bytes: int, n_streams: int, max_batch: int) -> int:
    h = lib().ds_server_create(int(mem_budget_bytes), n_streams, max_batch)
    if not h:
        raise DsError(DS_ERR_ARG, ds_last_error())
    return h


def ds_server_run(server: int, requests, flags: int):
    """requests: a ds_request array (or a sequence of (plan, in_ptr, out_ptr,
    arrival_s)); returns (latency_ms numpy array, stats dict)."""
    if not isinstance(requests, ctypes.Array):
        requests = (ds_request * len(requests))(*[ds_request(_ptr(p), _ptr(a), _ptr(b), float(t))
                                                  for p, a, b, t in requests])
    n = len(requests)
    lat = np.zeros(max(n, 1), dtype=np.float64)
    st = ds_serve_stats()
    _check(lib().ds_server_run(_ptr(server), requests, n, flags,
                               lat.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(st)))
    return lat[:n], {f: getattr(st, f) for f, _ in ds_serve_stats._fields_}


def ds_server_destroy(server: int) -> None:
    lib().ds_server_destroy(_ptr(server))


def ds_debug_timeout_probe(limit_cycles: int, stream: int = 0) -> None:
    """Launch a warp whose bounded wait runs out after limit_cycles (nothing
    completes its barrier); the next ds_stream_check raises DS_ERR_TIMEOUT."""
    _check(lib().ds_debug_timeout_probe(limit_cycles, _ptr(stream)))


def ds_bounds_checked() -> bool:
    """Whether the loaded library is the DS_CHECK_BOUNDS build."""
    return bool(lib().ds_bounds_checked())


def ds_debug_bounds_probe(stream: int = 0) -> None:
    """DS_CHECK_BOUNDS builds: run the kernels' bounds check on an index one
    past a buffer (no access is made); the next ds_stream_check raises
    DS_ERR_BOUNDS."""
    _check(lib().ds_debug_bounds_probe(_ptr(stream)))


def use_library(path: str) -> None:
    """Load libds from `path` for the calls that follow (plans made with the
    previous library must not be used with the new one)."""
    global _lib, LIB_PATH
    _lib = None
    LIB_PATH = path


# ---------------------------------------------------------------------- running

def ds_run(plan: int, in_ptr: int, out_ptr: int, stream: int = 0) -> None:
    _check(lib().ds_run(_ptr(plan), _ptr(in_ptr), _ptr(out_ptr), _ptr(stream)))


def ds_run_frames(plan: int, in_ptr: int, out_ptr: int, n_frames: int, stream: int = 0) -> None:
    _check(lib().ds_run_frames(_ptr(plan), _ptr(in_ptr), _ptr(out_ptr), n_frames, _ptr(stream)))


def _jobs_array(jobs: Iterable):
    jobs = list(jobs)
    arr = (ds_job * max(1, len(jobs)))()
    for k, j in enumerate(jobs):
        plan, inp, out = j[0], j[1], j[2]
        nf = j[3] if len(j) > 3 else 1
        arr[k] = ds_job(plan, inp, out, nf)
    return arr, len(jobs)


def ds_batch_run(jobs: Iterable, stream: int = 0) -> None:
    """jobs: iterable of (plan, in_ptr, out_ptr[, n_frames])."""
    arr, n = _jobs_array(jobs)
    _check(lib().ds_batch_run(arr, n, _ptr(stream)))


def ds_batch_autotune(jobs: Iterable, stream: int = 0, iters: int = 10) -> dict:
    """Time schedules of the whole batch (as ds_batch_run) and keep the
    fastest in its plans; returns each job's plan schedule (in job order), the
    batch's time at it and at the default, and the candidates timed."""
    jobs = list(jobs)
    arr, n = _jobs_array(jobs)
    r = ds_tune_result()
    _check(lib().ds_batch_autotune(arr, n, _ptr(stream), iters, ctypes.byref(r)))
    return {"schedules": [ds_plan_get_schedule_ex(j[0]) for j in jobs], "us_per_launch": r.best_us,
            "default_us_per_launch": r.default_us, "candidates": r.candidates}


def ds_plan_workspace_bytes(plan: int) -> int:
    return int(lib().ds_plan_workspace_bytes(_ptr(plan)))


def ds_run_unfused(plan: int, in_ptr: int, out_ptr: int, n_frames: int, workspace: int, workspace_bytes: int,
                   stream: int = 0) -> None:
    _check(lib().ds_run_unfused(_ptr(plan), _ptr(in_ptr), _ptr(out_ptr), n_frames, _ptr(workspace),
                                workspace_bytes, _ptr(stream)))


def ds_debug_check_plan(plan: int) -> None:
    """Host-only check of the fused kernel's index arithmetic for this plan."""
    _check(lib().ds_debug_check_plan(_ptr(plan)))


def ds_static_workspace_bytes() -> int:
    """Size of the fixed device array ds_run_unfused_static uses."""
    return int(lib().ds_static_workspace_bytes())


def ds_run_unfused_static(plan: int, in_ptr: int, out_ptr: int, n_frames: int, stream: int = 0) -> None:
    """Unfused form with its intermediate in the library's fixed device array:
    for callers that cannot allocate device memory on the call path."""
    _check(lib().ds_run_unfused_static(_ptr(plan), _ptr(in_ptr), _ptr(out_ptr), n_frames, _ptr(stream)))


def ds_stream_check(stream: int = 0) -> None:
    _check(lib().ds_stream_check(_ptr(stream)))


# ----------------------------------------------------------------------- graphs

def ds_graph_create(jobs: Iterable) -> int:
    arr, n = _jobs_array(jobs)
    g = lib().ds_graph_create(arr, n)
    if not g:
        raise DsError(DS_ERR_CUDA, ds_last_error())
    return g


def ds_graph_launch(graph: int, stream: int = 0) -> None:
    _check(lib().ds_graph_launch(_ptr(graph), _ptr(stream)))


def ds_graph_destroy(graph: int) -> None:
    lib().ds_graph_destroy(_ptr(graph))


# --------------------------------------------------------------------- pipeline

def ds_pipeline_create(plan: int, chunk_frames: int, depth: int) -> int:
    p = lib().ds_pipeline_create(_ptr(plan), chunk_frames, depth)
    if not p:
        raise DsError(DS_ERR_NOMEM, ds_last_error())
    return p


def ds_pipeline_run(pipe: int, in_host_ptr: int, out_host_ptr: int, n_frames: int) -> None:
    _check(lib().ds_pipeline_run(_ptr(pipe), _ptr(in_host_ptr), _ptr(out_host_ptr), n_frames))


def ds_pipeline_destroy(pipe: int) -> None:
    lib().ds_pipeline_destroy(_ptr(pipe))
