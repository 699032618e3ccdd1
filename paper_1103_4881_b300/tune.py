"""Persistent cache of autotuned schedules (host-side file IO only).

The tuning itself is ``ds_plan_autotune_ex`` in the library: CUDA events over
the compiled tile shapes of the plan's class, band heights and resident CTAs
per SM (the launch topology that the paper derives from thresholds, Sec.
3.B.1).  The cache keeps its choice per GPU model, SM count, dtype, the ratio
and taps of both axes, frame size and batch size, in the JSON file named by
``DS_TUNE_CACHE`` (default ``~/.cache/ds_tune.json``), so a process that has
tuned once reuses the result.
"""
from __future__ import annotations

import json
import os
import threading

import paper_1103_4881_b300 as ds

_lock = threading.Lock()


def cache_path() -> str:
    return os.environ.get("DS_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "ds_tune.json"))


def _device_tag() -> str:
    import torch

    p = torch.cuda.get_device_properties(torch.cuda.current_device())
    return "%s|%d" % (p.name, p.multi_processor_count)


def key(plan: int, n_frames: int, device_tag: str | None = None) -> str:
    in_h, in_w, p, q, taps, dtype = ds.ds_plan_get_params(plan)
    _, (pv, qv, kv), bnd = ds.ds_plan_get_axes(plan)
    return "%s|dt%d|%d/%d|K%d|v%d/%dK%d|b%d|%dx%d|n%d" % (device_tag or _device_tag(), dtype, p, q, taps, pv, qv, kv,
                                                         bnd, in_h, in_w, n_frames)


def load() -> dict:
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save(cache: dict) -> None:
    path = cache_path()
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = path + ".tmp%d" % os.getpid()
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def apply_or_tune(plan: int, in_ptr: int, out_ptr: int, n_frames: int, stream: int = 0, iters: int = 10,
                  device_tag: str | None = None) -> dict:
    """Set the plan's schedule from the cache, tuning (and caching) on a miss.
    Returns the schedule in use: row_blocks (0 = adaptive default band),
    ctas_per_sm (0 = as many as fit), shape, and on a miss the measured
    times (us per launch) of it and of the default schedule.  device_tag:
    the GPU part of the cache key (default: the current device's)."""
    k = key(plan, n_frames, device_tag)
    with _lock:
        e = load().get(k)
    if e and all(f in e for f in ("row_blocks", "ctas_per_sm", "shape")):
        try:
            ds.ds_plan_set_schedule_ex(plan, int(e["row_blocks"]), int(e["ctas_per_sm"]), int(e["shape"]))
            return dict(e, cached=True)
        except (ds.DsError, TypeError, ValueError):
            pass  # an entry this library cannot take (another build's tile shapes): tune again
    r = ds.ds_plan_autotune_ex(plan, in_ptr, out_ptr, n_frames, stream, iters)
    with _lock:
        cache = load()
        cache[k] = r
        save(cache)
    return dict(r, cached=False)


def batch_key(jobs, device_tag: str | None = None) -> str:
    """The cache key of a batch: its jobs' plan keys (with their frame
    counts), in job order."""
    tag = device_tag or _device_tag()
    return "batch[" + ";".join(key(j[0], j[3] if len(j) > 3 else 1, tag) for j in jobs) + "]"


def apply_or_tune_batch(jobs, stream: int = 0, iters: int = 10, device_tag: str | None = None) -> dict:
    """Set the schedules of a batch's plans from the cache, tuning the batch
    as a whole (``ds_batch_autotune``: its jobs share one launch per kernel
    class) on a miss.  jobs: (plan, in_ptr, out_ptr, n_frames) tuples, as for
    ``ds_batch_run``.  Returns the schedule of each job's plan (in job order)
    and, on a miss, the batch's time at it and at the default schedule."""
    jobs = list(jobs)
    k = batch_key(jobs, device_tag)
    with _lock:
        e = load().get(k)
    if e and isinstance(e.get("schedules"), list) and len(e["schedules"]) == len(jobs):
        try:
            for j, sc in zip(jobs, e["schedules"]):
                ds.ds_plan_set_schedule_ex(j[0], int(sc["row_blocks"]), int(sc["ctas_per_sm"]), int(sc["shape"]))
            return dict(e, cached=True)
        except (ds.DsError, TypeError, ValueError, KeyError):
            pass  # an entry this library cannot take: tune again
    r = ds.ds_batch_autotune(jobs, stream, iters)
    with _lock:
        cache = load()
        cache[k] = r
        save(cache)
    return dict(r, cached=False)
