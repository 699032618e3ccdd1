"""Persistent cache of autotuned tile schedules (host-side file IO only).

The tuning itself is ``ds_plan_autotune`` in the library (CUDA events over
candidate band heights).  The cache keeps its choice per GPU model, SM count,
dtype, ratio, taps, frame size and batch size, in the JSON file named by
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
    return "%s|dt%d|%d/%d|K%d|%dx%d|n%d" % (device_tag or _device_tag(), dtype, p, q, taps, in_h, in_w, n_frames)


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


def apply_or_tune(plan: int, in_ptr: int, out_ptr: int, n_frames: int, stream: int = 0, iters: int = 10) -> int:
    """Set the plan's band height from the cache, tuning (and caching) on a miss.
    Returns the band height in use."""
    k = key(plan, n_frames)
    with _lock:
        cache = load()
        if k in cache:
            ds.ds_plan_set_schedule(plan, int(cache[k]["row_blocks"]), 0)
            return int(cache[k]["row_blocks"])
    rb, us = ds.ds_plan_autotune(plan, in_ptr, out_ptr, n_frames, stream, iters)
    with _lock:
        cache = load()
        cache[k] = {"row_blocks": rb, "us_per_launch": us}
        save(cache)
    return rb
