"""Continuous-batching request loop over the libds C ABI (host-side control only).

Requests (one frame each, of any size / ratio / dtype) arrive on an open-loop
schedule.  The loop keeps one plan per request shape resident, admits queued
requests while their device memory fits a budget and a stream slot is free,
and launches every admitted group with one ``ds_batch_run`` (one persistent
launch per kernel class) on that stream, optionally wrapped in the
host-to-device copy of the inputs and the device-to-host copy of the results.
Requests that arrive while earlier batches run are admitted as memory and
stream slots free up, and run on other streams concurrently.  Per-request
latency is arrival -> observed completion.

All filtering happens in the library's kernels; this module only moves
pointers, streams and events (PyTorch supplies memory and streams).

    python -m paper_1103_4881_b300.serve --requests 2000 --rate 5000
"""
from __future__ import annotations

import argparse
import collections
import json
import time
from dataclasses import dataclass, field

import numpy as np

import paper_1103_4881_b300 as ds
from paper_1103_4881_b300 import synth

TORCH_DTYPE_NAMES = {synth.DS_F32: "float32", synth.DS_F16: "float16", synth.DS_U8: "uint8", synth.DS_U8_RGB: "uint8"}


def _torch():
    import torch

    return torch


@dataclass
class Batch:
    stream: object
    event: object
    reqs: list
    outs: list
    host_outs: list
    nbytes: int
    t_launch: float


@dataclass
class Result:
    latency_ms: list = field(default_factory=list)
    completed: int = 0
    wall_s: float = 0.0
    batches: int = 0
    max_batch: int = 0
    max_queue: int = 0
    peak_bytes: int = 0
    alloc_retries: int = 0

    def summary(self) -> dict:
        lat = np.array(self.latency_ms) if self.latency_ms else np.zeros(1)
        return {"requests": self.completed, "frames_per_s": self.completed / max(self.wall_s, 1e-9),
                "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "mean_ms": float(lat.mean()), "batches": self.batches, "max_batch": self.max_batch,
                "max_queue": self.max_queue, "peak_admitted_mb": self.peak_bytes / 1e6, "wall_s": self.wall_s,
                "alloc_retries": self.alloc_retries}


class Server:
    """Resident plans, a device-memory budget and a pool of streams.

    alloc(shape, dtype) -> device tensor allocates every buffer of a batch
    (default torch.empty on the GPU).  When it raises out-of-memory, the
    batch's requests go back to the front of the queue and are admitted again
    once an in-flight batch has completed (or, with nothing in flight, after a
    short wait, up to max_alloc_retries times in a row)."""

    def __init__(self, mem_budget_bytes: int = 4 << 30, n_streams: int = 4, max_batch: int = 64, alloc=None,
                 max_alloc_retries: int = 100):
        torch = _torch()
        self.budget = int(mem_budget_bytes)
        self.max_batch = int(max_batch)
        self.streams = [torch.cuda.Stream() for _ in range(n_streams)]
        self.plans = {}
        self.alloc = alloc or (lambda shape, dtype: torch.empty(shape, dtype=dtype, device="cuda"))
        self.max_alloc_retries = int(max_alloc_retries)

    def close(self):
        for pl in self.plans.values():
            ds.ds_destroy(pl)
        self.plans.clear()

    def plan(self, req) -> int:
        k = (req.height, req.width, req.ratio, req.taps, req.dtype)
        pl = self.plans.get(k)
        if pl is None:
            pl = ds.ds_plan_create(req.height, req.width, req.ratio, req.taps, req.dtype)
            self.plans[k] = pl
        return pl

    def out_shape(self, req):
        oh, ow, c = ds.ds_plan_out_shape(self.plan(req))
        return (oh, ow) if c == 1 else (oh, ow, c)

    def request_bytes(self, req, copies: bool) -> int:
        fin, fout = ds.ds_plan_frame_bytes(self.plan(req))
        return fout + (fin if copies else 0)

    def run(self, requests, inputs, copies: bool = False, realtime: bool = True, keep_outputs: bool = False):
        """Serve `requests` (synth.Request list, arrival order).

        inputs(req) -> tensor: a device tensor (copies=False: inputs already on
        the GPU, the kernel-only mode) or a pinned host tensor (copies=True:
        the copy in, the kernel and the copy out are all part of the request).
        realtime=False makes every request arrive at t=0 (saturation run).
        Returns (Result, {rid: output tensor} if keep_outputs).
        """
        torch = _torch()
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival_s))
        queue = collections.deque()
        free_streams = list(range(len(self.streams)))
        inflight = []
        admitted = 0
        blocked = False  # an allocation failed: admit again after a completion
        failures = 0     # consecutive allocation failures
        res = Result()
        outputs = {}
        for r in requests:  # resident plans before the clock starts
            self.plan(r)
            if self.request_bytes(r, copies) > self.budget:
                raise ValueError("request %d needs more device memory than the budget" % r.rid)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        while pending or queue or inflight:
            now = time.perf_counter() - t0
            while pending and (not realtime or pending[0].arrival_s <= now):
                queue.append(pending.popleft())
            res.max_queue = max(res.max_queue, len(queue))
            # completions
            still = []
            for b in inflight:
                if b.event.query():
                    blocked = False
                    t_done = time.perf_counter() - t0
                    for r in b.reqs:
                        arrival = r.arrival_s if realtime else 0.0
                        res.latency_ms.append(1e3 * (t_done - arrival))
                    res.completed += len(b.reqs)
                    admitted -= b.nbytes
                    free_streams.append(self.streams.index(b.stream))
                    if keep_outputs:
                        for r, o, h in zip(b.reqs, b.outs, b.host_outs):
                            outputs[r.rid] = h if h is not None else o
                else:
                    still.append(b)
            inflight = still
            # admission and launch
            if queue and free_streams and not blocked:
                group, nbytes = [], 0
                while queue and len(group) < self.max_batch:
                    need = self.request_bytes(queue[0], copies)
                    if admitted + nbytes + need > self.budget:
                        break
                    group.append(queue.popleft())
                    nbytes += need
                if group:
                    si = free_streams.pop()
                    st = self.streams[si]
                    try:
                        batch = self._launch(group, st, inputs, copies, nbytes, time.perf_counter() - t0)
                    except (torch.cuda.OutOfMemoryError, MemoryError):
                        # nothing of the batch was launched: requeue it in order
                        free_streams.append(si)
                        queue.extendleft(reversed(group))
                        res.alloc_retries += 1
                        failures += 1
                        if failures > self.max_alloc_retries:
                            raise
                        blocked = bool(inflight)
                        if not inflight:
                            time.sleep(1e-3)
                        continue
                    failures = 0
                    admitted += nbytes
                    res.peak_bytes = max(res.peak_bytes, admitted)
                    inflight.append(batch)
                    res.batches += 1
                    res.max_batch = max(res.max_batch, len(group))
                    continue
            if not (queue and free_streams) or blocked:
                time.sleep(20e-6)
        res.wall_s = time.perf_counter() - t0
        return res, outputs

    def _launch(self, group, st, inputs, copies, nbytes, t_launch) -> Batch:
        torch = _torch()
        jobs, outs, host_outs, keep = [], [], [], []
        with torch.cuda.stream(st):
            # every device buffer first, so an allocation failure launches nothing
            staged = []
            for r in group:
                x = inputs(r)
                xd = self.alloc(x.shape, x.dtype) if copies else x
                out = self.alloc(self.out_shape(r), xd.dtype)
                staged.append((r, x, xd, out))
            for r, x, xd, out in staged:
                if copies:
                    xd.copy_(x, non_blocking=True)
                    keep.append(xd)
                jobs.append((self.plan(r), xd.data_ptr(), out.data_ptr(), 1))
                outs.append(out)
            ds.ds_batch_run(jobs, st.cuda_stream)
            for o in outs:
                if copies:
                    h = torch.empty(o.shape, dtype=o.dtype, pin_memory=True)
                    h.copy_(o, non_blocking=True)
                    host_outs.append(h)
                else:
                    host_outs.append(None)
            ev = torch.cuda.Event()
            ev.record(st)
        # the caching allocator keeps the inputs' blocks until the stream passes them
        for xd in keep:
            xd.record_stream(st)
        for o in outs:
            o.record_stream(st)
        return Batch(st, ev, list(group), outs, host_outs, nbytes, t_launch)

    def per_frame(self, requests, inputs):
        """Baseline: one plain ds_run per request, in arrival order, one stream."""
        torch = _torch()
        outs = []
        st = self.streams[0]
        for r in requests:
            self.plan(r)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with torch.cuda.stream(st):
            for r in requests:
                x = inputs(r)
                out = torch.empty(self.out_shape(r), dtype=x.dtype, device="cuda")
                ds.ds_run(self.plan(r), x.data_ptr(), out.data_ptr(), st.cuda_stream)
                outs.append(out)
        st.synchronize()
        return len(requests) / (time.perf_counter() - t0)


class FramePool:
    """Seeded request content: a few distinct frames per (size, dtype), reused
    by request id, resident on the device (and pinned on the host for the
    end-to-end mode)."""

    def __init__(self, requests, per_class: int = 4, host: bool = False, seed: int = 6000):
        torch = _torch()
        self.dev, self.host = {}, {}
        g = torch.Generator(device="cuda")
        for r in requests:
            k = (r.height, r.width, r.dtype)
            if k in self.dev:
                continue
            shape = (r.height, r.width) if synth.CHANNELS[r.dtype] == 1 else (r.height, r.width, 3)
            frames = []
            for i in range(per_class):
                g.manual_seed(seed + 7919 * len(self.dev) + i)
                if r.dtype in (synth.DS_U8, synth.DS_U8_RGB):
                    t = torch.randint(0, 256, shape, generator=g, device="cuda", dtype=torch.uint8)
                else:
                    t = torch.rand(shape, generator=g, device="cuda").to(getattr(torch, TORCH_DTYPE_NAMES[r.dtype]))
                frames.append(t)
            self.dev[k] = frames
            if host:
                self.host[k] = [f.cpu().pin_memory() for f in frames]
        self.per_class = per_class

    def device(self, r):
        return self.dev[(r.height, r.width, r.dtype)][r.rid % self.per_class]

    def pinned(self, r):
        return self.host[(r.height, r.width, r.dtype)][r.rid % self.per_class]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--requests", type=int, default=2000)
    ap.add_argument("--rate", type=float, default=5000.0)
    ap.add_argument("--streams", type=int, default=4)
    ap.add_argument("--max-batch", type=int, default=64)
    ap.add_argument("--budget-gb", type=float, default=8.0)
    args = ap.parse_args()
    reqs = synth.serving_requests(args.requests, args.rate)
    pool = FramePool(reqs, host=True)
    srv = Server(int(args.budget_gb * (1 << 30)), args.streams, args.max_batch)
    try:
        # warm-up: one request of every (size, ratio, dtype) in the mix, so that
        # each plan is made and each kernel class loaded before the timed runs
        kinds = {}
        for r in reqs:
            kinds.setdefault((r.height, r.width, tuple(r.ratio), r.taps, r.dtype), r)
        srv.run(list(kinds.values()), pool.device, realtime=False)
        srv.run(reqs[:64], pool.device, realtime=False)  # and the allocator at batch sizes
        out = {"config": {"workload": "serving mix", "requests": args.requests, "rate_hz": args.rate,
                          "streams": args.streams, "max_batch": args.max_batch, "budget_gb": args.budget_gb}}
        r, _ = srv.run(reqs, pool.device, realtime=True)
        out["open_loop_kernel_only"] = r.summary()
        r, _ = srv.run(reqs, pool.pinned, copies=True, realtime=True)
        out["open_loop_end_to_end"] = r.summary()
        r, _ = srv.run(reqs, pool.device, realtime=False)
        out["saturation_batched"] = r.summary()
        out["saturation_per_frame_fps"] = srv.per_frame(reqs, pool.device)
        print(json.dumps(out), flush=True)
    finally:
        srv.close()


if __name__ == "__main__":
    main()
