#!/usr/bin/env python3
"""Benchmark of the fused horizontal + vertical decimating FIR (the downscaler
filter stage of arXiv:1103.4881, Sec. 3) on one B300 per rank.

Workload (default): 64 fp32 frames of 1080x1920, uniform [0,1) plus a seeded
smooth gradient, 3/8 decimation with 8 Lanczos-3 taps per phase -> 405x720.
One step = one batched persistent launch over the 64 frames, replayed from a
CUDA graph.  Inputs (531 MB per step) are larger than the 126 MB L2, so every
step streams them from HBM.

Prints one JSON line (rank 0): frames/s, with the roofline of the fused
kernel, the clocks seen during the timed region, the end-to-end figure
through the host-buffer pipeline, the plain per-frame and unfused forms, and
the CPU oracle as a baseline.  --impl reference times the CPU oracle alone.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

FALLBACK_HBM_GBS = 6400.0


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="batch64_1080x1920_f32")
    ap.add_argument("--frames", type=int, default=0, help="override the workload's frame count (profiling)")
    ap.add_argument("--no-extras", action="store_true", help="skip per-frame / unfused / e2e / cpu legs")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs: torch copy, read+write)"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback (no MEASURED_PEAKS.json)"


def kernel_source_hash():
    import hashlib

    h = hashlib.sha256()
    for name in ("fused_fast.cu", "pixel.cuh", "internal.h", "plan.cpp"):  # kernels and their schedule
        with open(os.path.join(ROOT, "paper_1103_4881_b300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_traffic(workload: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on
    the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        e = d.get(workload)
        if e and e.get("kernel_source_hash") == kernel_source_hash():
            return int(e["dram_bytes_per_launch"])
    except Exception:
        pass
    return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(0.1)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if not self.path or not os.path.exists(self.path):
            return out
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        if sm:
            out.update(sm_mhz=statistics.median(sm), sm_max_mhz=max(smax), reasons=sorted(reasons), samples=len(sm))
        return out


def oracle_filter(w, x, threads=0):
    """The oracle on one plane of workload w (its ratio and taps per axis)."""
    import oracle
    from paper_1103_4881_b300 import synth

    if w.dtype in (synth.DS_U8, synth.DS_U8_RGB):
        return oracle.filter_ex(x, w.ratio, w.taps, w.vratio, w.vtaps, threads=threads)
    return oracle.filter_ex(x.astype("float64"), w.ratio, w.taps, w.vratio, w.vtaps, threads=threads)


def time_cpu_oracle(w, budget_s=15.0):
    """The oracle as it stands on this host's cores: whole frames of the
    workload (every plane), OpenMP over frames, as many frames as fit the
    time budget."""
    import oracle
    from paper_1103_4881_b300 import synth

    cores = max(1, oracle.max_threads())
    first = synth.plane_frames(w, range(1))
    for x in first:  # once untimed: the first call pays for loading and first touches
        oracle_filter(w, x, threads=1)
    t = time.perf_counter()
    for x in first:
        oracle_filter(w, x, threads=1)
    one = time.perf_counter() - t
    del first
    # as many distinct frames as a pass of half the budget allows (so the
    # sample streams through memory like the workload, not from the host's caches)
    n = int(max(1, min(w.frames, cores * max(1, int(0.5 * budget_s / max(one, 1e-4) / max(cores, 1))))))
    n = max(1, min(n, w.frames))
    xs = synth.plane_frames(w, range(n))
    # whole passes over the sample until about the time budget is spent
    passes, t = 0, time.perf_counter()
    while True:
        for x in xs:
            oracle_filter(w, x, threads=0)
        passes += 1
        dt = time.perf_counter() - t
        if dt >= 0.66 * budget_s or passes >= 1000:
            break
    del xs
    return {"value": passes * n / dt, "unit": "frames/s", "cores": cores, "kind": "oracle",
            "sample": "%d pass(es) over %d of the workload's %d frames (whole frames, FP64 / int64 loop nest, "
                      "OpenMP over frames)" % (passes, n, w.frames),
            "seconds": round(dt, 3),
            "one_core": {"value": 1.0 / max(one, 1e-9), "unit": "frames/s", "sample": "frame 0, one thread"}}


def reference_arm(args, w, rank, world):
    """--impl reference: the CPU oracle, timed alone, on the same metric."""
    if rank != 0:
        return
    import oracle
    from paper_1103_4881_b300 import synth

    cores = max(1, oracle.max_threads())
    # one step = a band of rows from `cores` frames (one band per thread) of
    # every plane, sized so that warmup + steps take about a minute in total
    planes = synth.plane_frames(w, range(min(cores, w.frames)))
    qv = w.vratio[1]
    t = time.perf_counter()
    for x in planes:
        oracle_filter(w, x[:1, : 8 * qv], threads=1)
    per_row = (time.perf_counter() - t) / (8 * qv)  # per row of the first plane, all planes
    total = max(1, args.steps + args.warmup)
    rows = int(60.0 / total / max(per_row, 1e-9))
    rows = max(qv, min(w.height, rows - rows % qv))
    frac = rows / w.height
    samples = []
    for x in planes:
        r = max(qv, int(round(x.shape[1] * frac)) // qv * qv)
        samples.append(x[:, : min(r, x.shape[1])])
    for _ in range(args.warmup):
        for x in samples:
            oracle_filter(w, x, threads=0)
    t = time.perf_counter()
    for _ in range(args.steps):
        for x in samples:
            oracle_filter(w, x, threads=0)
    dt = time.perf_counter() - t
    frames_per_step = samples[0].shape[0] * rows / w.height
    value = frames_per_step * args.steps / dt
    line = {
        "impl": "reference", "metric": "frames/s", "value": value, "unit": "frames/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if w.dtype in (0, 1) else "int64", "data": "synthetic",
        "config": workload_config(w, w.frames),
        "cpu_baseline": {"value": value, "unit": "frames/s", "cores": cores, "kind": "oracle",
                         "sample": "per step: the first %d rows of %d frames (all planes), one band per thread"
                                   % (rows, samples[0].shape[0])},
        "e2e": {"value": value, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def workload_config(w, n):
    """The config block of the JSON line."""
    cfg = {"workload": w.name, "frames_per_step": n, "in": [w.height, w.width, w.channels],
           "out": list(w.out_frame_shape()) + ([1] if w.channels == 1 else []),
           "ratio": "%d/%d" % w.ratio, "taps": w.taps}
    if w.ratio_v:
        cfg["ratio_v"] = "%d/%d" % w.vratio
        cfg["taps_v"] = w.vtaps
    if w.planes:
        cfg["planes"] = [list(hw) for hw in w.plane_shapes()]
    return cfg


def main():
    args = parse_args()
    rank, world, local = dist_env()
    from paper_1103_4881_b300 import synth

    w = synth.WORKLOADS[args.workload]
    if args.frames > 0:
        import dataclasses

        w = dataclasses.replace(w, frames=args.frames)
    if args.impl == "reference":
        reference_arm(args, w, rank, world)
        return

    import numpy as np
    import torch

    import paper_1103_4881_b300 as ds
    from paper_1103_4881_b300 import build

    if rank == 0:
        build.build()
    torch.cuda.set_device(local)
    pg = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        pg = dist
        dist.barrier()
    dev_index = torch.cuda.current_device()

    # one plan per plane (a single plane unless the workload is planar)
    shapes = w.plane_shapes()
    plans = [ds.ds_plan_create_ex(h, ww, w.ratio, w.taps, w.vratio, w.vtaps, w.dtype) for h, ww in shapes]
    plan = plans[0]
    fbytes = [ds.ds_plan_frame_bytes(pl) for pl in plans]
    fin, fout = fbytes[0]
    # weak scaling: the job is world x w.frames frames, each rank filters its own
    # contiguous share (global frame indices, so no two ranks hold the same frame)
    from paper_1103_4881_b300 import shard

    a, b = shard.frame_range(w.frames * world, world, rank)
    n = b - a
    xs = synth.plane_frames(w, range(a, b))
    xins = [torch.from_numpy(x).cuda() for x in xs]
    outs = [torch.empty((n,) + w.plane_out_shape(hw), dtype=xins[0].dtype, device="cuda") for hw in shapes]
    x, xin, out = xs[0], xins[0], outs[0]
    stream = torch.cuda.current_stream()
    st = stream.cuda_stream

    # the step: one batched persistent launch over the n frames (of every
    # plane), replayed as a CUDA graph
    job = [(pl, xi.data_ptr(), o.data_ptr(), n) for pl, xi, o in zip(plans, xins, outs)]
    graph = ds.ds_graph_create(job)

    def step():
        ds.ds_graph_launch(graph, st)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    ds.ds_stream_check(st)

    def clock_warm(fn, ms=20.0):
        # keep the GPU busy right before a timed region: after an idle gap
        # (a sync, the clock sampler starting) its clocks take a moment to
        # come back up, which would land inside a short timed region
        t = time.perf_counter()
        while (time.perf_counter() - t) * 1e3 < ms:
            fn()
            torch.cuda.synchronize()

    def timed(fn, k):
        clock_warm(fn)
        if pg:
            pg.barrier()
        torch.cuda.synchronize()
        ds.ds_launch_count()  # count the timed steps' launches only
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(k):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        if pg:
            t = torch.tensor([ms], device="cuda")
            pg.all_reduce(t, op=pg.ReduceOp.MAX)
            ms = float(t.item())
        return ms

    with ClockSampler(dev_index) as clocks:
        ms = timed(step, args.steps)
    launches = ds.ds_launch_count()
    ds.ds_stream_check(st)
    clk = clocks.summary()

    frames_total = n * world * args.steps
    value = frames_total / (ms / 1e3)
    alg_bytes = n * sum(fi + fo for fi, fo in fbytes)  # input read once + output written once, per launch
    launch_s = ms / 1e3 / args.steps
    achieved = alg_bytes / launch_s / 1e9
    peak, peak_src = measured_peak()
    # the committed capture is of the full workload's launch: none for a resized one
    traffic = profiled_traffic(w.name) if n == synth.WORKLOADS[w.name].frames else None

    line = {
        "metric": "frames/s", "value": value, "unit": "frames/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {0: "f32", 1: "f16", 2: "u8", 3: "u8"}[w.dtype], "data": "synthetic",
        "config": dict(workload_config(w, n), **{
                   "form": "batched persistent fused H+V kernel, CUDA graph replay",
                   "warm": "W warm-up steps, then about 20 ms more of untimed steps right before the timed region",
                   "l2": ("inputs larger than L2 (%.0f MB per step vs 126 MB)" if n * sum(f[0] for f in fbytes) > 126e6
                          else "inputs smaller than L2 (%.0f MB per step vs 126 MB): not an HBM figure")
                         % (n * sum(f[0] for f in fbytes) / 1e6),
                   "parallelism": ("dp%d: frames sharded over ranks, no data-path collective" % world) if world > 1 else "single"}),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": traffic, "peak_source": peak_src,
                     "alg_bytes_per_launch": alg_bytes, "kernel_us": launch_s * 1e6},
        "clocks": clk,
        "gpu_launches": launches,
    }

    if rank == 0 and not args.no_extras:
        # enough repetitions for at least 256 frames per form (a 1-frame workload
        # would otherwise time a few launches, dominated by host jitter)
        k2 = max(5, min(args.steps // 50, 50), -(-256 // n))
        # plain per-frame: one ds_run per frame (and plane)
        def per_frame():
            for i in range(n):
                for pl, xi, o, (fi, fo) in zip(plans, xins, outs, fbytes):
                    ds.ds_run(pl, xi.data_ptr() + i * fi, o.data_ptr() + i * fo, st)
        per_frame()
        ms_pf = timed(per_frame, k2)
        # unfused two-kernel form over the batch
        wsb = max(ds.ds_plan_workspace_bytes(pl) for pl in plans) * n
        ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
        def unfused():
            for pl, xi, o in zip(plans, xins, outs):
                ds.ds_run_unfused(pl, xi.data_ptr(), o.data_ptr(), n, ws.data_ptr(), wsb, st)
        unfused()
        ms_uf = timed(unfused, k2)
        del ws
        # batched without the graph (direct launch)
        def direct():
            ds.ds_batch_run(job, st)
        direct()
        ms_dl = timed(direct, k2)
        line["forms"] = {
            "batched_graph_fps": value / world,
            "batched_direct_fps": n * k2 / (ms_dl / 1e3),
            "per_frame_fused_fps": n * k2 / (ms_pf / 1e3),
            "unfused_two_kernel_fps": n * k2 / (ms_uf / 1e3),
            "unfused_alg_gbs": alg_bytes * k2 / (ms_uf / 1e3) / 1e9,
        }
        # end to end through the C ABI with pinned host buffers (copies in the timed region)
        host_ins = [torch.from_numpy(xx).pin_memory() for xx in xs]
        host_outs = [torch.empty((n,) + w.plane_out_shape(hw), dtype=xin.dtype).pin_memory() for hw in shapes]
        chunk = 4 if fin > (1 << 20) else 64  # frames per pipeline chunk
        pipes = [ds.ds_pipeline_create(pl, chunk, 3) for pl in plans]
        def e2e_step():
            for pp, hi, ho in zip(pipes, host_ins, host_outs):
                ds.ds_pipeline_run(pp, hi.data_ptr(), ho.data_ptr(), n)
        e2e_step()
        k3 = 5
        t = time.perf_counter()
        for _ in range(k3):
            e2e_step()
        dt = time.perf_counter() - t
        for pp in pipes:
            ds.ds_pipeline_destroy(pp)
        line["e2e"] = {"value": n * k3 / dt, "unit": "frames/s", "h2d_bytes_per_step": n * sum(f[0] for f in fbytes),
                       "d2h_bytes_per_step": n * sum(f[1] for f in fbytes),
                       "api": "ds_pipeline_run (%d-frame chunks, 3 streams, per plane)" % chunk}
        ok = all(np.array_equal(ho.numpy(), o.cpu().numpy()) for ho, o in zip(host_outs, outs))
        line["e2e"]["matches_device_path"] = bool(ok)
        del host_ins, host_outs
        if world == 1:
            line["cpu_baseline"] = time_cpu_oracle(w)
    elif world > 1:
        line["e2e"] = None

    ds.ds_graph_destroy(graph)
    for pl in plans:
        ds.ds_destroy(pl)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
