#!/usr/bin/env python3
"""Benchmark of the fused horizontal + vertical decimating FIR (the downscaler
filter stage of arXiv:1103.4881, Sec. 3) on one B300 per rank.

Headline workload (default): 128 fp16-storage frames of 2160x3840, uniform
[0,1) plus N(0, 0.05) noise, clipped; 3/8 decimation with 8 Lanczos-3 taps
per phase on both axes -> 810x1440 fp16, FP32 accumulation.  The plan's
schedule (tile shape, band, CTAs per SM) comes from the autotuner (cached
per GPU and workload).  One step = one batched persistent launch over the
128 frames, replayed from a CUDA graph; inputs (2.1 GB per step) are far
larger than the 126 MB L2, so every step streams them from HBM.

Prints one JSON line (rank 0): frames/s, with the roofline of the fused
kernel, the clocks seen during the timed region, the error against the FP64
oracle on a seeded sample of frames, the end-to-end figure through the
host-buffer pipeline, the plain per-frame and unfused forms, the CPU oracle
as a baseline, and (key "workloads") the same device-timed batched figures,
roofline and error for the other workloads: 64 x 1080p fp32 3/8, 300 x
1080p uint8 RGB 1/2, and the paper's 2000 CIF frames as RGB and as YUV
4:2:0.  --impl reference times the CPU oracle alone.
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
HEADLINE = "uhd128_2160x3840_f16"
SIDE_WORKLOADS = ("batch64_1080x1920_f32", "rgb300_1080x1920_u8", "cif2000_352x288_u8rgb", "cif2000_yuv420_u8")


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=HEADLINE)
    ap.add_argument("--frames", type=int, default=0, help="override the workload's frame count (profiling)")
    ap.add_argument("--no-extras", action="store_true", help="skip per-frame / unfused / e2e / cpu legs")
    ap.add_argument("--no-side", action="store_true", help="skip the other workloads (key workloads)")
    ap.add_argument("--no-tune", action="store_true", help="the plan's default schedule, not the autotuner's")
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
    import glob

    csrc = os.path.join(ROOT, "paper_1103_4881_b300", "csrc")
    names = sorted(os.path.basename(f) for f in glob.glob(os.path.join(csrc, "rows*")))
    for name in names + ["fused_fast.cu", "pixel.cuh", "internal.h", "plan.cpp"]:  # kernels and their schedule
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_capture(workload: str, schedule=None):
    """The committed one-pass ncu capture of a workload's launch (DRAM bytes,
    warp instructions) taken on the current kernel source with the same
    schedule, or None."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        entries = d.get(workload) or []
        if isinstance(entries, dict):
            entries = [entries]
        h = kernel_source_hash()
        for e in entries:
            if e.get("kernel_source_hash") != h:
                continue
            if schedule is not None and e.get("schedule") is not None and e["schedule"] != schedule:
                continue
            return e
    except Exception:
        pass
    return None


def profiled_traffic(workload: str, schedule=None):
    """DRAM bytes per launch from the committed ncu captures (one entry per
    workload and schedule), if one was taken on the current kernel source
    with the same schedule (else None)."""
    e = profiled_capture(workload, schedule)
    return int(e["dram_bytes_per_launch"]) if e else None


def issue_roofline(workload: str, schedule, launch_s: float, clocks: dict, sms: int):
    """Instruction issue against its peak: the launch's warp instructions
    (committed capture) per second of the CUDA-event launch time, against
    4 schedulers x 1 warp instruction per clock x the SM count x the median
    SM clock sampled during the timed region.  The bound of the uint8
    classes, whose HBM fraction alone understates how busy they are."""
    e = profiled_capture(workload, schedule)
    mhz = clocks.get("sm_mhz")
    if not e or "warp_instructions_per_launch" not in e or not mhz or launch_s <= 0:
        return None
    inst = int(e["warp_instructions_per_launch"])
    peak = 4.0 * sms * mhz * 1e6 / 1e9
    achieved = inst / launch_s / 1e9
    return {"bound": "issue", "achieved": achieved, "peak": peak, "unit": "G warp instructions/s",
            "frac": achieved / peak, "warp_instructions_per_launch": inst,
            "peak_source": "4 schedulers x 1 warp instruction per clock x %d SMs x %.0f MHz (median SM clock of "
                           "the timed region)" % (sms, mhz)}


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
        "config": workload_config(w, w.frames, world),
        "cpu_baseline": {"value": value, "unit": "frames/s", "cores": cores, "kind": "oracle",
                         "sample": "per step: the first %d rows of %d frames (all planes), one band per thread"
                                   % (rows, samples[0].shape[0])},
        "e2e": {"value": value, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def workload_config(w, n, world=1):
    """The config block of the JSON line (the same in both arms)."""
    from paper_1103_4881_b300 import synth

    in_bytes = n * sum(h * ww * w.channels * synth.NP_DTYPE[w.dtype]().itemsize for h, ww in w.plane_shapes())
    cfg = {"workload": w.name, "frames_per_step": n, "in": [w.height, w.width, w.channels],
           "out": list(w.out_frame_shape()) + ([1] if w.channels == 1 else []),
           "ratio": "%d/%d" % w.ratio, "taps": w.taps,
           "l2": ("inputs larger than L2 (%.0f MB per step vs 126 MB)" if in_bytes > 126e6 else
                  "inputs smaller than L2 (%.0f MB per step vs 126 MB): not an HBM figure") % (in_bytes / 1e6),
           "parallelism": ("dp%d: frames sharded over ranks, no data-path collective" % world) if world > 1
           else "single"}
    if w.ratio_v:
        cfg["ratio_v"] = "%d/%d" % w.vratio
        cfg["taps_v"] = w.vtaps
    if w.planes:
        cfg["planes"] = [list(hw) for hw in w.plane_shapes()]
    return cfg


def sample_frames(n: int, k: int = 16, seed: int = 12345):
    """A seeded sample of k frames plus the first and the last."""
    import numpy as np

    if n <= k + 2:
        return list(range(n))
    mid = np.random.default_rng(seed).choice(np.arange(1, n - 1), size=k, replace=False)
    return sorted({0, n - 1, *mid.tolist()})


def accuracy(w, xs, outs, a):
    """Error against the FP64 / integer oracle on a seeded sample of frames of
    every plane (outside any timed region): max |err| for float data (full
    scale 1.0), mismatched bytes for uint8."""
    import numpy as np
    from paper_1103_4881_b300 import synth

    n = xs[0].shape[0]
    idx = sample_frames(n)
    u8 = w.dtype in (synth.DS_U8, synth.DS_U8_RGB)
    err, bad, total = 0.0, 0, 0
    for x, o in zip(xs, outs):
        got = o[idx].cpu().numpy()
        want = oracle_filter(w, x[idx])
        total += got.size
        if u8:
            bad += int(np.count_nonzero(got != want))
        else:
            err = max(err, float(np.abs(got.astype(np.float64) - want).max()))
    out = {"vs": "oracle (FP64 loop nest; int64 for uint8)", "frames": [a + i for i in idx],
           "sample": "%d seeded frames plus the first and the last, every plane" % max(0, len(idx) - 2)}
    if u8:
        out.update(mismatched_bytes=bad, compared_bytes=total, bound="bit-exact")
    else:
        out.update(max_abs_err=err, compared_values=total, bound=1e-6 if w.dtype == synth.DS_F32 else 2e-3,
                   full_scale=1.0)
    return out


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
    from paper_1103_4881_b300 import build, shard, tune

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
    peak, peak_src = measured_peak()
    stream = torch.cuda.current_stream()
    st = stream.cuda_stream

    def resident(wl, a, b):
        """Plans (one per plane), the frames [a, b) on the host and on the
        device, and their output buffers."""
        shapes = wl.plane_shapes()
        plans = [ds.ds_plan_create_ex(h, ww, wl.ratio, wl.taps, wl.vratio, wl.vtaps, wl.dtype) for h, ww in shapes]
        xs = synth.plane_frames(wl, range(a, b))
        xins = [torch.from_numpy(x).cuda() for x in xs]
        outs = [torch.empty((b - a,) + wl.plane_out_shape(hw), dtype=xins[0].dtype, device="cuda") for hw in shapes]
        return plans, xs, xins, outs

    def clock_warm(fn, ms=20.0):
        # keep the GPU busy right before a timed region: after an idle gap
        # (a sync, the clock sampler starting) its clocks take a moment to
        # come back up, which would land inside a short timed region
        t = time.perf_counter()
        while (time.perf_counter() - t) * 1e3 < ms:
            fn()
            torch.cuda.synchronize()

    def timed(fn, k, barrier=True):
        clock_warm(fn)
        if pg and barrier:
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
        if pg and barrier:
            t = torch.tensor([ms], device="cuda")
            pg.all_reduce(t, op=pg.ReduceOp.MAX)
            ms = float(t.item())
        return ms

    # weak scaling: the job is world x w.frames frames, each rank filters its own
    # contiguous share (global frame indices, so no two ranks hold the same frame)
    a, b = shard.frame_range(w.frames * world, world, rank)
    n = b - a
    plans, xs, xins, outs = resident(w, a, b)
    fbytes = [ds.ds_plan_frame_bytes(pl) for pl in plans]
    fin = fbytes[0][0]

    # the schedule: the autotuner's choice for this GPU and workload (cached)
    schedule = tuned_schedules(args, ds, tune, plans, xins, outs, n, st)
    for sc, pl in zip(schedule, plans):
        sc["describe"] = json.loads(ds.ds_plan_describe(pl))

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
    sched_key = [{k: sc[k] for k in ("row_blocks", "ctas_per_sm", "shape")} for sc in schedule]
    # the committed capture is of the full workload's launch: none for a resized one
    traffic = profiled_traffic(w.name, sched_key) if n == synth.WORKLOADS[w.name].frames else None

    line = {
        "metric": "frames/s", "value": value, "unit": "frames/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {0: "f32", 1: "f16", 2: "u8", 3: "u8"}[w.dtype], "data": "synthetic",
        "config": workload_config(w, n, world),
        "timing": {"form": "batched persistent fused H+V kernel, CUDA graph replay",
                   "warm": "W warm-up steps, then about 20 ms more of untimed steps right before the timed region",
                   "events": "CUDA events on the launching stream around the K steps"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": traffic, "peak_source": peak_src,
                     "alg_bytes_per_launch": alg_bytes, "kernel_us": launch_s * 1e6},
        "clocks": clk,
        "gpu_launches": launches,
        "schedule": schedule,
    }
    if n == synth.WORKLOADS[w.name].frames:
        line["issue_roofline"] = issue_roofline(w.name, sched_key, launch_s, clk,
                                                torch.cuda.get_device_properties(dev_index).multi_processor_count)

    if rank == 0:
        line["accuracy"] = accuracy(w, xs, outs, a)
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
        ms_pf = timed(per_frame, k2, barrier=False)
        # unfused two-kernel form over the batch
        wsb = max(ds.ds_plan_workspace_bytes(pl) for pl in plans) * n
        ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
        def unfused():
            for pl, xi, o in zip(plans, xins, outs):
                ds.ds_run_unfused(pl, xi.data_ptr(), o.data_ptr(), n, ws.data_ptr(), wsb, st)
        unfused()
        ms_uf = timed(unfused, k2, barrier=False)
        del ws
        # batched without the graph (direct launch)
        def direct():
            ds.ds_batch_run(job, st)
        direct()
        ms_dl = timed(direct, k2, barrier=False)
        line["forms"] = {
            "batched_graph_fps": value / world,
            "batched_direct_fps": n * k2 / (ms_dl / 1e3),
            "per_frame_fused_fps": n * k2 / (ms_pf / 1e3),
            "unfused_two_kernel_fps": n * k2 / (ms_uf / 1e3),
            "unfused_alg_gbs": alg_bytes * k2 / (ms_uf / 1e3) / 1e9,
        }
        # end to end through the C ABI with pinned host buffers (copies in the timed region)
        host_ins = [torch.from_numpy(xx).pin_memory() for xx in xs]
        host_outs = [torch.empty(tuple(o.shape), dtype=o.dtype).pin_memory() for o in outs]
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
    del xins, outs, xs

    if rank == 0 and world == 1 and not args.no_side:
        line["workloads"] = side_workloads(args, ds, synth, resident, timed, dev_index, peak)

    if rank == 0:
        print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()


def tuned_schedules(args, ds, tune, plans, xins, outs, n, st):
    """The autotuner's schedule for a workload's plans (cached per GPU): one
    plan is tuned alone, the planes of a planar workload as one batch (they
    share a launch, whose bands and tail a plan tuned alone does not see);
    with --no-tune, the plans' defaults.  One entry per plan."""
    if args.no_tune:
        return [dict(ds.ds_plan_get_schedule_ex(pl), tuned=False) for pl in plans]
    if len(plans) > 1:
        r = tune.apply_or_tune_batch([(pl, xi.data_ptr(), o.data_ptr(), n) for pl, xi, o in zip(plans, xins, outs)],
                                     st, 10)
        extra = {k: r[k] for k in ("us_per_launch", "default_us_per_launch", "candidates", "cached") if k in r}
        return [dict(sc, tuned=True, batch=True, **extra) for sc in r["schedules"]]
    pl, xi, o = plans[0], xins[0], outs[0]
    return [dict(tune.apply_or_tune(pl, xi.data_ptr(), o.data_ptr(), n, st, 10), tuned=True)]


def side_workloads(args, ds, synth, resident, timed, dev_index, peak):
    """The other workloads, each as its own batched graph launch at the
    autotuner's schedule (as the headline; the default with --no-tune):
    device time per launch, roofline against the measured copy peak, DRAM
    traffic from the committed capture, the clocks during its timed region
    and its error against the oracle."""
    import torch

    from paper_1103_4881_b300 import tune

    st = torch.cuda.current_stream().cuda_stream
    res = {}
    for name in SIDE_WORKLOADS:
        if name == args.workload:
            continue
        wl = synth.WORKLOADS[name]
        plans, xs, xins, outs = resident(wl, 0, wl.frames)
        fbytes = [ds.ds_plan_frame_bytes(pl) for pl in plans]
        alg = wl.frames * sum(fi + fo for fi, fo in fbytes)
        tuned = tuned_schedules(args, ds, tune, plans, xins, outs, wl.frames, st)
        g = ds.ds_graph_create([(pl, xi.data_ptr(), o.data_ptr(), wl.frames) for pl, xi, o in zip(plans, xins, outs)])
        step = lambda: ds.ds_graph_launch(g, st)
        for _ in range(max(3, args.warmup)):
            step()
        torch.cuda.synchronize()
        ds.ds_stream_check(st)
        # at least a quarter of a second of steps, so the clock sampler sees the region
        est = timed(step, 5, barrier=False) / 5
        k = max(args.steps, int(250.0 / max(est, 1e-3)))
        with ClockSampler(dev_index) as clocks:
            ms = timed(step, k, barrier=False)
        ds.ds_stream_check(st)
        us = ms * 1e3 / k
        sched = [{k_: v for k_, v in ds.ds_plan_get_schedule_ex(pl).items()} for pl in plans]
        res[name] = {
            "frames_per_launch": wl.frames, "steps": k, "kernel_us": us, "frames_per_s": wl.frames / (us * 1e-6),
            "alg_bytes_per_launch": alg, "achieved_gbs": alg / (us * 1e-6) / 1e9,
            "frac": alg / (us * 1e-6) / 1e9 / peak, "traffic": profiled_traffic(name, sched),
            "clocks": clocks.summary(), "schedule": tuned,
            "accuracy": accuracy(wl, xs, outs, 0),
        }
        res[name]["issue_roofline"] = issue_roofline(name, sched, us * 1e-6, res[name]["clocks"],
                                                     torch.cuda.get_device_properties(dev_index).multi_processor_count)
        ds.ds_graph_destroy(g)
        for pl in plans:
            ds.ds_destroy(pl)
        del xs, xins, outs
        torch.cuda.empty_cache()
    return res


if __name__ == "__main__":
    main()
