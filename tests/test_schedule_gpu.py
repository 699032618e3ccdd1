"""Schedules on the GPU: every compiled tile shape of every fast class gives
the oracle's results and the same bits as the default shape; the autotuner
never picks a schedule slower than the default on the full-size 1080p fp32
and 4K fp16 batches, nor the batch tuner on the 4:2:0 CIF planes; more direct launches in flight than there are
scheduling slots (queued behind a busy stream) all complete correctly; a
fused launch inside a capture the caller started is refused."""
import numpy as np
import pytest

import paper_1103_4881_b300 as ds
from paper_1103_4881_b300 import synth
from tests.gpu_util import assert_parity, finish, frames, oracle_out, out_buffer, run_fused, stream, to_dev

pytestmark = pytest.mark.gpu

AXES = [((3, 8), 8, (3, 8), 8), ((1, 2), 6, (1, 2), 6), ((2, 3), 6, (2, 3), 6)]
CIF = ((3, 8), 8, (4, 9), 8)
CASES = [(a, dt) for a in AXES for dt in (ds.DS_F32, ds.DS_F16, ds.DS_U8_RGB, ds.DS_U8)] + \
        [(CIF, ds.DS_U8_RGB), (CIF, ds.DS_U8)]


def _oracle(oracle, x, axes, dt):
    rh, Kh, rv, Kv = axes
    xo = x if dt in (ds.DS_U8, ds.DS_U8_RGB) else x.astype(np.float64)
    return oracle.filter_ex(xo, rh, Kh, rv, Kv)


@pytest.mark.parametrize("axes,dt", CASES)
@pytest.mark.parametrize("H,W,n", [(72, 528, 3), (200, 784, 2), (41, 272, 5), (288, 352, 3)])
def test_every_tile_shape_matches_the_oracle_and_shape_0(oracle, axes, dt, H, W, n):
    rh, Kh, rv, Kv = axes
    pl = ds.ds_plan_create_ex(H, W, rh, Kh, rv, Kv, dt)
    try:
        shapes = ds.ds_plan_tile_shapes(pl)
        assert shapes >= 2
        x = frames((H, W), dt, n, H + W + n)
        want = _oracle(oracle, x, axes, dt)
        base = run_fused(pl, x)
        assert_parity(base, want, dt, "shape 0")
        for shape in range(1, shapes):
            for band in (0, 3):  # adaptive, and a short fixed band (several tiles per frame)
                ds.ds_plan_set_schedule_ex(pl, band, 0, shape)
                got = run_fused(pl, x)
                np.testing.assert_array_equal(got, base, err_msg="shape %d band %d" % (shape, band))
    finally:
        ds.ds_destroy(pl)


def _time(fn, st, reps):
    import torch

    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    fn()
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) * 1e3 / reps


@pytest.mark.parametrize("name", ["batch64_1080x1920_f32", "uhd128_2160x3840_f16"])
def test_tuned_schedule_is_no_slower_than_the_default(name):
    import torch

    w = synth.WORKLOADS[name]
    pl = ds.ds_plan_create(w.height, w.width, w.ratio, w.taps, w.dtype)
    try:
        xd = torch.from_numpy(synth.frames(w)).cuda()
        out = out_buffer(pl, w.frames)
        st = stream()
        ds.ds_run_frames(pl, xd.data_ptr(), out.data_ptr(), w.frames, st)
        finish()
        want = out.cpu().numpy()
        r = ds.ds_plan_autotune_ex(pl, xd.data_ptr(), out.data_ptr(), w.frames, st, 10)
        finish()
        assert r["candidates"] >= 10 and r["us_per_launch"] <= r["default_us_per_launch"]
        tuned = (r["row_blocks"], r["ctas_per_sm"], r["shape"])
        run = lambda: ds.ds_run_frames(pl, xd.data_ptr(), out.data_ptr(), w.frames, st)
        t_default, t_tuned = [], []
        for _ in range(5):  # alternate, so drifts of the clock hit both
            ds.ds_plan_set_schedule_ex(pl, 0, 0, 0)
            t_default.append(_time(run, st, 20))
            ds.ds_plan_set_schedule_ex(pl, *tuned)
            t_tuned.append(_time(run, st, 20))
        finish()
        np.testing.assert_array_equal(out.cpu().numpy(), want)
        md, mt = float(np.median(t_default)), float(np.median(t_tuned))
        print("%s: default %.1f us, tuned %s %.1f us" % (name, md, tuned, mt))
        assert mt <= md * 1.03, (md, mt, tuned)
    finally:
        ds.ds_destroy(pl)


def test_batch_tuned_schedule_is_no_slower_than_the_default():
    """The batch tuner on the 2000-frame 4:2:0 CIF workload (Y, U and V planes
    in one launch): the same bits at the tuned schedules, and the batch no
    slower than at the default when the two are re-timed alternately."""
    import torch

    w = synth.WORKLOADS["cif2000_yuv420_u8"]
    plans = [ds.ds_plan_create_ex(h, ww, w.ratio, w.taps, w.vratio, w.vtaps, w.dtype) for h, ww in w.plane_shapes()]
    try:
        ins = [torch.from_numpy(x).cuda() for x in synth.plane_frames(w)]
        outs = [out_buffer(pl, w.frames) for pl in plans]
        jobs = [(pl, i.data_ptr(), o.data_ptr(), w.frames) for pl, i, o in zip(plans, ins, outs)]
        st = stream()
        ds.ds_batch_run(jobs, st)
        finish()
        want = [o.cpu().numpy() for o in outs]
        r = ds.ds_batch_autotune(jobs, st, 10)
        finish()
        assert r["candidates"] >= 10 and r["us_per_launch"] <= r["default_us_per_launch"]
        assert len(r["schedules"]) == 3
        run = lambda: ds.ds_batch_run(jobs, st)
        t_default, t_tuned = [], []
        for _ in range(5):  # alternate, so drifts of the clock hit both
            for pl in plans:
                ds.ds_plan_set_schedule_ex(pl, 0, 0, 0)
            t_default.append(_time(run, st, 20))
            for pl, sc in zip(plans, r["schedules"]):
                ds.ds_plan_set_schedule_ex(pl, sc["row_blocks"], sc["ctas_per_sm"], sc["shape"])
            t_tuned.append(_time(run, st, 20))
        finish()
        for o, x in zip(outs, want):
            np.testing.assert_array_equal(o.cpu().numpy(), x)
        md, mt = float(np.median(t_default)), float(np.median(t_tuned))
        print("yuv batch: default %.1f us, tuned %s %.1f us" % (md, r["schedules"], mt))
        assert mt <= md * 1.03, (md, mt, r["schedules"])
    finally:
        for pl in plans:
            ds.ds_destroy(pl)


def test_batch_autotune_on_a_mixed_batch(oracle):
    """A batch of two fused classes and a plan on the general kernels: the
    tuner sets schedules on the fused plans only, the general plan keeps its
    own, and every output keeps its bits (and matches the oracle)."""
    specs = [((120, 528), (3, 8), 8, ds.DS_F32, 5), ((90, 256), (1, 2), 6, ds.DS_U8_RGB, 7),
             ((77, 100), (3, 4), 4, ds.DS_F32, 3)]
    plans = [ds.ds_plan_create(h, w, r, k, dt) for (h, w), r, k, dt, _ in specs]
    try:
        xs = [frames(hw, dt, n, 300 + j) for j, (hw, _, _, dt, n) in enumerate(specs)]
        ins = [to_dev(x) for x in xs]
        outs = [out_buffer(pl, n) for pl, (_, _, _, _, n) in zip(plans, specs)]
        jobs = [(pl, i.data_ptr(), o.data_ptr(), n) for pl, i, o, (_, _, _, _, n) in zip(plans, ins, outs, specs)]
        st = stream()
        ds.ds_batch_run(jobs, st)
        finish()
        want = [o.cpu().numpy() for o in outs]
        r = ds.ds_batch_autotune(jobs, st, 3)
        finish()
        assert r["candidates"] >= 3 and r["us_per_launch"] <= r["default_us_per_launch"]
        assert ds.ds_plan_get_schedule_ex(plans[2]) == {"row_blocks": 0, "ctas_per_sm": 0, "shape": 0}
        ds.ds_batch_run(jobs, st)
        finish()
        for o, w_, x, ((h, ww), rr, k, dt, n) in zip(outs, want, xs, specs):
            got = o.cpu().numpy()
            np.testing.assert_array_equal(got, w_)
            assert_parity(got, oracle_out(oracle, x, rr[0], rr[1], k, dt), dt, "mixed batch")
    finally:
        for pl in plans:
            ds.ds_destroy(pl)


def test_more_launches_in_flight_than_slots(oracle):
    """640 one-frame fused launches over 4 streams, queued behind a busy
    kernel on each stream, so that more of them are in flight than there are
    direct scheduling slots (512): every output equals the oracle's."""
    import torch

    H, W, n_launch, n_in = 72, 528, 640, 16
    pl = ds.ds_plan_create(H, W, (3, 8), 8, ds.DS_F32)
    try:
        x = frames((H, W), ds.DS_F32, n_in, 640)
        xd = to_dev(x)
        out = out_buffer(pl, n_launch)
        fin, fout = ds.ds_plan_frame_bytes(pl)
        streams = [torch.cuda.Stream() for _ in range(4)]
        ds.ds_run(pl, xd.data_ptr(), out.data_ptr(), stream())  # plan and kernel set-up before the queue
        finish()
        for s in streams:
            with torch.cuda.stream(s):
                torch.cuda._sleep(20_000_000)  # ~10 ms of spinning (a fixed cycle count) per stream
        for k in range(n_launch):
            s = streams[k % 4]
            ds.ds_run(pl, xd.data_ptr() + (k % n_in) * fin, out.data_ptr() + k * fout, s.cuda_stream)
        torch.cuda.synchronize()
        for s in streams:
            ds.ds_stream_check(s.cuda_stream)
        got = out.cpu().numpy()
        want = oracle_out(oracle, x, 3, 8, 8, ds.DS_F32)
        for k in range(n_launch):
            assert_parity(got[k], want[k % n_in], ds.DS_F32, "launch %d" % k)
    finally:
        ds.ds_destroy(pl)


def test_fused_launch_in_a_callers_capture_is_refused():
    import torch

    pl = ds.ds_plan_create(72, 528, (3, 8), 8, ds.DS_F32)
    try:
        x = to_dev(frames((72, 528), ds.DS_F32, 1, 3))
        out = out_buffer(pl, 1)
        ds.ds_run(pl, x.data_ptr(), out.data_ptr(), stream())  # every lookup done before the capture
        finish()
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream()
        refused = None
        with torch.cuda.stream(s):
            with torch.cuda.graph(g, stream=s):
                try:
                    ds.ds_run(pl, x.data_ptr(), out.data_ptr(), s.cuda_stream)
                except ds.DsError as e:
                    refused = e
        assert refused is not None and refused.status == ds.DS_ERR_UNSUPPORTED
        assert "ds_graph_create" in str(refused)
        ds.ds_run(pl, x.data_ptr(), out.data_ptr(), stream())  # the library still works
        finish()
    finally:
        ds.ds_destroy(pl)
