"""Full-size workloads on the GPU, in the launch configuration the benchmark
uses (one batched launch over all frames of the workload), checked against
the CPU oracle on every frame (fp32 batch) or on a seeded sample of 16
frames plus the first and the last (the large uint8 / fp16 batches).
"""
import numpy as np
import pytest

import paper_1103_4881_b300 as ds
from paper_1103_4881_b300 import synth
from tests.gpu_util import assert_parity, finish, oracle_out, out_buffer, stream

pytestmark = pytest.mark.gpu


def _run_workload(w, graph=False):
    import torch

    pl = ds.ds_plan_create(w.height, w.width, w.ratio, w.taps, w.dtype)
    x = synth.frames(w)
    xd = torch.from_numpy(x).cuda()
    out = out_buffer(pl, w.frames)
    if graph:
        g = ds.ds_graph_create([(pl, xd.data_ptr(), out.data_ptr(), w.frames)])
        try:
            ds.ds_graph_launch(g, stream())
            finish()
        finally:
            ds.ds_graph_destroy(g)
    else:
        ds.ds_run_frames(pl, xd.data_ptr(), out.data_ptr(), w.frames, stream())
        finish()
    return pl, x, xd, out


def _sample(w, k, seed):
    rng = np.random.default_rng(seed)
    mid = rng.choice(np.arange(1, w.frames - 1), size=min(k, w.frames - 2), replace=False)
    return sorted({0, w.frames - 1, *mid.tolist()})


def test_plain_480x640_f32(oracle):
    w = synth.WORKLOADS["plain_480x640_f32"]
    pl, x, xd, out = _run_workload(w)
    try:
        want = oracle_out(oracle, x, w.ratio[0], w.ratio[1], w.taps, w.dtype)
        assert out.shape == (1, 180, 240)
        err = assert_parity(out.cpu().numpy(), want, w.dtype, w.name)
        print("%s max |err| = %.3g" % (w.name, err))
    finally:
        ds.ds_destroy(pl)


def test_batch64_1080x1920_f32_all_frames(oracle):
    import torch

    w = synth.WORKLOADS["batch64_1080x1920_f32"]
    pl, x, xd, out = _run_workload(w, graph=True)
    try:
        got = out.cpu().numpy()
        want = oracle_out(oracle, x, w.ratio[0], w.ratio[1], w.taps, w.dtype)
        err = assert_parity(got, want, w.dtype, w.name)
        print("%s max |err| = %.3g over %d frames" % (w.name, err, w.frames))
        # plain per-frame launches and the unfused form give the same bits
        fin, fout = ds.ds_plan_frame_bytes(pl)
        o2 = torch.zeros_like(out)
        for i in (0, 17, 63):
            ds.ds_run(pl, xd.data_ptr() + i * fin, o2.data_ptr() + i * fout, stream())
        nb = ds.ds_plan_workspace_bytes(pl) * w.frames
        ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
        o3 = torch.zeros_like(out)
        ds.ds_run_unfused(pl, xd.data_ptr(), o3.data_ptr(), w.frames, ws.data_ptr(), nb, stream())
        finish()
        for i in (0, 17, 63):
            np.testing.assert_array_equal(o2[i].cpu().numpy(), got[i])
        np.testing.assert_array_equal(o3.cpu().numpy(), got)
    finally:
        ds.ds_destroy(pl)


def test_rgb300_1080x1920_u8_sampled(oracle):
    w = synth.WORKLOADS["rgb300_1080x1920_u8"]
    pl, x, xd, out = _run_workload(w)
    try:
        idx = _sample(w, 16, 3)
        got = out[idx].cpu().numpy()
        want = oracle_out(oracle, x[idx], w.ratio[0], w.ratio[1], w.taps, w.dtype)
        assert_parity(got, want, w.dtype, w.name)
        assert got.shape[1:] == (540, 960, 3)
    finally:
        ds.ds_destroy(pl)


def test_uhd128_2160x3840_f16_sampled(oracle):
    w = synth.WORKLOADS["uhd128_2160x3840_f16"]
    pl, x, xd, out = _run_workload(w)
    try:
        idx = _sample(w, 16, 4)
        got = out[idx].cpu().numpy()
        want = oracle_out(oracle, x[idx], w.ratio[0], w.ratio[1], w.taps, w.dtype)
        err = assert_parity(got, want, w.dtype, w.name)
        print("%s max |err| = %.3g on frames %s" % (w.name, err, idx))
        assert got.shape[1:] == (810, 1440)
    finally:
        ds.ds_destroy(pl)


@pytest.mark.parametrize("ratio,K,dt", [((1, 2), 6, ds.DS_U8_RGB), ((3, 8), 8, ds.DS_F32), ((3, 8), 8, ds.DS_F16),
                                        ((2, 3), 6, ds.DS_U8)])
def test_one_8k_frame_against_the_oracle(oracle, ratio, K, dt):
    """A single 8192x8192 frame (201 MB of RGB bytes, 268 MB of floats, 134 MB
    of halves, 67 MB of one-channel bytes): 64-bit offsets, many strips per
    row and the adaptive band for one frame, every output compared."""
    from tests.gpu_util import assert_parity, frames, run_fused

    pl = ds.ds_plan_create(8192, 8192, ratio, K, dt)
    try:
        x = frames((8192, 8192), dt, 1, 8192)
        got = run_fused(pl, x)
        if dt in (ds.DS_U8_RGB, ds.DS_U8):
            want = oracle.filter_u8(x, ratio[0], ratio[1], K)
        else:
            want = oracle.filter_f64(x.astype(np.float64), ratio[0], ratio[1], K)
        assert_parity(got, want, dt, "8192x8192")
    finally:
        ds.ds_destroy(pl)


@pytest.mark.parametrize("name", ["cif2000_352x288_u8rgb", "cif2000_yuv420_u8"])
def test_cif2000_every_frame_in_the_bench_configuration(oracle, name):
    """The paper's case (Sec. 3): 2000 CIF frames (RGB, or YUV 4:2:0 as three
    plane jobs), one plan per plane, the whole batch in one captured graph as
    the benchmark runs it; every output byte of every plane against the
    oracle."""
    import torch

    w = synth.WORKLOADS[name]
    shapes = w.plane_shapes()
    plans = [ds.ds_plan_create_ex(h, ww, w.ratio, w.taps, w.vratio, w.vtaps, w.dtype) for h, ww in shapes]
    try:
        xs = synth.plane_frames(w)
        ins = [torch.from_numpy(x).cuda() for x in xs]
        outs = [out_buffer(pl, w.frames) for pl in plans]
        g = ds.ds_graph_create([(pl, i.data_ptr(), o.data_ptr(), w.frames) for pl, i, o in zip(plans, ins, outs)])
        try:
            ds.ds_graph_launch(g, stream())
            finish()
        finally:
            ds.ds_graph_destroy(g)
        for x, o in zip(xs, outs):
            want = oracle.filter_ex(x, w.ratio, w.taps, w.vratio, w.vtaps)
            assert_parity(o.cpu().numpy(), want, w.dtype, "%s plane %s" % (name, x.shape[1:]))
    finally:
        for pl in plans:
            ds.ds_destroy(pl)
