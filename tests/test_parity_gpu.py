"""GPU parity of libds against the CPU oracle, through the C ABI.

Shapes span several strips and tiles with ragged right and bottom edges,
tiny frames smaller than the halo, widths that break the TMA alignment
(general kernel), and ratios / tap counts outside the fast path.  uint8 must
match bit for bit; FP32 within 1e-6 and FP16 within 2e-3 of the FP64 oracle.
The fused TMA kernel, the general fused kernel and the unfused two-kernel
form must agree bit for bit (same FMA order, same rounding)."""
import numpy as np
import pytest

import paper_1103_4881_b300 as ds
from tests.gpu_util import (assert_parity, finish, frames, general_kernel, oracle_out, out_buffer, run_fused,
                            run_unfused, stream, to_dev)

pytestmark = pytest.mark.gpu

FAST = [((3, 8), 8), ((1, 2), 6), ((2, 3), 6)]
DTYPES = [ds.DS_F32, ds.DS_F16, ds.DS_U8_RGB, ds.DS_U8]
# (H, W): widths multiple of 16 keep every dtype on the TMA path
FAST_SHAPES = [(72, 528), (8, 16), (16, 16), (3, 16), (41, 272), (200, 784), (3, 32)]


def _case(oracle, H, W, ratio, K, dt, n=2, schedule=None, seed=0):
    try:
        pl = ds.ds_plan_create(H, W, ratio, K, dt)
    except ds.DsError:
        pytest.skip("empty output")
    try:
        if schedule:
            ds.ds_plan_set_schedule(pl, *schedule)
        x = frames((H, W), dt, n, seed + H * 7 + W)
        got = run_fused(pl, x)
        want = oracle_out(oracle, x, ratio[0], ratio[1], K, dt)
        assert_parity(got, want, dt, "fused %dx%d %s K=%d dt=%d" % (H, W, ratio, K, dt))
        return pl, x, got
    except Exception:
        ds.ds_destroy(pl)
        raise


@pytest.mark.parametrize("dt", DTYPES)
@pytest.mark.parametrize("ratio,K", FAST)
@pytest.mark.parametrize("H,W", FAST_SHAPES)
def test_fast_path_parity(oracle, H, W, ratio, K, dt):
    pl, x, got = _case(oracle, H, W, ratio, K, dt, schedule=(2, 0))
    try:
        assert '"fused_tma"' in ds.ds_plan_describe(pl)
        # unfused two-kernel form: identical bits
        np.testing.assert_array_equal(run_unfused(pl, x), got)
    finally:
        ds.ds_destroy(pl)
    with general_kernel():
        pg = ds.ds_plan_create(H, W, ratio, K, dt)
    try:
        assert '"fused_general"' in ds.ds_plan_describe(pg)
        np.testing.assert_array_equal(run_fused(pg, x), got)
    finally:
        ds.ds_destroy(pg)


@pytest.mark.parametrize("rb", [1, 3, 12, 1000])
def test_schedule_does_not_change_bits(oracle, rb):
    H, W = 130, 784
    ref = None
    for dt in DTYPES:
        pl = ds.ds_plan_create(H, W, (2, 3), 6, dt)
        try:
            x = frames((H, W), dt, 1, 77)
            ds.ds_plan_set_schedule(pl, rb, 1)
            a = run_fused(pl, x)
            ds.ds_plan_set_schedule(pl, 7, 0)
            b = run_fused(pl, x)
            np.testing.assert_array_equal(a, b)
            assert_parity(a, oracle_out(oracle, x, 2, 3, 6, dt), dt)
        finally:
            ds.ds_destroy(pl)


@pytest.mark.parametrize("ratio,K", FAST)
@pytest.mark.parametrize("W", [356, 364, 1924, 100, 260, 268])
def test_right_border_where_the_last_packet_ends(oracle, W, ratio, K):
    """The right border fix covers only what the frame's last lane with
    outputs reads.  fp32 rows of 4 (mod 8) pixels take the fast kernel and put
    the end of that lane's last packet past the row's end (3/8), on it (1/2)
    or before it (2/3 at widths 1 (mod 3)): every output matches the oracle,
    and the fused, general and unfused forms agree bit for bit."""
    H = 23
    pl, x, got = _case(oracle, H, W, ratio, K, ds.DS_F32, n=3, seed=W)
    try:
        assert '"fused_tma"' in ds.ds_plan_describe(pl)
        np.testing.assert_array_equal(run_unfused(pl, x), got)
    finally:
        ds.ds_destroy(pl)
    with general_kernel():
        pg = ds.ds_plan_create(H, W, ratio, K, ds.DS_F32)
    try:
        np.testing.assert_array_equal(run_fused(pg, x), got)
    finally:
        ds.ds_destroy(pg)


@pytest.mark.parametrize("H,W,ratio,K,dt", [
    (37, 61, (3, 8), 8, ds.DS_F32),      # odd width: general kernel
    (5, 7, (1, 2), 6, ds.DS_F16),
    (29, 22, (5, 7), 10, ds.DS_F32),     # ratio without a fast class
    (33, 48, (1, 4), 16, ds.DS_U8_RGB),
    (19, 40, (3, 8), 6, ds.DS_U8_RGB),   # K outside the fast class
    (64, 90, (3, 8), 8, ds.DS_U8),       # single-channel uint8, rows not 16-byte multiples
    (45, 50, (2, 3), 6, ds.DS_U8),
    (70, 130, (7, 16), 14, ds.DS_F16),
    (200, 70, (1, 64), 8, ds.DS_F32),    # q at its limit
    (17, 34, (16, 17), 16, ds.DS_F32),   # p at its limit
])
def test_general_path_parity(oracle, H, W, ratio, K, dt):
    pl, x, got = _case(oracle, H, W, ratio, K, dt)
    try:
        np.testing.assert_array_equal(run_unfused(pl, x), got)
    finally:
        ds.ds_destroy(pl)


def test_unaligned_input_pointer_uses_general_kernel(oracle):
    import torch

    H, W = 40, 256
    pl = ds.ds_plan_create(H, W, (3, 8), 8, ds.DS_F32)
    try:
        x = frames((H, W), ds.DS_F32, 1, 5)
        buf = torch.zeros(x.size + 1, dtype=torch.float32, device="cuda")
        buf[1:] = torch.from_numpy(x.ravel()).cuda()
        out = out_buffer(pl, 1)
        ds.ds_run(pl, buf.data_ptr() + 4, out.data_ptr(), stream())  # 4-byte aligned only
        finish()
        assert_parity(out.cpu().numpy(), oracle_out(oracle, x, 3, 8, 8, ds.DS_F32), ds.DS_F32)
    finally:
        ds.ds_destroy(pl)


def test_full_hd_single_frames(oracle):
    for dt, (ratio, K) in zip(DTYPES, FAST):
        pl, x, got = _case(oracle, 1080, 1920, ratio, K, dt, n=1, seed=11)
        ds.ds_destroy(pl)


def test_batch_mixed_plans_equal_solo_runs(oracle):
    """One ds_batch_run over jobs of different sizes, ratios and dtypes (one
    persistent launch for the fast ones) gives each job the bits of its solo run."""
    import torch

    specs = [(72, 528, (3, 8), 8, ds.DS_F32), (40, 256, (1, 2), 6, ds.DS_U8_RGB), (130, 784, (2, 3), 6, ds.DS_F16),
             (37, 61, (3, 8), 8, ds.DS_F32), (96, 320, (2, 3), 6, ds.DS_U8_RGB), (64, 64, (1, 2), 6, ds.DS_F32),
             (33, 48, (1, 4), 16, ds.DS_U8_RGB)]
    plans, ins, outs, solo, xs = [], [], [], [], []
    try:
        for k, (H, W, r, K, dt) in enumerate(specs):
            pl = ds.ds_plan_create(H, W, r, K, dt)
            plans.append(pl)
            x = frames((H, W), dt, 2, 100 + k)
            xs.append(x)
            solo.append(run_fused(pl, x))
            ins.append(to_dev(x))
            outs.append(out_buffer(pl, 2))
        ds.ds_launch_count()
        ds.ds_batch_run([(pl, i.data_ptr(), o.data_ptr(), 2) for pl, i, o in zip(plans, ins, outs)], stream())
        finish()
        launches = ds.ds_launch_count()
        assert launches == 5 + 2  # one launch per fast class present + two general-kernel jobs
        for k, (o, s) in enumerate(zip(outs, solo)):
            np.testing.assert_array_equal(o.cpu().numpy(), s, err_msg="job %d" % k)
        # graph replay of the same batch
        for o in outs:
            o.zero_()
        g = ds.ds_graph_create([(pl, i.data_ptr(), o.data_ptr(), 2) for pl, i, o in zip(plans, ins, outs)])
        try:
            ds.ds_graph_launch(g, stream())
            ds.ds_graph_launch(g, stream())
            finish()
        finally:
            ds.ds_graph_destroy(g)
        for k, (o, s) in enumerate(zip(outs, solo)):
            np.testing.assert_array_equal(o.cpu().numpy(), s, err_msg="graph job %d" % k)
        for (H, W, r, K, dt), x, s in zip(specs, xs, solo):
            assert_parity(s, oracle_out(oracle, x, r[0], r[1], K, dt), dt)
    finally:
        for pl in plans:
            ds.ds_destroy(pl)


def test_batch_more_jobs_than_one_launch_holds(oracle):
    H, W = 24, 64
    pl = ds.ds_plan_create(H, W, (3, 8), 8, ds.DS_F32)
    try:
        n = 150
        x = frames((H, W), ds.DS_F32, n, 9)
        xd = to_dev(x)
        out = out_buffer(pl, n)
        fb_in, fb_out = ds.ds_plan_frame_bytes(pl)
        ds.ds_batch_run([(pl, xd.data_ptr() + i * fb_in, out.data_ptr() + i * fb_out, 1) for i in range(n)], stream())
        finish()
        assert_parity(out.cpu().numpy(), oracle_out(oracle, x, 3, 8, 8, ds.DS_F32), ds.DS_F32)
    finally:
        ds.ds_destroy(pl)


def test_pipeline_host_buffers(oracle):
    import torch

    H, W = 120, 512
    pl = ds.ds_plan_create(H, W, (3, 8), 8, ds.DS_F16)
    try:
        n = 11
        x = frames((H, W), ds.DS_F16, n, 21)
        xin = torch.from_numpy(x).pin_memory()
        oh, ow, _ = ds.ds_plan_out_shape(pl)
        yout = torch.zeros((n, oh, ow), dtype=torch.float16).pin_memory()
        pp = ds.ds_pipeline_create(pl, 3, 2)
        try:
            ds.ds_pipeline_run(pp, xin.data_ptr(), yout.data_ptr(), n)
        finally:
            ds.ds_pipeline_destroy(pp)
        np.testing.assert_array_equal(yout.numpy(), run_fused(pl, x))
        assert_parity(yout.numpy(), oracle_out(oracle, x, 3, 8, 8, ds.DS_F16), ds.DS_F16)
    finally:
        ds.ds_destroy(pl)


@pytest.mark.parametrize("chunk", [1, 3, 5])
def test_pipeline_host_buffers_chroma_planes(oracle, chunk):
    """The host-buffer pipeline on 176x144 chroma planes (CIF axes): each
    chunk of 1, 3 or 5 frames is one launch whose tail strips run as a narrow
    job with a part-empty group of four; the result equals the device path
    and the oracle, bit for bit."""
    import torch

    pl = ds.ds_plan_create_ex(144, 176, (3, 8), 8, (4, 9), 8, ds.DS_U8)
    try:
        n = 13
        x = frames((144, 176), ds.DS_U8, n, 170 + chunk)
        xin = torch.from_numpy(x).pin_memory()
        oh, ow, _ = ds.ds_plan_out_shape(pl)
        yout = torch.zeros((n, oh, ow), dtype=torch.uint8).pin_memory()
        pp = ds.ds_pipeline_create(pl, chunk, 2)
        try:
            ds.ds_pipeline_run(pp, xin.data_ptr(), yout.data_ptr(), n)
        finally:
            ds.ds_pipeline_destroy(pp)
        np.testing.assert_array_equal(yout.numpy(), run_fused(pl, x))
        assert_parity(yout.numpy(), oracle.filter_ex(x, (3, 8), 8, (4, 9), 8), ds.DS_U8, "pipeline chunk %d" % chunk)
    finally:
        ds.ds_destroy(pl)


def test_constant_and_impulse_frames(oracle):
    H, W = 64, 256
    for dt in DTYPES:
        pl = ds.ds_plan_create(H, W, (3, 8), 8, dt)
        try:
            u8 = dt in (ds.DS_U8, ds.DS_U8_RGB)
            c = 200 if u8 else 0.625
            shape = (1, H, W, 3) if dt == ds.DS_U8_RGB else (1, H, W)
            x = np.full(shape, c, dtype={ds.DS_F32: np.float32, ds.DS_F16: np.float16, ds.DS_U8_RGB: np.uint8,
                                         ds.DS_U8: np.uint8}[dt])
            y = run_fused(pl, x).astype(np.float64)
            assert np.abs(y - c).max() <= (0 if u8 else 1e-6)
            x[...] = 0
            x[0, 31, 101] = 255 if u8 else 1
            assert_parity(run_fused(pl, x), oracle_out(oracle, x, 3, 8, 8, dt), dt)
        finally:
            ds.ds_destroy(pl)


def test_zero_frames_and_stream_check():
    pl = ds.ds_plan_create(64, 64, (3, 8), 8, ds.DS_F32)
    try:
        ds.ds_run_frames(pl, 16, 16, 0, stream())  # nothing launched
        ds.ds_stream_check(stream())
    finally:
        ds.ds_destroy(pl)


def test_graphs_and_direct_launches_on_several_streams(oracle):
    """Replays of two graphs and direct launches on three streams at once: each
    captured launch owns its tile-scheduling slot, so none disturbs another."""
    import torch

    H, W = 270, 480
    pl = ds.ds_plan_create(H, W, (3, 8), 8, ds.DS_F32)
    try:
        xs = [frames((H, W), ds.DS_F32, 3, 40 + k) for k in range(3)]
        want = [run_fused(pl, x) for x in xs]
        ins = [to_dev(x) for x in xs]
        outs = [out_buffer(pl, 3) for _ in xs]
        graphs = [ds.ds_graph_create([(pl, ins[k].data_ptr(), outs[k].data_ptr(), 3)]) for k in range(2)]
        streams = [torch.cuda.Stream() for _ in range(3)]
        torch.cuda.synchronize()
        try:
            for _ in range(20):
                ds.ds_graph_launch(graphs[0], streams[0].cuda_stream)
                ds.ds_graph_launch(graphs[1], streams[1].cuda_stream)
                ds.ds_run_frames(pl, ins[2].data_ptr(), outs[2].data_ptr(), 3, streams[2].cuda_stream)
            finish()
        finally:
            for g in graphs:
                ds.ds_graph_destroy(g)
        for k in range(3):
            np.testing.assert_array_equal(outs[k].cpu().numpy(), want[k], err_msg="stream %d" % k)
        assert_parity(want[0], oracle_out(oracle, xs[0], 3, 8, 8, ds.DS_F32), ds.DS_F32)
    finally:
        ds.ds_destroy(pl)
