"""Modular (Array-OL) tilers on the fast kernel: DS_WRAP plans whose rows are
at least a strip and its halo wide load every row of a stage with 1-D bulk
copies from frame row (y mod H), with the window's bytes past either end of
the row taken from its other end.  Every class (tile shape 0, the one
compiled for modular tilers), on frames
whose row counts and widths wrap the windows at the top, bottom, left and
right, against the oracle's modular tilers, bit-identical to the general
kernels; in batches with clamped plans of the same class; in the
bounds-checking build; and with guard bytes around the output."""
import numpy as np
import pytest

import paper_1103_4881_b300 as ds
from tests.gpu_util import (assert_parity, finish, frames, general_kernel, out_buffer, run_fused, stream, to_dev)

pytestmark = pytest.mark.gpu

AXES = [((3, 8), 8, (3, 8), 8), ((1, 2), 6, (1, 2), 6), ((2, 3), 6, (2, 3), 6), ((3, 8), 8, (4, 9), 8)]
DTYPES = [ds.DS_F32, ds.DS_F16, ds.DS_U8_RGB, ds.DS_U8]
# (H, W): ragged bottoms and right edges, a three-row frame, a frame exactly
# one 1024-pixel strip plus halo wide (the one-channel 1/2 class), CIF sizes
SHAPES = [(72, 528), (41, 272), (200, 784), (3, 1056), (130, 1104), (288, 352), (17, 1040)]
CASES = [(a, dt) for a in AXES for dt in DTYPES if a[2] != (4, 9) or dt in (ds.DS_U8_RGB, ds.DS_U8)]


def _oracle(oracle, x, axes, dt):
    rh, Kh, rv, Kv = axes
    xo = x if dt in (ds.DS_U8, ds.DS_U8_RGB) else x.astype(np.float64)
    return oracle.filter_ex(xo, rh, Kh, rv, Kv, wrap=True)


@pytest.mark.parametrize("axes,dt", CASES)
@pytest.mark.parametrize("H,W", SHAPES)
def test_modular_tilers_on_the_fast_kernel(oracle, axes, dt, H, W):
    rh, Kh, rv, Kv = axes
    try:
        pl = ds.ds_plan_create_ex(H, W, rh, Kh, rv, Kv, dt, ds.DS_WRAP)
    except ds.DsError:
        pytest.skip("empty output")
    try:
        x = frames((H, W), dt, 3, H * 11 + W)
        want = _oracle(oracle, x, axes, dt)
        fast = '"fused_tma"' in ds.ds_plan_describe(pl)
        got = run_fused(pl, x)
        assert_parity(got, want, dt, "wrap %dx%d %s dt=%d fast=%s" % (H, W, axes, dt, fast))
        if fast:
            for shape in range(ds.ds_plan_tile_shapes(pl)):
                for band in (0, 2):
                    ds.ds_plan_set_schedule_ex(pl, band, 0, shape)
                    np.testing.assert_array_equal(run_fused(pl, x), got, err_msg="shape %d band %d" % (shape, band))
        with general_kernel():
            pg = ds.ds_plan_create_ex(H, W, rh, Kh, rv, Kv, dt, ds.DS_WRAP)
        try:
            np.testing.assert_array_equal(run_fused(pg, x), got)
        finally:
            ds.ds_destroy(pg)
    finally:
        ds.ds_destroy(pl)


def test_wrap_takes_the_fast_kernel_where_it_fits():
    for H, W, fast in [(1080, 1920, True), (64, 260, True), (64, 256, False), (64, 64, False)]:
        pl = ds.ds_plan_create_ex(H, W, (3, 8), 8, (3, 8), 8, ds.DS_F32, ds.DS_WRAP)
        try:
            assert ('"fused_tma"' in ds.ds_plan_describe(pl)) == fast, (H, W)
        finally:
            ds.ds_destroy(pl)


def test_modular_and_clamped_plans_of_one_class_in_one_batch(oracle):
    """One batch (and one graph) with jobs of both boundaries: one launch per
    boundary; many frames, so that the launch's last tiles run in shorter
    bands and the job is split."""
    pw = ds.ds_plan_create_ex(270, 480, (3, 8), 8, (3, 8), 8, ds.DS_F32, ds.DS_WRAP)
    pc = ds.ds_plan_create(270, 480, (3, 8), 8, ds.DS_F32)
    try:
        xa, xb = frames((270, 480), ds.DS_F32, 97, 1), frames((270, 480), ds.DS_F32, 31, 2)
        ia, ib = to_dev(xa), to_dev(xb)
        oa, ob = out_buffer(pw, 97), out_buffer(pc, 31)
        for use_graph in (False, True):
            jobs = [(pw, ia.data_ptr(), oa.data_ptr(), 97), (pc, ib.data_ptr(), ob.data_ptr(), 31)]
            if use_graph:
                g = ds.ds_graph_create(jobs)
                ds.ds_graph_launch(g, stream())
                finish()
                ds.ds_graph_destroy(g)
            else:
                ds.ds_batch_run(jobs, stream())
                finish()
            assert_parity(oa.cpu().numpy(), oracle.filter_ex(xa.astype(np.float64), (3, 8), 8, (3, 8), 8, wrap=True),
                          ds.DS_F32, "wrap job")
            assert_parity(ob.cpu().numpy(), oracle.filter_f64(xb.astype(np.float64), 3, 8, 8), ds.DS_F32, "clamp job")
    finally:
        ds.ds_destroy(pw)
        ds.ds_destroy(pc)


@pytest.mark.parametrize("axes,dt", [(AXES[0], ds.DS_F32), (AXES[1], ds.DS_U8_RGB), (AXES[2], ds.DS_F16),
                                     (AXES[3], ds.DS_U8), (AXES[1], ds.DS_U8)])
def test_modular_tilers_leave_guard_bytes_alone(oracle, axes, dt):
    import torch

    rh, Kh, rv, Kv = axes
    H, W, n = 41, 1104, 3
    pl = ds.ds_plan_create_ex(H, W, rh, Kh, rv, Kv, dt, ds.DS_WRAP)
    try:
        assert '"fused_tma"' in ds.ds_plan_describe(pl)
        x = frames((H, W), dt, n, 5)
        xd = to_dev(x)
        fin, fout = ds.ds_plan_frame_bytes(pl)
        guard = 4096
        buf = torch.full((n * fout + 2 * guard,), 0xA5, dtype=torch.uint8, device="cuda")
        ds.ds_run_frames(pl, xd.data_ptr(), buf.data_ptr() + guard, n, stream())
        finish()
        b = buf.cpu().numpy()
        assert (b[:guard] == 0xA5).all() and (b[-guard:] == 0xA5).all()
        got = b[guard:-guard].view(x.dtype).reshape(_oracle(oracle, x, axes, dt).shape)
        assert_parity(got, _oracle(oracle, x, axes, dt), dt, "guarded wrap")
    finally:
        ds.ds_destroy(pl)
