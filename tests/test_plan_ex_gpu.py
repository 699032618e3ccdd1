"""GPU parity of extended plans: a ratio per axis (the paper's CIF case,
352x288 -> 132x128 with H 3/8 and V 4/9), modular tilers and caller-given
taps, against the oracle; the general fused kernel and the unfused form
agree bit for bit."""
import numpy as np
import pytest

import paper_1103_4881_b300 as ds
from tests.gpu_util import TOL, assert_parity, frames, run_fused, run_unfused

pytestmark = pytest.mark.gpu

RNG = np.random.default_rng(11)
W_H = RNG.normal(0, 0.3, (3, 8))
W_V = RNG.normal(0, 0.3, (4, 8))

CASES = [
    # (H, W, rh, Kh, rv, Kv, dtype, boundary, given)
    (288, 352, (3, 8), 8, (4, 9), 8, ds.DS_U8_RGB, ds.DS_CLAMP, False),   # the paper's CIF case
    (288, 352, (3, 8), 8, (4, 9), 8, ds.DS_U8, ds.DS_CLAMP, False),       # one plane
    (144, 176, (3, 8), 8, (4, 9), 8, ds.DS_U8, ds.DS_WRAP, False),        # a chroma plane, modular
    (97, 130, (1, 2), 6, (2, 3), 6, ds.DS_F32, ds.DS_CLAMP, False),
    (97, 130, (2, 3), 6, (1, 2), 6, ds.DS_F16, ds.DS_WRAP, False),
    (5, 7, (3, 8), 8, (4, 9), 8, ds.DS_F32, ds.DS_WRAP, False),           # windows wrap more than once
    (3, 16, (1, 2), 6, (1, 3), 6, ds.DS_U8_RGB, ds.DS_WRAP, False),
    (200, 256, (3, 8), 8, (3, 8), 8, ds.DS_F32, ds.DS_WRAP, False),       # equal axes, modular
    (120, 160, (3, 8), 8, (4, 9), 8, ds.DS_F32, ds.DS_CLAMP, True),       # given taps
    (120, 160, (3, 8), 8, (4, 9), 8, ds.DS_U8_RGB, ds.DS_WRAP, True),
    (64, 96, (3, 8), 8, (3, 8), 8, ds.DS_F16, ds.DS_CLAMP, True),
]


def _plan(H, W, rh, Kh, rv, Kv, dt, bnd, given):
    wh = W_H[: rh[0], :Kh] if given else None
    wv = W_V[: rv[0], :Kv] if given else None
    return ds.ds_plan_create_ex(H, W, rh, Kh, rv, Kv, dt, bnd, wh, wv), wh, wv


def _oracle(oracle, x, rh, Kh, rv, Kv, dt, bnd, wh, wv):
    if dt in (ds.DS_U8, ds.DS_U8_RGB):
        return oracle.filter_ex(x, rh, Kh, rv, Kv, wrap=bnd == ds.DS_WRAP, weights_h=wh, weights_v=wv)
    return oracle.filter_ex(x.astype(np.float64), rh, Kh, rv, Kv, wrap=bnd == ds.DS_WRAP, weights_h=wh,
                            weights_v=wv)


@pytest.mark.parametrize("H,W,rh,Kh,rv,Kv,dt,bnd,given", CASES)
def test_extended_plan_parity(oracle, H, W, rh, Kh, rv, Kv, dt, bnd, given):
    pl, wh, wv = _plan(H, W, rh, Kh, rv, Kv, dt, bnd, given)
    try:
        x = frames((H, W), dt, 3, H * 5 + W)
        got = run_fused(pl, x)
        want = _oracle(oracle, x, rh, Kh, rv, Kv, dt, bnd, wh, wv)
        assert got.shape == want.shape
        assert_parity(got, want, dt, "ex %dx%d %s/%s dt=%d bnd=%d given=%s" % (H, W, rh, rv, dt, bnd, given))
        np.testing.assert_array_equal(run_unfused(pl, x), got)
    finally:
        ds.ds_destroy(pl)


def test_cif_frames_in_one_batch_with_yuv_planes(oracle):
    """The paper's CIF workload as 4:2:0 planes: Y 352x288 and U, V 176x144,
    each H 3/8 and V 4/9 (outputs 132x128 and 66x64), one ds_batch_run."""
    import torch

    from tests.gpu_util import out_buffer, stream, to_dev, finish
    py = ds.ds_plan_create_ex(288, 352, (3, 8), 8, (4, 9), 8, ds.DS_U8)
    pc = ds.ds_plan_create_ex(144, 176, (3, 8), 8, (4, 9), 8, ds.DS_U8)
    try:
        assert ds.ds_plan_out_shape(py) == (128, 132, 1) and ds.ds_plan_out_shape(pc) == (64, 66, 1)
        n = 4
        ys, us, vs = frames((288, 352), ds.DS_U8, n, 1), frames((144, 176), ds.DS_U8, n, 2), frames((144, 176), ds.DS_U8, n, 3)
        ins = [to_dev(a) for a in (ys, us, vs)]
        outs = [out_buffer(py, n), out_buffer(pc, n), out_buffer(pc, n)]
        ds.ds_batch_run([(py, ins[0].data_ptr(), outs[0].data_ptr(), n), (pc, ins[1].data_ptr(), outs[1].data_ptr(), n),
                         (pc, ins[2].data_ptr(), outs[2].data_ptr(), n)], stream())
        finish()
        for o, x in zip(outs, (ys, us, vs)):
            assert_parity(o.cpu().numpy(), oracle.filter_ex(x, (3, 8), 8, (4, 9), 8), ds.DS_U8)
    finally:
        ds.ds_destroy(py)
        ds.ds_destroy(pc)


CIF_PLANES = [(288, 352, ds.DS_U8_RGB), (288, 352, ds.DS_U8), (144, 176, ds.DS_U8)]


@pytest.mark.parametrize("H,W,dt", CIF_PLANES)
@pytest.mark.parametrize("n", [1, 2, 3, 7])
def test_cif_frame_groups(oracle, H, W, dt, n):
    """The CIF classes filter two frames per warp (half a warp each): odd
    counts leave the last group half empty, and its missing frame must be
    neither loaded nor written."""
    pl = ds.ds_plan_create_ex(H, W, (3, 8), 8, (4, 9), 8, dt)
    try:
        assert ds.ds_plan_describe(pl).find("fused_tma") >= 0
        x = frames((H, W), dt, n, 100 + n)
        got = run_fused(pl, x)
        assert_parity(got, oracle.filter_ex(x, (3, 8), 8, (4, 9), 8), dt, "cif groups %dx%d n=%d" % (H, W, n))
    finally:
        ds.ds_destroy(pl)


def test_cif_frame_groups_guarded_output(oracle):
    """A half-empty last group writes nothing past its one frame: the output
    buffer's next frame (a sentinel) is untouched."""
    import torch

    from tests.gpu_util import finish, stream, to_dev
    pl = ds.ds_plan_create_ex(288, 352, (3, 8), 8, (4, 9), 8, ds.DS_U8_RGB)
    try:
        n = 5
        x = frames((288, 352), ds.DS_U8_RGB, n, 77)
        xd = to_dev(x)
        out = torch.full((n + 1, 128, 132, 3), 201, dtype=torch.uint8, device="cuda")
        ds.ds_run_frames(pl, xd.data_ptr(), out.data_ptr(), n, stream())
        finish()
        got = out.cpu().numpy()
        assert_parity(got[:n], oracle.filter_ex(x, (3, 8), 8, (4, 9), 8), ds.DS_U8_RGB)
        assert (got[n] == 201).all()
    finally:
        ds.ds_destroy(pl)


def test_cif_frame_groups_split_tail(oracle):
    """1201 CIF frames: long enough that the launch's last units run in
    shorter bands, the job being split at a whole group of frames; the odd
    count leaves the tail's last group half empty."""
    pl = ds.ds_plan_create_ex(288, 352, (3, 8), 8, (4, 9), 8, ds.DS_U8_RGB)
    try:
        x = frames((288, 352), ds.DS_U8_RGB, 1201, 1201)
        got = run_fused(pl, x)
        assert_parity(got, oracle.filter_ex(x, (3, 8), 8, (4, 9), 8), ds.DS_U8_RGB, "cif 1201 frames")
    finally:
        ds.ds_destroy(pl)


def test_cif_planes_odd_counts_in_one_batch(oracle):
    """Y, U and V jobs of odd frame counts in one launch (each job's groups
    are its own: a group never spans two jobs)."""
    from tests.gpu_util import finish, out_buffer, stream, to_dev
    py = ds.ds_plan_create_ex(288, 352, (3, 8), 8, (4, 9), 8, ds.DS_U8)
    pc = ds.ds_plan_create_ex(144, 176, (3, 8), 8, (4, 9), 8, ds.DS_U8)
    try:
        counts = (3, 5, 1)
        xs = [frames((288, 352), ds.DS_U8, counts[0], 31), frames((144, 176), ds.DS_U8, counts[1], 32),
              frames((144, 176), ds.DS_U8, counts[2], 33)]
        ins = [to_dev(a) for a in xs]
        outs = [out_buffer(py, counts[0]), out_buffer(pc, counts[1]), out_buffer(pc, counts[2])]
        plans = (py, pc, pc)
        ds.ds_batch_run([(plans[i], ins[i].data_ptr(), outs[i].data_ptr(), counts[i]) for i in range(3)], stream())
        finish()
        for o, x in zip(outs, xs):
            assert_parity(o.cpu().numpy(), oracle.filter_ex(x, (3, 8), 8, (4, 9), 8), ds.DS_U8)
    finally:
        ds.ds_destroy(py)
        ds.ds_destroy(pc)


@pytest.mark.parametrize("dt", [ds.DS_U8_RGB, ds.DS_U8])
@pytest.mark.parametrize("H", [3, 5, 10, 30])
@pytest.mark.parametrize("W", [16, 48, 272])
@pytest.mark.parametrize("n", [1, 3])
def test_cif_classes_on_tiny_and_ragged_frames(oracle, dt, H, W, n):
    """The CIF classes' lead blocks on frames shorter than a window (every
    row clamped), strips narrower than a half warp, and half-empty groups."""
    pl = ds.ds_plan_create_ex(H, W, (3, 8), 8, (4, 9), 8, dt)
    try:
        assert '"fused_tma"' in ds.ds_plan_describe(pl)
        x = frames((H, W), dt, n, H * 1000 + W * 10 + n)
        assert_parity(run_fused(pl, x), oracle.filter_ex(x, (3, 8), 8, (4, 9), 8), dt,
                      "cif %dx%d n=%d dt=%d" % (H, W, n, dt))
    finally:
        ds.ds_destroy(pl)


GIVEN_FAST = [
    # (H, W, rh, Kh, rv, Kv, dtype): fast classes with caller-given taps
    (72, 528, (3, 8), 8, (3, 8), 8, ds.DS_F32),
    (64, 256, (1, 2), 6, (1, 2), 6, ds.DS_U8_RGB),
    (41, 272, (2, 3), 6, (2, 3), 6, ds.DS_F16),
    (288, 352, (3, 8), 8, (4, 9), 8, ds.DS_U8_RGB),
    (144, 176, (3, 8), 8, (4, 9), 8, ds.DS_U8),
    (9, 16, (3, 8), 8, (3, 8), 8, ds.DS_U8),
]


def _given(rh, Kh, rv, Kv, seed):
    rng = np.random.default_rng(seed)
    wh, wv = rng.normal(0, 0.3, (rh[0], Kh)), rng.normal(0, 0.3, (rv[0], Kv))
    wh[:, Kh // 2] += 1.0  # a dominant centre tap, like a smoothing filter
    wv[:, Kv // 2] += 1.0
    return wh, wv


@pytest.mark.parametrize("H,W,rh,Kh,rv,Kv,dt", GIVEN_FAST)
def test_given_taps_on_the_fast_kernel(oracle, H, W, rh, Kh, rv, Kv, dt):
    wh, wv = _given(rh, Kh, rv, Kv, H + W)
    pl = ds.ds_plan_create_ex(H, W, rh, Kh, rv, Kv, dt, ds.DS_CLAMP, wh, wv)
    try:
        assert '"fused_tma"' in ds.ds_plan_describe(pl)
        x = frames((H, W), dt, 3, H * 13 + W)
        got = run_fused(pl, x)
        assert_parity(got, _oracle(oracle, x, rh, Kh, rv, Kv, dt, ds.DS_CLAMP, wh, wv), dt,
                      "given taps %dx%d %s/%s dt=%d" % (H, W, rh, rv, dt))
        np.testing.assert_array_equal(run_unfused(pl, x), got)
    finally:
        ds.ds_destroy(pl)


def test_batch_mixes_given_and_library_taps_of_one_class(oracle):
    """Plans of one class with different tap tables in one ds_batch_run and in
    one graph: each launch group carries its own tables."""
    from tests.gpu_util import finish, out_buffer, stream, to_dev
    wa, wb = _given((3, 8), 8, (3, 8), 8, 1), _given((3, 8), 8, (3, 8), 8, 2)
    plans = [ds.ds_plan_create(96, 528, (3, 8), 8, ds.DS_U8_RGB),
             ds.ds_plan_create_ex(96, 528, (3, 8), 8, (3, 8), 8, ds.DS_U8_RGB, ds.DS_CLAMP, *wa),
             ds.ds_plan_create_ex(96, 528, (3, 8), 8, (3, 8), 8, ds.DS_U8_RGB, ds.DS_CLAMP, *wb),
             ds.ds_plan_create(96, 528, (3, 8), 8, ds.DS_U8_RGB)]
    weights = [(None, None), wa, wb, (None, None)]
    try:
        xs = [frames((96, 528), ds.DS_U8_RGB, 2, 60 + k) for k in range(4)]
        ins = [to_dev(a) for a in xs]
        for use_graph in (False, True):
            outs = [out_buffer(pl, 2) for pl in plans]
            jobs = [(pl, i.data_ptr(), o.data_ptr(), 2) for pl, i, o in zip(plans, ins, outs)]
            if use_graph:
                g = ds.ds_graph_create(jobs)
                ds.ds_graph_launch(g, stream())
                finish()
                ds.ds_graph_destroy(g)
            else:
                ds.ds_batch_run(jobs, stream())
                finish()
            for o, a, (wh, wv) in zip(outs, xs, weights):
                want = oracle.filter_ex(a, (3, 8), 8, (3, 8), 8, weights_h=wh, weights_v=wv)
                assert_parity(o.cpu().numpy(), want, ds.DS_U8_RGB, "graph=%s" % use_graph)
    finally:
        for pl in plans:
            ds.ds_destroy(pl)


# One-plane CIF frames whose last strip has at most 6 packets (width mod 128
# in {16, 32, 48}): the launch gives that strip a job of its own, filtered
# four frames per warp in groups of 8 lanes, two frames' windows side by
# side in each TMA box.
NARROW_W = [16, 32, 48, 144, 160, 176, 304]


@pytest.mark.parametrize("W", NARROW_W)
@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6, 9])
def test_narrow_tail_strips(oracle, W, n):
    """Counts that leave the last group of four 1-3 frames short: the missing
    frames are neither loaded nor written (the output frame after the last,
    a sentinel, stays untouched), and every output matches the oracle."""
    import torch

    from tests.gpu_util import finish, stream, to_dev
    H = 144 if W != 304 else 37  # 37 rows: a ragged last block
    pl = ds.ds_plan_create_ex(H, W, (3, 8), 8, (4, 9), 8, ds.DS_U8)
    try:
        oh, ow, _ = ds.ds_plan_out_shape(pl)
        x = frames((H, W), ds.DS_U8, n, 500 + W + n)
        xd = to_dev(x)
        out = torch.full((n + 1, oh, ow), 201, dtype=torch.uint8, device="cuda")
        ds.ds_run_frames(pl, xd.data_ptr(), out.data_ptr(), n, stream())
        finish()
        got = out.cpu().numpy()
        assert_parity(got[:n], oracle.filter_ex(x, (3, 8), 8, (4, 9), 8), ds.DS_U8, "narrow %dx%d n=%d" % (H, W, n))
        assert (got[n] == 201).all()
    finally:
        ds.ds_destroy(pl)


def test_narrow_tail_strips_in_one_batch(oracle):
    """Jobs with and without narrow tail strips, of several frame counts, in
    one launch; then the same jobs again, each alone, give the same bytes."""
    from tests.gpu_util import finish, out_buffer, stream, to_dev
    shapes = [(144, 176, 5), (30, 48, 3), (288, 352, 2), (70, 160, 7), (144, 176, 1)]
    plans = [ds.ds_plan_create_ex(h, w, (3, 8), 8, (4, 9), 8, ds.DS_U8) for h, w, _ in shapes]
    try:
        xs = [frames((h, w), ds.DS_U8, n, 900 + k) for k, (h, w, n) in enumerate(shapes)]
        ins = [to_dev(a) for a in xs]
        outs = [out_buffer(pl, n) for pl, (_, _, n) in zip(plans, shapes)]
        ds.ds_batch_run([(pl, i.data_ptr(), o.data_ptr(), n) for pl, i, o, (_, _, n) in zip(plans, ins, outs, shapes)],
                        stream())
        finish()
        for pl, x, o in zip(plans, xs, outs):
            got = o.cpu().numpy()
            assert_parity(got, oracle.filter_ex(x, (3, 8), 8, (4, 9), 8), ds.DS_U8)
            np.testing.assert_array_equal(run_fused(pl, x), got)
    finally:
        for pl in plans:
            ds.ds_destroy(pl)


def test_narrow_tail_strips_split_tail(oracle):
    """1201 chroma planes: the launch's last units run in shorter bands, the
    job split by frames, and each part gets its own narrow tail-strip job."""
    pl = ds.ds_plan_create_ex(144, 176, (3, 8), 8, (4, 9), 8, ds.DS_U8)
    try:
        x = frames((144, 176), ds.DS_U8, 1201, 1202)
        assert_parity(run_fused(pl, x), oracle.filter_ex(x, (3, 8), 8, (4, 9), 8), ds.DS_U8, "narrow 1201 frames")
    finally:
        ds.ds_destroy(pl)
