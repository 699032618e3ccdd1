"""The bounds-checking build (libds_check.so, -DDS_CHECK_BOUNDS): every fast
class, on ragged and tiny frames, in single and batched launches, runs with
all of the kernel's own index checks passing (ds_stream_check would raise
DS_ERR_BOUNDS otherwise) and gives the oracle's results; the check's report
path works (a probe that checks an index one past a buffer, with no
access)."""
import numpy as np
import pytest

import paper_1103_4881_b300 as ds
from tests.gpu_util import assert_parity, finish, frames, out_buffer, run_fused, stream, to_dev

pytestmark = pytest.mark.gpu

FAST_AXES = [((3, 8), 8, (3, 8), 8), ((1, 2), 6, (1, 2), 6), ((2, 3), 6, (2, 3), 6), ((3, 8), 8, (4, 9), 8)]
# (130, 1100): two 1024-pixel strips of the one-channel 1/2 class, the second
# ragged, with interior units in both
SHAPES = [(72, 528), (9, 16), (41, 272), (3, 48), (200, 784), (130, 1100)]


@pytest.fixture(scope="module")
def checked():
    from paper_1103_4881_b300 import build

    build.build(check_bounds=True)
    previous = ds.LIB_PATH
    ds.use_library(ds.CHECK_LIB_PATH)
    assert ds.ds_bounds_checked()
    yield
    ds.use_library(previous)


def _oracle(oracle, x, rh, Kh, rv, Kv, dt):
    xo = x if dt in (ds.DS_U8, ds.DS_U8_RGB) else x.astype(np.float64)
    return oracle.filter_ex(xo, rh, Kh, rv, Kv)


# every compiled tile shape of every class (the CIF axes have fast classes
# for uint8 data only; float plans on them run the general kernel, shape 0)
CLASSES = [(a, dt, shape) for a in FAST_AXES for dt in (ds.DS_F32, ds.DS_F16, ds.DS_U8_RGB, ds.DS_U8)
           for shape in (0, 1) if shape == 0 or a[2] != (4, 9) or dt in (ds.DS_U8_RGB, ds.DS_U8)]


@pytest.mark.parametrize("axes,dt,shape", CLASSES)
@pytest.mark.parametrize("H,W", SHAPES)
def test_checked_build_every_class(checked, oracle, H, W, axes, dt, shape):
    rh, Kh, rv, Kv = axes
    pl = ds.ds_plan_create_ex(H, W, rh, Kh, rv, Kv, dt)
    try:
        ds.ds_plan_set_schedule_ex(pl, 0, 0, shape)
        x = frames((H, W), dt, 3, H * 31 + W)
        got = run_fused(pl, x)  # ds_stream_check inside: raises on a failed bounds check
        assert_parity(got, _oracle(oracle, x, rh, Kh, rv, Kv, dt), dt, ds.ds_plan_describe(pl))
    finally:
        ds.ds_destroy(pl)


def test_checked_build_large_batch_with_tail_split(checked, oracle):
    """Enough frames that the launch's last tiles run in shorter bands, the job
    split in two, plus the CIF planes of odd counts in one launch."""
    pl = ds.ds_plan_create(270, 480, (3, 8), 8, ds.DS_F32)
    py = ds.ds_plan_create_ex(288, 352, (3, 8), 8, (4, 9), 8, ds.DS_U8)
    pc = ds.ds_plan_create_ex(144, 176, (3, 8), 8, (4, 9), 8, ds.DS_U8)
    try:
        x = frames((270, 480), ds.DS_F32, 97, 5)
        got = run_fused(pl, x)
        assert_parity(got, oracle.filter_ex(x.astype(np.float64), (3, 8), 8, (3, 8), 8), ds.DS_F32)
        counts = (5, 3, 3)
        xs = [frames((288, 352), ds.DS_U8, 5, 6), frames((144, 176), ds.DS_U8, 3, 7), frames((144, 176), ds.DS_U8, 3, 8)]
        ins = [to_dev(a) for a in xs]
        outs = [out_buffer(py, 5), out_buffer(pc, 3), out_buffer(pc, 3)]
        ds.ds_batch_run([(p, i.data_ptr(), o.data_ptr(), n) for p, i, o, n in zip((py, pc, pc), ins, outs, counts)],
                        stream())
        finish()
        for o, a in zip(outs, xs):
            assert_parity(o.cpu().numpy(), oracle.filter_ex(a, (3, 8), 8, (4, 9), 8), ds.DS_U8)
    finally:
        for p in (pl, py, pc):
            ds.ds_destroy(p)


def test_bounds_probe_is_reported_and_the_context_stays_usable(checked, oracle):
    ds.ds_debug_bounds_probe(stream())
    with pytest.raises(ds.DsError) as e:
        ds.ds_stream_check(stream())
    assert e.value.status == ds.DS_ERR_BOUNDS
    ds.ds_stream_check(stream())  # the read cleared the word
    pl = ds.ds_plan_create(72, 528, (1, 2), 6, ds.DS_U8_RGB)
    try:
        x = frames((72, 528), ds.DS_U8_RGB, 2, 9)
        assert_parity(run_fused(pl, x), oracle.filter_u8(x, 1, 2, 6), ds.DS_U8_RGB)
    finally:
        ds.ds_destroy(pl)


@pytest.mark.parametrize("rh,Kh,rv,Kv,dt", [((3, 8), 8, (3, 8), 8, ds.DS_F32), ((1, 2), 6, (1, 2), 6, ds.DS_U8_RGB),
                                            ((3, 8), 8, (4, 9), 8, ds.DS_U8)])
def test_checked_build_given_taps(checked, oracle, rh, Kh, rv, Kv, dt):
    """Given tap tables on the fast kernel, with every index check passing."""
    rng = np.random.default_rng(Kh + Kv)
    wh, wv = rng.normal(0, 0.3, (rh[0], Kh)), rng.normal(0, 0.3, (rv[0], Kv))
    wh[:, Kh // 2] += 1.0
    wv[:, Kv // 2] += 1.0
    pl = ds.ds_plan_create_ex(100, 272, rh, Kh, rv, Kv, dt, ds.DS_CLAMP, wh, wv)
    try:
        assert '"fused_tma"' in ds.ds_plan_describe(pl)
        x = frames((100, 272), dt, 3, 77)
        xo = x if dt in (ds.DS_U8, ds.DS_U8_RGB) else x.astype(np.float64)
        want = oracle.filter_ex(xo, rh, Kh, rv, Kv, weights_h=wh, weights_v=wv)
        assert_parity(run_fused(pl, x), want, dt, "given taps, checked build")
    finally:
        ds.ds_destroy(pl)


@pytest.mark.parametrize("axes,dt", [(c[0], c[1]) for c in CLASSES
                                     if c[2] == 0 and (c[0][2] != (4, 9) or c[1] in (ds.DS_U8, ds.DS_U8_RGB))])
@pytest.mark.parametrize("H,W", [(41, 1104), (3, 1056), (97, 1040)])
def test_checked_build_modular_tilers(checked, oracle, H, W, axes, dt):
    """The row copies of modular tilers (tile shape 0, the one compiled for
    them) with every index check passing."""
    rh, Kh, rv, Kv = axes
    pl = ds.ds_plan_create_ex(H, W, rh, Kh, rv, Kv, dt, ds.DS_WRAP)
    try:
        assert '"fused_tma"' in ds.ds_plan_describe(pl) and ds.ds_plan_tile_shapes(pl) == 1
        x = frames((H, W), dt, 3, H + W)
        xo = x if dt in (ds.DS_U8, ds.DS_U8_RGB) else x.astype(np.float64)
        assert_parity(run_fused(pl, x), oracle.filter_ex(xo, rh, Kh, rv, Kv, wrap=True), dt, "checked wrap")
    finally:
        ds.ds_destroy(pl)
