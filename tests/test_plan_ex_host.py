"""Extended plans on the host: per-axis ratios, the boundary and caller-given
tap tables -- argument checks and tap tables against the oracle (no GPU)."""
import numpy as np
import pytest

import paper_1103_4881_b300 as ds


def _ex(**kw):
    args = dict(in_h=64, in_w=64, ratio_h=(3, 8), taps_h=8, ratio_v=(4, 9), taps_v=8, dtype=ds.DS_F32)
    args.update(kw)
    return ds.ds_plan_create_ex(**args)


@pytest.mark.parametrize("kw", [
    dict(ratio_v=(2, 4)), dict(ratio_h=(9, 4)), dict(taps_v=7), dict(taps_h=18), dict(boundary=2),
    dict(dtype=7), dict(in_h=2), dict(in_w=0),
    dict(weights_h=np.full((3, 8), np.nan)),
    dict(dtype=ds.DS_U8_RGB, weights_v=np.full((4, 8), 3.0)),    # Q14 taps of 49152: outside int16
    dict(dtype=ds.DS_U8, weights_h=np.full((3, 8), 0.6)),       # row magnitudes 8 x 9830 > 65535
])
def test_create_ex_rejects(kw):
    with pytest.raises(ds.DsError) as e:
        _ex(**kw)
    assert e.value.status == ds.DS_ERR_ARG


def test_axes_shapes_and_taps_match_the_oracle(oracle):
    pl = _ex(in_h=288, in_w=352, dtype=ds.DS_U8_RGB)
    try:
        assert ds.ds_plan_out_shape(pl) == (128, 132, 3)
        assert ds.ds_plan_get_axes(pl) == ((3, 8, 8), (4, 9, 8), ds.DS_CLAMP)
        assert '"fused_tma"' in ds.ds_plan_describe(pl) and "u8rgb_h3_8_v4_9_k8" in ds.ds_plan_describe(pl)
        for axis, (p, q, K) in enumerate([(3, 8, 8), (4, 9, 8)]):
            t = ds.ds_plan_get_axis_taps(pl, axis)
            np.testing.assert_allclose(t["fp64"], oracle.taps_f64(p, q, K), rtol=0, atol=1e-15)
            np.testing.assert_array_equal(t["q14"], oracle.taps_q14(p, q, K))
            np.testing.assert_array_equal(t["fp32"], oracle.taps_f64(p, q, K).astype(np.float32))
            np.testing.assert_array_equal(t["window_start"], oracle.phase_windows(p, q, K)[0])
        np.testing.assert_array_equal(ds.ds_plan_get_taps(pl)["q14"], oracle.taps_q14(3, 8, 8))
    finally:
        ds.ds_destroy(pl)
    with pytest.raises(ds.DsError):
        ds.ds_plan_get_axis_taps(pl := _ex(), 2)
    ds.ds_destroy(pl)


def test_given_taps_are_copied_and_quantised_like_the_oracle(oracle):
    rng = np.random.default_rng(2)
    wh = rng.normal(0, 0.3, (1, 6))
    wv = rng.normal(0, 0.3, (2, 6))
    pl = ds.ds_plan_create_ex(40, 48, (1, 2), 6, (2, 3), 6, ds.DS_U8, ds.DS_WRAP, wh, wv)
    try:
        wh[:] = 0  # the plan holds its own copy
        th, tv = ds.ds_plan_get_axis_taps(pl, 0), ds.ds_plan_get_axis_taps(pl, 1)
        np.testing.assert_array_equal(th["q14"], oracle.quantize_q14(th["fp64"]))
        np.testing.assert_array_equal(tv["q14"], oracle.quantize_q14(wv))
        assert np.abs(th["fp64"]).sum() > 0
        d = ds.ds_plan_describe(pl)
        assert '"boundary": "wrap"' in d and '"given_taps": true' in d and '"fused_general"' in d
    finally:
        ds.ds_destroy(pl)


def test_equal_axes_keep_the_fast_kernel():
    pl = ds.ds_plan_create_ex(1080, 1920, (3, 8), 8, (3, 8), 8, ds.DS_F32)
    try:
        assert '"fused_tma"' in ds.ds_plan_describe(pl)
    finally:
        ds.ds_destroy(pl)
    # modular tilers on a frame at least a strip wide and given taps keep the
    # fast kernel (given taps: the launch carries the plan's own tap tables)
    for kw, kernel in ((dict(boundary=ds.DS_WRAP), '"fused_tma"'),
                       (dict(weights_h=None, weights_v=np.eye(3, 8)), '"fused_tma"')):
        pl = ds.ds_plan_create_ex(1080, 1920, (3, 8), 8, (3, 8), 8, ds.DS_F32, **kw)
        try:
            assert kernel in ds.ds_plan_describe(pl)
        finally:
            ds.ds_destroy(pl)


def test_cif_classes_take_the_fast_kernel_and_pass_the_host_check():
    checked = 0
    for dt in (ds.DS_U8_RGB, ds.DS_U8):
        for H, W in [(288, 352), (144, 176), (9, 16), (30, 48), (100, 272), (1080, 1920), (17, 512), (288, 368)]:
            pl = ds.ds_plan_create_ex(H, W, (3, 8), 8, (4, 9), 8, dt)
            try:
                assert '"fused_tma"' in ds.ds_plan_describe(pl)
                for rb in (1, 2, 3, 7, 12, 1000):
                    ds.ds_plan_set_schedule(pl, rb, 0)
                    ds.ds_debug_check_plan(pl)
                    checked += 1
            finally:
                ds.ds_destroy(pl)
    assert checked == 2 * 8 * 6


def test_modular_tilers_take_the_fast_kernel_when_a_strip_fits():
    """DS_WRAP plans run on the fast kernel when a row is at least a strip and
    its halo wide (the row copies then reach at most one period past either
    end), else on the general kernels; the host replay of the kernel's index
    arithmetic passes on both sides of that limit and on ragged frames."""
    checked = fast = 0
    specs = [((3, 8), 8, (3, 8), 8), ((1, 2), 6, (1, 2), 6), ((2, 3), 6, (2, 3), 6), ((3, 8), 8, (4, 9), 8)]
    dts = (ds.DS_F32, ds.DS_F16, ds.DS_U8_RGB, ds.DS_U8)
    for rh, kh, rv, kv in specs:
        for dt in dts:
            for H, W in [(1, 1056), (5, 272), (41, 272), (200, 784), (288, 352), (144, 176), (9, 1040), (130, 1104)]:
                try:
                    pl = ds.ds_plan_create_ex(H, W, rh, kh, rv, kv, dt, ds.DS_WRAP)
                except ds.DsError:
                    continue
                try:
                    if '"fused_tma"' not in ds.ds_plan_describe(pl):
                        continue
                    fast += 1
                    for shape in range(ds.ds_plan_tile_shapes(pl)):
                        for rb in (1, 2, 5, 16, 1000):
                            ds.ds_plan_set_schedule_ex(pl, rb, 0, shape)
                            ds.ds_debug_check_plan(pl)
                            checked += 1
                finally:
                    ds.ds_destroy(pl)
    assert fast > 40 and checked == fast * 5  # modular tilers: tile shape 0 only
    # too narrow for the row copies: the general kernels
    pl = ds.ds_plan_create_ex(64, 64, (3, 8), 8, (3, 8), 8, ds.DS_F32, ds.DS_WRAP)
    try:
        assert '"fused_general"' in ds.ds_plan_describe(pl)
    finally:
        ds.ds_destroy(pl)
