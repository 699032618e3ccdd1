"""Seeded random plans on the GPU against the oracle: random frame sizes
(including tiny and ragged ones), ratios, tap counts, per-axis ratios,
boundaries and dtypes, through whichever kernel each plan selects."""
import math

import numpy as np
import pytest

import paper_1103_4881_b300 as ds
from tests.gpu_util import assert_parity, frames, run_fused, run_unfused

pytestmark = pytest.mark.gpu

FAST_AXES = [((3, 8), 8), ((1, 2), 6), ((2, 3), 6)]
DTYPES = [ds.DS_F32, ds.DS_F16, ds.DS_U8, ds.DS_U8_RGB]


def _random_axis(rng):
    if rng.random() < 0.5:
        return FAST_AXES[rng.integers(len(FAST_AXES))]
    while True:
        q = int(rng.integers(2, 17))
        p = int(rng.integers(1, q))
        if math.gcd(p, q) == 1 and p <= 16:
            return (p, q), int(rng.choice([2, 4, 6, 8, 10, 12, 16]))


def _cases(n, seed):
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < n:
        (rh, kh) = _random_axis(rng)
        (rv, kv) = (rh, kh) if rng.random() < 0.6 else _random_axis(rng)
        H = int(rng.integers(1, 300))
        W = int(rng.choice([16, 32, 48, 64, 96, 128, 256, 272, 512])) if rng.random() < 0.6 else int(rng.integers(1, 400))
        if H * rv[0] // rv[1] < 1 or W * rh[0] // rh[1] < 1:
            continue
        out.append((H, W, rh, kh, rv, kv, DTYPES[rng.integers(len(DTYPES))], int(rng.random() < 0.2)))
    return out


@pytest.mark.parametrize("H,W,rh,Kh,rv,Kv,dt,wrap", _cases(40, 2024))
def test_random_plans_match_the_oracle(oracle, H, W, rh, Kh, rv, Kv, dt, wrap):
    pl = ds.ds_plan_create_ex(H, W, rh, Kh, rv, Kv, dt, ds.DS_WRAP if wrap else ds.DS_CLAMP)
    try:
        x = frames((H, W), dt, 2, H * 7919 + W)
        got = run_fused(pl, x)
        xo = x if dt in (ds.DS_U8, ds.DS_U8_RGB) else x.astype(np.float64)
        want = oracle.filter_ex(xo, rh, Kh, rv, Kv, wrap=bool(wrap))
        assert_parity(got, want, dt, ds.ds_plan_describe(pl))
        np.testing.assert_array_equal(run_unfused(pl, x), got)
    finally:
        ds.ds_destroy(pl)


EXTREME = [((1, 64), 2), ((1, 64), 16), ((16, 17), 16), ((15, 64), 16), ((16, 33), 2), ((1, 2), 16), ((16, 63), 16)]


@pytest.mark.parametrize("ratio,K", EXTREME)
@pytest.mark.parametrize("dt", [ds.DS_F32, ds.DS_U8_RGB])
def test_extreme_ratios_and_tap_counts(oracle, ratio, K, dt):
    """The ends of the supported range (q up to 64, p up to 16, K from 2 to
    16) on ragged frames, both axes, through the general kernels."""
    H, W = 131, 197
    pl = ds.ds_plan_create_ex(H, W, ratio, K, ratio, K, dt)
    try:
        x = frames((H, W), dt, 2, ratio[0] * 100 + ratio[1] + K)
        got = run_fused(pl, x)
        xo = x if dt == ds.DS_U8_RGB else x.astype(np.float64)
        assert_parity(got, oracle.filter_ex(xo, ratio, K, ratio, K), dt, ds.ds_plan_describe(pl))
        np.testing.assert_array_equal(run_unfused(pl, x), got)
    finally:
        ds.ds_destroy(pl)


def _cif_cases(n, seed):
    """The paper's CIF axes (H 3/8 K=8, V 4/9 K=8): random heights, widths on
    and off the fast path's 16-byte rows (widths mod 128 in {16, 32, 48} give
    one-plane frames a narrow tail strip), 1-9 frames, both boundaries, and
    caller-given taps for some."""
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < n:
        H = int(rng.integers(3, 320))
        W = 16 * int(rng.integers(1, 50)) if rng.random() < 0.8 else int(rng.integers(3, 500))
        if W * 3 // 8 < 1 or H * 4 // 9 < 1:
            continue
        dt = ds.DS_U8 if rng.random() < 0.6 else ds.DS_U8_RGB
        out.append((H, W, dt, int(rng.integers(1, 10)), int(rng.random() < 0.2), int(rng.random() < 0.25),
                    int(rng.integers(1 << 30))))
    return out


@pytest.mark.parametrize("H,W,dt,n,wrap,given,seed", _cif_cases(30, 4881))
def test_random_cif_plans_match_the_oracle(oracle, H, W, dt, n, wrap, given, seed):
    rng = np.random.default_rng(seed)
    wh = wv = None
    if given:
        wh, wv = rng.normal(0, 0.2, (3, 8)), rng.normal(0, 0.2, (4, 8))
        wh[:, 3] += 1.0
        wv[:, 4] += 1.0
    pl = ds.ds_plan_create_ex(H, W, (3, 8), 8, (4, 9), 8, dt, ds.DS_WRAP if wrap else ds.DS_CLAMP, wh, wv)
    try:
        x = frames((H, W), dt, n, seed % 100000)
        got = run_fused(pl, x)
        want = oracle.filter_ex(x, (3, 8), 8, (4, 9), 8, wrap=bool(wrap), weights_h=wh, weights_v=wv)
        assert_parity(got, want, dt, ds.ds_plan_describe(pl))
        np.testing.assert_array_equal(run_unfused(pl, x), got)
    finally:
        ds.ds_destroy(pl)
