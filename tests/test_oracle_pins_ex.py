"""Pins for the extended oracle: a ratio and tap table per axis, and the
modular (wrap) boundary of Array-OL tilers.  The facts they check do not
come from the oracle itself:

* the Lanczos taps of the vertical 4/9 axis of the paper's CIF case, in
  closed form (sines of multiples of pi/96 from square roots by half angles);
* a dense-matrix restatement Y = M_v X M_h^T with separate axes and the
  boundary folded into the matrices by clamping or by modulo;
* the periodic extension: a modular tiler on a frame equals the clamped
  tiler on the 3 x 3 tiling of the frame, centre block;
* one-hot tap tables reduce the filter to exact sampling at floor(centre);
* Q14 quantisation of arbitrary tables: row sums, rounding, residual tap;
* the paper's CIF shape 352 x 288 -> 132 x 128 (Sec. 3) with H 3/8, V 4/9.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

# --------------------------------------------------------------------------
# sin / cos of pi * x for x with denominator 2^k or 3 * 2^k, from square
# roots only: a table of multiples of pi/12, then half angles
# --------------------------------------------------------------------------
_S2, _S3, _S6 = math.sqrt(2.0), math.sqrt(3.0), math.sqrt(6.0)
_SIN12 = [0.0, (_S6 - _S2) / 4, 0.5, _S2 / 2, _S3 / 2, (_S6 + _S2) / 4, 1.0]


def _sc_base(n):
    """(sin, cos) of n pi / 12, any integer n."""
    n %= 24
    def s(m):  # sin(m pi/12), 0 <= m < 24
        sign = 1.0
        if m >= 12:
            m -= 12
            sign = -1.0
        return sign * (_SIN12[m] if m <= 6 else _SIN12[12 - m])
    return s(n), s((n + 6) % 24)


def _sc(x: Fraction):
    """(sin pi x, cos pi x) by half angles down from the pi/12 table."""
    x = x % 2
    if (12 * x).denominator == 1:
        return _sc_base(int(12 * x))
    assert x.denominator % 2 == 0, x
    y = 2 * x  # angle pi x = (pi y) / 2, y in [0, 4)
    _, cy = _sc(y)
    half = float(x)  # x in [0, 2): pi x in [0, 2 pi)
    s = math.sqrt(max(0.0, (1.0 - cy) / 2.0))
    c = math.sqrt(max(0.0, (1.0 + cy) / 2.0))
    if half >= 1.0:  # pi x in [pi, 2 pi)
        s = -s
    if 0.5 < half < 1.5:  # pi x in (pi/2, 3pi/2)
        c = -c
    return s, c


def _lanczos3(x: Fraction):
    if x == 0:
        return 1.0
    if abs(x) >= 3:
        return 0.0
    xf = float(x)
    return (_sc(x)[0] / (math.pi * xf)) * (_sc(x / 3)[0] / (math.pi * xf / 3))


def test_half_angle_sines():
    for n in range(-200, 200):
        x = Fraction(n, 96)
        assert _sc(x)[0] == pytest.approx(math.sin(math.pi * n / 96), abs=1e-14)
        assert _sc(x)[1] == pytest.approx(math.cos(math.pi * n / 96), abs=1e-14)


# Vertical axis of the paper's CIF case, 4/9 with K=8 (sigma = 3/4): centres
# c_j = ((2j+1) 9 - 4) / 8 = 5/8, 23/8, 41/8, 59/8, window starts
# b_j = floor(c_j) - 3 = -3, -1, 2, 4, kernel arguments 3/4 (b_j + t - c_j):
ARGS_4_9_K8 = [[Fraction(24 * t - 87, 32) for t in range(8)],
               [Fraction(24 * t - 93, 32) for t in range(8)],
               [Fraction(24 * t - 75, 32) for t in range(8)],
               [Fraction(24 * t - 81, 32) for t in range(8)]]


def test_taps_4_9_closed_form(oracle):
    want = []
    for args in ARGS_4_9_K8:
        v = np.array([_lanczos3(a) for a in args])
        want.append(v / v.sum())
    np.testing.assert_allclose(oracle.taps_f64(4, 9, 8), np.array(want), rtol=0, atol=2e-15)
    b, _ = oracle.phase_windows(4, 9, 8)
    assert list(b) == [-3, -1, 2, 4]


def test_paper_cif_shape_per_axis(oracle):
    rows = [l.split() for l in open(os.path.join(GOLDEN, "paper_cif_shapes.txt"))
            if l.strip() and not l.startswith("#")]
    h = [r for r in rows if r[0] == "horizontal"][0]
    v = [r for r in rows if r[0] == "vertical"][0]
    x = np.zeros((1, int(v[1]), int(h[1]), 3), np.uint8)
    y = oracle.filter_ex(x, (int(h[3]), int(h[4])), 8, (int(v[3]), int(v[4])), 8)
    assert y.shape == (1, int(v[2]), int(h[2]), 3) == (1, 128, 132, 3)


# --------------------------------------------------------------------------
# Dense restatement with separate axes and a boundary
# --------------------------------------------------------------------------

def _window(o, p, q, K):
    centre = Fraction(2 * o + 1, 2) * Fraction(q, p) - Fraction(1, 2)
    lo = math.floor(centre)
    return list(range(lo - K // 2 + 1, lo + K // 2 + 1))


def _dense(n_in, p, q, taps, wrap):
    K = taps.shape[1]
    n_out = (n_in * p) // q
    M = np.zeros((n_out, n_in), taps.dtype)
    for o in range(n_out):
        for t, i in enumerate(_window(o, p, q, K)):
            M[o, i % n_in if wrap else min(max(i, 0), n_in - 1)] += taps[o % p, t]
    return M


def _dense_ex(x, rh, rv, th, tv, wrap):
    n, H, W, C = x.shape
    if x.dtype == np.uint8:
        Mh = _dense(W, rh[0], rh[1], th.astype(np.int64), wrap)
        Mv = _dense(H, rv[0], rv[1], tv.astype(np.int64), wrap)
        y = np.empty((n, Mv.shape[0], Mh.shape[0], C), np.uint8)
        for f in range(n):
            for ch in range(C):
                h = np.clip((x[f, :, :, ch].astype(np.int64) @ Mh.T + 8192) // 16384, 0, 255)
                y[f, :, :, ch] = np.clip((Mv @ h + 8192) // 16384, 0, 255)
        return y
    Mh, Mv = _dense(W, rh[0], rh[1], th, wrap), _dense(H, rv[0], rv[1], tv, wrap)
    y = np.empty((n, Mv.shape[0], Mh.shape[0], C))
    for f in range(n):
        for ch in range(C):
            y[f, :, :, ch] = Mv @ x[f, :, :, ch] @ Mh.T
    return y


EX_CASES = [
    # (rh, Kh, rv, Kv, H, W, C, wrap)
    ((3, 8), 8, (4, 9), 8, 36, 40, 1, False), ((3, 8), 8, (4, 9), 8, 27, 33, 3, True),
    ((1, 2), 6, (2, 3), 6, 17, 30, 3, False), ((1, 2), 6, (2, 3), 6, 18, 22, 1, True),
    ((2, 3), 6, (3, 8), 8, 40, 25, 1, True), ((5, 7), 10, (1, 4), 16, 29, 22, 1, False),
    ((3, 8), 8, (3, 8), 8, 5, 9, 1, True), ((1, 2), 2, (1, 3), 4, 7, 6, 2, True),
]


@pytest.mark.parametrize("rh,Kh,rv,Kv,H,W,C,wrap", EX_CASES)
def test_ex_matches_dense_form(oracle, rh, Kh, rv, Kv, H, W, C, wrap):
    rng = np.random.default_rng(H * 131 + W)
    x = rng.random((2, H, W, C))
    got = oracle.filter_ex(x, rh, Kh, rv, Kv, wrap=wrap)
    want = _dense_ex(x, rh, rv, oracle.taps_f64(*rh, Kh), oracle.taps_f64(*rv, Kv), wrap)
    assert got.shape == want.shape
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-13)
    xu = rng.integers(0, 256, (2, H, W, C), dtype=np.uint8)
    got = oracle.filter_ex(xu, rh, Kh, rv, Kv, wrap=wrap)
    want = _dense_ex(xu, rh, rv, oracle.taps_q14(*rh, Kh), oracle.taps_q14(*rv, Kv), wrap)
    np.testing.assert_array_equal(got, want)


@pytest.mark.parametrize("rh,Kh,rv,Kv", [((3, 8), 8, (4, 9), 8), ((1, 2), 6, (2, 3), 6), ((2, 3), 6, (3, 8), 8)])
def test_wrap_is_the_periodic_extension(oracle, rh, Kh, rv, Kv):
    # frame extents multiples of q so the output grids of the tiling line up
    H, W = rv[1] * 4, rh[1] * 5
    rng = np.random.default_rng(7)
    for x in (rng.random((1, H, W, 2)), rng.integers(0, 256, (1, H, W, 2), dtype=np.uint8)):
        got = oracle.filter_ex(x, rh, Kh, rv, Kv, wrap=True)
        big = np.tile(x, (1, 3, 3, 1))
        ref = oracle.filter_ex(big, rh, Kh, rv, Kv, wrap=False)
        OH, OW = got.shape[1], got.shape[2]
        np.testing.assert_array_equal(got, ref[:, OH:2 * OH, OW:2 * OW])


def test_same_axes_equal_the_plain_filter(oracle):
    rng = np.random.default_rng(3)
    x = rng.random((2, 37, 41, 3))
    np.testing.assert_array_equal(oracle.filter_ex(x, (2, 3), 6, (2, 3), 6), oracle.filter_f64(x, 2, 3, 6))
    xu = rng.integers(0, 256, (2, 37, 41, 3), dtype=np.uint8)
    np.testing.assert_array_equal(oracle.filter_ex(xu, (3, 8), 8, (3, 8), 8), oracle.filter_u8(xu, 3, 8, 8))


def test_axes_swap_with_transpose_fp64(oracle):
    rng = np.random.default_rng(4)
    x = rng.random((1, 45, 52, 1))
    a = oracle.filter_ex(x, (3, 8), 8, (4, 9), 8)
    b = oracle.filter_ex(np.ascontiguousarray(x.transpose(0, 2, 1, 3)), (4, 9), 8, (3, 8), 8)
    np.testing.assert_allclose(a, b.transpose(0, 2, 1, 3), rtol=0, atol=1e-12)


def test_constant_frames_stay_constant_with_wrap(oracle):
    for x, tol in ((np.full((1, 30, 44, 3), 0.375), 1e-14), (np.full((1, 30, 44, 3), 201, np.uint8), 0)):
        y = oracle.filter_ex(x, (3, 8), 8, (4, 9), 8, wrap=True)
        assert np.abs(y.astype(np.float64) - x.flat[0]).max() <= tol


# --------------------------------------------------------------------------
# Caller-given tap tables
# --------------------------------------------------------------------------

def _one_hot(p, K):
    w = np.zeros((p, K))
    w[:, K // 2 - 1] = 1.0  # the tap at floor(centre)
    return w


@pytest.mark.parametrize("wrap", [False, True])
def test_one_hot_taps_sample_at_the_floor_of_the_centre(oracle, wrap):
    rh, rv, Kh, Kv = (3, 8), (4, 9), 8, 6
    H, W = 31, 45
    rng = np.random.default_rng(5)
    x = rng.random((1, H, W, 2))
    got = oracle.filter_ex(x, rh, Kh, rv, Kv, wrap=wrap, weights_h=_one_hot(3, Kh), weights_v=_one_hot(4, Kv))
    OH, OW = H * 4 // 9, W * 3 // 8
    ys = [math.floor(Fraction(2 * o + 1, 2) * Fraction(9, 4) - Fraction(1, 2)) for o in range(OH)]
    xs = [math.floor(Fraction(2 * o + 1, 2) * Fraction(8, 3) - Fraction(1, 2)) for o in range(OW)]
    fix = (lambda i, n: i % n) if wrap else (lambda i, n: min(max(i, 0), n - 1))
    want = x[:, [fix(i, H) for i in ys]][:, :, [fix(i, W) for i in xs]]
    np.testing.assert_array_equal(got, want)
    xu = rng.integers(0, 256, (1, H, W, 2), dtype=np.uint8)
    got = oracle.filter_ex(xu, rh, Kh, rv, Kv, wrap=wrap, weights_h=_one_hot(3, Kh), weights_v=_one_hot(4, Kv))
    np.testing.assert_array_equal(got, xu[:, [fix(i, H) for i in ys]][:, :, [fix(i, W) for i in xs]])


def test_given_taps_scale_linearly_fp64(oracle):
    rng = np.random.default_rng(6)
    x = rng.random((1, 40, 48, 1))
    wh, wv = oracle.taps_f64(1, 2, 6), oracle.taps_f64(2, 3, 6)
    a = oracle.filter_ex(x, (1, 2), 6, (2, 3), 6, weights_h=wh, weights_v=wv)
    b = oracle.filter_ex(x, (1, 2), 6, (2, 3), 6, weights_h=2 * wh, weights_v=-0.5 * wv)
    np.testing.assert_allclose(b, -a, rtol=0, atol=1e-13)
    np.testing.assert_array_equal(a, oracle.filter_ex(x, (1, 2), 6, (2, 3), 6))


def test_quantize_q14_of_arbitrary_tables(oracle):
    rng = np.random.default_rng(8)
    for _ in range(200):
        p, K = int(rng.integers(1, 6)), int(rng.choice([2, 4, 6, 8]))
        w = rng.normal(0.0, 0.6, (p, K))
        qt = oracle.quantize_q14(w).astype(np.int64)
        naive = np.floor(w * 16384 + 0.5).astype(np.int64)
        for j in range(p):
            assert qt[j].sum() == math.floor(w[j].sum() * 16384 + 0.5)
            big = int(np.argmax(w[j]))
            others = [t for t in range(K) if t != big]
            assert np.array_equal(qt[j, others], naive[j, others])
    for p, q, K in [(3, 8, 8), (1, 2, 6), (2, 3, 6), (4, 9, 8)]:
        np.testing.assert_array_equal(oracle.quantize_q14(oracle.taps_f64(p, q, K)), oracle.taps_q14(p, q, K))


def test_ex_rejects_bad_arguments(oracle):
    x = np.zeros((1, 20, 20), np.float64)
    for args in [((2, 4), 6, (1, 2), 6), ((1, 2), 5, (1, 2), 6), ((1, 2), 6, (3, 2), 6), ((1, 2), 18, (1, 2), 6)]:
        with pytest.raises(ValueError):
            oracle.filter_ex(x, *args)
    with pytest.raises(ValueError):
        oracle.filter_ex(x, (1, 2), 6, (1, 2), 6, weights_h=np.array([[0.5, np.nan, 0.5, 0, 0, 0]]))
