"""Pins for the CPU oracle against facts that do not come from the oracle itself.

* shape facts the paper prints (Sec. 3, Sec. 3.A) -- tests/golden/paper_cif_shapes.txt;
* tap values in closed form: Lanczos-3 at rational offsets, evaluated through
  sines of special angles built from square roots only (no libm sine), with
  the sample offsets derived by hand for each ratio;
* exact rational Q14 taps of the 1/2 ratio;
* a dense-matrix restatement Y = M_v X M_h^T evaluated with numpy matmul,
  with each window found as "the K/2 integers at or below the centre and the
  K/2 above it";
* invariants: impulse response, constant frames, linearity, mirror
  equivariance, separability (order of the passes), uint8 vs FP64 error bound.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

# --------------------------------------------------------------------------
# sin(pi * n / 24) from square roots only (half-angle and special angles)
# --------------------------------------------------------------------------
_S2, _S3, _S6 = math.sqrt(2.0), math.sqrt(3.0), math.sqrt(6.0)
# sin(j pi / 12), j = 0..6
_SIN12 = [0.0, (_S6 - _S2) / 4, 0.5, _S2 / 2, _S3 / 2, (_S6 + _S2) / 4, 1.0]


def _sin12(j):
    """sin(j pi/12) for 0 <= j <= 12 (first two quadrants)."""
    return _SIN12[j] if j <= 6 else _SIN12[12 - j]


def _sin_pi24(n):
    """sin(n pi / 24) for any integer n, from square roots only."""
    n %= 48
    sign = 1.0
    if n >= 24:
        n -= 24
        sign = -1.0
    if n > 12:
        n = 24 - n  # sin(pi - a) = sin(a)
    if n % 2 == 0:
        return sign * _sin12(n // 2)
    # odd n: half-angle, sin(a/2) = sqrt((1 - cos a) / 2), a = n pi/12 in (0, pi)
    cos_a = _sin12(6 - n) if n <= 6 else -_sin12(n - 6)
    return sign * math.sqrt((1.0 - cos_a) / 2.0)


def _sin_pi(x: Fraction):
    """sin(pi x) for x with a denominator dividing 24."""
    assert (24 % x.denominator) == 0, x
    return _sin_pi24(int(x * 24))


def _lanczos3(x: Fraction):
    if x == 0:
        return 1.0
    if abs(x) >= 3:
        return 0.0
    xf = float(x)
    return (_sin_pi(x) / (math.pi * xf)) * (_sin_pi(x / 3) / (math.pi * xf / 3))


# Hand-derived kernel arguments sigma * (b_j + t - c_j), t = 0..K-1, per phase.
#   3/8, K=8, sigma=3/4: c = 5/6, 7/2, 37/6; b = -3, 0, 3
#     -> (6t-23)/8, (6t-21)/8, (6t-19)/8
#   1/2, K=6, sigma=1: c = 1/2, b = -2 -> (2t-5)/2
#   2/3, K=6, sigma=1: c = 1/4, 7/4; b = -2, -1 -> (4t-9)/4, (4t-11)/4
#   1/3, K=12, sigma=1/2: c = 1, b = -4 -> (t-5)/2
#   1/3, K=6, sigma=1: c = 1, b = -1 -> t-2   (integer offsets: a pure sample)
HAND_ARGS = {
    (3, 8, 8): [[Fraction(6 * t - 23, 8) for t in range(8)],
                [Fraction(6 * t - 21, 8) for t in range(8)],
                [Fraction(6 * t - 19, 8) for t in range(8)]],
    (1, 2, 6): [[Fraction(2 * t - 5, 2) for t in range(6)]],
    (2, 3, 6): [[Fraction(4 * t - 9, 4) for t in range(6)],
                [Fraction(4 * t - 11, 4) for t in range(6)]],
    (1, 3, 12): [[Fraction(t - 5, 2) for t in range(12)]],
    (1, 3, 6): [[Fraction(t - 2) for t in range(6)]],
}


def _closed_form_taps(key):
    rows = []
    for args in HAND_ARGS[key]:
        v = np.array([_lanczos3(a) for a in args])
        rows.append(v / v.sum())
    return np.array(rows)


def test_radical_sines_match_special_values():
    # the helper itself: known values
    assert _sin_pi(Fraction(1, 2)) == pytest.approx(1.0, abs=1e-15)
    assert _sin_pi(Fraction(1, 6)) == pytest.approx(0.5, abs=1e-15)
    assert _sin_pi(Fraction(1, 8)) == pytest.approx(math.sqrt(2 - math.sqrt(2)) / 2, abs=1e-15)
    assert _sin_pi(Fraction(-7, 8)) == pytest.approx(-math.sqrt(2 - math.sqrt(2)) / 2, abs=1e-15)
    assert _sin_pi(Fraction(5, 4)) == pytest.approx(-math.sqrt(2) / 2, abs=1e-15)
    # sin^2 + cos^2 = 1 on the whole 1/24 grid (cos a = sin(a + pi/2))
    for n in range(-48, 49):
        s = _sin_pi24(n)
        c = _sin_pi24(n + 12)
        assert s * s + c * c == pytest.approx(1.0, abs=1e-14)


@pytest.mark.parametrize("key", sorted(HAND_ARGS))
def test_taps_closed_form(oracle, key):
    p, q, K = key
    got = oracle.taps_f64(p, q, K)
    want = _closed_form_taps(key)
    np.testing.assert_allclose(got, want, rtol=0, atol=2e-15)


def test_taps_half_ratio_exact_rational(oracle):
    # L(1/2) = 6/pi^2, L(3/2) = -4/(3 pi^2), L(5/2) = 6/(25 pi^2): after
    # normalisation the pi^2 cancels, leaving [18, -100, 450, 450, -100, 18]/736.
    want = [Fraction(v, 736) for v in (18, -100, 450, 450, -100, 18)]
    got = oracle.taps_f64(1, 2, 6)[0]
    np.testing.assert_allclose(got, [float(v) for v in want], rtol=0, atol=1e-15)
    # Q14 = floor(16384 w + 1/2) exactly; the sum is 16384 with no residual
    q14 = [math.floor(v * 16384 + Fraction(1, 2)) for v in want]
    assert q14 == [401, -2226, 10017, 10017, -2226, 401]
    assert list(oracle.taps_q14(1, 2, 6)[0]) == q14


def test_taps_integer_offsets_are_a_pure_sample(oracle):
    # 1/3 with K=6: the centre falls on an input pixel and the sinc zeros on
    # every other tap -> decimation by plain sampling.
    np.testing.assert_allclose(oracle.taps_f64(1, 3, 6), [[0, 0, 1, 0, 0, 0]], atol=1e-16)
    assert list(oracle.taps_q14(1, 3, 6)[0]) == [0, 0, 16384, 0, 0, 0]


@pytest.mark.parametrize("p,q,K", [(3, 8, 8), (1, 2, 6), (2, 3, 6), (3, 8, 6), (1, 2, 8),
                                   (2, 3, 8), (5, 7, 10), (1, 4, 16), (3, 4, 4), (1, 2, 2)])
def test_taps_sum_symmetry_q14(oracle, p, q, K):
    w = oracle.taps_f64(p, q, K)
    np.testing.assert_allclose(w.sum(axis=1), 1.0, atol=1e-15)
    # phases mirror: w_{p-1-j} = reverse(w_j).  A phase whose centre is an
    # integer has the even-K window one tap longer on the right, where the
    # kernel argument is sigma*K/2 = 3 and the weight is exactly 0: there the
    # mirror holds for the first K-1 taps.
    _, c = oracle.phase_windows(p, q, K)
    for j in range(p):
        if float(c[j]).is_integer():
            assert w[j, K - 1] == 0.0
            np.testing.assert_allclose(w[j, :K - 1], w[p - 1 - j, :K - 1][::-1], atol=1e-15)
        else:
            np.testing.assert_allclose(w[p - 1 - j, ::-1], w[j], atol=1e-15)
    q14 = oracle.taps_q14(p, q, K)
    assert (q14.sum(axis=1) == 16384).all()
    assert np.abs(q14 - np.floor(w * 16384 + 0.5)).max() <= 2  # only the residual tap moves


def test_phase_windows_are_centred(oracle):
    # window = the K/2 integers at or below the centre and the K/2 above it
    for p, q, K in [(3, 8, 8), (1, 2, 6), (2, 3, 6), (5, 7, 10), (1, 3, 12)]:
        b, c = oracle.phase_windows(p, q, K)
        for j in range(p):
            cj = Fraction((2 * j + 1) * q - p, 2 * p)
            assert c[j] == pytest.approx(float(cj), abs=1e-15)
            window = list(range(b[j], b[j] + K))
            assert sum(1 for i in window if i <= cj) == K // 2
            assert sum(1 for i in window if i > cj) == K // 2


def test_paper_shapes_golden(oracle):
    rows = []
    with open(os.path.join(GOLDEN, "paper_cif_shapes.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append(line.split())
    h = [r for r in rows if r[0] == "horizontal"][0]
    n_in, n_out, p, q, lines, packets = int(h[1]), int(h[2]), int(h[3]), int(h[4]), int(h[5]), int(h[6])
    assert oracle.out_extent(n_in, p, q) == n_out
    # repetition space of the horizontal task: lines x packets of q pixels
    assert -(-n_out // p) == packets == n_in // q
    assert lines == 288
    v = [r for r in rows if r[0] == "vertical"][0]
    assert oracle.out_extent(int(v[1]), int(v[3]), int(v[4])) == int(v[2])


# --------------------------------------------------------------------------
# Dense-matrix restatement of the separable filter
# --------------------------------------------------------------------------

def _window(o, p, q, K):
    """Input indices of output o: K/2 integers <= centre, K/2 above (unclamped)."""
    centre = Fraction(2 * o + 1, 2) * Fraction(q, p) - Fraction(1, 2)
    lo = math.floor(centre)
    return list(range(lo - K // 2 + 1, lo + K // 2 + 1))


def _dense(n_in, p, q, taps):
    K = taps.shape[1]
    n_out = (n_in * p) // q
    M = np.zeros((n_out, n_in), taps.dtype)
    for o in range(n_out):
        for t, i in enumerate(_window(o, p, q, K)):
            M[o, min(max(i, 0), n_in - 1)] += taps[o % p, t]
    return M


def _dense_filter_f64(x, p, q, K, taps):
    n, H, W, C = x.shape
    Mh, Mv = _dense(W, p, q, taps), _dense(H, p, q, taps)
    y = np.empty((n, Mv.shape[0], Mh.shape[0], C))
    for f in range(n):
        for ch in range(C):
            y[f, :, :, ch] = Mv @ x[f, :, :, ch] @ Mh.T
    return y


def _dense_filter_u8(x, p, q, K, q14):
    n, H, W, C = x.shape
    Mh, Mv = _dense(W, p, q, q14.astype(np.int64)), _dense(H, p, q, q14.astype(np.int64))
    y = np.empty((n, Mv.shape[0], Mh.shape[0], C), np.uint8)
    for f in range(n):
        for ch in range(C):
            h = np.clip((x[f, :, :, ch].astype(np.int64) @ Mh.T + 8192) // 16384, 0, 255)
            y[f, :, :, ch] = np.clip((Mv @ h + 8192) // 16384, 0, 255)
    return y


SMALL_CASES = [
    # (p, q, K, H, W, C, n)
    (3, 8, 8, 40, 37, 1, 2), (3, 8, 8, 8, 8, 1, 1), (3, 8, 8, 3, 11, 1, 1),
    (1, 2, 6, 17, 30, 3, 2), (1, 2, 6, 2, 2, 1, 1), (2, 3, 6, 25, 31, 1, 1),
    (2, 3, 6, 2, 5, 3, 1), (5, 7, 10, 29, 22, 1, 1), (1, 4, 16, 33, 12, 1, 1),
    (3, 4, 4, 9, 14, 2, 1), (1, 2, 2, 6, 7, 1, 1), (3, 8, 6, 19, 40, 3, 1),
]


@pytest.mark.parametrize("p,q,K,H,W,C,n", SMALL_CASES)
def test_f64_matches_dense_matrix_form(oracle, p, q, K, H, W, C, n):
    rng = np.random.default_rng(H * 1000 + W)
    x = rng.random((n, H, W, C))
    got = oracle.filter_f64(x, p, q, K)
    want = _dense_filter_f64(x, p, q, K, oracle.taps_f64(p, q, K))
    assert got.shape == want.shape == (n, H * p // q, W * p // q, C)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-13)


@pytest.mark.parametrize("p,q,K,H,W,C,n", SMALL_CASES)
def test_u8_matches_dense_integer_form(oracle, p, q, K, H, W, C, n):
    rng = np.random.default_rng(H * 1000 + W + 7)
    x = rng.integers(0, 256, (n, H, W, C), dtype=np.uint8)
    got = oracle.filter_u8(x, p, q, K)
    want = _dense_filter_u8(x, p, q, K, oracle.taps_q14(p, q, K))
    np.testing.assert_array_equal(got, want)


@pytest.mark.parametrize("p,q,K", [(3, 8, 8), (1, 2, 6), (2, 3, 6)])
def test_impulse_gives_outer_product_of_taps(oracle, p, q, K):
    H, W = 48, 64
    y0, x0 = 21, 30
    x = np.zeros((H, W))
    x[y0, x0] = 1.0
    y = oracle.filter_f64(x, p, q, K)
    w = oracle.taps_f64(p, q, K)
    # the response column: tap of output o that lands on input index i (interior)
    def column(n_in, i):
        n_out = n_in * p // q
        col = np.zeros(n_out)
        for o in range(n_out):
            win = _window(o, p, q, K)
            if i in win:
                col[o] = w[o % p, win.index(i)]
        return col
    want = np.outer(column(H, y0), column(W, x0))
    np.testing.assert_allclose(y, want, atol=1e-15)
    assert np.count_nonzero(np.abs(y) > 1e-18) == np.count_nonzero(want)


@pytest.mark.parametrize("p,q,K", [(3, 8, 8), (1, 2, 6), (2, 3, 6), (5, 7, 10)])
def test_constant_frame_stays_constant(oracle, p, q, K):
    x = np.full((2, 30, 41, 3), 0.3125)
    np.testing.assert_allclose(oracle.filter_f64(x, p, q, K), 0.3125, atol=1e-15)
    for v in (0, 1, 77, 254, 255):
        xu = np.full((1, 30, 41, 3), v, np.uint8)
        assert (oracle.filter_u8(xu, p, q, K) == v).all()


def test_linearity(oracle):
    rng = np.random.default_rng(5)
    a, b = rng.random((2, 33, 50)), rng.random((2, 33, 50))
    fa, fb = oracle.filter_f64(a, 3, 8, 8), oracle.filter_f64(b, 3, 8, 8)
    np.testing.assert_allclose(oracle.filter_f64(2.5 * a - 0.75 * b, 3, 8, 8),
                               2.5 * fa - 0.75 * fb, atol=1e-13)


@pytest.mark.parametrize("p,q,K,H,W", [(3, 8, 8, 48, 64), (1, 2, 6, 30, 22), (2, 3, 6, 27, 33)])
def test_mirror_equivariance(oracle, p, q, K, H, W):
    # with n*p/q integral the centre map is symmetric about the frame middle
    assert (H * p) % q == 0 and (W * p) % q == 0
    x = np.random.default_rng(9).random((H, W))
    y = oracle.filter_f64(x, p, q, K)
    np.testing.assert_allclose(oracle.filter_f64(x[:, ::-1], p, q, K), y[:, ::-1], atol=1e-14)
    np.testing.assert_allclose(oracle.filter_f64(x[::-1, :], p, q, K), y[::-1, :], atol=1e-14)


def test_separable_order_fp64(oracle):
    # FP64: horizontal-then-vertical equals vertical-then-horizontal
    x = np.random.default_rng(3).random((45, 62))
    hv = oracle.filter_f64(x, 3, 8, 8)
    vh = oracle.filter_f64(x.T.copy(), 3, 8, 8).T
    np.testing.assert_allclose(hv, vh, atol=1e-13)


@pytest.mark.parametrize("p,q,K", [(3, 8, 8), (1, 2, 6), (2, 3, 6)])
def test_u8_within_rounding_of_fp64(oracle, p, q, K):
    # inputs in [64, 191]: Lanczos overshoot (sum |w| < 1.55) never reaches the
    # clamp, so the integer path differs from the exact filter only by the Q14
    # quantisation and two roundings: |err| <= 0.6 + 1.55 * 0.6 < 1.6
    x = np.random.default_rng(11).integers(64, 192, (3, 40, 56, 3), dtype=np.uint8)
    yu = oracle.filter_u8(x, p, q, K).astype(np.float64)
    yf = oracle.filter_f64(x, p, q, K)
    assert np.abs(yu - yf).max() < 1.6


def test_bad_arguments_rejected(oracle):
    with pytest.raises(ValueError):
        oracle.taps_f64(2, 4, 8)  # not lowest terms
    with pytest.raises(ValueError):
        oracle.taps_f64(3, 8, 7)  # odd K
    with pytest.raises(ValueError):
        oracle.taps_f64(8, 3, 8)  # upsampling
    with pytest.raises(ValueError):
        oracle.filter_f64(np.zeros((2, 2)), 3, 8, 8)  # empty output
