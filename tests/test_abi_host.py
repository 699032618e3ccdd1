"""Host-side tests of libds (no GPU needed): the library loads and exports every
ABI symbol, plans validate their arguments, the plan layer's tap tables agree
with the oracle's (computed by separate code), and the fused kernel's index
arithmetic passes its host self-check for a sweep of shapes."""
import ctypes
import itertools
import os
import re

import numpy as np
import pytest

import paper_1103_4881_b300 as ds

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1103_4881_b300 import build

    build.build()


def header_functions():
    text = open(os.path.join(ROOT, "include", "ds.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ds_[a-z0-9_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    names = header_functions()
    assert len(names) >= 20
    L = ctypes.CDLL(ds.LIB_PATH)
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing
    assert set(names) == set(ds.ABI_SYMBOLS)


def test_version_and_error_string():
    assert "sm_103a" in ds.ds_version()
    with pytest.raises(ds.DsError):
        ds.ds_plan_create(0, 10, (3, 8), 8, ds.DS_F32)
    assert "1x1" in ds.ds_last_error()


@pytest.mark.parametrize("args", [
    (0, 64, (3, 8), 8, ds.DS_F32),      # empty frame
    (64, 64, (2, 4), 8, ds.DS_F32),     # ratio not in lowest terms
    (64, 64, (8, 3), 8, ds.DS_F32),     # upsampling
    (64, 64, (0, 3), 8, ds.DS_F32),
    (64, 64, (3, 8), 7, ds.DS_F32),     # odd taps
    (64, 64, (3, 8), 18, ds.DS_F32),    # too many taps
    (64, 64, (3, 8), 0, ds.DS_F32),
    (64, 64, (3, 8), 8, 9),             # unknown dtype
    (2, 2, (3, 8), 8, ds.DS_F32),       # empty output
    (64, 64, (17, 64), 8, ds.DS_F32),   # p beyond the limit
    (64, 200, (1, 65), 8, ds.DS_F32),   # q beyond the limit
])
def test_plan_create_rejects(args):
    with pytest.raises(ds.DsError) as e:
        ds.ds_plan_create(*args)
    assert e.value.status == ds.DS_ERR_ARG


def test_plan_shapes_and_params():
    pl = ds.ds_plan_create(288, 352, (3, 8), 8, ds.DS_U8_RGB)
    try:
        assert ds.ds_plan_get_params(pl) == (288, 352, 3, 8, 8, ds.DS_U8_RGB)
        assert ds.ds_plan_out_shape(pl) == (108, 132, 3)   # 352 -> 132 (paper Sec. 3)
        assert ds.ds_plan_frame_bytes(pl) == (288 * 352 * 3, 108 * 132 * 3)
        assert ds.ds_plan_workspace_bytes(pl) == 288 * 132 * 3
        d = ds.ds_plan_describe(pl)
        assert '"kernel": "fused_tma"' in d and "u8rgb_3_8_k8" in d
        ds.ds_plan_set_schedule(pl, 5, 1)
        assert ds.ds_plan_get_schedule(pl) == (5, 1)
        with pytest.raises(ds.DsError):
            ds.ds_plan_set_schedule(pl, 0, 0)
    finally:
        ds.ds_destroy(pl)


@pytest.mark.parametrize("p,q,K", [(3, 8, 8), (1, 2, 6), (2, 3, 6), (5, 7, 10), (1, 4, 16), (3, 4, 4),
                                   (1, 3, 12), (1, 2, 2), (7, 16, 14), (16, 17, 16), (1, 64, 8)])
def test_plan_taps_agree_with_oracle(oracle, p, q, K):
    pl = ds.ds_plan_create(200, 200, (p, q), K, ds.DS_F32)
    try:
        t = ds.ds_plan_get_taps(pl)
    finally:
        ds.ds_destroy(pl)
    b, _ = oracle.phase_windows(p, q, K)
    np.testing.assert_array_equal(t["window_start"], b)
    np.testing.assert_allclose(t["fp64"], oracle.taps_f64(p, q, K), rtol=0, atol=2e-15)
    np.testing.assert_array_equal(t["fp32"], oracle.taps_f64(p, q, K).astype(np.float32))
    np.testing.assert_array_equal(t["q14"].astype(np.int32), oracle.taps_q14(p, q, K))


def test_null_arguments_rejected():
    with pytest.raises(ds.DsError):
        ds.ds_run(0, 0, 0, 0)
    with pytest.raises(ds.DsError):
        ds.ds_plan_out_shape(0)
    with pytest.raises(ds.DsError):
        ds.ds_batch_run([(0, 0, 0)])
    pl = ds.ds_plan_create(64, 64, (3, 8), 8, ds.DS_F32)
    try:
        with pytest.raises(ds.DsError):
            ds.ds_run_unfused(pl, 16, 16, 1, 16, 10)  # workspace too small
        ds.ds_batch_run([])  # empty batch: nothing to do
    finally:
        ds.ds_destroy(pl)


SHAPES = [(8, 8), (16, 16), (8, 32), (24, 40), (17, 64), (33, 100), (480, 640), (720, 1280),
          (1080, 1920), (288, 352), (3, 16), (1, 16), (2, 48), (100, 4), (129, 2048), (7, 520), (300, 1568),
          (2160, 3840)]
RATIOS = [((3, 8), 8), ((1, 2), 6), ((2, 3), 6)]
DTYPES = [ds.DS_F32, ds.DS_F16, ds.DS_U8_RGB, ds.DS_U8]


def test_fused_kernel_index_arithmetic_host_check():
    checked = 0
    for (H, W), (r, K), dt in itertools.product(SHAPES, RATIOS, DTYPES):
        try:
            pl = ds.ds_plan_create(H, W, r, K, dt)
        except ds.DsError:
            continue
        try:
            for rb in (1, 2, 3, 7, 12, 32, 1000):
                ds.ds_plan_set_schedule(pl, rb, 0)
                ds.ds_debug_check_plan(pl)
                checked += 1
        finally:
            ds.ds_destroy(pl)
    assert checked > 300


def test_fast_kernel_host_check_on_random_shapes():
    """ds_debug_check_plan over seeded random frame sizes, bands, tile shapes
    and boundaries for every fast class (host replay of the kernel's index
    arithmetic, no GPU)."""
    rng = np.random.default_rng(77)
    specs = [((3, 8), 8, (3, 8), 8), ((1, 2), 6, (1, 2), 6), ((2, 3), 6, (2, 3), 6), ((3, 8), 8, (4, 9), 8)]
    checked = 0
    for _ in range(200):
        rh, kh, rv, kv = specs[rng.integers(len(specs))]
        dt = [ds.DS_F32, ds.DS_F16, ds.DS_U8, ds.DS_U8_RGB][rng.integers(4)]
        bnd = ds.DS_WRAP if rng.random() < 0.3 else ds.DS_CLAMP
        H = int(rng.integers(1, 700))
        W = 16 * int(rng.integers(1, 160))
        try:
            pl = ds.ds_plan_create_ex(H, W, rh, kh, rv, kv, dt, bnd)
        except ds.DsError:
            continue
        try:
            if '"fused_tma"' not in ds.ds_plan_describe(pl):
                continue
            ds.ds_plan_set_schedule_ex(pl, int(rng.integers(1, 40)), 0, int(rng.integers(ds.ds_plan_tile_shapes(pl))))
            ds.ds_debug_check_plan(pl)
            checked += 1
        finally:
            ds.ds_destroy(pl)
    assert checked > 80


def test_host_check_passes_rows_the_fast_kernel_never_takes():
    """A plan whose rows are not whole 16-byte units keeps its fast class
    (ds_plan_describe) but every launch of it takes the general kernel, so
    the replay has nothing to check: a 200-pixel one-plane row with modular
    tilers, whose strip copies could not start on 16-byte boundaries."""
    pl = ds.ds_plan_create_ex(17, 200, (3, 8), 8, (4, 9), 8, ds.DS_U8, ds.DS_WRAP)
    try:
        ds.ds_debug_check_plan(pl)
    finally:
        ds.ds_destroy(pl)


def test_normal_build_is_not_bounds_checked():
    """The normal library has no index checks; its bounds probe is refused
    before any launch (so this runs without a GPU)."""
    assert not ds.ds_bounds_checked()
    with pytest.raises(ds.DsError) as e:
        ds.ds_debug_bounds_probe(0)
    assert e.value.status == ds.DS_ERR_UNSUPPORTED


def test_env_selects_the_bounds_checking_build():
    """DS_CHECK_BOUNDS=1 in the environment makes the binding load the
    bounds-checking library for the whole process (no GPU needed to ask)."""
    import subprocess
    import sys

    from paper_1103_4881_b300 import build

    build.build(check_bounds=True)
    code = ("import paper_1103_4881_b300 as ds; "
            "assert ds.LIB_PATH == ds.CHECK_LIB_PATH, ds.LIB_PATH; "
            "assert ds.ds_bounds_checked(); print('checked')")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, DS_CHECK_BOUNDS="1")
    r = subprocess.run([sys.executable, "-c", code], cwd=root, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and "checked" in r.stdout, r.stderr
    env["DS_CHECK_BOUNDS"] = "0"
    code0 = "import paper_1103_4881_b300 as ds; assert not ds.ds_bounds_checked(); print('normal')"
    r = subprocess.run([sys.executable, "-c", code0], cwd=root, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and "normal" in r.stdout, r.stderr


def test_server_arguments_are_checked_before_any_device_work():
    for args in [(0, 2, 64), (1 << 20, 0, 64), (1 << 20, 65, 64), (1 << 20, 2, 0), (1 << 20, 2, 5000)]:
        with pytest.raises(ds.DsError):
            ds.ds_server_create(*args)
    with pytest.raises(ds.DsError) as e:
        ds.ds_server_run(0, [], 0)
    assert e.value.status == ds.DS_ERR_ARG
