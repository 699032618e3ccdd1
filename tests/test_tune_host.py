"""Host side of the autotuner: argument checks (no GPU work) and the cache file."""
import pytest

import paper_1103_4881_b300 as ds
from paper_1103_4881_b300 import tune


def test_autotune_rejects_bad_arguments():
    pl = ds.ds_plan_create(64, 64, (3, 8), 8, ds.DS_F32)
    try:
        for args in [(pl, 0, 16, 1), (pl, 16, 0, 1), (pl, 16, 16, 0)]:
            with pytest.raises(ds.DsError):
                ds.ds_plan_autotune(*args, 0, 1)
        with pytest.raises(ds.DsError):
            ds.ds_plan_autotune(pl, 16, 16, 1, 0, 0)
        assert ds.ds_plan_get_schedule(pl) == ds.ds_plan_get_schedule(pl)
    finally:
        ds.ds_destroy(pl)


def test_cache_key_and_round_trip(tmp_path, monkeypatch):
    monkeypatch.setenv("DS_TUNE_CACHE", str(tmp_path / "sub" / "tune.json"))
    assert tune.load() == {}
    a = ds.ds_plan_create(1080, 1920, (3, 8), 8, ds.DS_F32)
    b = ds.ds_plan_create(1080, 1920, (3, 8), 8, ds.DS_F16)
    c = ds.ds_plan_create_ex(1080, 1920, (3, 8), 8, (4, 9), 8, ds.DS_F32)
    try:
        assert tune.key(a, 64, "GPU|148") != tune.key(c, 64, "GPU|148")  # the vertical axis is in the key
        ka, kb = tune.key(a, 64, "GPU|148"), tune.key(b, 64, "GPU|148")
        assert ka != kb and ka != tune.key(a, 1, "GPU|148") and ka != tune.key(a, 64, "GPU|132")
        assert "1080x1920" in ka and "3/8" in ka
        tune.save({ka: {"row_blocks": 8, "ctas_per_sm": 0, "shape": 1, "us_per_launch": 130.0}})
        assert tune.load()[ka]["row_blocks"] == 8
        # a hit sets the plan's whole schedule without touching a GPU
        got = tune.apply_or_tune(a, 0, 0, 64, device_tag="GPU|148")
        assert got["cached"] and ds.ds_plan_get_schedule_ex(a) == {"row_blocks": 8, "ctas_per_sm": 0, "shape": 1}
        (tmp_path / "sub" / "tune.json").write_text("{not json")
        assert tune.load() == {}
    finally:
        ds.ds_destroy(a)
        ds.ds_destroy(b)
        ds.ds_destroy(c)


def test_schedule_ex_round_trip_and_checks():
    pl = ds.ds_plan_create(1080, 1920, (3, 8), 8, ds.DS_F16)
    gp = ds.ds_plan_create(100, 100, (3, 4), 4, ds.DS_F32)  # general kernels: no compiled shapes
    try:
        assert ds.ds_plan_tile_shapes(pl) >= 2 and ds.ds_plan_tile_shapes(gp) == 0
        assert ds.ds_plan_get_schedule_ex(pl) == {"row_blocks": 0, "ctas_per_sm": 0, "shape": 0}
        ds.ds_plan_set_schedule_ex(pl, 12, 3, 1)
        assert ds.ds_plan_get_schedule_ex(pl) == {"row_blocks": 12, "ctas_per_sm": 3, "shape": 1}
        assert '"index": 1' in ds.ds_plan_describe(pl) and '"band": "fixed"' in ds.ds_plan_describe(pl)
        ds.ds_plan_set_schedule_ex(pl, 0, 0, 0)  # back to the default, adaptive band
        assert '"band": "adaptive"' in ds.ds_plan_describe(pl)
        for bad in [(-1, 0, 0), (0, -1, 0), (0, 0, -1), (0, 0, ds.ds_plan_tile_shapes(pl))]:
            with pytest.raises(ds.DsError):
                ds.ds_plan_set_schedule_ex(pl, *bad)
        with pytest.raises(ds.DsError):
            ds.ds_plan_set_schedule_ex(gp, 0, 0, 1)
        ds.ds_plan_set_schedule_ex(gp, 0, 0, 0)
    finally:
        ds.ds_destroy(pl)
        ds.ds_destroy(gp)


def test_a_cache_entry_the_library_cannot_take_is_tuned_again(tmp_path, monkeypatch):
    """A stale entry (a tile shape this build does not have) is not applied:
    apply_or_tune falls through to tuning, which needs the caller's buffers
    (here NULL, so the library refuses with DS_ERR_ARG before any device work)."""
    monkeypatch.setenv("DS_TUNE_CACHE", str(tmp_path / "tune.json"))
    pl = ds.ds_plan_create(1080, 1920, (3, 8), 8, ds.DS_F32)
    try:
        k = tune.key(pl, 8, "GPU|148")
        tune.save({k: {"row_blocks": 8, "ctas_per_sm": 0, "shape": 7}})
        with pytest.raises(ds.DsError) as e:
            tune.apply_or_tune(pl, 0, 0, 8, device_tag="GPU|148")
        assert e.value.status == ds.DS_ERR_ARG
        assert ds.ds_plan_get_schedule_ex(pl)["shape"] == 0
    finally:
        ds.ds_destroy(pl)


def test_batch_autotune_rejects_bad_arguments():
    """Checked before any GPU work: no jobs, iters < 1, a NULL buffer, and a
    batch with no job on the fused kernel."""
    pl = ds.ds_plan_create_ex(288, 352, (3, 8), 8, (4, 9), 8, ds.DS_U8)
    gp = ds.ds_plan_create(100, 100, (3, 4), 4, ds.DS_F32)  # general kernels only
    try:
        with pytest.raises(ds.DsError) as e:
            ds.ds_batch_autotune([], 0, 10)
        assert e.value.status == ds.DS_ERR_ARG
        with pytest.raises(ds.DsError) as e:
            ds.ds_batch_autotune([(pl, 16, 16, 1)], 0, 0)
        assert e.value.status == ds.DS_ERR_ARG
        with pytest.raises(ds.DsError) as e:
            ds.ds_batch_autotune([(pl, 16, 16, 1), (pl, 0, 16, 1)], 0, 10)
        assert e.value.status == ds.DS_ERR_ARG
        with pytest.raises(ds.DsError) as e:
            ds.ds_batch_autotune([(gp, 16, 16, 1)], 0, 10)
        assert e.value.status == ds.DS_ERR_UNSUPPORTED
        assert ds.ds_plan_get_schedule_ex(pl) == {"row_blocks": 0, "ctas_per_sm": 0, "shape": 0}
    finally:
        ds.ds_destroy(pl)
        ds.ds_destroy(gp)


def test_batch_cache_key_and_hit(tmp_path, monkeypatch):
    """A batch is cached under its jobs' keys in order; a hit sets every
    job's plan schedule without touching a GPU."""
    monkeypatch.setenv("DS_TUNE_CACHE", str(tmp_path / "tune.json"))
    y = ds.ds_plan_create_ex(288, 352, (3, 8), 8, (4, 9), 8, ds.DS_U8)
    c = ds.ds_plan_create_ex(144, 176, (3, 8), 8, (4, 9), 8, ds.DS_U8)
    try:
        jobs = [(y, 16, 16, 2000), (c, 16, 16, 2000), (c, 16, 16, 2000)]
        k = tune.batch_key(jobs, "GPU|148")
        assert k != tune.batch_key(jobs[:2], "GPU|148") and k != tune.batch_key(list(reversed(jobs)), "GPU|148")
        assert k != tune.batch_key([(y, 16, 16, 1000)] + jobs[1:], "GPU|148")
        assert k.count("288x352") == 1 and k.count("144x176") == 2
        sc = [{"row_blocks": 0, "ctas_per_sm": 20, "shape": 0}, {"row_blocks": 0, "ctas_per_sm": 20, "shape": 0},
              {"row_blocks": 0, "ctas_per_sm": 20, "shape": 0}]
        tune.save({k: {"schedules": sc, "us_per_launch": 90.5}})
        got = tune.apply_or_tune_batch(jobs, device_tag="GPU|148")
        assert got["cached"]
        assert ds.ds_plan_get_schedule_ex(y) == sc[0] and ds.ds_plan_get_schedule_ex(c) == sc[1]
    finally:
        ds.ds_destroy(y)
        ds.ds_destroy(c)
