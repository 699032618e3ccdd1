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
    try:
        ka, kb = tune.key(a, 64, "GPU|148"), tune.key(b, 64, "GPU|148")
        assert ka != kb and ka != tune.key(a, 1, "GPU|148") and ka != tune.key(a, 64, "GPU|132")
        assert "1080x1920" in ka and "3/8" in ka
        tune.save({ka: {"row_blocks": 8, "us_per_launch": 130.0}})
        assert tune.load()[ka]["row_blocks"] == 8
        (tmp_path / "sub" / "tune.json").write_text("{not json")
        assert tune.load() == {}
    finally:
        ds.ds_destroy(a)
        ds.ds_destroy(b)
