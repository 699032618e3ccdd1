"""DS_LOG: the library logs plan choices and errors (level 1) and launches
(level 2) to stderr, and nothing when the variable is unset.  Plans are
host-only, so this runs without a GPU."""
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SCRIPT = """
import sys
sys.path.insert(0, %r)
import paper_1103_4881_b300 as ds
pl = ds.ds_plan_create(64, 96, (3, 8), 8, ds.DS_U8_RGB)
ds.ds_destroy(pl)
try:
    ds.ds_plan_create(1, 8, (3, 8), 8, ds.DS_F32)
except ds.DsError:
    pass
""" % ROOT


def _run(level):
    env = dict(os.environ)
    env.pop("DS_LOG", None)
    if level is not None:
        env["DS_LOG"] = str(level)
    r = subprocess.run([sys.executable, "-c", SCRIPT], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    return r.stderr


def test_log_level_one_reports_plans_and_errors():
    err = _run(1)
    assert "[ds] plan 64x96x3" in err and "fused_tma" in err
    assert "[ds] error: ds_plan_create: 1x8" in err


def test_no_log_without_the_variable():
    assert "[ds]" not in _run(None)
    assert "[ds]" not in _run(0)
