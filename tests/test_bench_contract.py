"""bench.py's output contract on the host: the reference arm (the CPU
oracle) prints one JSON line with the keys the driver reads."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                          "plain_480x640_f32", "--steps", "3", "--warmup", "1"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 3
    assert d["config"]["workload"] == "plain_480x640_f32"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0


def test_reference_arm_on_a_planar_per_axis_workload():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                          "cif2000_yuv420_u8", "--steps", "2", "--warmup", "1"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    d = json.loads([l for l in out.stdout.splitlines() if l.startswith("{")][0])
    assert d["config"]["ratio_v"] == "4/9" and len(d["config"]["planes"]) == 3


def test_committed_traffic_capture_matches_the_kernel_source():
    """profiles/traffic.json holds a one-pass ncu capture of the headline
    workload's launch taken on the current kernel source (bench.py reports it
    as roofline.traffic), at the default schedule the tuner keeps there."""
    sys.path.insert(0, ROOT)
    import bench

    sched = [{"row_blocks": 0, "ctas_per_sm": 0, "shape": 0}]
    t = bench.profiled_traffic(bench.HEADLINE, sched)
    assert t is not None, "re-capture the headline's DRAM traffic on the current kernel source"
    from paper_1103_4881_b300 import synth

    w = synth.WORKLOADS[bench.HEADLINE]
    alg = w.frames * w.bytes_per_frame()
    assert 0.95 * alg < t < 1.2 * alg  # traffic near the algorithmic bytes: no wasted re-reads
    assert bench.profiled_traffic(bench.HEADLINE, [{"row_blocks": 3, "ctas_per_sm": 1, "shape": 1}]) is None


def test_issue_roofline_from_the_committed_capture():
    """The headline's committed capture also holds the launch's warp
    instructions; the issue roofline divides them by the launch time and
    compares with 4 warp instructions per SM per clock at the sampled clock."""
    sys.path.insert(0, ROOT)
    import bench

    sched = [{"row_blocks": 0, "ctas_per_sm": 0, "shape": 0}]
    e = bench.profiled_capture(bench.HEADLINE, sched)
    assert e is not None and e["warp_instructions_per_launch"] > 0
    r = bench.issue_roofline(bench.HEADLINE, sched, 400e-6, {"sm_mhz": 2000.0}, 148)
    assert r["peak"] == 4 * 148 * 2000.0 * 1e6 / 1e9
    assert abs(r["achieved"] - e["warp_instructions_per_launch"] / 400e-6 / 1e9) < 1e-6
    assert 0.0 < r["frac"] < 1.0 and r["bound"] == "issue"
    assert bench.issue_roofline(bench.HEADLINE, sched, 400e-6, {"sm_mhz": None}, 148) is None
    assert bench.issue_roofline(bench.HEADLINE, [{"row_blocks": 3, "ctas_per_sm": 1, "shape": 1}], 400e-6,
                                {"sm_mhz": 2000.0}, 148) is None
