"""Serving loop and autotuner on the GPU.

The native continuous-batching loop (ds_server_run) groups requests of
different sizes, ratios and dtypes into ds_batch_run launches on several
streams; every request must come back with the bits of its solo ds_run,
whatever group it landed in and in both the kernel-only and the copy mode,
and within the oracle's tolerance.  The autotuner times band heights that all compute the
same bits, so its choice must not change the output."""
import numpy as np
import pytest

import paper_1103_4881_b300 as ds
from paper_1103_4881_b300 import serve, synth, tune
from tests.gpu_util import assert_parity, finish, frames, oracle_out, out_buffer, run_fused, stream, to_dev

pytestmark = pytest.mark.gpu

SIZES = ((72, 528), (120, 256), (200, 784), (41, 272), (37, 61))


def _requests(n, seed=3):
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(2e-4, n))
    out = []
    for k in range(n):
        h, w = SIZES[rng.integers(len(SIZES))]
        ratio, taps = synth.SERVE_RATIOS[rng.integers(len(synth.SERVE_RATIOS))]
        dt = synth.SERVE_DTYPES[rng.integers(len(synth.SERVE_DTYPES))]
        out.append(synth.Request(k, float(t[k]), h, w, ratio, taps, dt))
    return out


def _solo(srv, r, x):
    import torch

    out = torch.empty(srv.out_shape(r), dtype=x.dtype, device="cuda")
    ds.ds_run(srv.plan(r), x.data_ptr(), out.data_ptr(), stream())
    finish()
    return out.cpu().numpy()


@pytest.mark.parametrize("copies", [False, True])
def test_served_requests_equal_solo_runs(oracle, copies):
    reqs = _requests(48)
    pool = serve.FramePool(reqs, per_class=3, host=copies)
    # a budget of a few frames forces many small groups and waits on admission
    srv = serve.Server(mem_budget_bytes=3 << 20, n_streams=3, max_batch=6)
    try:
        outs = serve.OutputPool(srv, reqs, per_request=True, host=copies)
        res = srv.run(reqs, pool.pinned if copies else pool.device, outs, copies=copies, realtime=True)
        finish()
        s = res.stats
        assert res.completed == len(reqs)
        assert s["peak_admitted_bytes"] <= srv.budget and s["max_batch"] <= 6 and s["batches"] >= len(reqs) // 6
        assert len(res.latency_ms) == len(reqs) and res.latency_ms.min() >= 0 and s["launches"] >= s["batches"]
        checked = set()
        for r in reqs:
            got = outs(r).cpu().numpy()
            x = pool.device(r)
            np.testing.assert_array_equal(got, _solo(srv, r, x), err_msg="request %d" % r.rid)
            k = (r.height, r.width, r.ratio, r.dtype, r.rid % pool.per_class)
            if k not in checked:  # each distinct input once against the oracle
                checked.add(k)
                xn = x.cpu().numpy()[None]
                assert_parity(got[None], oracle_out(oracle, xn, r.ratio[0], r.ratio[1], r.taps, r.dtype), r.dtype,
                              "request %d" % r.rid)
    finally:
        srv.close()


def test_saturation_groups_requests_and_the_plain_baseline_matches():
    """All requests at t=0: groups up to the batch limit; the plain per-frame
    baseline (one fused launch per request) writes the same bits."""
    reqs = _requests(64, seed=5)
    pool = serve.FramePool(reqs, per_class=2)
    srv = serve.Server(mem_budget_bytes=256 << 20, n_streams=2, max_batch=16)
    try:
        a = serve.OutputPool(srv, reqs, per_request=True)
        b = serve.OutputPool(srv, reqs, per_request=True)
        res = srv.run(reqs, pool.device, a, realtime=False)
        assert res.completed == len(reqs) and res.stats["max_batch"] == 16 and res.stats["batches"] == 4
        fps = srv.per_frame(reqs, pool.device, b)
        finish()
        assert fps > 0
        for r in reqs:
            np.testing.assert_array_equal(a(r).cpu().numpy(), b(r).cpu().numpy(), err_msg="request %d" % r.rid)
    finally:
        srv.close()


def test_budget_too_small_for_one_request_is_rejected():
    reqs = _requests(2)
    pool = serve.FramePool(reqs, per_class=1)
    srv = serve.Server(mem_budget_bytes=1024, n_streams=1)
    try:
        outs = serve.OutputPool(srv, reqs, per_request=True)
        with pytest.raises(ds.DsError) as e:
            srv.run(reqs, pool.device, outs)
        assert e.value.status == ds.DS_ERR_ARG
    finally:
        srv.close()


def test_copy_mode_arena_allocation_failure_is_reported_and_the_server_recovers():
    """Arenas the device cannot hold: DS_ERR_NOMEM, nothing launched; the same
    server then serves in the kernel-only mode."""
    reqs = _requests(4, seed=11)
    pool = serve.FramePool(reqs, per_class=1, host=True)
    srv = serve.Server(mem_budget_bytes=1 << 52, n_streams=2, max_batch=4)  # 2 PiB per arena
    try:
        host_outs = serve.OutputPool(srv, reqs, per_request=True, host=True)
        with pytest.raises(ds.DsError) as e:
            srv.run(reqs, pool.pinned, host_outs, copies=True)
        assert e.value.status == ds.DS_ERR_NOMEM
        outs = serve.OutputPool(srv, reqs, per_request=True)
        res = srv.run(reqs, pool.device, outs, realtime=False)
        finish()
        assert res.completed == len(reqs)
        for r in reqs:
            np.testing.assert_array_equal(outs(r).cpu().numpy(), _solo(srv, r, pool.device(r)))
    finally:
        srv.close()


@pytest.mark.parametrize("dt", [ds.DS_F32, ds.DS_F16, ds.DS_U8_RGB])
def test_autotune_keeps_bits_and_caches(oracle, dt, tmp_path, monkeypatch):
    monkeypatch.setenv("DS_TUNE_CACHE", str(tmp_path / "tune.json"))
    H, W, n = 270, 480, 3
    pl = ds.ds_plan_create(H, W, (3, 8), 8, dt)
    try:
        x = frames((H, W), dt, n, 31)
        want = run_fused(pl, x)
        xd = to_dev(x)
        out = out_buffer(pl, n)
        rb, us = ds.ds_plan_autotune(pl, xd.data_ptr(), out.data_ptr(), n, stream(), 3)
        finish()
        nby = (ds.ds_plan_out_shape(pl)[0] + 2) // 3
        assert 1 <= rb <= max(nby, 3) and us > 0
        assert ds.ds_plan_get_schedule(pl)[0] == rb
        np.testing.assert_array_equal(out.cpu().numpy(), want)
        np.testing.assert_array_equal(run_fused(pl, x), want)
        assert_parity(want, oracle_out(oracle, x, 3, 8, 8, dt), dt)
        # cache: a second plan of the same key takes the stored schedule without timing
        first = tune.apply_or_tune(pl, xd.data_ptr(), out.data_ptr(), n, stream(), 2)  # miss: tunes
        assert not first["cached"] and first["us_per_launch"] <= first["default_us_per_launch"]
        np.testing.assert_array_equal(run_fused(pl, x), want)
        pl2 = ds.ds_plan_create(H, W, (3, 8), 8, dt)
        try:
            ds.ds_plan_set_schedule(pl2, 1, 0)
            got = tune.apply_or_tune(pl2, 0, 0, n)  # a cache hit touches no buffer
            stored = tune.load()[tune.key(pl2, n)]
            assert got["cached"] and got["shape"] == stored["shape"] and got["row_blocks"] == stored["row_blocks"]
            assert ds.ds_plan_get_schedule_ex(pl2) == {k: stored[k] for k in ("row_blocks", "ctas_per_sm", "shape")}
            np.testing.assert_array_equal(run_fused(pl2, x), want)
        finally:
            ds.ds_destroy(pl2)
    finally:
        ds.ds_destroy(pl)
