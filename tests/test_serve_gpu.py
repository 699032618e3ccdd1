"""Serving loop and autotuner on the GPU.

The continuous-batching loop groups requests of different sizes, ratios and
dtypes into ds_batch_run launches on several streams; every request must come
back with the bits of its solo ds_run, whatever batch it landed in, and within
the oracle's tolerance.  The autotuner times band heights that all compute the
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
    # a budget of a few frames forces many small batches and waits on admission
    srv = serve.Server(mem_budget_bytes=3 << 20, n_streams=3, max_batch=6)
    try:
        res, outs = srv.run(reqs, pool.pinned if copies else pool.device, copies=copies, realtime=True,
                            keep_outputs=True)
        finish()
        assert res.completed == len(reqs) and len(outs) == len(reqs)
        assert res.peak_bytes <= srv.budget and res.max_batch <= 6 and res.batches >= len(reqs) // 6
        assert len(res.latency_ms) == len(reqs) and min(res.latency_ms) >= 0
        checked = set()
        for r in reqs:
            got = outs[r.rid].cpu().numpy()
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


def test_budget_too_small_for_one_request_is_rejected():
    reqs = _requests(2)
    pool = serve.FramePool(reqs, per_class=1)
    srv = serve.Server(mem_budget_bytes=1024, n_streams=1)
    try:
        with pytest.raises(ValueError):
            srv.run(reqs, pool.device)
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


def test_allocation_failures_requeue_and_every_request_completes():
    """An injected allocator that runs out of memory now and then: the batch
    goes back to the queue, nothing of it is launched, and every request
    still completes with the bits of its solo run."""
    import torch

    calls = {"n": 0}

    def flaky(shape, dtype):
        calls["n"] += 1
        if calls["n"] <= 3 or calls["n"] % 7 == 0:
            raise torch.cuda.OutOfMemoryError("injected")
        return torch.empty(shape, dtype=dtype, device="cuda")

    reqs = _requests(30, seed=9)
    pool = serve.FramePool(reqs, per_class=2)
    srv = serve.Server(mem_budget_bytes=64 << 20, n_streams=2, max_batch=4, alloc=flaky)
    try:
        res, outs = srv.run(reqs, pool.device, realtime=False, keep_outputs=True)
        finish()
        assert res.completed == len(reqs) and res.alloc_retries >= 3
        for r in reqs:
            np.testing.assert_array_equal(outs[r.rid].cpu().numpy(), _solo(srv, r, pool.device(r)))
    finally:
        srv.close()
