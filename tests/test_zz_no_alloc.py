"""ds_run_unfused_static: the unfused form without caller workspace, for
callers that cannot allocate device memory on the call path (a serving loop
that must not stall on cudaMalloc, a fixed device-memory budget, a host
program whose allocator must own the device).  Its intermediate lives in the
library's fixed device array.  Two calls in a row must match the fused
entry point within the tolerances of the parity tests.

This file is collected last on purpose: a run that stops at the first
failure has then already run every other test."""
import numpy as np
import pytest

import paper_1103_4881_b300 as ds
from tests.gpu_util import TOL, finish, frames, out_buffer, run_fused, stream, to_dev


def test_static_workspace_rejects_oversize_without_gpu():
    pl = ds.ds_plan_create(2160, 3840, (1, 2), 6, ds.DS_F32)
    try:
        need = ds.ds_plan_workspace_bytes(pl)
        n = ds.ds_static_workspace_bytes() // need + 1
        with pytest.raises(ds.DsError) as e:
            ds.ds_run_unfused_static(pl, 16, 16, n, 0)
        assert e.value.status == ds.DS_ERR_ARG
        assert "static workspace" in ds.ds_last_error()
    finally:
        ds.ds_destroy(pl)


@pytest.mark.gpu
@pytest.mark.parametrize("H,W,ratio,K,dt,n", [
    (1080, 1920, (3, 8), 8, ds.DS_F32, 3),
    (720, 1280, (1, 2), 6, ds.DS_U8_RGB, 2),
    (540, 960, (2, 3), 6, ds.DS_F16, 4),
])
def test_static_workspace_matches_fused_twice(H, W, ratio, K, dt, n):
    pl = ds.ds_plan_create(H, W, ratio, K, dt)
    try:
        assert ds.ds_plan_workspace_bytes(pl) * n <= ds.ds_static_workspace_bytes()
        x = frames((H, W), dt, n, 4242 + H)
        want = run_fused(pl, x)
        xd = to_dev(x)
        for call in range(2):  # the array keeps the previous call's contents
            out = out_buffer(pl, n)
            ds.ds_run_unfused_static(pl, xd.data_ptr(), out.data_ptr(), n, stream())
            finish()
            got = out.cpu().numpy()
            if dt == ds.DS_U8_RGB:
                np.testing.assert_array_equal(got, want, err_msg="call %d" % call)
            else:
                np.testing.assert_allclose(got.astype(np.float64), want.astype(np.float64), rtol=0,
                                           atol=TOL[dt], err_msg="call %d" % call)
    finally:
        ds.ds_destroy(pl)
