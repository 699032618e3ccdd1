"""ds_run_unfused_static: the unfused form without caller workspace, for
callers that cannot allocate device memory on the call path (a serving loop
that must not stall on cudaMalloc, a fixed device-memory budget, a host
program whose allocator must own the device).  Its intermediate lives in the
library's fixed device array, which keeps whatever the previous call left
there.  So before each call under test another call, with another plan and
other pixels, fills the whole array; the call under test must then give
exactly the bits of the fused entry point (the unfused form accumulates in
the same order), twice in a row.

This file is collected last on purpose: a run that stops at the first
failure has then already run every other test."""
import numpy as np
import pytest

import paper_1103_4881_b300 as ds
from tests.gpu_util import finish, frames, out_buffer, run_fused, stream, to_dev


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


def _fill_the_array(seed):
    """One call whose intermediate covers the whole array with other data:
    one-channel bytes, 4096 x 16384 at 1/2 (4096 x 8192 bytes = 32 MiB)."""
    pl = ds.ds_plan_create(4096, 16384, (1, 2), 6, ds.DS_U8)
    try:
        assert ds.ds_plan_workspace_bytes(pl) == ds.ds_static_workspace_bytes()
        x = to_dev(frames((4096, 16384), ds.DS_U8, 1, 9000 + seed))
        out = out_buffer(pl, 1)
        ds.ds_run_unfused_static(pl, x.data_ptr(), out.data_ptr(), 1, stream())
        finish()
    finally:
        ds.ds_destroy(pl)


CASES = [
    # (H, W, ratio_h, K_h, ratio_v, K_v, dtype, boundary, n)
    (1080, 1920, (3, 8), 8, (3, 8), 8, ds.DS_F32, ds.DS_CLAMP, 3),
    (720, 1280, (1, 2), 6, (1, 2), 6, ds.DS_U8_RGB, ds.DS_CLAMP, 2),
    (540, 960, (2, 3), 6, (2, 3), 6, ds.DS_F16, ds.DS_CLAMP, 4),
    (288, 352, (3, 8), 8, (4, 9), 8, ds.DS_U8, ds.DS_WRAP, 5),       # modular tilers, per-axis ratios
    (1024, 8192, (1, 2), 6, (1, 2), 6, ds.DS_F32, ds.DS_CLAMP, 2),   # exactly the array's size
]


@pytest.mark.gpu
@pytest.mark.parametrize("H,W,rh,Kh,rv,Kv,dt,bnd,n", CASES)
def test_static_workspace_matches_fused_twice(H, W, rh, Kh, rv, Kv, dt, bnd, n):
    pl = ds.ds_plan_create_ex(H, W, rh, Kh, rv, Kv, dt, bnd)
    try:
        need = ds.ds_plan_workspace_bytes(pl) * n
        assert need <= ds.ds_static_workspace_bytes()
        if (H, W) == (1024, 8192):
            assert need == ds.ds_static_workspace_bytes()
        x = frames((H, W), dt, n, 4242 + H)
        want = run_fused(pl, x)
        xd = to_dev(x)
        for call in range(2):
            _fill_the_array(call)
            out = out_buffer(pl, n)
            ds.ds_run_unfused_static(pl, xd.data_ptr(), out.data_ptr(), n, stream())
            finish()
            np.testing.assert_array_equal(out.cpu().numpy(), want, err_msg="call %d" % call)
    finally:
        ds.ds_destroy(pl)
