"""Guard bytes around every output: each fast class and the general kernel,
on ragged shapes, writes exactly its output region (the device-side
counterpart of ds_debug_check_plan's host replay of the index arithmetic)."""
import numpy as np
import pytest

import paper_1103_4881_b300 as ds
from tests.gpu_util import finish, frames, run_fused, stream, to_dev

pytestmark = pytest.mark.gpu

GUARD = 4096
CASES = [
    # (H, W, rh, Kh, rv, Kv, dtype)
    (72, 528, (3, 8), 8, (3, 8), 8, ds.DS_F32), (41, 272, (1, 2), 6, (1, 2), 6, ds.DS_F32),
    (130, 784, (2, 3), 6, (2, 3), 6, ds.DS_F32), (200, 784, (3, 8), 8, (3, 8), 8, ds.DS_F16),
    (37, 528, (1, 2), 6, (1, 2), 6, ds.DS_F16), (97, 400, (2, 3), 6, (2, 3), 6, ds.DS_F16),
    (65, 272, (3, 8), 8, (3, 8), 8, ds.DS_U8_RGB), (99, 400, (1, 2), 6, (1, 2), 6, ds.DS_U8_RGB),
    (77, 336, (2, 3), 6, (2, 3), 6, ds.DS_U8_RGB), (289, 352, (3, 8), 8, (4, 9), 8, ds.DS_U8_RGB),
    (145, 176, (3, 8), 8, (4, 9), 8, ds.DS_U8), (37, 61, (3, 8), 8, (3, 8), 8, ds.DS_F32),  # general kernel
]


@pytest.mark.parametrize("H,W,rh,Kh,rv,Kv,dt", CASES)
def test_outputs_stay_inside_their_region(H, W, rh, Kh, rv, Kv, dt):
    import torch

    pl = ds.ds_plan_create_ex(H, W, rh, Kh, rv, Kv, dt)
    try:
        n = 3
        x = frames((H, W), dt, n, H + W)
        want = run_fused(pl, x)
        _, fout = ds.ds_plan_frame_bytes(pl)
        buf = torch.full((GUARD + n * fout + GUARD,), 0xA5, dtype=torch.uint8, device="cuda")
        xd = to_dev(x)
        ds.ds_run_frames(pl, xd.data_ptr(), buf.data_ptr() + GUARD, n, stream())
        finish()
        host = buf.cpu().numpy()
        assert np.all(host[:GUARD] == 0xA5) and np.all(host[GUARD + n * fout:] == 0xA5)
        got = host[GUARD:GUARD + n * fout].view(want.dtype).reshape(want.shape)
        np.testing.assert_array_equal(got, want)
    finally:
        ds.ds_destroy(pl)
