"""Helpers shared by the GPU tests: device buffers via torch, calls through the
C ABI, comparison against the oracle with the stated tolerances."""
import contextlib
import os

import numpy as np

import paper_1103_4881_b300 as ds
from paper_1103_4881_b300 import synth

# Tolerances against the FP64 oracle, full scale 1.0 for float data:
# FP32 storage and accumulation 1e-6; FP16 storage (FP32 accumulation) 2e-3;
# uint8 bit-exact.
TOL = {ds.DS_F32: 1e-6, ds.DS_F16: 2e-3}


def torch_dtype(dtype):
    import torch

    return {ds.DS_F32: torch.float32, ds.DS_F16: torch.float16, ds.DS_U8: torch.uint8,
            ds.DS_U8_RGB: torch.uint8}[dtype]


def to_dev(x: np.ndarray):
    import torch

    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def stream():
    import torch

    return torch.cuda.current_stream().cuda_stream


def out_buffer(plan, n):
    import torch

    oh, ow, c = ds.ds_plan_out_shape(plan)
    _, _, _, _, _, dt = ds.ds_plan_get_params(plan)
    shape = (n, oh, ow) if c == 1 else (n, oh, ow, c)
    return torch.full(shape, 0, dtype=torch_dtype(dt), device="cuda")


def finish():
    import torch

    torch.cuda.synchronize()
    ds.ds_stream_check(stream())


def run_fused(plan, x: np.ndarray):
    """ds_run_frames over the stacked frames x (n, H, W[, C]) -> numpy."""
    xd = to_dev(x)
    out = out_buffer(plan, x.shape[0])
    ds.ds_run_frames(plan, xd.data_ptr(), out.data_ptr(), x.shape[0], stream())
    finish()
    return out.cpu().numpy()


def run_unfused(plan, x: np.ndarray):
    import torch

    xd = to_dev(x)
    out = out_buffer(plan, x.shape[0])
    nbytes = ds.ds_plan_workspace_bytes(plan) * x.shape[0]
    ws = torch.empty(max(1, nbytes), dtype=torch.uint8, device="cuda")
    ds.ds_run_unfused(plan, xd.data_ptr(), out.data_ptr(), x.shape[0], ws.data_ptr(), nbytes, stream())
    finish()
    return out.cpu().numpy()


@contextlib.contextmanager
def general_kernel():
    """Plans created inside use the general fused kernel (no TMA)."""
    old = os.environ.get("DS_NO_TMA")
    os.environ["DS_NO_TMA"] = "1"
    try:
        yield
    finally:
        if old is None:
            del os.environ["DS_NO_TMA"]
        else:
            os.environ["DS_NO_TMA"] = old


def oracle_out(oracle, x, p, q, K, dtype):
    if dtype in (ds.DS_U8, ds.DS_U8_RGB):
        return oracle.filter_u8(x, p, q, K)
    return oracle.filter_f64(x, p, q, K)


def assert_parity(got, want, dtype, what=""):
    if dtype in (ds.DS_U8, ds.DS_U8_RGB):
        bad = np.count_nonzero(got != want)
        assert bad == 0, "%s: %d of %d bytes differ from the oracle" % (what, bad, got.size)
    else:
        err = np.abs(got.astype(np.float64) - want).max() if got.size else 0.0
        assert err <= TOL[dtype], "%s: max |err| %.3g > %.3g" % (what, err, TOL[dtype])
        return err


def frames(shape, dtype, n, seed):
    c = synth.CHANNELS[dtype]
    full = (n,) + tuple(shape) + ((c,) if c > 1 else ())
    return synth.random_frames(full, dtype, seed)
