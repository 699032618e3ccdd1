"""Several host threads launching at once, each on its own stream with its
own plans (per-thread launch parameters, per-launch scheduling slots, the
class tap tables built once): every result equals the oracle's, as if each
thread ran alone.  ctypes drops the GIL around library calls, so the calls
really overlap."""
import threading

import numpy as np
import pytest

import paper_1103_4881_b300 as ds
from tests.gpu_util import assert_parity, frames, to_dev

pytestmark = pytest.mark.gpu

JOBS = [
    ((96, 528), (3, 8), 8, ds.DS_F32),
    ((64, 256), (1, 2), 6, ds.DS_U8_RGB),
    ((72, 384), (2, 3), 6, ds.DS_F16),
    ((48, 512), (3, 8), 8, ds.DS_U8),
    ((97, 130), (3, 4), 8, ds.DS_F32),  # general kernel
    ((288, 352), (3, 8), 8, ds.DS_U8_RGB),
]


def test_threads_on_own_streams_match_the_oracle(oracle):
    import torch

    inputs = [frames(shape, dt, 3, 50 + k) for k, (shape, _, _, dt) in enumerate(JOBS)]
    results = [None] * len(JOBS)
    errors = []

    def work(k):
        try:
            shape, ratio, K, dt = JOBS[k]
            st = torch.cuda.Stream()
            pl = ds.ds_plan_create(shape[0], shape[1], ratio, K, dt)
            try:
                oh, ow, c = ds.ds_plan_out_shape(pl)
                x = to_dev(inputs[k])
                out = torch.zeros((3, oh, ow) + ((c,) if c > 1 else ()), dtype=x.dtype, device="cuda")
                for _ in range(20):  # many launches, interleaved with the other threads'
                    ds.ds_run_frames(pl, x.data_ptr(), out.data_ptr(), 3, st.cuda_stream)
                st.synchronize()
                ds.ds_stream_check(st.cuda_stream)
                results[k] = out.cpu().numpy()
            finally:
                ds.ds_destroy(pl)
        except Exception as e:  # reported by the main thread
            errors.append((k, repr(e)))

    threads = [threading.Thread(target=work, args=(k,)) for k in range(len(JOBS))]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors
    for k, (shape, ratio, K, dt) in enumerate(JOBS):
        x = inputs[k]
        if dt in (ds.DS_U8, ds.DS_U8_RGB):
            want = oracle.filter_u8(x, ratio[0], ratio[1], K)
        else:
            want = oracle.filter_f64(x.astype(np.float64), ratio[0], ratio[1], K)
        assert_parity(results[k], want, dt, "thread %d" % k)
