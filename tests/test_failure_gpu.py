"""Failure detection on the GPU without a fault: a bounded device wait that
nothing completes runs out, the kernel records the timeout in the status
word, the host reads it as DS_ERR_TIMEOUT, and the context keeps working."""
import pytest

import paper_1103_4881_b300 as ds
from tests.gpu_util import assert_parity, finish, frames, oracle_out, run_fused, stream


@pytest.mark.gpu
def test_bounded_wait_reports_timeout_and_context_survives(oracle):
    ds.ds_stream_check(stream())  # nothing pending
    ds.ds_debug_timeout_probe(20_000_000, stream())  # about 10 ms at 2 GHz
    with pytest.raises(ds.DsError) as err:
        ds.ds_stream_check(stream())
    assert err.value.status == ds.DS_ERR_TIMEOUT
    ds.ds_stream_check(stream())  # the read cleared the word
    pl = ds.ds_plan_create(96, 256, (3, 8), 8, ds.DS_F32)
    try:
        x = frames((96, 256), ds.DS_F32, 2, 8)
        assert_parity(run_fused(pl, x), oracle_out(oracle, x, 3, 8, 8, ds.DS_F32), ds.DS_F32)
    finally:
        ds.ds_destroy(pl)
    finish()


def test_timeout_probe_rejects_bad_limits_without_gpu():
    for bad in (-1, 5_000_000_000):
        with pytest.raises(ds.DsError) as err:
            ds.ds_debug_timeout_probe(bad, 0)
        assert err.value.status == ds.DS_ERR_ARG
