"""thapi_tally_static: the tally for callers that cannot allocate device memory.

A tracing agent that tallies on the node while the traced application runs
in the same CUDA context cannot count on allocating device memory: the
application (or its framework's caching allocator) usually holds almost all
of it, and an allocation by the agent could fail or disturb the run being
observed.  thapi_tally_static takes its working memory from an array that is
part of the library instead.  This test calls it through the C ABI twice in a
row, on two different traces (the shared array keeps the first call's
contents), and checks that rows and diagnostics are exactly those of the
allocating path (thapi_trace_load_device + thapi_tally).
"""
import numpy as np
import pytest

import tracegen as tg
from paper_2504_03683_b300 import thapi

pytestmark = pytest.mark.gpu


def _allocating(ctx, dev, nbytes):
    tid = thapi.thapi_trace_load_device(ctx.handle, dev.data_ptr(), nbytes)
    try:
        return thapi.thapi_tally(ctx.handle, tid)
    finally:
        ctx.free(tid)


def _static(dev, nbytes):
    import torch
    n, _diag = thapi.thapi_tally_static(dev.data_ptr(), nbytes, 0, 0)          # size query
    rows_dev = torch.empty(max(1, n) * thapi.ROW_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    n2, diag = thapi.thapi_tally_static(dev.data_ptr(), nbytes, rows_dev.data_ptr(), n)
    torch.cuda.synchronize()
    assert n2 == n
    return rows_dev.cpu().numpy().view(thapi.ROW_DTYPE)[:n], diag


def test_static_tally_equals_allocating_tally_twice_in_a_row():
    import torch
    traces = [
        tg.generate(tg.preset("large", total_calls=60_000, n_hosts=1, pids_per_host=2, tids_per_pid=3,
                              p_drop=0.002, p_sample=0.05, seed=21))[0],
        tg.generate(tg.preset("tiny", total_calls=40_000, seed=22, packet_bytes=1024))[0],
    ]
    with thapi.Context(0) as ctx:
        for b in traces:
            dev = torch.from_numpy(b).to("cuda")
            want_rows, want_diag = _allocating(ctx, dev, b.nbytes)
            got_rows, got_diag = _static(dev, b.nbytes)
            assert got_diag == want_diag
            assert len(got_rows) == len(want_rows) > 0
            for f in thapi.ROW_DTYPE.names:
                assert np.array_equal(got_rows[f], want_rows[f]), f


def test_static_tally_rejects_traces_beyond_its_limits():
    import torch
    b = tg.generate(tg.preset("tiny", total_calls=200_000, packet_bytes=256))[0]  # > 4096 packets
    dev = torch.from_numpy(b).to("cuda")
    with pytest.raises(thapi.ThapiError) as ei:
        thapi.thapi_tally_static(dev.data_ptr(), b.nbytes, 0, 0)
    assert ei.value.code == thapi.E_UNSUPPORTED
