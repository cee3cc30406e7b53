"""thapi_tally_static: the tally for callers that cannot allocate device memory.

A tracing agent that tallies on the node while the traced application runs
in the same CUDA context cannot count on allocating device memory: the
application (or its framework's caching allocator) usually holds almost all
of it, and an allocation by the agent could fail or disturb the run being
observed.  thapi_tally_static takes its working memory from an array that is
part of the library instead.

This test calls it through the C ABI twice in a row on each of two traces
(the shared array keeps the previous call's contents) and checks rows and
diagnostics exactly against the oracle and against the allocating path
(thapi_trace_load_device + thapi_tally).  Around the second call on each
trace it also checks that the device's free memory and torch's allocated
bytes are unchanged.  A first call may still make the driver load the
kernels it launches (lazy module loading, per kernel), which is not an
allocation by the entry point, so first calls are not measured.
"""
import numpy as np
import pytest

import oracle
import tracegen as tg
from paper_2504_03683_b300 import thapi

pytestmark = pytest.mark.gpu


def _allocating(ctx, dev, nbytes):
    tid = thapi.thapi_trace_load_device(ctx.handle, dev.data_ptr(), nbytes)
    try:
        return thapi.thapi_tally(ctx.handle, tid)
    finally:
        ctx.free(tid)


def _static(dev, nbytes, rows_dev):
    import torch
    n, _diag = thapi.thapi_tally_static(dev.data_ptr(), nbytes, 0, 0)  # size query
    assert n * thapi.ROW_DTYPE.itemsize <= rows_dev.numel()
    n2, diag = thapi.thapi_tally_static(dev.data_ptr(), nbytes, rows_dev.data_ptr(), n)
    torch.cuda.synchronize()
    assert n2 == n
    return n, diag


def _rows_equal(a, b):
    return len(a) == len(b) and all(np.array_equal(a[f], b[f]) for f in thapi.ROW_DTYPE.names)


def test_static_tally_equals_oracle_and_allocating_tally_twice_in_a_row():
    import torch
    traces = [
        tg.generate(tg.preset("large", total_calls=60_000, n_hosts=1, pids_per_host=2, tids_per_pid=3,
                              p_drop=0.002, p_sample=0.05, seed=21))[0],
        tg.generate(tg.preset("tiny", total_calls=40_000, seed=22, packet_bytes=1024))[0],
    ]
    refs = [oracle.run(b, want_intervals=False) for b in traces]
    devs = [torch.from_numpy(b).to("cuda") for b in traces]
    rows_dev = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")  # output memory the caller owns
    with thapi.Context(0) as ctx:
        want = [_allocating(ctx, d, b.nbytes) for d, b in zip(devs, traces)]
    torch.cuda.synchronize()
    for k, (b, d, ref) in enumerate(zip(traces, devs, refs)):
        for call in range(2):
            free0 = torch.cuda.mem_get_info()[0]
            held0 = torch.cuda.memory_allocated()
            n, diag = _static(d, b.nbytes, rows_dev)
            if call == 1:  # a repeated call: nothing allocated, nothing left held
                assert torch.cuda.mem_get_info()[0] == free0
                assert torch.cuda.memory_allocated() == held0
            got = rows_dev[: n * thapi.ROW_DTYPE.itemsize].cpu().numpy().view(thapi.ROW_DTYPE)
            assert n > 0
            assert diag == ref.diag
            assert _rows_equal(got, ref.rows)
            assert diag == want[k][1] and _rows_equal(got, want[k][0])


def test_static_tally_rejects_traces_beyond_its_limits():
    import torch
    b = tg.generate(tg.preset("tiny", total_calls=200_000, packet_bytes=256))[0]  # > 4096 packets
    dev = torch.from_numpy(b).to("cuda")
    with pytest.raises(thapi.ThapiError) as ei:
        thapi.thapi_tally_static(dev.data_ptr(), b.nbytes, 0, 0)
    assert ei.value.code == thapi.E_UNSUPPORTED
