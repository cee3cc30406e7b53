"""Batches of traces loaded as one (thapi_trace_load_batch) vs the oracle on
the union trace that the batch defines (tolerance 0)."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import tracegen as tg
from tests._concat import concat_batch
from tests._percpu import to_per_cpu
from tests._util import intervals_equal, rows_equal, stream_table
from tests.test_gpu_parity import assert_parity, gpu_run

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    from paper_2504_03683_b300 import thapi
    assert torch.cuda.is_available()
    c = thapi.Context(0)
    yield c
    c.close()


def _traces():
    out = []
    for k, (calls, seed, over) in enumerate([(3_000, 50, {}), (40_000, 51, dict(p_drop=0.01)), (200, 52, {}),
                                             (25_000, 53, dict(p_ext=0.02)), (9_000, 54, dict(tids_per_pid=3))]):
        cfg = dict(total_calls=calls, n_hosts=1, pids_per_host=1, tids_per_pid=4, seed=seed, packet_bytes=4096)
        cfg.update(over)
        out.append(tg.generate(tg.preset("large", **cfg))[0])
    out.append(to_per_cpu(out[1], n_cpus=2, seed=55))  # per-CPU buffers in the batch as well
    return out


def _run_batch(ctx, traces, device=False):
    if device:
        import torch
        bufs = [torch.from_numpy(np.frombuffer(bytes(t), dtype=np.uint8).copy()).cuda() for t in traces]
        tid = ctx.load_batch_device([(b.data_ptr(), b.numel()) for b in bufs])
    else:
        tid = ctx.load_batch(traces)
    try:
        rows, diag = ctx.tally(tid)
        ivs = ctx.timeline(tid)
        info = ctx.info(tid)
    finally:
        ctx.free(tid)
    return rows, diag, ivs, info


@pytest.mark.parametrize("device", [False, True])
def test_batch_equals_oracle_on_the_union(ctx, device):
    traces = _traces()
    union = concat_batch(traces)
    o = oracle.run(union)
    assert o.code == oracle.OK
    rows, diag, ivs, info = _run_batch(ctx, traces, device)
    for k in oracle.DIAG_FIELDS:
        assert diag[k] == o.diag[k], k
    assert rows_equal(rows, o.rows)
    assert intervals_equal(ivs, o.intervals)
    assert info["n_streams"] == sum(len(stream_table(t)) for t in traces)
    # the union also goes through the plain path
    assert_parity(ctx, union)


def test_batch_of_one_equals_a_plain_load(ctx):
    t = _traces()[1]
    rows, diag, ivs, _info = _run_batch(ctx, [t])
    rows2, diag2, ivs2, _w, _i = gpu_run(ctx, t)
    assert rows_equal(rows, rows2) and intervals_equal(ivs, ivs2) and diag == diag2


def test_batch_self_time_and_device_activity(ctx):
    from paper_2504_03683_b300 import thapi
    traces = [tg.generate(tg.preset("device", total_calls=8_000, n_hosts=1, pids_per_host=2, tids_per_pid=2,
                                    n_device_streams=3, seed=60 + k))[0] for k in range(3)]
    union = concat_batch(traces)
    o = oracle.run(union)
    with thapi.Context(0) as c:
        c.set_self_time(True)
        tid = c.load_batch(traces)
        try:
            rows, _d = c.tally(tid)
            dev_rows, dev_diag = c.device_tally(tid)
            srows = c.self_tally(tid)
            ivs = c.timeline(tid)
        finally:
            c.free(tid)
    assert rows_equal(rows, o.rows) and rows_equal(srows, o.self_rows) and rows_equal(dev_rows, o.dev_rows)
    assert intervals_equal(ivs, o.intervals)
    for k in oracle.DEV_DIAG_FIELDS:
        assert dev_diag[k] == o.dev_diag[k], k


def test_batch_needs_one_packet_size(ctx):
    from paper_2504_03683_b300 import thapi
    a = tg.generate(tg.preset("large", total_calls=500, n_hosts=1, pids_per_host=1, tids_per_pid=2, seed=1,
                              packet_bytes=4096))[0]
    b = tg.generate(tg.preset("large", total_calls=500, n_hosts=1, pids_per_host=1, tids_per_pid=2, seed=2,
                              packet_bytes=8192))[0]
    with pytest.raises(thapi.ThapiError) as ei:
        ctx.load_batch([a, b])
    assert ei.value.code == thapi.E_UNSUPPORTED


def test_batch_errors_name_the_trace_or_the_packet(ctx):
    from paper_2504_03683_b300 import thapi
    traces = [np.frombuffer(bytes(t), dtype=np.uint8).copy() for t in _traces()[:3]]
    bad = [t.copy() for t in traces]
    bad[2][0] ^= 0xFF  # trace 2's file magic
    with pytest.raises(thapi.ThapiError) as ei:
        ctx.load_batch(bad)
    assert ei.value.code == thapi.E_FORMAT and ei.value.location == (0, 2, 0)
    # a packet header error in trace 1: located by the packet's index in the batch
    bad = [t.copy() for t in traces]
    import struct
    pk_off = struct.unpack_from("<Q", bytes(bad[1][:128]), 88)[0]
    P = struct.unpack_from("<I", bytes(bad[1][:16]), 8)[0]
    bad[1][pk_off + 3 * P] ^= 0xFF  # the magic of its fourth packet
    o = oracle.run(concat_batch(bad))
    with pytest.raises(thapi.ThapiError) as ei:
        ctx.load_batch(bad)
    assert ei.value.code == o.code and ei.value.location == o.loc


def _named_trace(host: str, funcs=("alpha", "beta", "gamma"), seed: int = 0):
    """A small hand-built trace with one host of the given name and three call
    functions; its tables equal those of any other trace built with the same
    functions (a batch takes the head of such a trace without parsing its
    tables again)."""
    from tracegen.handbuilt import Ev, TraceBuilder
    tb = TraceBuilder(packet_bytes=1024)
    h = tb.add_host(host)
    fs = [tb.add_call_func(f) for f in funcs]
    for k in range(2):
        s = tb.add_stream(h, 10 + seed, 100 + k)
        evs, t = [], 1_000 + 7 * seed
        for i in range(40):
            _f, e, x = fs[(i + k + seed) % len(fs)]
            evs += [Ev(e, t), Ev(x, t + 5 + i, result=i % 7 == 0)]
            t += 20
        tb.place(tb.stream_events(s, evs, ts_begin=1_000))
    return np.frombuffer(tb.build(), dtype=np.uint8).copy()


def test_batch_host_names_and_head_checks(ctx):
    """Traces whose class and function tables equal the first trace's: each
    keeps its own host name, rows and intervals equal the oracle's on the
    union, and a bad host-name offset or stream-row host in a later trace is
    reported at that trace, as a full parse reports it.  A trace whose
    function names differ still makes the batch unsupported."""
    import struct
    from paper_2504_03683_b300 import thapi
    names = ["node-a", "n-b", "a-much-longer-host-name", "z"]
    traces = [_named_trace(n, seed=k) for k, n in enumerate(names)]
    union = concat_batch(traces)
    o = oracle.run(union)
    assert o.code == oracle.OK
    tid = ctx.load_batch(traces)
    try:
        rows, diag = ctx.tally(tid)
        ivs = ctx.timeline(tid)
        assert [thapi.thapi_trace_strings(ctx.handle, tid, 0, h) for h in range(len(names))] == names
        assert [thapi.thapi_trace_strings(ctx.handle, tid, 1, f) for f in range(3)] == ["alpha", "beta", "gamma"]
    finally:
        ctx.free(tid)
    assert rows_equal(rows, o.rows) and intervals_equal(ivs, o.intervals)
    for k in oracle.DIAG_FIELDS:
        assert diag[k] == o.diag[k], k

    def head(t):
        b = bytes(t[:128])
        return {k: struct.unpack_from("<Q", b, off)[0] for k, off in (("st", 40), ("ho", 64), ("sb", 80))}

    # trace 2's host name offset past its string block
    bad = [t.copy() for t in traces]
    h2 = head(bad[2])
    struct.pack_into("<I", bad[2], h2["ho"], h2["sb"] + 3)
    with pytest.raises(thapi.ThapiError) as ei:
        ctx.load_batch(bad)
    assert ei.value.code == thapi.E_FORMAT and ei.value.location == (0, 2, 0)
    # trace 3's second stream names host 1 of a trace with one host
    bad = [t.copy() for t in traces]
    struct.pack_into("<I", bad[3], head(bad[3])["st"] + 16, 1)
    with pytest.raises(thapi.ThapiError) as ei:
        ctx.load_batch(bad)
    assert ei.value.code == thapi.E_FORMAT and ei.value.location == (0, 3, 0)
    # the same errors in a batch whose tables all differ from the first trace's are reported alike
    other = [_named_trace(n, funcs=("alpha", "beta", "delta"), seed=k) for k, n in enumerate(names)]
    with pytest.raises(thapi.ThapiError) as ei:
        ctx.load_batch([traces[0]] + other[1:])
    assert ei.value.code == thapi.E_UNSUPPORTED
    bad = [traces[0]] + [t.copy() for t in other[1:]]
    struct.pack_into("<I", bad[2], head(bad[2])["ho"], head(bad[2])["sb"] + 3)
    with pytest.raises(thapi.ThapiError) as ei:
        ctx.load_batch(bad)
    assert ei.value.code == thapi.E_FORMAT and ei.value.location == (0, 2, 0)
