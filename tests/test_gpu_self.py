"""Self (exclusive) time through the CUDA path vs the oracle (tolerance 0):
warp and CTA analysis kernels, second-pass dense packets, pairs across
packets, nesting past 255 levels, per-CPU buffers, device workloads."""
from __future__ import annotations

import pytest

import oracle
import tracegen as tg
from tests._percpu import to_per_cpu
from tests._util import intervals_equal, rows_equal
from tests.test_gpu_parity import _builder
from tracegen.handbuilt import Ev, TraceBuilder

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sctx():
    import torch
    from paper_2504_03683_b300 import thapi
    assert torch.cuda.is_available()
    c = thapi.Context(0)
    c.set_self_time(True)
    yield c
    c.close()


def assert_self(ctx, trace):
    o = oracle.run(trace)
    assert o.code == oracle.OK
    tid = ctx.load(trace)
    try:
        rows, diag = ctx.tally(tid)
        ivs = ctx.timeline(tid)
        srows = ctx.self_tally(tid)
        info = ctx.info(tid)
    finally:
        ctx.free(tid)
    for k in oracle.DIAG_FIELDS:
        assert diag[k] == o.diag[k], k
    assert rows_equal(rows, o.rows)
    assert intervals_equal(ivs, o.intervals)
    assert info["self_time"] == 1
    assert rows_equal(srows, o.self_rows)
    return o


@pytest.mark.parametrize("over", [
    dict(total_calls=40_000, n_hosts=2, pids_per_host=2, tids_per_pid=2, seed=31, p_drop=0.01),
    dict(total_calls=30_000, n_hosts=1, pids_per_host=2, tids_per_pid=2, seed=32, packet_bytes=256, p_ext=0.02),
    dict(total_calls=30_000, n_hosts=1, pids_per_host=1, tids_per_pid=3, seed=33, packet_bytes=1024, p_sample=0.05,
         p_drop=0.003),
    dict(total_calls=60_000, n_hosts=1, pids_per_host=1, tids_per_pid=2, seed=34, packet_bytes=65536, p_drop=0.002),
])
def test_self_generated(sctx, over):
    o = assert_self(sctx, tg.generate(tg.preset("large", **over))[0])
    assert int(o.intervals["level"].max()) >= 2


def test_self_layered_worked_case(sctx):
    tb = TraceBuilder(packet_bytes=256)
    h = tb.add_host("h")
    hip, eh, xh = tb.add_call_func("hipDeviceSynchronize", layer=0)
    ze, ez, xz = tb.add_call_func("zeEventHostSynchronize", layer=1)
    lf, el, xl = tb.add_call_func("leaf", layer=1)
    s = tb.add_stream(h, 1, 1)
    evs = [Ev(eh, 1000), Ev(ez, 1010), Ev(el, 1012), Ev(xl, 1020, result=0), Ev(xz, 1040, result=0),
           Ev(ez, 1050), Ev(xz, 1095, result=0), Ev(xh, 1100, result=2)]
    tb.place(tb.stream_events(s, evs, ts_begin=1000))
    o = assert_self(sctx, tb.build())
    assert sorted(int(v) for v in o.self_rows["total_ns"]) == [8, 25, 67]


def test_self_dense_packets(sctx):
    # minimum-size events: nested calls fill 16 KB packets past the fast-path capacity
    tb, h, ids = _builder(P=16384)
    for s in (tb.add_stream(h, 7, 7), tb.add_stream(h, 7, 8)):
        evs, t = [], 1000
        for k in range(3000):
            evs += [Ev(ids[0][1], t), Ev(ids[1][1], t + 1), Ev(ids[1][2], t + 2, result=k % 5 == 0),
                    Ev(ids[2][1], t + 3), Ev(ids[2][2], t + 5), Ev(ids[0][2], t + 9 + k % 3)]
            t += 20
        tb.place(tb.stream_events(s, evs, ts_begin=1000))
    assert_self(sctx, tb.build())


def test_self_deep_nesting_across_packets(sctx):
    """300 levels over 256-byte packets, each level with a leaf child and a
    sibling pair, a dropped exit in the middle and an unmatched exit at the end:
    parents and children are paired across packets and levels pass 255."""
    tb, h, ids = _builder(P=256)
    s = tb.add_stream(h, 3, 3)
    depth, t, evs = 300, 100, []
    for d in range(depth):
        evs.append(Ev(ids[d % 3][1], t))
        evs += [Ev(ids[2][1], t + 1), Ev(ids[2][2], t + 2 + d % 4, result=0)]
        t += 10
    for d in reversed(range(depth)):
        if d == 150:
            t += 10
            continue  # its exit is dropped: the levels below pair with shifted entries
        evs.append(Ev(ids[d % 3][2], t, result=d % 11 == 0))
        t += 7 + d % 5
    evs += [Ev(ids[0][2], t + 100), Ev(ids[1][1], t + 101)]
    tb.place(tb.stream_events(s, evs, ts_begin=100))
    o = assert_self(sctx, tb.build())
    assert o.diag["mismatched_pairs"] > 0


def test_self_per_cpu(sctx):
    b, _c, _e = tg.generate(tg.preset("large", total_calls=30_000, n_hosts=2, pids_per_host=2, tids_per_pid=2,
                                      seed=35, p_drop=0.005))
    assert_self(sctx, to_per_cpu(b, n_cpus=3, seed=35))


def test_self_per_cpu_and_per_thread_mixed(sctx):
    tb = TraceBuilder(packet_bytes=512)
    h = tb.add_host("h")
    f, ef, xf = tb.add_call_func("f")
    g, eg, xg = tb.add_call_func("g")
    s_t = tb.add_stream(h, 5, 7)
    c0, c1 = tb.add_stream(h, 0, 0, 2), tb.add_stream(h, 0, 1, 2)
    tb.place(tb.stream_events(s_t, [Ev(ef, 10), Ev(eg, 12), Ev(xg, 15, result=0), Ev(xf, 20, result=0)], ts_begin=10))
    ev0, ev1, t = [], [], 100
    for k in range(200):
        ctxk = (5, 7 + (k % 3))
        a, b = (ev0, ev1) if (k // 5) % 2 == 0 else (ev1, ev0)
        a += [Ev(ef, t, ctx=ctxk), Ev(eg, t + 1, ctx=ctxk)]
        b += [Ev(xg, t + 2 + k % 3, result=0, ctx=ctxk)]          # the child exits on the other CPU
        a += [Ev(xf if k % 13 else xg, t + 6, result=k % 2, ctx=ctxk)]
        t += 10
    ev0.sort(key=lambda e: e.ts)
    ev1.sort(key=lambda e: e.ts)
    tb.place(tb.stream_events(c0, ev0, ts_begin=100))
    tb.place(tb.stream_events(c1, ev1, ts_begin=100))
    assert_self(sctx, tb.build())


def test_self_device_workload(sctx):
    b, _c, _e = tg.generate(tg.preset("device", total_calls=30_000, n_hosts=1, pids_per_host=2, tids_per_pid=2,
                                      n_device_streams=3, seed=36))
    assert_self(sctx, b)


def test_self_time_off_has_no_rows():
    from paper_2504_03683_b300 import thapi
    b, _c, _e = tg.generate(tg.preset("tiny", seed=37))
    with thapi.Context(0) as c:
        tid = c.load(b)
        try:
            assert c.info(tid)["self_time"] == 0
            with pytest.raises(thapi.ThapiError) as ei:
                c.self_tally(tid)
            assert ei.value.code == thapi.E_INVALID
        finally:
            c.free(tid)
