"""Per-CPU buffers through the CUDA path vs the oracle (tolerance 0): threads
regrouped across buffers, paired, tallied and merged into the timeline."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import tracegen as tg
from tests._percpu import to_per_cpu
from tests.test_gpu_parity import _windows, assert_parity
from tracegen.handbuilt import Ev, TraceBuilder

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    from paper_2504_03683_b300 import thapi
    assert torch.cuda.is_available()
    c = thapi.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("over,n_cpus", [
    (dict(total_calls=30_000, n_hosts=2, pids_per_host=2, tids_per_pid=2, seed=3, p_drop=0.005), 3),
    (dict(total_calls=20_000, n_hosts=1, pids_per_host=2, tids_per_pid=4, seed=4, p_ext=0.02, packet_bytes=1024), 2),
    (dict(total_calls=20_000, n_hosts=1, pids_per_host=1, tids_per_pid=3, seed=5, packet_bytes=256), 4),
    (dict(total_calls=40_000, n_hosts=1, pids_per_host=2, tids_per_pid=2, seed=6, packet_bytes=32768), 2),
])
def test_per_cpu_workloads(ctx, over, n_cpus):
    b, _c, _e = tg.generate(tg.preset("large", **over))
    pc = to_per_cpu(b, n_cpus=n_cpus, seed=over["seed"])
    o = assert_parity(ctx, pc, _windows(oracle.run(pc), seed=over["seed"]))
    ref = oracle.run(b)
    assert o.diag["pairs"] == ref.diag["pairs"]


def test_per_cpu_migration_case(ctx):
    tb = TraceBuilder(packet_bytes=256)
    h = tb.add_host("h")
    f, ef, xf = tb.add_call_func("f")
    g, eg, xg = tb.add_call_func("g")
    c0, c1 = tb.add_stream(h, 0, 0, 2), tb.add_stream(h, 0, 1, 2)
    A, B = (5, 7), (5, 8)
    cpu0 = [Ev(ef, 100, ctx=A), Ev(ef, 105, ctx=B), Ev(eg, 110, ctx=A), Ev(xf, 130, result=3, ctx=B)]
    cpu1 = [Ev(xg, 140, result=0, ctx=A), Ev(xf, 170, result=0, ctx=A)]
    tb.place(tb.stream_events(c0, cpu0, ts_begin=100))
    tb.place(tb.stream_events(c1, cpu1, ts_begin=100))
    o = assert_parity(ctx, tb.build())
    assert [tuple(int(v) for v in x) for x in o.intervals.tolist()] == [
        (100, 170, c0, f, 0, 0), (105, 130, c0, f, 0, 1), (110, 140, c0, g, 1, 0)]


def test_per_cpu_and_per_thread_streams_mixed(ctx):
    """Per-thread streams and per-CPU buffers in one trace, some thread keys in both
    (their rows combine), unmatched and mismatched calls on the per-CPU side."""
    tb = TraceBuilder(packet_bytes=512)
    h = tb.add_host("h")
    f, ef, xf = tb.add_call_func("f")
    g, eg, xg = tb.add_call_func("g")
    s_t = tb.add_stream(h, 5, 7)                    # thread (5, 7) as its own stream
    c0, c1 = tb.add_stream(h, 0, 0, 2), tb.add_stream(h, 0, 1, 2)
    tb.place(tb.stream_events(s_t, [Ev(ef, 10), Ev(xf, 20, result=0), Ev(eg, 30), Ev(xg, 35, result=1)], ts_begin=10))
    ev0, ev1 = [], []
    t = 100
    for k in range(300):
        ctxk = (5, 7 + (k % 3))                      # threads (5,7), (5,8), (5,9)
        lst = ev0 if (k // 7) % 2 == 0 else ev1
        lst.append(Ev(ef if k % 5 else eg, t, ctx=ctxk))
        t += 3
        other = ev1 if lst is ev0 else ev0           # some exits on the other CPU
        (other if k % 4 == 0 else lst).append(Ev(xf if k % 5 else (xf if k % 11 == 0 else xg), t, result=k % 2,
                                                  ctx=ctxk))
        t += 2
    ev0.append(Ev(ef, t + 5, ctx=(5, 9)))            # never closed
    ev1.append(Ev(xg, t + 7, result=0, ctx=(6, 1)))  # exit on an empty stack
    ev0.sort(key=lambda e: e.ts)
    ev1.sort(key=lambda e: e.ts)
    tb.place(tb.stream_events(c0, ev0, ts_begin=100))
    tb.place(tb.stream_events(c1, ev1, ts_begin=100))
    o = assert_parity(ctx, tb.build())
    assert o.diag["unmatched_entries"] >= 1 and o.diag["unmatched_exits"] >= 1 and o.diag["mismatched_pairs"] > 0


def test_per_cpu_decode(ctx):
    b, _c, _e = tg.generate(tg.preset("large", total_calls=10_000, n_hosts=1, pids_per_host=2, tids_per_pid=2, seed=8))
    pc = to_per_cpu(b, n_cpus=3, seed=8)
    got = ctx.decode(pc)
    ref = oracle.decode(pc)
    for fld in ("ts", "cmd", "stream_id", "class_id", "var_len", "result", "ext", "kind", "func_id", "vpid", "vtid"):
        assert np.array_equal(got[fld], ref[fld]), fld


def test_per_cpu_header_errors_match_oracle(ctx):
    from paper_2504_03683_b300 import thapi
    tb = TraceBuilder(packet_bytes=256)
    h = tb.add_host("h")
    f, e, x = tb.add_call_func("f")
    c0 = tb.add_stream(h, 0, 0, 2)
    ok = tb.encode_event(e, 1, ctx=(1, 1))
    tb.raw_packet(c0, 0, [ok, ok[:12]], n_events=2)
    trace = tb.build()
    o = oracle.run(trace)
    for call in (ctx.load, ctx.decode):
        with pytest.raises(thapi.ThapiError) as ei:
            call(trace)
        assert ei.value.code == o.code and ei.value.location == o.loc


def test_per_cpu_needs_packets_of_at_most_32k(ctx):
    from paper_2504_03683_b300 import thapi
    tb = TraceBuilder(packet_bytes=65536)
    h = tb.add_host("h")
    f, e, x = tb.add_call_func("f")
    c0 = tb.add_stream(h, 0, 0, 2)
    tb.place(tb.stream_events(c0, [Ev(e, 1, ctx=(1, 1)), Ev(x, 2, result=0, ctx=(1, 1))], ts_begin=1))
    with pytest.raises(thapi.ThapiError) as ei:
        ctx.load(tb.build())
    assert ei.value.code == thapi.E_UNSUPPORTED


def test_per_cpu_many_threads_take_the_sort_path(ctx):
    """40,000 threads (more than the thread table takes) in two per-CPU buffers:
    the order comes from the fallback sorts; results as the oracle's."""
    tb = TraceBuilder(packet_bytes=4096)
    h = tb.add_host("h")
    f, ef, xf = tb.add_call_func("f")
    g, eg, xg = tb.add_call_func("g")
    c0, c1 = tb.add_stream(h, 0, 0, 2), tb.add_stream(h, 0, 1, 2)
    ev0, ev1 = [], []
    t = 1000
    for k in range(40_000):
        th = (7 + k % 3, 100 + k)
        (ev0 if k % 2 else ev1).append(Ev(ef, t, ctx=th))
        (ev1 if k % 5 == 0 else (ev0 if k % 2 else ev1)).append(Ev(eg, t + 1, ctx=th))
        (ev0 if k % 2 else ev1).append(Ev(xg, t + 2, result=0, ctx=th))
        (ev0 if k % 2 else ev1).append(Ev(xf if k % 17 else xg, t + 4, result=k % 2, ctx=th))
        t += 3
    ev0.sort(key=lambda e: e.ts)
    ev1.sort(key=lambda e: e.ts)
    tb.place(tb.stream_events(c0, ev0, ts_begin=1000))
    tb.place(tb.stream_events(c1, ev1, ts_begin=1000))
    o = assert_parity(ctx, tb.build())
    assert len(o.rows) > 40_000
