"""Time-window queries (thapi_timeline with [t0, t1), the timeline view of a
time range) against the oracle on a trace built to stress the window index:
one call that spans the whole trace (its interval sits in the first block
yet belongs to every window), calls nested inside it, thousands of short
calls on other streams (many index blocks of 2048 intervals), zero-length
calls and equal starts; windows before, after and inside the trace, empty
ones (t0 = t1, which still catches the calls open at t0), one-nanosecond
ones, and windows whose edges sit on interval starts and ends."""
from __future__ import annotations

import random

import numpy as np
import pytest

import oracle
from paper_2504_03683_b300 import thapi
from tests._util import intervals_equal
from tracegen.handbuilt import Ev, TraceBuilder

pytestmark = pytest.mark.gpu

T0 = 5_000_000_000


def _trace():
    rng = random.Random(17)
    tb = TraceBuilder(packet_bytes=2048)
    h = tb.add_host("node0")
    funcs = [tb.add_call_func("f%d" % k) for k in range(6)]
    streams = [tb.add_stream(h, 100, 100 + k) for k in range(4)]
    span = 2_000_000
    for s in streams:
        evs = []
        t = T0 + rng.randrange(50)
        if s == streams[0]:  # the long call: open from the first event to the last
            _f, e, x = funcs[0]
            evs.append(Ev(e, T0))
        n = 6000 if s != streams[0] else 3000
        for i in range(n):
            _f, e, x = funcs[1 + rng.randrange(5)]
            d = 0 if rng.random() < 0.05 else rng.randrange(1, 400)
            evs += [Ev(e, t), Ev(x, t + d, result=0 if rng.random() < 0.99 else 5)]
            t += d + (0 if rng.random() < 0.05 else rng.randrange(1, span // n))
        if s == streams[0]:
            evs.append(Ev(funcs[0][2], t + 10, result=0))
        tb.place(tb.stream_events(s, evs, ts_begin=T0))
    return np.frombuffer(tb.build(), dtype=np.uint8)


def test_windows_equal_the_oracle():
    import torch
    b = _trace()
    ref = oracle.run(b)
    ivs = ref.intervals
    assert len(ivs) > 10 * 2048
    lo_t, hi_t = int(ivs["start_ns"].min()), int(ivs["end_ns"].max())
    rng = random.Random(3)
    windows = [(0, lo_t), (hi_t + 1, 2**64 - 1), (lo_t, lo_t), (hi_t, hi_t), (hi_t, hi_t + 1), (0, 1),
               (lo_t - 5, lo_t + 1), (0, 2**64 - 2), (1, 2**64 - 1)]
    for _ in range(40):
        a = rng.randrange(lo_t, hi_t)
        w = rng.choice([0, 1, 7, 1000, 50_000, 400_000, hi_t - lo_t])
        windows.append((a, a + w))
    for _ in range(10):  # edges on interval boundaries
        k = ivs[rng.randrange(len(ivs))]
        windows.append((int(k["end_ns"]), int(k["start_ns"]) + 1))
        windows.append((int(k["start_ns"]), int(k["end_ns"])))
    with thapi.Context(0) as ctx:
        tid = ctx.load(b)
        dev = torch.empty(len(ivs) * 24 + 24, dtype=torch.uint8, device="cuda")
        for (t0, t1) in windows:
            want = oracle.run(b, t0=t0, t1=t1).intervals
            got = ctx.timeline(tid, t0, t1)
            assert intervals_equal(got, want), (t0, t1)
            n = thapi.thapi_timeline_device(ctx.handle, tid, t0, t1, dev.data_ptr(), len(ivs) + 1)
            torch.cuda.synchronize()
            assert n == len(want)
            assert intervals_equal(dev[: n * 24].cpu().numpy().view(thapi.INTERVAL_DTYPE), want), (t0, t1)
        # the long call belongs to every window inside its span, its first index block's
        # running maximum reaching even the windows near its end
        long_iv = ivs[(ivs["end_ns"] - ivs["start_ns"]) == (ivs["end_ns"] - ivs["start_ns"]).max()][0]
        e = int(long_iv["end_ns"])
        got = ctx.timeline(tid, e - 3, e - 2)
        assert any(int(g["start_ns"]) == int(long_iv["start_ns"]) for g in got)
        ctx.free(tid)
