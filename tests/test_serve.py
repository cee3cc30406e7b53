"""Host logic of serving without a GPU: the seeded schedule (Poisson arrivals,
loads, frees of the oldest trace, queries only on resident traces), its
translation to serving-loop requests, the one-at-a-time baseline's order and
latency accounting (fake clock and backend), and the percentile."""
from __future__ import annotations

import math

import numpy as np

from paper_2504_03683_b300 import thapi
from paper_2504_03683_b300.serve import Step, make_schedule, percentile, serve_serial, summary, to_requests

SPANS = [(1000, 1000 + 10**9), (5, 5 + 10**6), (0, 10**7)]


def test_schedule_is_poisson_and_mixed():
    steps = make_schedule(200.0, 20.0, [0, 1, 2, 0], SPANS, seed=3, p_load=0.05, p_free=0.05)
    assert abs(len(steps) - 4000) < 4 * math.sqrt(4000)  # Poisson count, 4 sigma
    arr = [s.arrival for s in steps]
    assert arr == sorted(arr) and 0 < arr[0] and arr[-1] < 20.0
    gaps = np.diff([0.0] + arr)
    assert abs(gaps.mean() - 1 / 200.0) < 0.1 / 200.0
    kinds = [s.kind for s in steps]
    for k, p in (("load", 0.05), ("free", 0.05), ("tally", 0.45), ("window", 0.45)):
        assert abs(kinds.count(k) / len(kinds) - p) < 0.03, k
    assert make_schedule(200.0, 2.0, [0, 1], SPANS, seed=3) == make_schedule(200.0, 2.0, [0, 1], SPANS, seed=3)


def test_schedule_names_only_resident_traces():
    resident = [0, 1, 2, 0]
    steps = make_schedule(500.0, 4.0, resident, SPANS, seed=9, p_load=0.1, p_free=0.1, min_resident=2)
    live = list(range(len(resident)))
    src = list(resident)
    for s in steps:
        if s.kind == "load":
            assert s.handle == len(src) and 0 <= s.source < len(SPANS)
            src.append(s.source)
            live.append(s.handle)
        elif s.kind == "free":
            assert s.handle == live[0] and len(live) > 2  # the oldest leaves, never below min_resident
            live.pop(0)
        else:
            assert s.handle in live
            if s.kind == "window":
                a, b = SPANS[src[s.handle]]
                assert a <= s.t0 < s.t1 <= max(b, a + 1)
    fr = [(s.t1 - s.t0) / (SPANS[src[s.handle]][1] - SPANS[src[s.handle]][0]) for s in steps if s.kind == "window"]
    assert min(fr) >= 0.9e-4 and max(fr) <= 1.0 and np.median(np.log10(fr)) < -1.5  # log-uniform 1e-4..1


def test_requests_name_the_load_that_brings_a_trace_in():
    steps = [Step(0.0, "tally", 0), Step(0.1, "load", 2, source=1), Step(0.2, "window", 2, t0=5, t1=9),
             Step(0.3, "free", 2), Step(0.4, "free", 1)]
    reqs = to_requests(steps, ids=[11, 12], sources=[(0x1000, 64, False), (0x2000, 128, True)])
    assert [r.kind for r in reqs] == [thapi.REQ_TALLY, thapi.REQ_LOAD, thapi.REQ_WINDOW, thapi.REQ_FREE,
                                      thapi.REQ_FREE]
    assert reqs[0].trace == 11 and reqs[0].after == 0
    assert reqs[1].bytes == 0x2000 and reqs[1].nbytes == 128 and reqs[1].on_device == 1
    assert reqs[2].after == 2 and (reqs[2].t0, reqs[2].t1) == (5, 9)
    assert reqs[3].after == 2 and reqs[4].trace == 12 and reqs[4].after == 0


class _Fake:
    """Plain-path backend on a fake clock: every request takes `service`
    seconds; loads are refused by the cap while `full` is set."""

    def __init__(self):
        self.now = 0.0
        self.service = 0.01
        self.full = False
        self.next_id = 100
        self.log = []

    def clock(self):
        return self.now

    def sleep(self, d):
        self.now += d

    def do(self, st, trace):
        self.log.append((st.kind, st.handle))
        if st.kind == "load" and self.full:
            return thapi.E_NOMEM, 0, 0, 0
        self.now += self.service
        if st.kind == "load":
            self.next_id += 1
            return thapi.OK, self.next_id, 0, 10
        if st.kind == "free":
            self.full = False
        return thapi.OK, trace, 3, 10


def test_serial_baseline_counts_queueing():
    f = _Fake()
    steps = [Step(0.0, "tally", 0), Step(0.001, "window", 1, t0=0, t1=10), Step(0.5, "tally", 0)]
    out = serve_serial(None, steps, [7, 8], [], None, None, clock=f.clock, sleep=f.sleep, backend=f)
    lat = [o.t_done - o.t_arrival for o in out]
    # the second request waits for the first (arrives at 1 ms, served from 10 ms to 20 ms)
    assert abs(lat[0] - 0.01) < 1e-9 and abs(lat[1] - 0.019) < 1e-9 and abs(lat[2] - 0.01) < 1e-9
    assert [o.trace for o in out] == [7, 8, 7]


def test_serial_baseline_admission_order():
    """A load the cap refuses waits for the next free; a query on its trace waits
    for it; queries on other traces go ahead; a free waits for earlier queries."""
    f = _Fake()
    f.full = True
    steps = [Step(0.0, "load", 2, source=0), Step(0.001, "tally", 2), Step(0.002, "tally", 0),
             Step(0.003, "free", 1), Step(0.004, "window", 2, t0=0, t1=5)]
    out = serve_serial(None, steps, [7, 8], [(0, 0, True)], None, None, clock=f.clock, sleep=f.sleep, backend=f)
    assert all(o.status == thapi.OK for o in out)
    assert f.log == [("load", 2), ("tally", 0), ("free", 1), ("load", 2), ("tally", 2), ("window", 2)]
    assert out[1].trace == out[4].trace == out[0].trace == 101
    s = summary(out)
    assert s["failed"] == 0 and s["load"]["n"] == 1 and s["queries"]["n"] == 3


def test_percentile_nearest_rank():
    xs = list(range(1, 101))
    assert percentile(xs, 50) == 50 and percentile(xs, 99) == 99 and percentile(xs, 100) == 100
    assert percentile([7.0], 99) == 7.0
    assert percentile([3, 1, 2], 0) == 1
