"""The serving loop's host logic without a GPU: the arrival schedule, the
latency accounting (a fake clock and backend) and the percentile."""
from __future__ import annotations

import math

import numpy as np

from paper_2504_03683_b300.serve import Request, Server, percentile, poisson_requests


def test_poisson_schedule():
    spans = [(1000, 1000 + 10**9), (5, 5 + 10**6)]
    reqs = poisson_requests(200.0, 20.0, spans, seed=3)
    assert abs(len(reqs) - 4000) < 4 * math.sqrt(4000)  # Poisson count, 4 sigma
    arr = [r.arrival for r in reqs]
    assert arr == sorted(arr) and 0 < arr[0] and arr[-1] < 20.0
    gaps = np.diff([0.0] + arr)
    assert abs(gaps.mean() - 1 / 200.0) < 0.1 / 200.0
    kinds = [r.kind for r in reqs]
    assert abs(kinds.count("tally") / len(kinds) - 0.5) < 0.05
    for r in reqs:
        if r.kind == "window":
            a, b = spans[r.trace]
            assert a <= r.t0 < r.t1 <= max(b, a + 1)
            assert (r.t1 - r.t0) >= 1
    assert poisson_requests(200.0, 2.0, spans, seed=3) == poisson_requests(200.0, 2.0, spans, seed=3)
    fr = [(r.t1 - r.t0) / (spans[r.trace][1] - spans[r.trace][0]) for r in reqs if r.kind == "window"]
    assert min(fr) >= 0.9e-4 and max(fr) <= 1.0 and np.median(np.log10(fr)) < -1.5  # log-uniform 1e-4..1


def test_percentile_nearest_rank():
    xs = list(range(1, 101))
    assert percentile(xs, 50) == 50 and percentile(xs, 99) == 99 and percentile(xs, 100) == 100
    assert percentile([7.0], 99) == 7.0
    assert percentile([3, 1, 2], 0) == 1


class _FakeServer(Server):
    """Answers from a list; each answer takes `service` seconds of fake time."""

    def __post_init__(self):
        self.traces = [None, None]
        self.now = 0.0
        self.service = 0.01

    def answer(self, r):
        self.now += self.service
        return [0] * (3 if r.kind == "tally" else 5)


def test_latency_counts_queueing():
    s = _FakeServer()

    def clock():
        return s.now

    def sleep(d):
        s.now += d

    reqs = [Request(0.0, "tally", 0), Request(0.001, "window", 1, 0, 10), Request(0.5, "tally", 0)]
    out = s.run(reqs, clock=clock, sleep=sleep)
    lat = [o[0] for o in out]
    # the second request waits for the first (arrives at 1 ms, served from 10 ms to 20 ms)
    assert abs(lat[0] - 0.01) < 1e-9 and abs(lat[1] - 0.019) < 1e-9 and abs(lat[2] - 0.01) < 1e-9
    assert [o[1] for o in out] == [3, 5, 3]
