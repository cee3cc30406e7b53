"""A query-serving loop over device-resident traces.

Traces are loaded once and stay decoded in device memory (tally rows and the
ordered timeline); requests arrive over time and are answered from them:
``tally`` returns a trace's tally rows, ``window`` the intervals of a time
window [t0, t1) of its timeline.  Admission is by device-memory footprint: the
context is created with a cap, and a trace whose load would pass it is
refused (the library's E_NOMEM), not queued.

Window results land in one pinned host buffer, sized at admission for the
largest resident timeline and reused (a result is valid until the next
window answer): copies from pinned memory run at the link's speed, where a
fresh pageable array would both allocate and copy slower.

The loop answers requests in arrival order on one CUDA stream; a request's
latency runs from its scheduled arrival to its result in host memory, so
time spent waiting behind earlier requests counts.  ``poisson_requests``
draws the seeded arrival schedule (exponential gaps, a kind per request, and
for windows a width log-uniform over a range of fractions of the trace's
span, at a uniform start).
"""
from __future__ import annotations

import math
import random
import time
from dataclasses import dataclass, field

from . import thapi


@dataclass
class Request:
    arrival: float   # seconds from the start of the run
    kind: str        # "tally" or "window"
    trace: int       # index into the server's admitted traces
    t0: int = 0
    t1: int = 2**64 - 1


@dataclass
class Resident:
    trace_id: int
    events: int
    t_min: int
    t_max: int
    device_bytes: int


@dataclass
class Server:
    device: int = 0
    hbm_cap_bytes: int = 120 * 10**9
    ctx: thapi.Context = field(init=False)
    traces: list = field(default_factory=list)
    refused: int = 0
    _pinned: object = None   # torch pinned buffer (host memory plumbing only)
    _window: object = None   # its INTERVAL_DTYPE view

    def __post_init__(self):
        self.ctx = thapi.Context(self.device, self.hbm_cap_bytes)

    def _reserve(self, intervals: int):
        if self._window is not None and len(self._window) >= intervals:
            return
        import torch
        self._pinned = torch.empty(max(intervals, 1) * thapi.INTERVAL_DTYPE.itemsize, dtype=torch.uint8,
                                   pin_memory=True)
        self._window = self._pinned.numpy().view(thapi.INTERVAL_DTYPE)

    def admit(self, trace=None, device_ptr: tuple | None = None) -> int | None:
        """Loads a trace (host bytes, or (device pointer, nbytes)); its index,
        or None when the device-memory cap refuses it."""
        try:
            tid = self.ctx.load_device(*device_ptr) if device_ptr is not None else self.ctx.load(trace)
        except thapi.ThapiError as e:
            if e.code == thapi.E_NOMEM:
                self.refused += 1
                return None
            raise
        info = self.ctx.info(tid)
        self._reserve(info["intervals"])
        self.traces.append(Resident(tid, info["events"], info["t_min"], info["t_max"], info["device_bytes"]))
        return len(self.traces) - 1

    def answer(self, r: Request):
        t = self.traces[r.trace]
        if r.kind == "tally":
            rows, _diag = self.ctx.tally(t.trace_id)
            return rows
        return thapi.thapi_timeline(self.ctx.handle, t.trace_id, r.t0, r.t1, out=self._window)

    def run(self, requests, clock=time.perf_counter, sleep=time.sleep):
        """Answers the requests in arrival order; returns per request
        (latency in seconds, result rows)."""
        out = []
        start = clock()
        for r in sorted(requests, key=lambda q: q.arrival):
            now = clock() - start
            if now < r.arrival:
                sleep(r.arrival - now)
            res = self.answer(r)
            out.append((clock() - start - r.arrival, len(res)))
        return out

    def close(self):
        for t in self.traces:
            self.ctx.free(t.trace_id)
        self.traces = []
        self.ctx.close()


def poisson_requests(rate: float, duration: float, spans, seed: int = 0, p_tally: float = 0.5,
                     frac_range=(1e-4, 1.0)):
    """Arrivals of mean rate `rate` per second over `duration` seconds; spans:
    (t_min, t_max) per trace.  Each request picks a trace uniformly; a window
    request's width is a log-uniform fraction of the trace's span."""
    rng = random.Random(seed)
    out, t = [], 0.0
    lo, hi = math.log(frac_range[0]), math.log(frac_range[1])
    while True:
        t += rng.expovariate(rate)
        if t >= duration:
            return out
        k = rng.randrange(len(spans))
        if rng.random() < p_tally:
            out.append(Request(t, "tally", k))
            continue
        a, b = spans[k]
        span = max(b - a, 1)
        w = max(1, int(span * math.exp(rng.uniform(lo, hi))))
        t0 = a + rng.randrange(max(span - w, 0) + 1)
        out.append(Request(t, "window", k, t0, t0 + w))


def percentile(xs, q: float) -> float:
    """Nearest-rank percentile (q in [0, 100]) of a non-empty list."""
    s = sorted(xs)
    k = max(0, min(len(s) - 1, math.ceil(q / 100.0 * len(s)) - 1))
    return s[k]
