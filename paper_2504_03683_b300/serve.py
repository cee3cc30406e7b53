"""Serving traces: a schedule of requests, served two ways.

The paper's analysis runs on the traced job's node, beside it (on-node
processing, Sec. 3.7), and answers with the tally and timeline views
(Sec. 3.4, Sec. 3.6).  Served, that is a stream of requests over time:

* ``load``   a trace arrives and is decoded into resident tally rows and a
             resident ordered timeline (admitted against the context's HBM cap);
* ``tally``  the tally rows of a resident trace;
* ``window`` the intervals of a time range [t0, t1) of a resident timeline;
* ``free``   a trace leaves.

``make_schedule`` draws a seeded schedule: Poisson arrivals; each request a
load, a free (the oldest resident trace leaves), or a query on a resident
trace chosen uniformly (a tally, or a window whose width is a log-uniform
fraction of the trace's span, at a uniform start).  Traces are named by
*handles*: the traces resident at the start, then one per load of the
schedule.

``Server`` serves a schedule with the library's serving loop
(thapi_server_*, continuous batching: requests that arrive while others run
start as slots and device memory free up, on their own CUDA streams, so
their work overlaps on the device).  ``serve_serial`` serves the same
schedule one request at a time in arrival order with the plain entry points
on one stream, the per-request baseline.  Both report, per request, the
latency from its scheduled arrival to its result in host memory.
"""
from __future__ import annotations

import ctypes
import math
import random
import time
from dataclasses import dataclass

from . import thapi

KINDS = ("load", "tally", "window", "free")


@dataclass
class Step:
    arrival: float        # seconds from the start of the schedule
    kind: str             # one of KINDS
    handle: int           # the trace: load -> the new handle; others -> an existing handle
    source: int = -1      # load: index of the trace source (pool) it loads
    t0: int = 0
    t1: int = 2**64 - 1


def make_schedule(rate: float, duration: float, resident, spans, seed: int = 0, p_load: float = 0.05,
                  p_free: float = 0.05, p_tally: float = 0.5, frac_range=(1e-4, 1.0), min_resident: int = 1):
    """Seeded schedule of Poisson arrivals (mean `rate` per second) over
    `duration` seconds.  resident: source index of each trace resident at the
    start (handles 0..len-1); spans: (t_min, t_max) per source.  A request is
    a load of a uniformly drawn source (probability p_load), a free of the
    oldest resident handle (p_free; never below min_resident traces), else a
    query on a uniformly drawn resident handle: a tally (p_tally) or a window
    of log-uniform width (fraction of the span in frac_range) at a uniform
    start.  Returns the list of Step."""
    rng = random.Random(seed)
    live = list(range(len(resident)))     # resident handles, oldest first
    src = list(resident)                  # handle -> source
    lo, hi = math.log(frac_range[0]), math.log(frac_range[1])
    out, t = [], 0.0
    while True:
        t += rng.expovariate(rate)
        if t >= duration:
            return out
        u = rng.random()
        if u < p_load:
            s = rng.randrange(len(spans))
            src.append(s)
            live.append(len(src) - 1)
            out.append(Step(t, "load", len(src) - 1, source=s))
            continue
        if u < p_load + p_free and len(live) > min_resident:
            out.append(Step(t, "free", live.pop(0)))
            continue
        if not live:
            continue
        h = live[rng.randrange(len(live))]
        if rng.random() < p_tally:
            out.append(Step(t, "tally", h))
            continue
        a, b = spans[src[h]]
        span = max(b - a, 1)
        w = max(1, int(span * math.exp(rng.uniform(lo, hi))))
        t0 = a + rng.randrange(max(span - w, 0) + 1)
        out.append(Step(t, "window", h, t0=t0, t1=t0 + w))


def percentile(xs, q: float) -> float:
    """Nearest-rank percentile (q in [0, 100]) of a non-empty list."""
    s = sorted(xs)
    k = max(0, min(len(s) - 1, math.ceil(q / 100.0 * len(s)) - 1))
    return s[k]


def to_requests(steps, ids, sources):
    """The schedule as thapi_request records for thapi_server_replay.

    ids: trace id of each handle resident at the start; sources: per source,
    (pointer, nbytes, on_device).  A request on a handle that a load of the
    schedule brings in names that load (`after` = its index + 1)."""
    load_at = {}
    reqs = []
    for i, st in enumerate(steps):
        r = thapi.Request()
        r.kind = KINDS.index(st.kind)
        if st.kind == "load":
            ptr, nbytes, on_dev = sources[st.source]
            r.bytes, r.nbytes, r.on_device = ptr, nbytes, 1 if on_dev else 0
            load_at[st.handle] = i
        elif st.handle in load_at:
            r.after = load_at[st.handle] + 1
        else:
            r.trace = ids[st.handle]
        if st.kind == "window":
            r.t0, r.t1 = st.t0, st.t1
        reqs.append(r)
    return reqs


class Server:
    """The library's serving loop on a context (thapi_server_*).

    Results of queries land in pinned host memory the loop owns (replay
    returns them as soon as each request completes unless `keep`)."""

    def __init__(self, ctx: thapi.Context, load_slots: int = 2, query_slots: int = 6, result_bytes: int = 0):
        self.ctx = ctx
        self.handle = thapi.thapi_server_create(ctx.handle, load_slots, query_slots, result_bytes)

    def replay(self, steps, ids, sources, keep: bool = False):
        """Serves the schedule; returns one thapi.Result per step (times on the
        server's clock, t_arrival the scheduled arrival)."""
        reqs = to_requests(steps, ids, sources)
        return thapi.thapi_server_replay(self.handle, reqs, [s.arrival for s in steps], keep=keep)

    def submit(self, req: thapi.Request) -> int:
        return thapi.thapi_server_submit(self.handle, req)

    def wait(self, ticket: int):
        return thapi.thapi_server_poll(self.handle, ticket)

    def release(self, ticket: int) -> None:
        thapi.thapi_server_release(self.handle, ticket)

    def stats(self) -> dict:
        return thapi.thapi_server_stats_get(self.handle)

    def close(self) -> None:
        if self.handle:
            thapi.thapi_server_destroy(self.handle)
            self.handle = None


@dataclass
class Outcome:
    """One request served by serve_serial (fields as thapi.Result's)."""
    status: int
    kind: int
    trace: int
    n: int
    events: int
    t_arrival: float
    t_admit: float
    t_done: float


def serve_serial(ctx: thapi.Context, steps, ids, sources, rows_out, ivs_out, stream=None,
                 clock=time.perf_counter, sleep=time.sleep, backend=None):
    """The same schedule one request at a time with the plain entry points
    (thapi_trace_load / _load_device, thapi_tally, thapi_timeline,
    thapi_trace_free) on one stream: the serving loop's order with a single
    slot.  Of the requests that have arrived, the first that may start runs
    to completion: loads in arrival order, each once the cap has room (a load
    the cap refuses is tried again after the next free), queries once their
    trace is loaded, a free after the earlier queries of its trace.
    rows_out / ivs_out: reused host result buffers (pinned for speed).
    Returns one Outcome per step, in step order."""
    b = backend or _PlainBackend(ctx, sources, rows_out, ivs_out, stream)
    handle_id = dict(enumerate(ids))   # handle -> trace id, once loaded
    bad = set()                        # handles whose load failed
    out = [None] * len(steps)
    queue = []                         # arrived, not run, in arrival order
    refused_at = {}                    # load step -> frees seen when the cap refused it
    frees = 0
    nxt = 0
    start = clock()

    def may_start(i):
        st = steps[i]
        if st.kind == "load":
            return refused_at.get(i, -1) < frees
        if st.handle in bad:
            return True
        if st.handle not in handle_id:
            return False
        if st.kind == "free":
            return not any(steps[k].handle == st.handle and steps[k].kind in ("tally", "window")
                           for k in queue if k < i)
        return True

    while nxt < len(steps) or queue:
        now = clock() - start
        while nxt < len(steps) and steps[nxt].arrival <= now:
            queue.append(nxt)
            nxt += 1
        pick, load_seen = None, False
        for i in queue:
            if steps[i].kind == "load":
                if load_seen:
                    continue
                load_seen = True
            if may_start(i):
                pick = i
                break
        if pick is None:
            if nxt < len(steps):
                sleep(max(0.0, steps[nxt].arrival - (clock() - start)))
                continue
            break
        queue.remove(pick)
        st = steps[pick]
        t_admit = clock() - start
        if st.kind != "load" and st.handle in bad:
            status, trace, n, events = thapi.E_INVALID, 0, 0, 0
        else:
            status, trace, n, events = b.do(st, handle_id.get(st.handle))
        if st.kind == "load" and status == thapi.E_NOMEM:
            refused_at[pick] = frees
            queue.insert(next((k for k, q in enumerate(queue) if q > pick), len(queue)), pick)
            continue
        if st.kind == "load":
            if status == thapi.OK:
                handle_id[st.handle] = trace
            else:
                bad.add(st.handle)
        if st.kind == "free" and status == thapi.OK:
            frees += 1
        out[pick] = Outcome(status, KINDS.index(st.kind), trace, n, events, st.arrival, t_admit, clock() - start)
    for i in queue:   # never admitted
        out[i] = Outcome(thapi.E_NOMEM, KINDS.index(steps[i].kind), 0, 0, 0, steps[i].arrival, clock() - start,
                         clock() - start)
    return out


class _PlainBackend:
    """One request through the plain entry points."""

    def __init__(self, ctx, sources, rows_out, ivs_out, stream):
        self.ctx, self.sources, self.rows_out, self.ivs_out, self.stream = ctx, sources, rows_out, ivs_out, stream

    def do(self, st, trace):
        h = self.ctx.handle
        try:
            if st.kind == "load":
                ptr, nbytes, on_dev = self.sources[st.source]
                tid = (thapi.thapi_trace_load_device(h, ptr, nbytes, self.stream) if on_dev
                       else thapi.thapi_trace_load(h, (ptr, nbytes), self.stream))
                return thapi.OK, tid, 0, thapi.thapi_trace_info_get(h, tid)["events"]
            if st.kind == "free":
                thapi.thapi_trace_free(h, trace)
                return thapi.OK, trace, 0, 0
            info = thapi.thapi_trace_info_get(h, trace)
            if st.kind == "tally":
                n = ctypes.c_uint64()
                rc = thapi.library().thapi_tally(h, trace, self.rows_out.ctypes.data, len(self.rows_out),
                                                 ctypes.byref(n), None)
                return rc, trace, int(n.value), info["events"]
            n = ctypes.c_uint64()
            rc = thapi.library().thapi_timeline(h, trace, st.t0, st.t1, self.ivs_out.ctypes.data, len(self.ivs_out),
                                                ctypes.byref(n))
            return rc, trace, int(n.value), info["events"]
        except thapi.ThapiError as e:
            return e.code, trace or 0, 0, 0


def summary(outcomes, kinds=KINDS):
    """Latency percentiles (ms) per kind and overall, from Results or Outcomes:
    arrival to result, and its two parts, the wait before the request started
    and its service time."""
    lat = {k: [] for k in kinds}
    failed = 0
    for o in outcomes:
        if o is None or o.status != thapi.OK:
            failed += 1
            continue
        lat[KINDS[o.kind]].append(((o.t_done - o.t_arrival) * 1e3, (o.t_admit - o.t_arrival) * 1e3,
                                   (o.t_done - o.t_admit) * 1e3))
    allq = [x for k in ("tally", "window") for x in lat.get(k, [])]
    out = {"failed": failed}
    for k, xs in list(lat.items()) + [("queries", allq)]:
        if xs:
            tot, wait, svc = ([x[j] for x in xs] for j in range(3))
            out[k] = {"n": len(xs), "p50": percentile(tot, 50), "p99": percentile(tot, 99), "max": max(tot),
                      "wait_p50": percentile(wait, 50), "wait_p99": percentile(wait, 99),
                      "service_p50": percentile(svc, 50), "service_p99": percentile(svc, 99)}
    return out
