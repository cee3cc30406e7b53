"""The serving loop on the GPU (thapi_server_*): every result of a mix of
overlapping requests equals the oracle's and equals the result of the same
request served alone; admission waits for device memory; a free waits for
the queries of its trace submitted before it; the one-at-a-time baseline
gives the same answers."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import tracegen as tg
from paper_2504_03683_b300 import serve, thapi
from tests._util import intervals_equal, rows_equal

pytestmark = pytest.mark.gpu


def _pool():
    """Traces of different sizes and packet sizes (the large workload's API mix)."""
    specs = [(2_000, 4096, 1), (30_000, 4096, 4), (9_000, 16384, 2), (60_000, 16384, 8), (500, 1024, 1),
             (15_000, 8192, 3)]
    return [tg.generate(tg.preset("large", total_calls=c, n_hosts=1, pids_per_host=1, tids_per_pid=t, seed=70 + k,
                                  packet_bytes=p, p_drop=0.001))[0] for k, (c, p, t) in enumerate(specs)]


def _sources(traces):
    """Each trace in pinned host memory and in device memory: (ptr, nbytes, on_device)."""
    import torch
    keep, host_src, dev_src = [], [], []
    for t in traces:
        h = torch.from_numpy(t).pin_memory()
        d = h.to("cuda")
        keep += [h, d]
        host_src.append((h.data_ptr(), t.nbytes, False))
        dev_src.append((d.data_ptr(), t.nbytes, True))
    torch.cuda.synchronize()
    return keep, host_src, dev_src


def _check_against_oracle(steps, results, src_of, traces, refs):
    for st, res in zip(steps, results):
        assert res.status == thapi.OK, (st, res.status)
        if st.kind == "tally":
            assert rows_equal(thapi.result_rows(res), refs[src_of[st.handle]].rows)
        elif st.kind == "window":
            want = oracle.run(traces[src_of[st.handle]], t0=st.t0, t1=st.t1).intervals
            assert intervals_equal(thapi.result_intervals(res), want)
        elif st.kind == "load":
            assert res.events == refs[st.source % len(traces)].diag["events"]


def test_mix_and_alone_equal_the_oracle():
    import torch
    traces = _pool()
    refs = [oracle.run(t) for t in traces]
    keep, host_src, dev_src = _sources(traces)
    sources = host_src + dev_src  # loads from host memory and from device memory
    spans = [(int(r.intervals["start_ns"].min()), int(r.intervals["end_ns"].max())) for r in refs] * 2
    with thapi.Context(0, 8 * 10**9, use_torch_allocator=False) as ctx:
        srv = serve.Server(ctx, load_slots=2, query_slots=6)
        try:
            ids = [thapi.thapi_trace_load(ctx.handle, traces[k]) for k in (0, 1, 3)]
            resident = [0, 1, 3]
            # ~60 requests within ~25 ms: they arrive while others are on the GPU
            steps = serve.make_schedule(2400.0, 0.025, resident, spans, seed=5, p_load=0.12, p_free=0.06,
                                        min_resident=2)
            assert len(steps) > 40 and {s.kind for s in steps} == set(serve.KINDS)
            src_of = dict(enumerate(resident))
            for s in steps:
                if s.kind == "load":
                    src_of[s.handle] = s.source % len(traces)
            mix = srv.replay(steps, ids, sources, keep=True)
            _check_against_oracle(steps, mix, src_of, traces, refs)
            st = srv.stats()
            assert st["peak_running"] >= 2  # requests were in flight at the same time
            # their device work overlapped: some request started before another finished
            spans_run = sorted((r.t_admit, r.t_done) for r in mix)
            assert any(b[0] < a[1] for a, b in zip(spans_run, spans_run[1:]))
            # each query alone, on a trace loaded alone, equals the oracle too
            for k, s in enumerate(steps):
                if s.kind not in ("tally", "window"):
                    continue
                tid = thapi.thapi_trace_load(ctx.handle, traces[src_of[s.handle]])
                req = thapi.Request()
                req.kind = serve.KINDS.index(s.kind)
                req.trace = tid
                req.t0, req.t1 = s.t0, s.t1
                t = srv.submit(req)
                alone = srv.wait(t)
                assert alone.status == thapi.OK and alone.n == mix[k].n
                if s.kind == "tally":
                    assert rows_equal(thapi.result_rows(alone), thapi.result_rows(mix[k]))
                else:
                    assert intervals_equal(thapi.result_intervals(alone), thapi.result_intervals(mix[k]))
                srv.release(t)
                thapi.thapi_trace_free(ctx.handle, tid)
        finally:
            srv.close()
    torch.cuda.synchronize()
    del keep


def test_results_into_caller_memory():
    """Queries into caller memory: pageable host, pinned host and device buffers,
    and a buffer too small (E_RANGE with the count needed)."""
    import torch
    t = _pool()[1]
    ref = oracle.run(t)
    mid = int(np.median(ref.intervals["start_ns"]))
    want = oracle.run(t, t0=mid, t1=mid + 50_000).intervals
    with thapi.Context(0, 0, use_torch_allocator=False) as ctx:
        tid = thapi.thapi_trace_load(ctx.handle, t)
        srv = serve.Server(ctx, 1, 2)
        try:
            bufs = {"pageable": np.zeros(len(want) + 5, dtype=thapi.INTERVAL_DTYPE),
                    "pinned": torch.empty((len(want) + 5) * 24, dtype=torch.uint8).pin_memory(),
                    "device": torch.empty((len(want) + 5) * 24, dtype=torch.uint8, device="cuda")}
            for name, b in bufs.items():
                req = thapi.Request()
                req.kind, req.trace, req.t0, req.t1 = thapi.REQ_WINDOW, tid, mid, mid + 50_000
                req.out = b.ctypes.data if name == "pageable" else b.data_ptr()
                req.cap = len(want) + 5
                r = srv.wait(srv.submit(req))
                assert r.status == thapi.OK and r.n == len(want), name
                got = b[: r.n] if name == "pageable" else b.cpu().numpy().view(thapi.INTERVAL_DTYPE)[: r.n]
                assert intervals_equal(got, want), name
            small = np.zeros(max(1, len(want) - 1), dtype=thapi.INTERVAL_DTYPE)
            req.out, req.cap = small.ctypes.data, len(small)
            r = srv.wait(srv.submit(req))
            assert r.status == thapi.E_RANGE and r.n == len(want)
            rows = np.zeros(len(ref.rows), dtype=thapi.ROW_DTYPE)
            req = thapi.Request()
            req.kind, req.trace, req.out, req.cap = thapi.REQ_TALLY, tid, rows.ctypes.data, len(rows)
            r = srv.wait(srv.submit(req))
            assert r.status == thapi.OK and rows_equal(rows, ref.rows)
        finally:
            srv.close()


def test_admission_waits_for_memory_and_free_order():
    traces = _pool()
    small, big = traces[4], traces[3]
    keep_big = np.ascontiguousarray(big)
    with thapi.Context(0, 0, use_torch_allocator=False) as probe:
        # what admission charges for the big trace (an idle server's peak commitment
        # after one load) and what its results keep resident
        ps = serve.Server(probe, 1, 1)
        r = thapi.Request()
        r.kind, r.bytes, r.nbytes = thapi.REQ_LOAD, keep_big.ctypes.data, big.nbytes
        res = ps.wait(ps.submit(r))
        charge = ps.stats()["peak_committed"]
        big_resident = thapi.thapi_trace_info_get(probe.handle, res.trace)["device_bytes"]
        ps.close()
    assert 0 < big_resident < charge
    # a cap with room for one load, but not for a second one next to the first's results
    cap = charge + big_resident // 2
    with thapi.Context(0, cap, use_torch_allocator=False) as ctx:
        srv = serve.Server(ctx, 1, 2)
        try:
            def req(kind, **kw):
                r = thapi.Request()
                r.kind = kind
                for k, v in kw.items():
                    setattr(r, k, v)
                return r
            first = srv.submit(req(thapi.REQ_LOAD, bytes=keep_big.ctypes.data, nbytes=big.nbytes))
            r1 = srv.wait(first)
            assert r1.status == thapi.OK
            second = srv.submit(req(thapi.REQ_LOAD, bytes=keep_big.ctypes.data, nbytes=big.nbytes))
            assert thapi.thapi_server_poll(srv.handle, second, 300) is None  # waits: no room
            q_before = srv.submit(req(thapi.REQ_TALLY, trace=r1.trace))
            fr = srv.submit(req(thapi.REQ_FREE, trace=r1.trace))
            q_after = srv.submit(req(thapi.REQ_TALLY, trace=r1.trace))
            assert srv.wait(q_before).status == thapi.OK       # submitted before the free
            assert srv.wait(fr).status == thapi.OK
            assert srv.wait(q_after).status == thapi.E_INVALID  # the trace had left
            r2 = srv.wait(second)                               # admitted once the free made room
            assert r2.status == thapi.OK and r2.t_admit >= srv.wait(fr).t_admit
            assert srv.stats()["load_waits"] >= 1
            # a query naming the waiting load's ticket runs after it
            q_dep = srv.submit(req(thapi.REQ_TALLY, after=second))
            assert srv.wait(q_dep).status == thapi.OK and srv.wait(q_dep).trace == r2.trace
            # a load larger than the whole cap is refused at once
            with thapi.Context(0, 1 << 20, use_torch_allocator=False) as tiny:
                s2 = serve.Server(tiny, 1, 1)
                try:
                    t = s2.submit(req(thapi.REQ_LOAD, bytes=keep_big.ctypes.data, nbytes=big.nbytes))
                    assert s2.wait(t).status == thapi.E_NOMEM
                    sm = np.ascontiguousarray(small)
                    t2 = s2.submit(req(thapi.REQ_LOAD, bytes=sm.ctypes.data, nbytes=small.nbytes))
                    assert s2.wait(t2).status in (thapi.OK, thapi.E_NOMEM)
                finally:
                    s2.close()
        finally:
            srv.close()


def test_serial_baseline_gives_the_same_answers():
    import torch
    traces = _pool()[:4]
    refs = [oracle.run(t) for t in traces]
    keep, host_src, _dev = _sources(traces)
    spans = [(int(r.intervals["start_ns"].min()), int(r.intervals["end_ns"].max())) for r in refs]
    rows_out = np.zeros(4096, dtype=thapi.ROW_DTYPE)
    ivs_out = np.zeros(max(len(r.intervals) for r in refs), dtype=thapi.INTERVAL_DTYPE)
    with thapi.Context(0, 8 * 10**9, use_torch_allocator=False) as ctx:
        ids = [thapi.thapi_trace_load(ctx.handle, traces[k]) for k in (0, 1)]
        steps = serve.make_schedule(1500.0, 0.03, [0, 1], spans, seed=8, p_load=0.1, p_free=0.05)
        out = serve.serve_serial(ctx, steps, ids, host_src, rows_out, ivs_out, torch.cuda.current_stream())
        src_of = {0: 0, 1: 1}
        for s in steps:
            if s.kind == "load":
                src_of[s.handle] = s.source
        for s, o in zip(steps, out):
            assert o is not None and o.status == thapi.OK, (s, o)
            if s.kind == "tally":
                assert o.n == len(refs[src_of[s.handle]].rows)
            elif s.kind == "window":
                assert o.n == len(oracle.run(traces[src_of[s.handle]], t0=s.t0, t1=s.t1).intervals)
    del keep


def test_whole_timeline_windows():
    """A window over the whole time range (t0 = 0, t1 = 2^64 - 1) returns the
    whole ordered timeline into every kind of destination: server-owned
    pinned memory, pageable and pinned host buffers, a device buffer; a
    buffer one interval short is refused with the count needed."""
    import torch
    t = _pool()[1]
    want = oracle.run(t).intervals
    with thapi.Context(0, 0, use_torch_allocator=False) as ctx:
        tid = thapi.thapi_trace_load(ctx.handle, t)
        srv = serve.Server(ctx, 1, 2)
        try:
            def window(out=None, cap=0):
                req = thapi.Request()
                req.kind, req.trace, req.t0, req.t1 = thapi.REQ_WINDOW, tid, 0, 2**64 - 1
                if out is not None:
                    req.out, req.cap = out, cap
                tk = srv.submit(req)
                return tk, srv.wait(tk)
            tk, r = window()
            assert r.status == thapi.OK and intervals_equal(thapi.result_intervals(r), want)
            srv.release(tk)
            n = len(want)
            bufs = {"pageable": np.zeros(n, dtype=thapi.INTERVAL_DTYPE),
                    "pinned": torch.empty(n * 24, dtype=torch.uint8).pin_memory(),
                    "device": torch.empty(n * 24, dtype=torch.uint8, device="cuda")}
            for name, b in bufs.items():
                _tk, r = window(b.ctypes.data if name == "pageable" else b.data_ptr(), n)
                assert r.status == thapi.OK and r.n == n, name
                got = b if name == "pageable" else b.cpu().numpy().view(thapi.INTERVAL_DTYPE)
                assert intervals_equal(got, want), name
            short = np.zeros(n - 1, dtype=thapi.INTERVAL_DTYPE)
            _tk, r = window(short.ctypes.data, n - 1)
            assert r.status == thapi.E_RANGE and r.n == n
        finally:
            srv.close()
