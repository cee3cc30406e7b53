"""CUDA path vs the CPU oracle, element by element (tolerance 0: integer ns).

Every case loads a trace through the C ABI (libthapi.so via the ctypes
binding), reads back the tally rows, diagnostics and timeline, and compares
them with the oracle on the same bytes.
"""
from __future__ import annotations

import random

import numpy as np
import pytest

import oracle
import tracegen as tg
from paper_2504_03683_b300 import thapi
from tests import _malformed
from tests._util import intervals_equal, rows_equal
from tracegen.handbuilt import DEV_BEGIN, ENTRY, EXIT, SAMPLE, Ev, TraceBuilder

pytestmark = pytest.mark.gpu
U64MAX = 2**64 - 1


@pytest.fixture(scope="module")
def ctx():
    import torch

    assert torch.cuda.is_available()
    c = thapi.Context(0)
    yield c
    c.close()


def gpu_run(ctx, trace, windows=(), device=False):
    tid = ctx.load(trace)
    try:
        rows, diag = ctx.tally(tid)
        ivs = ctx.timeline(tid)
        win = [ctx.timeline(tid, t0, t1) for (t0, t1) in windows]
        info = ctx.info(tid)
        dev = ctx.device_tally(tid)
    finally:
        ctx.free(tid)
    if device:
        return rows, diag, ivs, win, info, dev
    return rows, diag, ivs, win, info


def assert_parity(ctx, trace, windows=()):
    o = oracle.run(trace)
    assert o.code == oracle.OK
    rows, diag, ivs, win, info, (dev_rows, dev_diag) = gpu_run(ctx, trace, windows, device=True)
    for k in oracle.DIAG_FIELDS:
        assert diag[k] == o.diag[k], (k, diag[k], o.diag[k])
    assert rows_equal(rows, o.rows)
    assert intervals_equal(ivs, o.intervals)
    for (t0, t1), w in zip(windows, win):
        ow = oracle.run(trace, t0=t0, t1=t1)
        assert intervals_equal(w, ow.intervals), (t0, t1)
    assert info["intervals"] == len(o.intervals) and info["tally_rows"] == len(o.rows)
    # device-activity pairing
    assert dev_diag == o.dev_diag, (dev_diag, o.dev_diag)
    assert rows_equal(dev_rows, o.dev_rows)
    assert info["device_rows"] == len(o.dev_rows) and info["device_intervals"] == o.dev_diag["dev_intervals"]
    return o


def _windows(o, k=4, seed=0):
    if not len(o.intervals):
        return [(0, U64MAX), (5, 6)]
    rng = random.Random(seed)
    s = o.intervals["start_ns"]
    e = o.intervals["end_ns"]
    lo, hi = int(s.min()), int(e.max())
    out = [(0, U64MAX), (lo, lo + 1), (hi, hi + 1), (int(s[len(s) // 2]), int(e[len(e) // 2]))]
    for _ in range(k):
        a = rng.randrange(lo, hi + 1)
        out.append((a, a + rng.randrange(1, max(2, (hi - lo) // 50))))
    return out


# ------------------------------------------------------------- workloads
def test_tiny_workload(ctx):
    b, _c, _e = tg.generate(tg.preset("tiny"))
    o = oracle.run(b)
    assert_parity(ctx, b, _windows(o))


@pytest.mark.parametrize("over", [
    dict(total_calls=200_000, n_hosts=2, pids_per_host=2, tids_per_pid=4),
    dict(total_calls=100_000, n_hosts=1, pids_per_host=2, tids_per_pid=3, p_drop=0.002, p_sample=0.05,
         p_long_gap=0.01, p_ext=0.02, packet_bytes=1024, seed=5),
    dict(total_calls=30_000, n_hosts=1, pids_per_host=1, tids_per_pid=3, packet_bytes=256, seed=6, p_drop=0.01),
    dict(total_calls=60_000, n_hosts=1, pids_per_host=2, tids_per_pid=2, packet_bytes=32768, seed=7, p_drop=0.001),
    dict(total_calls=80_000, n_hosts=1, pids_per_host=1, tids_per_pid=2, packet_bytes=65536, seed=8, p_err=0.2),
])
def test_layered_workloads(ctx, over):
    b, _c, _e = tg.generate(tg.preset("large", **over))
    o = oracle.run(b)
    assert_parity(ctx, b, _windows(o, seed=over.get("seed", 1)))


def test_device_workload_counts_other_events(ctx):
    b, _c, _e = tg.generate(tg.preset("device", total_calls=20_000, n_hosts=1, pids_per_host=2, tids_per_pid=2,
                                      n_device_streams=3))
    o = assert_parity(ctx, b)
    assert o.diag["other_events"] > 0


# ------------------------------------------------ device-activity pairing
@pytest.mark.parametrize("packet_bytes", [256, 4096, 65536])
def test_device_pairing_handbuilt_cases(ctx, packet_bytes):
    from tests import _device_trace as dt
    b, ids = dt.build(packet_bytes=packet_bytes)
    o = assert_parity(ctx, b, [(0, U64MAX), (dt.T0 + 150, dt.T0 + 131), (dt.T0 + 138, dt.T0 + 139)])
    assert o.dev_diag == dt.EXPECTED_DEV_DIAG


@pytest.mark.parametrize("over", [
    # device streams with ~1000 events per 16 KB packet (warp kernel), drops, EXT timestamps
    dict(total_calls=120_000, n_hosts=1, pids_per_host=4, tids_per_pid=4, n_device_streams=8, seed=3),
    dict(total_calls=80_000, n_hosts=2, pids_per_host=2, tids_per_pid=2, n_device_streams=5, packet_bytes=1024,
         p_drop=0.01, p_ext=0.01, seed=4),
    # 32 KB packets: device packets hold ~2000 events, past the warp kernel's limit (the CTA kernel takes them)
    dict(total_calls=60_000, n_hosts=1, pids_per_host=2, tids_per_pid=2, n_device_streams=3, packet_bytes=32768,
         p_drop=0.002, seed=5),
    # 64 KB packets: every packet goes to the CTA kernel
    dict(total_calls=60_000, n_hosts=1, pids_per_host=2, tids_per_pid=2, n_device_streams=4, packet_bytes=65536,
         seed=6),
])
def test_device_workloads(ctx, over):
    b, calls, _e = tg.generate(tg.preset("device", **over), truth=True)
    o = oracle.run(b)
    assert_parity(ctx, b, _windows(o, seed=over["seed"]))
    assert o.dev_diag["dev_intervals"] > 0


def test_device_table_rebuilt_when_ids_do_not_repeat(ctx):
    """Every record has its own id (no begin, end or host record shares one), so the
    first command table (room for twice the largest record kind) overflows and the
    join rebuilds it for every record."""
    tb = TraceBuilder(packet_bytes=4096)
    h = tb.add_host("h")
    f = tb.add_func("launch")
    fd = tb.add_func("dev", 3)
    en = tb.add_class(f, ENTRY, 16, cmd_off=8)
    ex = tb.add_class(f, EXIT, 4, result_off=0)
    cb = tb.add_class(fd, DEV_BEGIN, 8, cmd_off=0)
    from tracegen.handbuilt import DEV_END
    ce = tb.add_class(fd, DEV_END, 8, cmd_off=0)
    sh, sd = tb.add_stream(h, 1, 1), tb.add_stream(h, 2, 2, 1)
    n = 3000
    host, dev = [], []
    for i in range(n):
        host += [Ev(en, 10_000 + 10 * i, cmd=3 * i + 1), Ev(ex, 10_000 + 10 * i + 5, result=0)]
        dev += [Ev(cb, 10_000 + 10 * i, cmd=3 * i + 2), Ev(ce, 10_000 + 10 * i + 3, cmd=3 * i + 3)]
    tb.place(tb.stream_events(sh, host, ts_begin=10_000))
    tb.place(tb.stream_events(sd, dev, ts_begin=10_000))
    o = assert_parity(ctx, tb.build())
    assert o.dev_diag["dev_unpaired"] == 2 * n and o.dev_diag["host_unjoined"] == n


def test_ground_truth_through_gpu(ctx):
    from tests._util import expected_from_truth
    b, calls, _e = tg.generate(tg.preset("large", total_calls=50_000, n_hosts=1, pids_per_host=2, tids_per_pid=2,
                                         seed=9), truth=True)
    rows, diag, ivs, _w, _i = gpu_run(ctx, b)
    er, ei = expected_from_truth(b, calls)
    assert rows_equal(rows, er) and intervals_equal(ivs, ei)


# ------------------------------------------------------------ edge cases
def _builder(P=256, n_funcs=3):
    tb = TraceBuilder(packet_bytes=P)
    h = tb.add_host("node")
    ids = [tb.add_call_func("fn%d" % i) for i in range(n_funcs)]
    return tb, h, ids


def test_empty_trace(ctx):
    tb, h, ids = _builder()
    tb.add_stream(h, 1, 1)
    assert_parity(ctx, tb.build())


def test_no_streams_no_packets(ctx):
    tb = TraceBuilder(packet_bytes=256)
    tb.add_host("h")
    tb.add_call_func("f")
    assert_parity(ctx, tb.build())


def test_packets_without_events(ctx):
    tb, h, ids = _builder()
    s = tb.add_stream(h, 1, 1)
    tb.raw_packet(s, 100, [], discarded=4)
    tb.raw_packet(s, 100, [tb.encode_event(ids[0][1], 5), tb.encode_event(ids[0][2], 5)])
    tb.raw_packet(s, 100, [], discarded=1)
    assert_parity(ctx, tb.build())


def test_dense_packets_take_second_pass(ctx):
    # minimum-size events (8-byte entries, 12-byte exits) fill 16 KB packets past the fast-path capacity
    tb, h, ids = _builder(P=16384)
    s0 = tb.add_stream(h, 7, 7)
    s1 = tb.add_stream(h, 7, 8)
    for s in (s0, s1):
        evs = []
        t = 1000
        for k in range(5000):
            evs.append(Ev(ids[k % 3][1], t))
            evs.append(Ev(ids[k % 3][2], t + 3 + k % 5, result=k % 7 == 0))
            t += 10
        tb.place(tb.stream_events(s, evs, ts_begin=1000))
    b = tb.build()
    o = assert_parity(ctx, b)
    assert o.diag["packets"] >= 2


def test_deep_nesting_across_packets_saturates_level(ctx):
    tb, h, ids = _builder(P=256)
    s = tb.add_stream(h, 3, 3)
    depth = 300
    evs = [Ev(ids[d % 3][1], 100 + d) for d in range(depth)]
    evs += [Ev(ids[d % 3][2], 100000 - d, result=d % 11 == 0) for d in reversed(range(depth))]
    evs += [Ev(ids[0][2], 200000)]  # one unmatched exit at the end
    evs += [Ev(ids[1][1], 200001)]  # one unmatched entry
    tb.place(tb.stream_events(s, evs, ts_begin=100))
    o = assert_parity(ctx, tb.build())
    assert o.intervals["level"].max() == 255


def test_other_kinds_and_ext(ctx):
    tb, h, ids = _builder(P=256)
    fs = tb.add_func("sample")
    cs = tb.add_class(fs, SAMPLE, 8)
    cb = tb.add_class(fs, DEV_BEGIN, 8, cmd_off=0)
    s = tb.add_stream(h, 1, 1)
    evs = [Ev(ids[0][1], 10), Ev(cs, 12), Ev(cb, 13, cmd=99), Ev(ids[0][2], 20, result=3),
           Ev(ids[1][1], 20 + (1 << 27)), Ev(ids[1][2], 21 + (1 << 27), force_ext=True),
           Ev(ids[2][1], 5), Ev(ids[2][2], 7)]  # timestamps going backwards use EXT
    tb.place(tb.stream_events(s, evs, ts_begin=5))
    assert_parity(ctx, tb.build())


def test_equal_start_ties_across_streams(ctx):
    tb, h, ids = _builder(P=256)
    streams = [tb.add_stream(h, 9, 9 + k) for k in range(5)]
    for k, s in reversed(list(enumerate(streams))):  # file order differs from stream order
        evs = [Ev(ids[0][1], 500), Ev(ids[1][1], 500), Ev(ids[1][2], 500), Ev(ids[0][2], 501 + k)]
        tb.place(tb.stream_events(s, evs, ts_begin=500))
    assert_parity(ctx, tb.build())


def test_crowded_start_bucket_takes_radix_sort(ctx):
    # 5000 zero-length calls starting at one instant fill one start bucket past
    # its shared-memory capacity: the timeline is ordered by the radix sort.
    tb, h, ids = _builder(P=4096)
    s0, s1 = tb.add_stream(h, 1, 1), tb.add_stream(h, 1, 2)
    evs = []
    for _ in range(5000):
        evs += [Ev(ids[0][1], 1000), Ev(ids[0][2], 1000)]
    tb.place(tb.stream_events(s0, evs, ts_begin=1000))
    tb.place(tb.stream_events(s1, [Ev(ids[1][1], 999), Ev(ids[1][2], 1000 + 10**6)], ts_begin=999))
    o = assert_parity(ctx, tb.build())
    assert len(o.intervals) == 5001


def test_spread_starts_many_buckets(ctx):
    # starts spread over a wide span with jitter and ties across streams: the
    # bucketed order must equal the oracle's (start, stream, position) order
    rng = random.Random(5)
    tb, h, ids = _builder(P=1024)
    streams = [tb.add_stream(h, 2, 10 + k) for k in range(24)]
    for s in streams:
        t, evs = 1 << 20, []
        for _ in range(900):
            t += rng.choice([0, 0, 1, 7, 300, 5000])
            f = rng.randrange(3)
            d = rng.choice([0, 1, 3, 40])
            evs += [Ev(ids[f][1], t), Ev(ids[f][2], t + d)]
            t += d
        tb.place(tb.stream_events(s, evs, ts_begin=1 << 20))
    o = assert_parity(ctx, tb.build())
    assert len(o.intervals) == 24 * 900


def test_crowded_bin_inside_a_bucket(ctx):
    # a burst of 700 calls at one instant among spread starts: the burst's
    # bucket fits in shared memory but one bin of its starts' top bits is
    # crowded, so that bucket is sorted by radix passes and the others by bin
    # insertion; the order must still be (start, stream, position)
    rng = random.Random(11)
    tb, h, ids = _builder(P=1024)
    streams = [tb.add_stream(h, 3, 20 + k) for k in range(12)]
    for k, s in enumerate(streams):
        t, evs = 1 << 22, []
        for j in range(1500):
            if k == 3 and j == 600:
                evs += [Ev(ids[0][1], t), Ev(ids[0][2], t)] * 700
            t += rng.choice([1, 13, 250, 4000])
            f = rng.randrange(3)
            d = rng.choice([0, 2, 90])
            evs += [Ev(ids[f][1], t), Ev(ids[f][2], t + d)]
            t += d
        tb.place(tb.stream_events(s, evs, ts_begin=1 << 22))
    o = assert_parity(ctx, tb.build())
    assert len(o.intervals) == 12 * 1500 + 700


def test_wide_span_buckets_take_64_bit_items(ctx):
    # starts spread over about 2^38 ns: a bucket's key needs more than 20 bits,
    # so the bucket sort's items are 64-bit.  One stream spreads its calls
    # (bins of the top key bits hold a few items: insertion path), another
    # bursts at the start (one crowded bin: radix passes over all key bits).
    rng = random.Random(3)
    tb, h, ids = _builder(P=1024)
    s0, s1 = tb.add_stream(h, 4, 1), tb.add_stream(h, 4, 2)
    evs, t = [], 1000
    for _ in range(3000):
        t += rng.randrange(1, 1 << 28)
        d = rng.randrange(0, 100)
        evs += [Ev(ids[0][1], t), Ev(ids[0][2], t + d)]
        t += d
    tb.place(tb.stream_events(s0, evs, ts_begin=1000))
    evs, t = [], 5000
    for _ in range(1500):
        t += rng.choice([0, 1, 2])
        evs += [Ev(ids[1][1], t), Ev(ids[1][2], t + 1)]
        t += 1
    tb.place(tb.stream_events(s1, evs, ts_begin=5000))
    o = assert_parity(ctx, tb.build())
    assert len(o.intervals) == 4500


def test_brute_force_sequences_in_one_trace(ctx):
    rng = random.Random(77)
    tb, h, ids = _builder(P=256, n_funcs=2)
    packed = []
    for k in range(300):
        s = tb.add_stream(h, 100 + k // 7, 1000 + k)
        n = rng.choice([1, 2, 5, 10, 17, 40, 90])
        evs, t = [], 1000 + k
        for j in range(n):
            t += rng.choice([0, 1, 5, 30])
            kind = rng.choice([ENTRY, ENTRY, EXIT, EXIT, EXIT])
            f = rng.randrange(2)
            evs.append(Ev(ids[f][1] if kind == ENTRY else ids[f][2], t, payload=b"\x07" * rng.choice([0, 4, 40]),
                          result=rng.choice([0, 0, 1]) if kind == EXIT else None))
        packed.append(tb.stream_events(s, evs, ts_begin=1000))
    # interleave packets of all streams, each stream's in order
    queues = [list(p) for p in packed]
    while any(queues):
        q = rng.choice([q for q in queues if q])
        tb.place([q.pop(0)])
    assert_parity(ctx, tb.build())


def test_payloads_that_look_like_headers(ctx):
    # payload words that parse as valid events make speculative walks go astray
    tb, h, ids = _builder(P=1024)
    import struct
    s = tb.add_stream(h, 1, 1)
    evs, t = [], 100
    for k in range(400):
        fake = struct.pack("<IHH", k % 9, ids[k % 3][1], 4 * (k % 5)) * (1 + k % 6)
        evs.append(Ev(ids[k % 3][1], t, payload=fake[: 4 * (k % 12)]))
        evs.append(Ev(ids[k % 3][2], t + 5, payload=fake[: 4 * (k % 7)]))
        t += 9
    tb.place(tb.stream_events(s, evs, ts_begin=100))
    assert_parity(ctx, tb.build())


# ---------------------------------------------------------------- errors
@pytest.mark.parametrize("name,trace", _malformed.cases(), ids=[c[0] for c in _malformed.cases()])
def test_errors_match_oracle(ctx, name, trace):
    o = oracle.run(trace)
    if o.code == oracle.OK:
        assert_parity(ctx, trace)
        return
    with pytest.raises(thapi.ThapiError) as ei:
        ctx.load(trace)
    assert ei.value.code == o.code, name
    if o.loc[0] > 0:
        assert ei.value.location == o.loc, name


# ------------------------------------------------------------ the paper
def test_paper_table_trace(ctx):
    from tests import _paper_trace as pt
    trace, golden, names = pt.build()
    o = oracle.run(trace, want_intervals=True)
    rows, diag, ivs, _w, _i = gpu_run(ctx, trace)
    assert rows_equal(rows, o.rows)
    assert intervals_equal(ivs, o.intervals)
    got = pt.render(rows, names)
    for g in golden:
        assert got[g["name"]] == (g["time"], g["pct"], str(g["calls"]), g["avg"], g["min"], g["max"])


# ---------------------------------------------------------- API surface
def test_device_load_and_device_outputs(ctx):
    import torch
    b, _c, _e = tg.generate(tg.preset("large", total_calls=40_000, n_hosts=1, pids_per_host=2, tids_per_pid=2,
                                      seed=12))
    o = oracle.run(b)
    stream = torch.cuda.Stream()
    dev = torch.from_numpy(b).to("cuda")
    tid = thapi.thapi_trace_load_device(ctx.handle, dev.data_ptr(), dev.numel(), stream)
    try:
        info = ctx.info(tid)
        rows_d = torch.empty(info["tally_rows"] * 56, dtype=torch.uint8, device="cuda")
        ivs_d = torch.empty(info["intervals"] * 24, dtype=torch.uint8, device="cuda")
        n, diag = thapi.thapi_tally_device(ctx.handle, tid, rows_d.data_ptr(), info["tally_rows"], stream)
        m = thapi.thapi_timeline_device(ctx.handle, tid, 0, U64MAX, ivs_d.data_ptr(), info["intervals"], stream)
        stream.synchronize()
        rows = rows_d.cpu().numpy().view(thapi.ROW_DTYPE)
        ivs = ivs_d.cpu().numpy().view(thapi.INTERVAL_DTYPE)
        assert n == len(o.rows) and m == len(o.intervals)
        assert rows_equal(rows, o.rows) and intervals_equal(ivs, o.intervals)
        # a window into device memory
        t0 = int(o.intervals["start_ns"][len(o.intervals) // 3])
        t1 = t0 + 500_000
        ow = oracle.run(b, t0=t0, t1=t1).intervals
        wd = torch.empty(max(1, len(ow)) * 24, dtype=torch.uint8, device="cuda")
        k = thapi.thapi_timeline_device(ctx.handle, tid, t0, t1, wd.data_ptr(), len(ow), stream)
        stream.synchronize()
        assert k == len(ow)
        assert intervals_equal(wd.cpu().numpy().view(thapi.INTERVAL_DTYPE)[:k], ow)
    finally:
        ctx.free(tid)


def test_capacity_and_names(ctx):
    b, _c, _e = tg.generate(tg.preset("tiny", total_calls=3000))
    tid = ctx.load(b)
    try:
        info = ctx.info(tid)
        with pytest.raises(thapi.ThapiError) as ei:
            buf = np.zeros(1, dtype=thapi.INTERVAL_DTYPE)
            thapi.thapi_timeline(ctx.handle, tid, out=buf)
        assert ei.value.code == thapi.E_RANGE
        assert thapi.thapi_trace_strings(ctx.handle, tid, 1, 0) == "apiFunc0"
        assert thapi.thapi_trace_strings(ctx.handle, tid, 0, 0).startswith("x4204")
        assert info["events"] == 6000
    finally:
        ctx.free(tid)
    with pytest.raises(thapi.ThapiError) as ei:
        ctx.tally(tid)
    assert ei.value.code == thapi.E_INVALID


def test_default_allocator_and_timing():
    b, _c, _e = tg.generate(tg.preset("tiny", total_calls=20_000))
    o = oracle.run(b)
    with thapi.Context(0, use_torch_allocator=False) as c:
        thapi.thapi_ctx_set_timing(c.handle, True)
        before = thapi.thapi_kernel_launches()
        tid = c.load(b)
        rows, diag = c.tally(tid)
        t = thapi.thapi_trace_timing(c.handle, tid)
        assert rows_equal(rows, o.rows)
        assert t["analyze_ms"] > 0 and t["launches"] > 5 and t["analyze_launches"] == 1
        assert thapi.thapi_kernel_launches() - before == t["launches"]
        assert t["analyze_read_bytes"] > 0


def test_hbm_cap_admission():
    b, _c, _e = tg.generate(tg.preset("tiny", total_calls=20_000))
    with thapi.Context(0, hbm_cap_bytes=1 << 16) as c:
        with pytest.raises(thapi.ThapiError) as ei:
            c.load(b)
        assert ei.value.code == thapi.E_NOMEM


def test_device_join_global_table_for_a_heavy_id(ctx):
    """6200 host calls share one command id, so that id's partition holds more
    records than a shared-memory partition table takes (3072) and the join uses
    one global table instead.  8192 begins and 8192 ends with ids of their own,
    and 100 more host ids, overflow that table's first size (twice the largest
    record kind, 16384 entries, for 16485 ids), so it is rebuilt for every record."""
    from tracegen.handbuilt import DEV_END
    tb = TraceBuilder(packet_bytes=4096)
    h = tb.add_host("h")
    f = tb.add_func("launch")
    fd = tb.add_func("dev", 3)
    en = tb.add_class(f, ENTRY, 16, cmd_off=8)
    ex = tb.add_class(f, EXIT, 4, result_off=0)
    cb = tb.add_class(fd, DEV_BEGIN, 8, cmd_off=0)
    ce = tb.add_class(fd, DEV_END, 8, cmd_off=0)
    sh, sd = tb.add_stream(h, 1, 1), tb.add_stream(h, 2, 2, 1)
    host, dev = [], []
    t = 10_000
    for i in range(6200):
        host += [Ev(en, t, cmd=0xABCDEF), Ev(ex, t + 5, result=0)]
        t += 10
    for i in range(100):
        host += [Ev(en, t, cmd=(1 << 40) + i), Ev(ex, t + 5, result=0)]
        t += 10
    t = 10_000
    for i in range(8192):
        dev += [Ev(cb, t, cmd=(2 << 40) + i), Ev(ce, t + 3, cmd=(3 << 40) + i)]
        t += 10
    tb.place(tb.stream_events(sh, host, ts_begin=10_000))
    tb.place(tb.stream_events(sd, dev, ts_begin=10_000))
    o = assert_parity(ctx, tb.build())
    assert o.dev_diag["dev_unpaired"] == 2 * 8192 and o.dev_diag["host_unjoined"] == 6300


def test_bounded_device_wait_runs_out_and_the_context_stays_usable(ctx):
    """An mbarrier wait that nothing completes gives up after its limit and
    reports THAPI_E_TIMEOUT through a status word; then a load on the same
    context still matches the oracle."""
    from paper_2504_03683_b300 import thapi
    assert thapi.thapi_check_device_wait(ctx.handle, 256) == thapi.E_TIMEOUT
    assert thapi.thapi_check_device_wait(ctx.handle, 0) == thapi.E_INVALID
    tb, h, ids = _builder()
    s = tb.add_stream(h, 1, 1)
    tb.place(tb.stream_events(s, [Ev(ids[0][1], 10), Ev(ids[0][2], 20, result=0)], ts_begin=10))
    assert_parity(ctx, tb.build())


def test_autotune_keeps_results_and_remembers_the_configuration():
    """With the autotuner on, the first load of a shape tries every candidate
    configuration and keeps the fastest; results equal the oracle's, and a
    later load of the same shape uses the same configuration."""
    from paper_2504_03683_b300 import thapi
    b, _c, _e = tg.generate(tg.preset("device", total_calls=30_000, n_hosts=1, pids_per_host=2, tids_per_pid=2,
                                      n_device_streams=3, seed=41))
    o = oracle.run(b)
    with thapi.Context(0) as c:
        thapi.thapi_ctx_set_autotune(c.handle, True)
        thapi.thapi_ctx_set_timing(c.handle, True)
        seen = []
        for _ in range(2):
            tid = c.load(b)
            try:
                rows, diag = c.tally(tid)
                drows, ddiag = c.device_tally(tid)
                ivs = c.timeline(tid)
                t = thapi.thapi_trace_timing(c.handle, tid)
            finally:
                c.free(tid)
            assert rows_equal(rows, o.rows) and rows_equal(drows, o.dev_rows) and intervals_equal(ivs, o.intervals)
            assert diag == o.diag and ddiag == o.dev_diag
            assert t["grid_mult"] in (1, 2, 4) and t["part_shift"] in (-1, 0, 1)
            seen.append((t["grid_mult"], t["part_shift"]))
        assert seen[0] == seen[1]
