"""A one-thread trace consistent with the paper's worked tally (Sec. 4.3).

The paper prints a partial tally of a HIP-over-Level-Zero run (1 host,
1 process, 1 thread): per function Time, Time(%), Calls, Average, Min, Max.
This module builds a trace whose tally, rendered at the paper's precision,
reproduces every printed value:

* per-call durations are chosen so that count, min, max and total fall in
  the rounding interval of each printed number (total is also constrained by
  Average x Calls);
* Time(%) uses one denominator for all rows of both layers, so the builder
  picks one grand total X inside every row's Time(%) interval and adds the
  unprinted remainder (the table is truncated) as a filler function;
* the Level-Zero calls are nested inside the HIP calls that issue them
  (zeEventHostSynchronize spins inside hipDeviceSynchronize, the memory copy
  inside hipMemcpy, module creation inside the first kernel launch), which is
  only consistent with the table if a call's Time includes its children.

Only the input is constructed here; the expected strings are the paper's.
"""
from __future__ import annotations

import os

import numpy as np

from tracegen.handbuilt import TraceBuilder, pack_stream_arrays

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "hiplz_lrn_tally.txt")
UNITS = [("ms", 1e6), ("us", 1e3), ("ns", 1.0), ("s", 1e9)]


def parse_ns(text: str):
    """'4.73s' -> (4.73e9, half of the last printed unit in ns)."""
    for suffix, scale in UNITS:
        if text.endswith(suffix):
            num = text[: -len(suffix)]
            decimals = len(num.split(".")[1]) if "." in num else 0
            return float(num) * scale, 0.5 * scale * 10.0 ** (-decimals)
    raise ValueError(text)


def fmt_ns(v) -> str:
    """The paper's duration format: 2 decimals with s/ms/us, integer or 2-decimal ns."""
    if v >= 1e9:
        return "%.2fs" % (v / 1e9)
    if v >= 1e6:
        return "%.2fms" % (v / 1e6)
    if v >= 1e3:
        return "%.2fus" % (v / 1e3)
    if isinstance(v, (int, np.integer)):
        return "%dns" % v
    return "%.2fns" % v


def fmt_pct(v: float) -> str:
    return "%.2f%%" % v


def load_golden():
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            if not line.strip() or line.startswith("#"):
                continue
            name, time, pct, calls, avg, mn, mx = [c.strip() for c in line.split("|")]
            rows.append(dict(name=name, time=time, pct=pct, calls=int(calls), avg=avg, min=mn, max=mx))
    return rows


def _choose_totals(golden):
    totals = {}
    for r in golden:
        t, th = parse_ns(r["time"])
        a, ah = parse_ns(r["avg"])
        n = r["calls"]
        lo = max(t - th, (a - ah) * n)
        hi = min(t + th, (a + ah) * n)
        assert lo < hi, r["name"]
        totals[r["name"]] = int(round((lo + hi) / 2))
    # one grand total X inside every row's Time(%) interval
    x_lo, x_hi = 0.0, float("inf")
    for r in golden:
        p = float(r["pct"].rstrip("%"))
        T = totals[r["name"]]
        x_lo = max(x_lo, T / ((p + 0.005) / 100.0))
        x_hi = min(x_hi, T / ((p - 0.005) / 100.0))
    assert x_lo < x_hi
    X = int(round((x_lo + x_hi) / 2))
    filler = X - sum(totals.values())
    assert filler > 0
    return totals, filler


def _durations(n, total, mn, mx):
    if n == 1:
        return np.array([total], dtype=np.uint64)
    rest = total - mn - mx
    k = n - 2
    out = np.empty(n, dtype=np.uint64)
    out[0], out[1] = mn, mx
    if k:
        q, r = divmod(rest, k)
        assert mn <= q and q + (1 if r else 0) <= mx
        out[2:] = q
        out[2: 2 + r] += 1
    assert int(out.sum()) == total
    return out


def build():
    """Returns (trace bytes, golden rows, {func_id: name})."""
    golden = load_golden()
    totals, filler = _choose_totals(golden)
    by = {r["name"]: r for r in golden}

    def durs(name):
        r = by[name]
        mn = int(round(parse_ns(r["min"])[0]))
        mx = int(round(parse_ns(r["max"])[0]))
        return _durations(r["calls"], totals[name], mn, mx)

    tb = TraceBuilder(packet_bytes=65536)
    h = tb.add_host("x4204c0s1b0n0")
    names = [r["name"] for r in golden] + ["otherApiCalls"]
    layer = {n: (1 if n.startswith("ze") else 0) for n in names}
    ids = {n: tb.add_call_func(n, layer[n]) for n in names}
    s = tb.add_stream(h, 124765, 124765)

    ts_parts, cls_parts = [], []
    t = 10 ** 18

    def leaf(name, d):
        nonlocal t
        f, e, x = ids[name]
        ts_parts.append(np.array([t, t + int(d)], dtype=np.uint64))
        cls_parts.append(np.array([e, x]))
        t += int(d) + 1000

    def parent_one_child(pname, pd, cname, cd):
        nonlocal t
        _, pe, px = ids[pname]
        _, ce, cx = ids[cname]
        a = (int(pd) - int(cd)) // 2
        ts_parts.append(np.array([t, t + a, t + a + int(cd), t + int(pd)], dtype=np.uint64))
        cls_parts.append(np.array([pe, ce, cx, px]))
        t += int(pd) + 1000

    launch = durs("hipLaunchKernel")
    parent_one_child("hipLaunchKernel", launch[1], "zeModuleCreate", durs("zeModuleCreate")[0])
    for d in np.concatenate([launch[:1], launch[2:]]):
        leaf("hipLaunchKernel", d)
    for pd, cd in zip(durs("hipMemcpy"), np.sort(durs("zeCommandListAppendMemoryCopy"))):
        parent_one_child("hipMemcpy", pd, "zeCommandListAppendMemoryCopy", cd)

    syncs = durs("hipDeviceSynchronize")
    spins = durs("zeEventHostSynchronize")
    _, se, sx = ids["hipDeviceSynchronize"]
    _, ze, zx = ids["zeEventHostSynchronize"]
    leaf("hipDeviceSynchronize", syncs[0])  # the 678 ns sync issues no spin
    csum = np.concatenate([[0], np.cumsum(spins.astype(np.int64))])
    first = 0
    long_syncs = np.concatenate([syncs[1:2], syncs[2:]])
    for k, pd in enumerate(long_syncs):
        pd = int(pd)
        if k == len(long_syncs) - 1:
            last = len(spins)
        else:
            last = int(np.searchsorted(csum, csum[first] + pd, side="right")) - 1
        used = int(csum[last] - csum[first])
        assert used <= pd
        lead = (pd - used) // 2
        starts = np.uint64(t + lead) + (csum[first:last] - csum[first]).astype(np.uint64)
        ends = starts + spins[first:last]
        inner_ts = np.empty(2 * (last - first), dtype=np.uint64)
        inner_ts[0::2], inner_ts[1::2] = starts, ends
        inner_cls = np.empty(2 * (last - first), dtype=np.int64)
        inner_cls[0::2], inner_cls[1::2] = ze, zx
        ts_parts.append(np.concatenate([[np.uint64(t)], inner_ts, [np.uint64(t + pd)]]).astype(np.uint64))
        cls_parts.append(np.concatenate([[se], inner_cls, [sx]]))
        t += pd + 1000
        first = last
    assert first == len(spins)

    leaf("__hipUnregisterFatBinary", durs("__hipUnregisterFatBinary")[0])
    q, r = divmod(filler, 5)
    for i in range(5):
        leaf("otherApiCalls", q + (1 if i < r else 0))

    ts = np.concatenate(ts_parts)
    cls = np.concatenate(cls_parts)
    assert np.all(ts[1:] >= ts[:-1])
    pack_stream_arrays(tb, s, ts, cls, ts_begin=10 ** 18)
    func_names = {ids[n][0]: n for n in names}
    return tb.build(), golden, func_names


def render(rows, func_names):
    """{name: (Time, Time%, Calls, Average, Min, Max)} strings at the paper's precision."""
    grand = float(sum(int(r["total_ns"]) for r in rows))
    out = {}
    for r in rows:
        total = int(r["total_ns"])
        n = int(r["count"])
        out[func_names[int(r["func_id"])]] = (
            fmt_ns(total), fmt_pct(100.0 * total / grand), str(n), fmt_ns(total / n),
            fmt_ns(int(r["min_ns"])), fmt_ns(int(r["max_ns"])))
    return out
