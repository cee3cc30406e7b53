"""Text rendering of tally rows, in the layout of the paper's summary table
(arxiv 2504.03683, Sec. 4.3: Name | Time | Time(%) | Calls | Average | Min |
Max, rows by Time descending, durations with s / ms / us / ns units and two
decimals).

Rendering is display only: Time(%) and Average are floating-point views of the
exact integer rows (total_ns / sum of all rows' totals, total_ns / count),
outside the bit-exact contract of the tally itself.  Names come from the
trace's string table (thapi_trace_strings).
"""
from __future__ import annotations

from collections import OrderedDict

import numpy as np


def fmt_ns(v) -> str:
    """A duration in the paper's format: two decimals in s, ms or us; ns as an integer when exact."""
    if v >= 1e9:
        return "%.2fs" % (v / 1e9)
    if v >= 1e6:
        return "%.2fms" % (v / 1e6)
    if v >= 1e3:
        return "%.2fus" % (v / 1e3)
    if isinstance(v, (int, np.integer)) or float(v).is_integer():
        return "%dns" % int(v)
    return "%.2fns" % v


def fmt_pct(v: float) -> str:
    return "%.2f%%" % v


def summarize(rows, func_names, by_group: bool = False):
    """Rows combined per function (or per (host_id, pid, tid, function) with by_group),
    as dicts of exact integers, ordered by total time descending then name."""
    acc = OrderedDict()
    for r in np.asarray(rows).tolist():
        host, pid, tid, func, count, total, mn, mx, err = r
        key = (host, pid, tid, func) if by_group else (func,)
        a = acc.get(key)
        if a is None:
            acc[key] = [count, total, mn, mx, err]
        else:
            a[0] += count
            a[1] = (a[1] + total) & ((1 << 64) - 1)
            a[2] = min(a[2], mn)
            a[3] = max(a[3], mx)
            a[4] += err
    out = []
    for key, (count, total, mn, mx, err) in acc.items():
        out.append(dict(key=key, name=func_names[key[-1]], count=count, total=total, min=mn, max=mx, err=err))
    out.sort(key=lambda d: (-d["total"], d["name"]))
    return out


def tally_table(rows, func_names, title: str | None = None, by_group: bool = False, host_names=None) -> str:
    """The summary table as text; Time(%) of each row against the sum over all rows shown."""
    items = summarize(rows, func_names, by_group)
    grand = float(sum(d["total"] for d in items)) or 1.0
    header = ["Name", "Time", "Time(%)", "Calls", "Average", "Min", "Max"]
    if by_group:
        header = ["Hostname", "Process", "Thread"] + header
    body = []
    for d in items:
        cells = [d["name"], fmt_ns(d["total"]), fmt_pct(100.0 * d["total"] / grand), str(d["count"]),
                 fmt_ns(d["total"] / d["count"]) if d["count"] else "-", fmt_ns(d["min"]), fmt_ns(d["max"])]
        if by_group:
            host, pid, tid = d["key"][:3]
            hname = host_names[host] if host_names is not None else str(host)
            cells = [hname, str(pid), str(tid)] + cells
        body.append(cells)
    widths = [max(len(header[i]), *(len(b[i]) for b in body)) if body else len(header[i]) for i in range(len(header))]
    lines = []
    if title:
        lines.append(title)
    lines.append(" | ".join(h.rjust(w) for h, w in zip(header, widths)) + " |")
    lines.append("-|-".join("-" * w for w in widths) + "-|")
    for b in body:
        lines.append(" | ".join(c.rjust(w) for c, w in zip(b, widths)) + " |")
    return "\n".join(lines) + "\n"


def trace_names(ctx, trace_id: int):
    """(function names, host names) of a loaded trace, from its string table."""
    from .thapi import thapi_trace_info_get, thapi_trace_strings
    h = ctx.handle if hasattr(ctx, "handle") else ctx
    info = thapi_trace_info_get(h, trace_id)
    funcs = [thapi_trace_strings(h, trace_id, 1, i) for i in range(info["n_funcs"])]
    hosts = [thapi_trace_strings(h, trace_id, 0, i) for i in range(info["n_hosts"])]
    return funcs, hosts


_KIND = {0: "entry", 1: "exit", 2: "device_begin", 3: "device_end", 4: "sample"}


def event_lines(events, func_names, host_names, stream_table, limit: int | None = None):
    """Decoded events (thapi_decode records) as text, one line per event, in the
    spirit of the paper's pretty-printed trace (Sec. 3.2: timestamp, hostname,
    process and thread, event name, then its fields).  The payload bytes are
    opaque in this layout, so the fields shown are the ones every class has:
    result, command id and payload size.  stream_table: (n_streams, 4) rows of
    host_id, pid, tid, flags; the thread is the record's vpid / vtid when it has
    them (per-CPU buffers), else its stream's pid / tid."""
    out = []
    ev = np.asarray(events)
    n = len(ev) if limit is None else min(limit, len(ev))
    has_ctx = ev.dtype.names is not None and "vtid" in ev.dtype.names
    for i in range(n):
        r = ev[i]
        sid = int(r["stream_id"])
        host, pid, tid = (int(v) for v in stream_table[sid][:3])
        if has_ctx:
            pid, tid = int(r["vpid"]), int(r["vtid"])
        kind, cmd = int(r["kind"]), int(r["cmd"])
        fields = []
        if kind == 1:
            fields.append("result: %d" % int(r["result"]))
        if cmd:
            fields.append("cmd: 0x%016x" % cmd)
        fields.append("payload_bytes: %d" % int(r["var_len"]))
        out.append("%d %s vpid: %d, vtid: %d - %s_%s: { %s }" % (
            int(r["ts"]), host_names[host], pid, tid, func_names[int(r["func_id"])], _KIND.get(kind, "event"),
            ", ".join(fields)))
    return out


def func_layers(ctx, trace_id: int):
    """Layer of every function of a loaded trace (thapi_trace_func_layer)."""
    from .thapi import thapi_trace_func_layer, thapi_trace_info_get
    h = ctx.handle if hasattr(ctx, "handle") else ctx
    n = thapi_trace_info_get(h, trace_id)["n_funcs"]
    return [thapi_trace_func_layer(h, trace_id, i) for i in range(n)]


def _table(header, body, title):
    widths = [max(len(header[i]), *(len(b[i]) for b in body)) if body else len(header[i]) for i in range(len(header))]
    lines = [title] if title else []
    lines.append(" | ".join(h.rjust(w) for h, w in zip(header, widths)) + " |")
    lines.append("-|-".join("-" * w for w in widths) + "-|")
    for b in body:
        lines.append(" | ".join(c.rjust(w) for c, w in zip(b, widths)) + " |")
    return "\n".join(lines) + "\n"


def self_table(rows, self_rows, func_names, func_layers=None, title: str | None = None) -> str:
    """Inclusive and self time side by side, per function, ordered by self time
    descending (the layering view of Sec. 4.3: how much of hipDeviceSynchronize
    is its own time and how much the zeEventHostSynchronize calls inside it
    take).  Self(%) = self / inclusive time of the same function; Average is
    the mean self time per call."""
    incl = {d["key"]: d for d in summarize(rows, func_names)}
    items = summarize(self_rows, func_names)
    items.sort(key=lambda d: (-d["total"], d["name"]))
    header = ["Name", "Layer", "Time", "Self", "Self(%)", "Calls", "Average"]
    body = []
    for d in items:
        t = incl.get(d["key"], {}).get("total", 0)
        layer = str(func_layers[d["key"][-1]]) if func_layers is not None else "-"
        body.append([d["name"], layer, fmt_ns(t), fmt_ns(d["total"]),
                     fmt_pct(100.0 * d["total"] / t) if t else "-", str(d["count"]),
                     fmt_ns(d["total"] / d["count"]) if d["count"] else "-"])
    return _table(header, body, title)


def layer_summary(self_rows, func_layers, layer_names=None, title: str | None = None):
    """Self time summed per layer (the time each API layer spends itself), as
    (text, {layer: (self_ns, calls)}); Self(%) of the sum over all layers."""
    acc = {}
    for r in np.asarray(self_rows).tolist():
        func, count, total = r[3], r[4], r[5]
        a = acc.setdefault(func_layers[func], [0, 0])
        a[0] = (a[0] + total) & ((1 << 64) - 1)
        a[1] += count
    grand = float(sum(v[0] for v in acc.values())) or 1.0
    body = []
    for layer in sorted(acc, key=lambda k: (-acc[k][0], k)):
        name = layer_names[layer] if layer_names is not None else str(layer)
        body.append([name, fmt_ns(acc[layer][0]), fmt_pct(100.0 * acc[layer][0] / grand), str(acc[layer][1])])
    return _table(["Layer", "Self", "Self(%)", "Calls"], body, title), {k: tuple(v) for k, v in acc.items()}
