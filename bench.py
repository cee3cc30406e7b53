#!/usr/bin/env python
"""Benchmark of the trace-analysis path on B300 (one JSON line on rank 0).

A step is one pass of the whole path over one synthetic trace already
resident in device memory: packet index + validation, warp/CTA-per-packet
decode with timestamp scan, in-packet and cross-packet entry/exit pairing,
per-(host, pid, tid, function) tally, and the sorted interval timeline
(thapi_trace_load_device), then both results copied out to device buffers
(thapi_tally_device, thapi_timeline_device) and the trace released.

Workload (default): 8 hosts x 8 pids x 8 threads, portable (60 fns) over
vendor (120 fns) plus a message-passing layer (30 fns), 100M calls = 200M
events (~8.4 GB), depth <= 6, log-normal durations (median 5 us), 1 % error
results, 16 KB packets.  Inputs are 8.4 GB, far larger than the 126 MB L2, so
no flush is needed between steps.

``--impl reference`` times the CPU oracle (the plain sequential definition)
on a bounded sample of the same trace instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "large": dict(preset="large", desc="8 hosts x 8 pids x 8 threads; portable(60)/vendor(120)/mpi(30) layers; "
                                       "100M calls = 200M events; depth<=6; 1% errors; 16 KB packets"),
    "tiny": dict(preset="tiny", desc="1 host x 1 pid x 4 threads; one API of 40 functions; 100k calls; "
                                     "depth<=3; 4 KB packets"),
    "device": dict(preset="device", desc="512 host streams (8x8x8) of launch/memcpy calls (16 fns) carrying unique "
                                         "random 64-bit command ids; 64 device streams of begin/end events; 50M "
                                         "commands = 200M events; device pairing + merged timeline; 16 KB packets"),
    "batch": dict(preset="large", desc="4096 per-rank traces (1 host x 1 pid x 8 threads each, the large workload's "
                                        "3-layer API mix, depth<=6), event counts log-uniform 10k-20M scaled to ~60 GB "
                                        "in total and clamped to [10k, 20M]; 16 KB packets; one batched load reading "
                                        "the device-resident traces in place vs 4096 plain loads of the same traces"),
    "serve": dict(preset="large", desc="serving loop: traces of the large workload's API mix (1 host x 1 pid x 8 "
                                        "threads each) sized log-uniform 1 MB-4 GB, decoded results kept "
                                        "device-resident under a 120 GB admission cap (100 GB resident at the "
                                        "start); Poisson arrivals at 200 req/s: 5% trace loads from pinned host "
                                        "memory, 5% frees of the oldest trace, the rest half tally and half "
                                        "time-window queries (width log-uniform 1e-4-1 of the span)"),
    "percpu": dict(preset="percpu", desc="the large workload's shape (8 hosts x 64 threads, 3 layers, depth<=6) "
                                         "written as per-CPU buffers: 32 CPUs per host, threads rotated over CPUs "
                                         "every 200 us (two threads interleaved per CPU); 50M calls = 100M events "
                                         "with 16-byte headers; 16 KB packets"),
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="large")
    ap.add_argument("--calls", type=int, default=0, help="override total calls (smaller runs)")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--cpu-streams", type=int, default=0, help="streams in the CPU-baseline sample (0 = auto)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--profile-once", action="store_true", help="one load only (for a profiler), no JSON")
    ap.add_argument("--self-time", action="store_true", help="every load also computes self (exclusive) time")
    ap.add_argument("--autotune", action="store_true", help="the context's autotuner picks the load configuration "
                                                             "(during the warm-up steps)")
    ap.add_argument("--batch-traces", type=int, default=4096, help="batch workload: traces")
    ap.add_argument("--batch-gb", type=float, default=60.0, help="batch workload: total trace bytes (GB)")
    ap.add_argument("--serve-sources", type=int, default=40, help="serve workload: distinct traces in the pool")
    ap.add_argument("--serve-cap-gb", type=float, default=120.0, help="serve workload: admission cap (GB)")
    ap.add_argument("--serve-resident-gb", type=float, default=100.0,
                    help="serve workload: device bytes of the results resident at the start (GB)")
    ap.add_argument("--serve-seconds", type=float, default=10.0, help="serve workload: arrival window (s)")
    ap.add_argument("--serve-rate", type=float, default=200.0, help="serve workload: mean arrivals per second")
    ap.add_argument("--serve-p-load", type=float, default=0.05, help="serve workload: share of loads (and of frees)")
    ap.add_argument("--serve-result-gb", type=float, default=8.0,
                    help="serve workload: pinned host memory the serving loop sets aside for results (GB)")
    ap.add_argument("--serve-load-slots", type=int, default=2)
    ap.add_argument("--serve-query-slots", type=int, default=6)
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return rank, world, local


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0}, "fallback"


def trace_config(args, rank):
    import tracegen as tg
    over = {}
    if args.calls:
        over["total_calls"] = args.calls
    cfg = tg.preset(WORKLOADS[args.workload]["preset"], **over)
    cfg.seed = cfg.seed + 1000 * rank
    return cfg


def generate_pinned(cfg):
    """Writes the trace straight into pinned host memory (a torch tensor)."""
    import torch
    import tracegen as tg
    plan = tg.Plan(cfg)
    host = torch.empty(plan.nbytes, dtype=torch.uint8, pin_memory=True)
    plan.write(host.data_ptr())
    meta = dict(nbytes=plan.nbytes, n_packets=plan.n_packets, n_streams=plan.n_streams)
    plan.close()
    return host, meta


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.QUERY, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def profile_traffic(kernel_file, kernel, workload):
    """DRAM traffic per launch recorded by the committed ncu summary, if it still matches the kernel source."""
    path = os.path.join(ROOT, "profiles", "%s_%s.md" % (kernel, workload))
    try:
        text = open(path).read()
    except OSError:
        return None
    src = hashlib.sha256(open(kernel_file, "rb").read()).hexdigest()[:16]
    rec = {}
    for line in text.splitlines():
        if line.startswith("traffic_bytes_per_launch:"):
            rec["traffic"] = float(line.split(":", 1)[1])
        if line.startswith("kernel_source_sha256_16:"):
            rec["sha"] = line.split(":", 1)[1].strip()
    if rec.get("sha") != src or "traffic" not in rec:
        return None
    return rec["traffic"]


def sample_streams(workload, n_streams, cpu_streams):
    """Streams of the bounded CPU sample (about 10-20 s of oracle time on one core)."""
    if workload == "device":  # the first host streams and the first device streams (ids 512..575)
        k = cpu_streams or 32
        return list(range(min(k, 512))) + list(range(512, min(n_streams, 514)))
    k = cpu_streams or {"large": 200, "percpu": 24}.get(workload, 64)
    return list(range(max(1, min(n_streams, k))))


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_sample(host_np, n_streams, streams, threads=1):
    """The oracle, as it stands, on a subset of the streams of the same trace:
    one thread, or `threads` std::threads over stream subsets (the all-cores
    baseline; traces whose pairing crosses streams run on one thread)."""
    import oracle
    t = time.perf_counter()
    r = oracle.run_threads(host_np, threads, streams=streams) if threads > 1 else oracle.run(host_np, streams=streams)
    dt = time.perf_counter() - t
    ranges, i = [], 0
    while i < len(streams):
        j = i
        while j + 1 < len(streams) and streams[j + 1] == streams[j] + 1:
            j += 1
        ranges.append("%d..%d" % (streams[i], streams[j]))
        i = j + 1
    whole = len(streams) == n_streams
    return dict(value=r.diag["events"] / dt, unit="events/s", cores=threads, kind="oracle",
                sample="%s of the same trace (%d events), decode+pair+tally%s+timeline, %s" % (
                    "all %d streams" % n_streams if whole else "streams %s of %d" % (", ".join(ranges), n_streams),
                    r.diag["events"], "+device pairing" if r.dev_diag["dev_events"] else "",
                    "one thread" if threads == 1 else "%d std::threads over stream subsets (host cores: %d)" % (
                        threads, host_cores())),
                seconds=round(dt, 3))


def e2e_pipelined(device, host, info, events, h2d, d2h, steps, depth=2, warm=2):
    """End to end through the serving loop (thapi_server_*), trace after
    trace with `depth` traces in flight: each step loads the trace from pinned
    host memory and reads its tally rows and whole timeline back into pinned
    host memory, then frees it, so that one trace's upload runs while the one
    before it is analysed and read back.  Steady-state time per step: between
    the completions of the last warm-up step and of the last step."""
    import collections
    import numpy as np
    import torch
    from paper_2504_03683_b300 import serve, thapi
    n_iv, n_rows = info["intervals"], info["tally_rows"]
    rows = [np.zeros(max(1, n_rows), dtype=thapi.ROW_DTYPE) for _ in range(depth)]
    ivs = [torch.empty(max(1, n_iv) * 24, dtype=torch.uint8, pin_memory=True) for _ in range(depth)]
    ctx = thapi.Context(device, use_torch_allocator=False)
    srv = serve.Server(ctx, load_slots=1, query_slots=2, result_bytes=64 << 20)

    def req(kind, **kw):
        r = thapi.Request()
        r.kind = kind
        for k, v in kw.items():
            setattr(r, k, v)
        return r

    inflight, done = collections.deque(), []
    try:
        for k in range(warm + steps + depth):
            if len(inflight) == depth or k >= warm + steps:
                if not inflight:
                    break
                tickets = inflight.popleft()
                res = [srv.wait(t) for t in tickets]
                done.append(time.perf_counter())
                ok = all(r.status == thapi.OK for r in res) and res[1].n == n_rows and res[2].n == n_iv
                for t in tickets:
                    srv.release(t)
                if not ok:
                    raise RuntimeError("pipelined end-to-end step failed: %s" % [r.status for r in res])
            if k >= warm + steps:
                continue
            b = k % depth
            tl = srv.submit(req(thapi.REQ_LOAD, bytes=host.data_ptr(), nbytes=host.numel()))
            tt = srv.submit(req(thapi.REQ_TALLY, after=tl, out=rows[b].ctypes.data, cap=len(rows[b])))
            tw = srv.submit(req(thapi.REQ_WINDOW, after=tl, t0=0, t1=2**64 - 1, out=ivs[b].data_ptr(),
                                cap=max(1, n_iv)))
            tf = srv.submit(req(thapi.REQ_FREE, after=tl))
            inflight.append((tl, tt, tw, tf))
    finally:
        srv.close()
        ctx.close()
    per = (done[warm + steps - 1] - done[warm - 1]) / steps
    return {"value": events / per, "unit": "events/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "ms_per_step": per * 1e3,
            "mode": "%d traces in flight through the serving loop (one load slot, two query slots): a trace's "
                    "upload overlaps the previous trace's analysis and read-back; steady state over %d steps"
                    % (depth, steps)}


def cpu_baseline(host_np, n_streams, workload, cpu_streams):
    """The reported CPU baseline: the oracle on all host cores over every stream
    (per-thread host workloads), with the one-thread oracle on a bounded stream
    sample beside it; other workloads (pairing across streams): one thread."""
    one = cpu_sample(host_np, n_streams, sample_streams(workload, n_streams, cpu_streams))
    if workload not in ("large", "tiny"):
        return one
    allc = cpu_sample(host_np, n_streams, list(range(n_streams)), threads=host_cores())
    allc["one_core"] = one
    return allc


def run_reference(args, rank, world):
    if rank != 0:
        return
    import numpy as np  # noqa: F401
    cfg = trace_config(args, 0)
    import tracegen as tg
    host, _c, _e = tg.generate(cfg)
    plan = tg.Plan(cfg)
    n_streams = plan.n_streams
    plan.close()
    streams = sample_streams(args.workload, n_streams,
                             args.cpu_streams or {"large": 128, "device": 16, "percpu": 8}.get(args.workload, 0))
    threads = host_cores() if args.workload in ("large", "tiny") else 1
    samples = []
    for i in range(args.warmup + args.steps):
        s = cpu_sample(host, n_streams, streams, threads=threads)
        if i >= args.warmup:
            samples.append(s)
    value = statistics.median(x["value"] for x in samples)
    ms = statistics.median(x["seconds"] for x in samples) * 1e3
    line = {
        "impl": "reference", "metric": "events/s decode+pair+tally+timeline", "value": value, "unit": "events/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": args.workload, "desc": WORKLOADS[args.workload]["desc"],
                   "calls": int(cfg.total_calls), "seed": int(cfg.seed)},
        "cpu_baseline": {"value": value, "unit": "events/s", "cores": threads, "kind": "oracle",
                         "sample": samples[0]["sample"]},
        "e2e": {"value": value, "unit": "events/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def batch_sizes(n, total_events, seed):
    """Event counts of the batch: log-uniform in [10k, 20M], scaled by one factor
    so that they sum to about total_events, then clamped to [10k, 20M]."""
    import numpy as np
    rng = np.random.default_rng(seed)
    x = np.exp(rng.uniform(np.log(1e4), np.log(2e7), n))
    x *= total_events / x.sum()
    return np.clip(x, 1e4, 2e7).astype(np.int64)


def batch_configs(args, rank):
    import tracegen as tg
    ev = batch_sizes(args.batch_traces, args.batch_gb * 1e9 / 40.2, 7 + rank)
    cfgs = []
    for i, e in enumerate(ev):
        cfgs.append(tg.preset("large", total_calls=int(e) // 2, n_hosts=1, pids_per_host=1, tids_per_pid=8,
                              seed=100000 * (rank + 1) + i))
    return cfgs


def run_batch(args, rank, world, local):
    """Config 3: many per-rank traces in one batched load vs one plain load each."""
    import numpy as np
    import torch
    import tracegen as tg
    from paper_2504_03683_b300 import thapi
    cfgs = batch_configs(args, rank)
    plans = [tg.Plan(c) for c in cfgs]
    offs, tot = [], 0
    for pl in plans:
        offs.append(tot)
        tot += (pl.nbytes + 255) // 256 * 256
    host = torch.empty(tot, dtype=torch.uint8, pin_memory=True)
    for pl, o in zip(plans, offs):
        pl.write(host.data_ptr() + o)
    sizes = [pl.nbytes for pl in plans]
    n_packets = sum(pl.n_packets for pl in plans)
    for pl in plans:
        pl.close()
    dev = host.to("cuda")
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    ctx = thapi.Context(local)
    thapi.thapi_ctx_set_timing(ctx.handle, True)
    if args.autotune:
        thapi.thapi_ctx_set_autotune(ctx.handle, True)
    dptr = [(dev.data_ptr() + o, n) for o, n in zip(offs, sizes)]
    tid = ctx.load_batch_device(dptr, stream)
    info = ctx.info(tid)
    ctx.free(tid)
    events = info["events"]
    rows_d = torch.empty(max(1, info["tally_rows"]) * 56, dtype=torch.uint8, device="cuda")
    ivs_d = torch.empty(max(1, info["intervals"]) * 24, dtype=torch.uint8, device="cuda")
    timings = []

    def batched(record=False):
        t = thapi.thapi_trace_load_batch(ctx.handle, dptr, stream, on_device=True)
        thapi.thapi_tally_device(ctx.handle, t, rows_d.data_ptr(), info["tally_rows"], stream)
        thapi.thapi_timeline_device(ctx.handle, t, 0, 2**64 - 1, ivs_d.data_ptr(), info["intervals"], stream)
        if record:
            timings.append(thapi.thapi_trace_timing(ctx.handle, t))
        thapi.thapi_trace_free(ctx.handle, t)

    def plain():  # one load per trace, each trace's results copied out
        for (p, n) in dptr:
            t = thapi.thapi_trace_load_device(ctx.handle, p, n, stream)
            i = ctx.info(t)
            thapi.thapi_tally_device(ctx.handle, t, rows_d.data_ptr(), i["tally_rows"], stream)
            thapi.thapi_timeline_device(ctx.handle, t, 0, 2**64 - 1, ivs_d.data_ptr(), i["intervals"], stream)
            thapi.thapi_trace_free(ctx.handle, t)

    for _ in range(args.warmup):
        batched()
    sampler = ClockSampler(local)
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.3)
    launches0 = thapi.thapi_kernel_launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        batched(record=True)
    e1.record(stream)
    torch.cuda.synchronize()
    launches = thapi.thapi_kernel_launches() - launches0
    ms = e0.elapsed_time(e1) / args.steps
    plain()  # warm
    torch.cuda.synchronize()
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    pl_launch0 = thapi.thapi_kernel_launches()
    p0.record(stream)
    plain()
    p1.record(stream)
    torch.cuda.synchronize()
    plain_launches = thapi.thapi_kernel_launches() - pl_launch0
    plain_ms = p0.elapsed_time(p1)
    clocks = sampler.stop()
    peaks, peak_src = measured_peaks()
    an_ms = statistics.mean(t["analyze_ms"] for t in timings)
    an_bytes = timings[0]["analyze_read_bytes"] + timings[0]["analyze_write_bytes"]
    achieved = an_bytes / (an_ms / 1e3) / 1e9
    peak = float(peaks.get("hbm_gbs", 6400.0))
    phase = {k: round(statistics.mean(t[k] for t in timings), 4)
             for k in ("index_ms", "analyze_ms", "frontier_ms", "tally_ms", "compact_ms", "sort_ms", "gather_ms",
                       "total_ms", "parse_ms", "call_ms")}
    # end to end: the batch from pinned host memory, results to the host
    e2e = None
    if not args.no_e2e:
        times = []
        for i in range(args.e2e_steps + 1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            t = ctx.load_batch([host[o:o + n].numpy() for o, n in zip(offs, sizes)], stream)
            thapi.thapi_tally(ctx.handle, t)
            thapi.thapi_timeline(ctx.handle, t)
            thapi.thapi_trace_free(ctx.handle, t)
            if i > 0:
                times.append(time.perf_counter() - t0)
        e2e_s = statistics.median(times)
        e2e = {"value": events / e2e_s, "unit": "events/s", "h2d_bytes_per_step": n_packets * 16384,
               "d2h_bytes_per_step": info["tally_rows"] * 56 + info["intervals"] * 24, "ms_per_step": e2e_s * 1e3}
    cpu = None
    if not args.no_cpu_baseline:
        import oracle
        k = sorted(range(len(sizes)), key=lambda i: sizes[i])[: max(1, len(sizes) // 8)]
        t0 = time.perf_counter()
        ev = 0
        for i in k:
            ev += oracle.run(host[offs[i]:offs[i] + sizes[i]].numpy()).diag["events"]
        dt = time.perf_counter() - t0
        cpu = {"value": ev / dt, "unit": "events/s", "cores": 1, "kind": "oracle",
               "sample": "the %d smallest of the %d traces (%d events), decode+pair+tally+timeline, one thread"
                         % (len(k), len(sizes), ev), "seconds": round(dt, 3)}
    ev_sorted = np.sort([c.total_calls * 2 for c in cfgs])
    line = {
        "metric": "events/s decode+pair+tally+timeline, batched", "value": events / (ms / 1e3), "unit": "events/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": "batch", "desc": WORKLOADS["batch"]["desc"], "traces": len(cfgs), "events": events,
                   "trace_bytes": int(sum(sizes)), "packets": int(n_packets),
                   "events_per_trace": {"min": int(ev_sorted[0]), "p50": int(ev_sorted[len(ev_sorted) // 2]),
                                        "max": int(ev_sorted[-1])},
                   "load_config": {"grid_mult": timings[0]["grid_mult"], "part_shift": timings[0]["part_shift"],
                                   "autotuned": bool(args.autotune)},
                   "l2": "inputs larger than L2; no flush"},
        "plain": {"value": events / (plain_ms / 1e3), "unit": "events/s", "ms_per_pass": plain_ms,
                  "gpu_launches": plain_launches, "desc": "one thapi_trace_load_device + tally + timeline per trace"},
        "batched_over_plain": plain_ms / ms,
        "phases_ms": phase,
        "roofline": {"kernel": "k_analyze_warp (decode+validate+pair+tally, interval slots)", "bound": "hbm",
                     "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "peak_source": peak_src + " hbm_gbs (MEASURED_PEAKS.json)" if peak_src == "measured"
                     else "fallback", "bytes_per_launch": an_bytes, "launch_ms": an_ms, "traffic": None},
        "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clocks,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()


def serve_pool(args, rank):
    """Trace sources of the serve workload: sizes log-uniform in 1 MB - 4 GB (the
    large workload's API mix, 1 host x 1 pid x 8 threads each), written into
    one pinned host buffer; returns (host tensor, [(offset, nbytes)])."""
    import numpy as np
    import torch
    import tracegen as tg
    rng = np.random.default_rng(11 + rank)
    sizes = [float(np.exp(rng.uniform(np.log(1e6), np.log(4e9)))) for _ in range(args.serve_sources)]
    plans = [tg.Plan(tg.preset("large", total_calls=max(1000, int(b / 40.2) // 2), n_hosts=1, pids_per_host=1,
                               tids_per_pid=8, seed=200000 + 1000 * rank + i)) for i, b in enumerate(sizes)]
    offs, tot = [], 0
    for pl in plans:
        offs.append((tot, pl.nbytes))
        tot += (pl.nbytes + 255) // 256 * 256
    host = torch.empty(tot, dtype=torch.uint8, pin_memory=True)
    for pl, (o, _n) in zip(plans, offs):
        pl.write(host.data_ptr() + o)
        pl.close()
    return host, offs


def run_serve(args, rank, world, local):
    """Config 5: a Poisson stream of trace loads, tally / window queries and trace
    frees over traces kept resident near the 120 GB admission cap, served by the
    serving loop (continuous batching, thapi_server_*) and, on the same
    schedule from the same resident set, one request at a time with plain
    launches on one stream."""
    import numpy as np
    import torch
    from paper_2504_03683_b300 import serve, thapi
    host, offs = serve_pool(args, rank)
    dev = host.to("cuda")
    torch.cuda.synchronize()
    host_src = [(host.data_ptr() + o, n, False) for o, n in offs]
    dev_src = [(dev.data_ptr() + o, n, True) for o, n in offs]
    cap = int(args.serve_cap_gb * 1e9)
    ctx = thapi.Context(local, cap, use_torch_allocator=False)
    stream = torch.cuda.current_stream()
    k_src = len(offs)

    def preload():
        """Loads sources round robin from device memory until the resident
        results reach the target; returns (trace ids, their sources)."""
        ids, srcs, k = [], [], 0
        target = int(args.serve_resident_gb * 1e9)
        used = 0
        while used < target:
            s = k % k_src
            tid = thapi.thapi_trace_load_device(ctx.handle, dev_src[s][0], dev_src[s][1], stream)
            ids.append(tid)
            srcs.append(s)
            used += thapi.thapi_trace_info_get(ctx.handle, tid)["device_bytes"]
            k += 1
        return ids, srcs, used

    def unload_all(ids_alive):
        for tid in ids_alive:
            thapi.thapi_trace_free(ctx.handle, tid)

    t_pre = time.perf_counter()
    ids, srcs, resident_bytes = preload()
    pre_s = time.perf_counter() - t_pre
    info = {}
    for tid, s in zip(ids, srcs):
        if s not in info:
            info[s] = thapi.thapi_trace_info_get(ctx.handle, tid)
    spans = [(info[s]["t_min"], info[s]["t_max"]) for s in range(k_src)]
    src_events = [info[s]["events"] for s in range(k_src)]
    max_iv = max(info[s]["intervals"] for s in range(k_src))
    steps = serve.make_schedule(args.serve_rate, args.serve_seconds, srcs, spans, seed=13 + rank,
                                p_load=args.serve_p_load, p_free=args.serve_p_load)
    warm = serve.make_schedule(args.serve_rate, 0.5, srcs, spans, seed=17 + rank, p_load=0.0, p_free=0.0)

    def answered(kind, n, events):
        return events if kind == "tally" else (2 * n if kind == "window" else (events if kind == "load" else 0))

    # ---- one request at a time with plain launches
    rows_out = np.zeros(1 << 16, dtype=thapi.ROW_DTYPE)
    ivs_pin = torch.empty(max(1, max_iv) * 24, dtype=torch.uint8, pin_memory=True)
    ivs_out = ivs_pin.numpy().view(thapi.INTERVAL_DTYPE)
    serve.serve_serial(ctx, warm, ids, host_src, rows_out, ivs_out, stream)
    t0 = time.perf_counter()
    serial = serve.serve_serial(ctx, steps, ids, host_src, rows_out, ivs_out, stream)
    serial_wall = time.perf_counter() - t0
    # the resident set as it was before the schedule: every trace now resident leaves, the preload is redone
    alive = {}
    for i, tid in enumerate(ids):
        alive[i] = tid
    for st, o in zip(steps, serial):
        if o is None or o.status != thapi.OK:
            continue
        if st.kind == "load":
            alive[st.handle] = o.trace
        elif st.kind == "free":
            alive.pop(st.handle, None)
    unload_all(alive.values())
    ids, srcs2, resident_bytes = preload()
    assert srcs2 == srcs

    # ---- the serving loop
    srv = serve.Server(ctx, args.serve_load_slots, args.serve_query_slots, int(args.serve_result_gb * 1e9))
    srv.replay(warm, ids, host_src)
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    launches0 = thapi.thapi_kernel_launches()
    t0 = time.perf_counter()
    res = srv.replay(steps, ids, host_src)
    wall = time.perf_counter() - t0
    launches = thapi.thapi_kernel_launches() - launches0
    clocks = sampler.stop()
    stats = srv.stats()
    srv.close()

    def totals(outs, wall_s):
        ev = {"load": 0, "tally": 0, "window": 0}
        h2d = d2h = 0
        for st, o in zip(steps, outs):
            if o is None or o.status != thapi.OK or st.kind == "free":
                continue
            ev[st.kind] += answered(st.kind, o.n, o.events)
            if st.kind == "load":
                h2d += offs[st.source][1]
            else:
                d2h += o.n * (56 if st.kind == "tally" else 24)
        # the last result, on the schedule's clock (each result's latency after its arrival)
        end = max((st.arrival + o.t_done - o.t_arrival for st, o in zip(steps, outs) if o is not None),
                  default=0.0)
        return {"answered_events_per_s": (ev["tally"] + ev["window"]) / wall_s,
                "loaded_events_per_s": ev["load"] / wall_s, "wall_s": wall_s, "h2d_bytes": h2d, "d2h_bytes": d2h,
                "last_result_s": end}

    srv_sum, ser_sum = serve.summary(res), serve.summary(serial)
    srv_tot, ser_tot = totals(res, wall), totals(serial, serial_wall)
    q99 = srv_sum["queries"]["p99"]
    line = {
        "metric": "p99 latency of tally / window queries at %g req/s with loads and frees, arrival to result "
                  "on the host" % args.serve_rate,
        "value": q99, "unit": "ms", "n_gpus": world, "steps": len(steps), "warmup": len(warm),
        "ms_per_step": float(np.mean([(o.t_done - o.t_arrival) * 1e3 for o in res if o.status == thapi.OK])),
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": "serve", "desc": WORKLOADS["serve"]["desc"], "sources": k_src,
                   "source_bytes": {"min": int(min(n for _o, n in offs)), "max": int(max(n for _o, n in offs)),
                                    "total": int(sum(n for _o, n in offs))},
                   "cap_bytes": cap, "resident_at_start": {"traces": len(ids), "device_bytes": resident_bytes},
                   "preload_s": round(pre_s, 2), "requests": len(steps),
                   "mix": {k: sum(1 for s in steps if s.kind == k) for k in serve.KINDS},
                   "seconds": args.serve_seconds, "slots": {"load": args.serve_load_slots,
                                                            "query": args.serve_query_slots},
                   "loads_from": "pinned host memory"},
        "latency_ms": srv_sum,
        "serial": {"latency_ms": ser_sum, **ser_tot,
                   "desc": "the same schedule one request at a time in arrival order with the plain entry points "
                           "(thapi_trace_load, thapi_tally, thapi_timeline, thapi_trace_free) on one stream"},
        "served_over_serial_p99": ser_sum["queries"]["p99"] / q99 if q99 else None,
        **srv_tot,
        "server_stats": stats,
        "e2e": {"value": q99, "unit": "ms", "h2d_bytes_per_step": srv_tot["h2d_bytes"] / len(steps),
                "d2h_bytes_per_step": srv_tot["d2h_bytes"] / len(steps),
                "note": "every latency is already arrival to result in host memory; loads read pinned host memory"},
        "gpu_launches": launches, "clocks": clocks, "cpu_baseline": None, "roofline": None,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    del dev, host


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.workload in ("batch", "serve"):
        import torch
        torch.cuda.set_device(local)
        return (run_batch if args.workload == "batch" else run_serve)(args, rank, world, local)

    import numpy as np
    import torch
    from paper_2504_03683_b300 import thapi

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    cfg = trace_config(args, rank)
    host, meta = generate_pinned(cfg)
    dev = host.to("cuda", non_blocking=False)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    ctx = thapi.Context(local)
    thapi.thapi_ctx_set_timing(ctx.handle, True)
    if args.self_time:
        thapi.thapi_ctx_set_self_time(ctx.handle, True)
    if args.autotune:
        thapi.thapi_ctx_set_autotune(ctx.handle, True)

    if args.profile_once:
        tid = thapi.thapi_trace_load_device(ctx.handle, dev.data_ptr(), dev.numel(), stream)
        torch.cuda.synchronize()
        ctx.free(tid)
        ctx.close()
        return

    # first load sizes the output buffers
    tid = thapi.thapi_trace_load_device(ctx.handle, dev.data_ptr(), dev.numel(), stream)
    info = ctx.info(tid)
    n_self_rows = len(thapi.thapi_self_tally(ctx.handle, tid)) if args.self_time else 0
    ctx.free(tid)
    rows_d = torch.empty(max(1, info["tally_rows"]) * 56, dtype=torch.uint8, device="cuda")
    ivs_d = torch.empty(max(1, info["intervals"]) * 24, dtype=torch.uint8, device="cuda")
    events = info["events"]
    timings = []

    def step(record=False):
        t = thapi.thapi_trace_load_device(ctx.handle, dev.data_ptr(), dev.numel(), stream)
        thapi.thapi_tally_device(ctx.handle, t, rows_d.data_ptr(), info["tally_rows"], stream)
        thapi.thapi_timeline_device(ctx.handle, t, 0, 2**64 - 1, ivs_d.data_ptr(), info["intervals"], stream)
        if record:
            timings.append(thapi.thapi_trace_timing(ctx.handle, t))
        thapi.thapi_trace_free(ctx.handle, t)

    for _ in range(args.warmup):
        step()
    barrier = (lambda: torch.distributed.barrier()) if world > 1 else (lambda: None)
    sampler = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.3)
    launches0 = thapi.thapi_kernel_launches()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step(record=True)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    launches = thapi.thapi_kernel_launches() - launches0
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1) / args.steps
    ms_max = ms
    total_events = events
    if world > 1:
        t = torch.tensor([ms], device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms_max = float(t.item())
        ev = torch.tensor([float(events)], device="cuda", dtype=torch.float64)
        torch.distributed.all_reduce(ev)
        total_events = float(ev.item())
        lt = torch.tensor([float(launches)], device="cuda", dtype=torch.float64)
        torch.distributed.all_reduce(lt)
        launches = int(lt.item())
    value = total_events / (ms_max / 1e3)

    # roofline of the dominant kernel, CUDA events inside the library: the analysis kernel
    # (decode + pair + tally), or for traces of per-CPU buffers their record-writing decode
    peaks, peak_src = measured_peaks()
    an_ms = statistics.mean(t["analyze_ms"] for t in timings)
    an_bytes = timings[0]["analyze_read_bytes"] + timings[0]["analyze_write_bytes"]
    kname = "k_analyze_warp"
    kdesc = "k_analyze_warp (decode+validate+pair+tally, interval slots%s)" % (
        ", command records" if args.workload == "device" else "")
    pd_ms = statistics.mean(t["percpu_decode_ms"] for t in timings)
    if pd_ms > an_ms:
        an_ms = pd_ms
        an_bytes = timings[0]["percpu_read_bytes"] + timings[0]["percpu_write_bytes"]
        kname = "k_percpu_decode"
        kdesc = "k_percpu_decode (decode+validate per-CPU buffers, 32-byte event records, entry slots)"
    achieved = an_bytes / (an_ms / 1e3) / 1e9
    peak = float(peaks.get("hbm_gbs", 6400.0))
    phase = {k: round(statistics.mean(t[k] for t in timings), 4)
             for k in ("index_ms", "analyze_ms", "frontier_ms", "join_ms", "percpu_ms", "percpu_decode_ms", "tally_ms",
                       "self_ms", "compact_ms", "sort_ms", "gather_ms", "total_ms", "parse_ms", "call_ms")}
    # a capture is per kernel variant: loads with self time run the variant with side records
    traffic = profile_traffic(os.path.join(ROOT, "paper_2504_03683_b300", "csrc", "analyze_warp.cu"), kname,
                              args.workload + ("_self" if args.self_time and kname == "k_analyze_warp" else ""))

    # end to end through the public API: host bytes in, host results out
    e2e = None
    if not args.no_e2e and rank == 0:
        rows_h = np.zeros(max(1, info["tally_rows"]), dtype=thapi.ROW_DTYPE)
        ivs_pinned = torch.empty(max(1, info["intervals"]) * 24, dtype=torch.uint8, pin_memory=True)
        ivs_h = ivs_pinned.numpy().view(thapi.INTERVAL_DTYPE)
        n_iv = info["intervals"]
        times = []
        for i in range(args.e2e_steps + 1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            tid = thapi.thapi_trace_load(ctx.handle, (host.data_ptr(), host.numel()), stream)
            rows, _d = thapi.thapi_tally(ctx.handle, tid)
            thapi.thapi_timeline(ctx.handle, tid, out=ivs_h)
            if args.self_time:
                thapi.thapi_self_tally(ctx.handle, tid)
            thapi.thapi_trace_free(ctx.handle, tid)
            dt = time.perf_counter() - t0
            if i > 0:
                times.append(dt)
        e2e_s = statistics.median(times)
        h2d = meta["n_packets"] * int(cfg.packet_bytes)
        d2h = (info["tally_rows"] + n_self_rows) * 56 + n_iv * 24
        e2e = {"value": events / e2e_s, "unit": "events/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "ms_per_step": e2e_s * 1e3}

        if not args.self_time:  # the serving loop has no self-time request
            serial = e2e
            try:
                e2e = e2e_pipelined(local, host, info, events, h2d, d2h, max(4, args.e2e_steps))
                e2e["serial"] = serial
            except Exception as exc:  # keep the one-at-a-time number, say why
                e2e = dict(serial, pipelined_error="%s: %s" % (type(exc).__name__, exc))

    cpu = None
    if not args.no_cpu_baseline and rank == 0:
        cpu = cpu_baseline(host.numpy(), meta["n_streams"], args.workload, args.cpu_streams)

    if rank == 0:
        line = {
            "metric": "events/s decode+pair+tally+timeline" + ("+self time" if args.self_time else ""),
            "value": value, "unit": "events/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": args.workload, "desc": WORKLOADS[args.workload]["desc"],
                       "self_time": bool(args.self_time),
                       "load_config": {"grid_mult": timings[0]["grid_mult"], "part_shift": timings[0]["part_shift"],
                                       "autotuned": bool(args.autotune)},
                       "calls": int(cfg.total_calls), "events_per_rank": events, "trace_bytes": meta["nbytes"],
                       "packets": meta["n_packets"], "seed": int(cfg.seed), "parallelism": "replicas" if world > 1
                       else "single",
                       "l2": "inputs larger than L2 (%.1f GB trace vs 126 MB L2); no flush" % (meta["nbytes"] / 1e9)},
            "trace_gbs": meta["nbytes"] / (ms_max / 1e3) / 1e9 * (world if world > 1 else 1),
            "phases_ms": phase,
            "roofline": {"kernel": kdesc, "bound": "hbm",
                         "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "peak_source": peak_src + " hbm_gbs (MEASURED_PEAKS.json)" if peak_src == "measured"
                         else "fallback",
                         "bytes_per_launch": an_bytes, "launch_ms": an_ms, "traffic": traffic},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
