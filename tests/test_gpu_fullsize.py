"""Full-size parity on the large layered workload (100M calls, 200M events,
~8.4 GB, 512 streams, 16 KB packets), in the launch configuration bench.py
times (trace resident in device memory, thapi_trace_load_device).

The oracle cannot redo 200M events within the test budget, so it analyses a
sample of whole streams (streams are independent) and the CUDA results for
those streams must match it exactly; properties that hold at any size are
checked on everything.
"""
from __future__ import annotations

import random

import numpy as np
import pytest

import oracle
import tracegen as tg
from paper_2504_03683_b300 import thapi
from tests._util import intervals_equal, rows_equal, stream_table

pytestmark = pytest.mark.gpu


def test_large_workload_sampled_parity():
    import torch

    cfg = tg.preset("large")
    plan = tg.Plan(cfg)
    host = torch.empty(plan.nbytes, dtype=torch.uint8, pin_memory=True)
    plan.write(host.data_ptr())
    n_streams = plan.n_streams
    plan.close()
    host_np = host.numpy()
    dev = host.to("cuda")
    with thapi.Context(0) as ctx:
        tid = thapi.thapi_trace_load_device(ctx.handle, dev.data_ptr(), dev.numel(), torch.cuda.current_stream())
        rows, diag = ctx.tally(tid)
        ivs = ctx.timeline(tid)
        info = ctx.info(tid)
        ctx.free(tid)
    del dev
    # properties at full size
    assert diag["events"] == 200_000_000
    assert diag["events"] == 2 * (diag["pairs"] + diag["mismatched_pairs"]) + diag["unmatched_entries"] + \
        diag["unmatched_exits"] + diag["other_events"]
    assert diag["pairs"] == 100_000_000 == int(rows["count"].sum()) == len(ivs) == info["intervals"]
    assert diag["unmatched_entries"] == diag["unmatched_exits"] == diag["mismatched_pairs"] == 0
    s = ivs["start_ns"]
    assert np.all(s[1:] >= s[:-1])
    dur = (ivs["end_ns"] - ivs["start_ns"]).astype(np.uint64)
    assert np.add.reduce(dur, dtype=np.uint64) == np.add.reduce(rows["total_ns"], dtype=np.uint64)
    assert int(((ivs["flags"] & 1) > 0).sum()) == int(rows["err_count"].sum())
    # exact parity on sampled streams
    rng = random.Random(2504)
    sample = sorted({0, n_streams - 1} | set(rng.sample(range(n_streams), 6)))
    o = oracle.run(host_np, streams=sample)
    assert o.code == oracle.OK
    st = stream_table(host_np)
    keys = {(int(st[k][0]), int(st[k][1]), int(st[k][2])) for k in sample}
    mask = np.array([(r["host_id"], r["pid"], r["tid"]) in keys for r in rows])
    assert rows_equal(rows[mask], o.rows)
    assert intervals_equal(ivs[np.isin(ivs["stream_id"], sample)], o.intervals)
