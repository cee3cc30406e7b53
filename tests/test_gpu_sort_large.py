"""Sorts of a million items and more take the one-sweep radix form (one
histogram pass, one decoupled look-back kernel per digit pass): per-CPU
thread order (64-bit keys), the timeline's radix order with record gather
(too many streams for the bucket sort), and self time's (stream, level)
order, each against the oracle (tolerance 0)."""
from __future__ import annotations

import pytest

import oracle
import tracegen as tg
from tests._util import intervals_equal, rows_equal
from tests.test_gpu_parity import assert_parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    from paper_2504_03683_b300 import thapi
    assert torch.cuda.is_available()
    c = thapi.Context(0)
    yield c
    c.close()


def test_per_cpu_million_records(ctx):
    b = tg.generate(tg.preset("large", total_calls=650_000, n_hosts=2, pids_per_host=2, tids_per_pid=4, n_cpus=4,
                              slice_ns=50_000.0, seed=90, p_drop=0.001))[0]
    o = assert_parity(ctx, b)
    assert o.diag["events"] >= 1_200_000


def test_timeline_radix_order_with_many_streams(ctx):
    b = tg.generate(tg.preset("large", total_calls=1_200_000, n_hosts=3, pids_per_host=30, tids_per_pid=25,
                              seed=91, packet_bytes=4096))[0]
    o = assert_parity(ctx, b)
    assert len(o.intervals) >= 1_100_000


def test_self_time_million_intervals():
    from paper_2504_03683_b300 import thapi
    b = tg.generate(tg.preset("large", total_calls=1_200_000, n_hosts=2, pids_per_host=4, tids_per_pid=4, seed=92))[0]
    o = oracle.run(b)
    with thapi.Context(0) as c:
        c.set_self_time(True)
        tid = c.load(b)
        try:
            rows, _d = c.tally(tid)
            srows = c.self_tally(tid)
            ivs = c.timeline(tid)
        finally:
            c.free(tid)
    assert rows_equal(rows, o.rows) and rows_equal(srows, o.self_rows) and intervals_equal(ivs, o.intervals)
