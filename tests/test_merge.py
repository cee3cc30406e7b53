"""Merge of tally rows across traces and ranks.

Pin (no GPU): the oracle's tally of one trace made of two traces' streams
(streams of the two halves share (host, pid, tid) keys) equals the plain
group-by merge of the two halves' oracle tallies — so merging aggregates is
exact.  The same merge over a two-rank gloo gather.  With a GPU:
thapi_tally_merge of the CUDA tallies of the halves against the oracle's
tally of the joined trace, and against the plain merge on random rows.
"""
from __future__ import annotations

import os
import random
from collections import defaultdict

import numpy as np
import pytest

import oracle
import tracegen as tg
from tests._concat import concat
from tests._util import ROW_DTYPE, U64, rows_equal

SMALL = dict(total_calls=15_000, n_hosts=1, pids_per_host=2, tids_per_pid=2, p_err=0.05)


def plain_merge(*parts):
    """Group-by over (host_id, pid, tid, func_id): sums (u64), min, max."""
    acc = defaultdict(lambda: [0, 0, U64, 0, 0])
    for rows in parts:
        for r in rows.tolist():
            a = acc[tuple(r[:4])]
            a[0] += r[4]
            a[1] = (a[1] + r[5]) & U64
            a[2] = min(a[2], r[6])
            a[3] = max(a[3], r[7])
            a[4] += r[8]
    keys = sorted(acc)
    out = np.zeros(len(keys), dtype=ROW_DTYPE)
    for i, k in enumerate(keys):
        out[i] = (*k, *acc[k])
    return out


def _halves(seed_a=3, seed_b=4):
    a, _, _ = tg.generate(tg.preset("large", seed=seed_a, **SMALL))
    b, _, _ = tg.generate(tg.preset("large", seed=seed_b, **dict(SMALL, total_calls=11_000)))
    return a, b


def test_oracle_tally_of_joined_trace_is_merge_of_halves():
    a, b = _halves()
    ra, rb, rab = oracle.run(a), oracle.run(b), oracle.run(concat(a, b))
    assert rab.code == oracle.OK
    assert len(rab.rows) < len(ra.rows) + len(rb.rows)  # the halves share keys
    assert rows_equal(rab.rows, plain_merge(ra.rows, rb.rows))


def _rank_main(rank, world, port, result):
    import torch.distributed as dist
    from paper_2504_03683_b300.dist import gather_rows
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    try:
        a, b = _halves()
        mine = oracle.run(a if rank == 0 else b).rows
        got = gather_rows(mine, dst=0)
        if rank == 0:
            result.put(got.tobytes())
        else:
            assert got is None
    finally:
        dist.destroy_process_group()


def test_gather_rows_two_ranks_gloo():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + random.randrange(2000)
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = np.frombuffer(q.get(timeout=120), dtype=ROW_DTYPE)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    a, b = _halves()
    assert rows_equal(plain_merge(got), oracle.run(concat(a, b)).rows)


# ------------------------------------------------------------------ GPU
@pytest.fixture(scope="module")
def ctx():
    import torch
    from paper_2504_03683_b300 import thapi
    assert torch.cuda.is_available()
    c = thapi.Context(0)
    yield c
    c.close()


@pytest.mark.gpu
def test_gpu_merge_of_halves_equals_joined_trace(ctx):
    a, b = _halves()
    ta, tb = ctx.load(a), ctx.load(b)
    try:
        ra, _ = ctx.tally(ta)
        rb, _ = ctx.tally(tb)
    finally:
        ctx.free(ta)
        ctx.free(tb)
    merged = ctx.tally_merge(np.concatenate([rb, ra]))
    assert rows_equal(merged, oracle.run(concat(a, b)).rows)


@pytest.mark.gpu
@pytest.mark.parametrize("n,keys,seed", [(0, 1, 0), (1, 1, 1), (5000, 1, 2), (20_000, 300, 3), (70_000, 60_000, 4)])
def test_gpu_merge_random_rows(ctx, n, keys, seed):
    rng = np.random.default_rng(seed)
    pool = rng.integers(0, 2**32, size=(keys, 4), dtype=np.uint64)
    pool[:, 0] %= 8  # few hosts: keys differ in the low words too
    pick = rng.integers(0, keys, size=n)
    rows = np.zeros(n, dtype=ROW_DTYPE)
    for j, f in enumerate(("host_id", "pid", "tid", "func_id")):
        rows[f] = pool[pick, j]
    rows["count"] = rng.integers(1, 1000, size=n)
    rows["total_ns"] = rng.integers(0, 2**64 - 1, size=n, dtype=np.uint64)  # sums wrap in u64
    rows["min_ns"] = rng.integers(0, 2**40, size=n)
    rows["max_ns"] = rows["min_ns"] + rng.integers(0, 2**40, size=n)
    rows["err_count"] = rng.integers(0, 5, size=n)
    assert rows_equal(ctx.tally_merge(rows), plain_merge(rows))
