"""The all-cores CPU baseline runs the oracle on disjoint stream subsets in
host threads and merges the results; on traces whose streams pair
independently that must equal the plain single-threaded oracle exactly, and
traces with per-CPU buffers or device activity must fall back to one thread
(their pairing crosses streams)."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import tracegen as tg


def _same(a, b):
    assert a.code == b.code == oracle.OK
    assert a.diag == b.diag
    for x, y in ((a.rows, b.rows), (a.intervals, b.intervals), (a.dev_rows, b.dev_rows)):
        assert len(x) == len(y) and all(np.array_equal(x[f], y[f]) for f in x.dtype.names)


@pytest.mark.parametrize("threads", [2, 3, 7])
def test_threaded_oracle_equals_the_plain_oracle(threads):
    b = tg.generate(tg.preset("large", total_calls=200_000, n_hosts=2, pids_per_host=2, tids_per_pid=4,
                              p_drop=0.002, p_sample=0.02, seed=31, packet_bytes=2048))[0]
    _same(oracle.run_threads(b, threads), oracle.run(b))
    sub = [1, 4, 5, 14]
    _same(oracle.run_threads(b, threads, streams=sub), oracle.run(b, streams=sub))


def test_threaded_oracle_keeps_cross_stream_pairing_on_one_thread():
    d = tg.generate(tg.preset("device", total_calls=4_000, n_hosts=1, pids_per_host=2, tids_per_pid=2,
                              n_device_streams=3, seed=32))[0]
    p = tg.generate(tg.preset("large", total_calls=6_000, n_hosts=1, pids_per_host=2, tids_per_pid=2, n_cpus=2,
                              slice_ns=20_000.0, packet_bytes=4096, seed=33))[0]
    for t in (d, p):
        _same(oracle.run_threads(t, 4), oracle.run(t))
