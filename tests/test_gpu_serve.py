"""The serving loop on the GPU: every answer equals the oracle's, and the
device-memory cap refuses a trace that does not fit."""
from __future__ import annotations

import pytest

import oracle
import tracegen as tg
from tests._util import intervals_equal, rows_equal

pytestmark = pytest.mark.gpu


def test_served_answers_equal_the_oracle():
    from paper_2504_03683_b300.serve import Server, poisson_requests
    traces = [tg.generate(tg.preset("large", total_calls=c, n_hosts=1, pids_per_host=1, tids_per_pid=4, seed=70 + k,
                                    packet_bytes=4096))[0] for k, c in enumerate((2_000, 30_000, 9_000))]
    s = Server(0, 8 * 10**9)
    try:
        for t in traces:
            assert s.admit(t) is not None
        spans = [(r.t_min, r.t_max) for r in s.traces]
        reqs = poisson_requests(2000.0, 0.05, spans, seed=5)
        assert len(reqs) > 40
        for r in reqs:
            got = s.answer(r)
            if r.kind == "tally":
                assert rows_equal(got, oracle.run(traces[r.trace]).rows)
            else:
                assert intervals_equal(got, oracle.run(traces[r.trace], t0=r.t0, t1=r.t1).intervals)
        out = s.run(reqs)
        assert len(out) == len(reqs) and all(lat >= 0 for lat, _n in out)
    finally:
        s.close()


def test_admission_refuses_past_the_cap():
    from paper_2504_03683_b300.serve import Server
    small = tg.generate(tg.preset("large", total_calls=1_000, n_hosts=1, pids_per_host=1, tids_per_pid=2, seed=80,
                                  packet_bytes=4096))[0]
    big = tg.generate(tg.preset("large", total_calls=400_000, n_hosts=1, pids_per_host=1, tids_per_pid=2, seed=81,
                                packet_bytes=4096))[0]
    s = Server(0, 40 * 10**6)  # 40 MB: room for the small trace only
    try:
        assert s.admit(small) == 0
        assert s.admit(big) is None and s.refused == 1
        assert len(s.traces) == 1
    finally:
        s.close()
