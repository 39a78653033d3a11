"""Continuous-batching service: every request's result equals the result of
the same contract computed alone (bit-identical: a contract's tiles and
their reduction order do not depend on the batch), with requests arriving
from several threads while earlier batches are on the GPU."""
import threading

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def q():
    from paper_2209_11337_gb300 import build, qmccpw
    build.build()
    return qmccpw


def mix(count, seed):
    book = W.book(count=count, seed=seed, R=4)
    out = []
    for i, c in enumerate(book):
        N = min(c.N, 2 ** 13) + (i % 3) * 17               # ragged sizes
        out.append(W.Contract(c.type, c.d, c.K, c.T, c.S0, c.r, c.sigma, N, 2 + i % 3,
                              W.PCA if i % 4 == 0 else W.BB))
    return out


@pytest.mark.parametrize("precision", [0, 1])
def test_results_same_alone_and_in_the_mix(q, precision):
    plan = q.qmccpw_plan(device=0, d_max=366, r_max=8, seed=W.SCRAMBLE_SEED)
    try:
        cs = mix(48, 11 + precision)
        alone = [q.qmccpw_greeks(plan, c.type, c.d, c.K, c.T, c.S0, c.r, c.sigma, c.N, c.R, c.construction, precision)
                 for c in cs]
        q.qmccpw_server_start(plan, precision=precision, max_inflight=3, max_batch_contracts=7,
                              max_batch_bytes=1 << 22)
        tickets = [None] * len(cs)

        def submit(idx):
            for i in idx:
                tickets[i] = q.qmccpw_submit(plan, cs[i])

        threads = [threading.Thread(target=submit, args=(range(k, len(cs), 2),)) for k in range(2)]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
        got = [q.qmccpw_wait(plan, tickets[i], cs[i].R, 120000) for i in range(len(cs))]
        stats = q.qmccpw_server_get_stats(plan)
        q.qmccpw_server_stop(plan)
        for c, (m, s, p), (m1, s1, p1) in zip(cs, got, alone):
            assert np.array_equal(p, p1), c.label()
            assert np.array_equal(m, m1) and np.array_equal(s, s1)
        assert stats["completed"] == len(cs) and stats["failed"] == 0
        assert stats["batches"] >= len(cs) // 7
        assert stats["point_dates"] == sum(c.N * c.R * c.d for c in cs)
    finally:
        q.qmccpw_free(plan)


def test_poll_semantics_and_errors(q):
    plan = q.qmccpw_plan(device=0, d_max=65, r_max=8, seed=W.SCRAMBLE_SEED)
    try:
        c = W.Contract(W.ARITH, 64, 100.0, 1.0, 100.0, 0.05, 0.2, 2 ** 12, 4, W.BB)
        with pytest.raises(q.QmcCpwError):
            q.qmccpw_submit(plan, c)                      # no server yet
        q.qmccpw_server_start(plan, precision=1)
        with pytest.raises(q.QmcCpwError):
            q.qmccpw_server_start(plan, precision=1)      # already running
        bad = W.Contract(W.ARITH, 99, 100.0, 1.0, 100.0, 0.05, 0.2, 16, 4, W.BB)   # d > d_max
        with pytest.raises(q.QmcCpwError) as e:
            q.qmccpw_submit(plan, bad)
        assert e.value.code == q.QMCCPW_ERR_INVALID_ARG
        t = q.qmccpw_submit(plan, c)
        res = None
        for _ in range(200000):
            res = q.qmccpw_poll(plan, t, c.R)
            if res is not None:
                break
        assert res is not None
        with pytest.raises(q.QmcCpwError):
            q.qmccpw_poll(plan, t, c.R)                   # collected tickets are forgotten
        q.qmccpw_server_stop(plan)
        q.qmccpw_server_stop(plan)                        # idempotent
        ref = q.qmccpw_greeks(plan, c.type, c.d, c.K, c.T, c.S0, c.r, c.sigma, c.N, c.R, c.construction, 1)
        assert np.array_equal(res[2], ref[2])
    finally:
        q.qmccpw_free(plan)
