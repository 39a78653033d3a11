"""Device-resident serving loop: every request's result equals the result of
the same contract computed alone (bit-identical: a contract's tiles and
their reduction order do not depend on what else runs), with requests
arriving from several threads while earlier ones are on the GPU, admitted
by device memory; the kernel leaves on its idle limit and is launched again
when work arrives, losing no work item."""
import threading
import time

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
        # 256 KiB of device scratch holds a few requests at a time (the largest,
        # d = 365 in FP64, about 66 KB): the rest wait for admission
        q.qmccpw_server_start(plan, precision=precision, max_inflight=8, max_inflight_bytes=1 << 18)
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
        assert stats["launches"] >= 1 and stats["inflight"] == 0 and stats["pending"] == 0
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


def test_tensor_core_precisions_are_not_served(q):
    plan = q.qmccpw_plan(device=0, d_max=65, r_max=8, seed=W.SCRAMBLE_SEED)
    try:
        for prec in (2, 3):
            with pytest.raises(q.QmcCpwError) as e:
                q.qmccpw_server_start(plan, precision=prec)
            assert e.value.code == q.QMCCPW_ERR_UNSUPPORTED
    finally:
        q.qmccpw_free(plan)


@pytest.mark.parametrize("precision", [0, 1])
def test_idle_limit_runs_out_and_the_kernel_is_launched_again(q, precision):
    """A 2 ms idle limit: after each burst the kernel's CTAs wait for a
    published work item, the limit runs out and the launch ends (idle_exits);
    the next burst launches it again, and the work items the leaving CTAs
    held are handed out first.  Every result is the one computed alone."""
    plan = q.qmccpw_plan(device=0, d_max=366, r_max=8, seed=W.SCRAMBLE_SEED)
    try:
        cs = mix(12, 31 + precision)
        alone = [q.qmccpw_greeks(plan, c.type, c.d, c.K, c.T, c.S0, c.r, c.sigma, c.N, c.R, c.construction, precision)
                 for c in cs]
        q.qmccpw_server_start(plan, precision=precision, idle_limit_us=2000)
        got = []
        for burst in range(3):
            part = cs[4 * burst:4 * burst + 4]
            tickets = [q.qmccpw_submit(plan, c) for c in part]
            got += [q.qmccpw_wait(plan, t, c.R, 60000) for t, c in zip(tickets, part)]
            deadline = time.time() + 5.0
            while q.qmccpw_server_get_stats(plan)["running"] and time.time() < deadline:
                time.sleep(0.005)
            st = q.qmccpw_server_get_stats(plan)
            assert st["running"] == 0, st
            # every launch so far ended on the idle limit (more than one per burst
            # only if a gap between two submissions passed the limit)
            assert st["idle_exits"] >= burst + 1 and st["launches"] == st["idle_exits"], st
        t0 = time.time()
        q.qmccpw_server_stop(plan)
        assert time.time() - t0 < 5.0
        for c, (m, s, p), (m1, s1, p1) in zip(cs, got, alone):
            assert np.array_equal(p, p1), c.label()
            assert np.array_equal(m, m1) and np.array_equal(s, s1)
    finally:
        q.qmccpw_free(plan)


def test_stop_ends_a_waiting_kernel(q):
    """With a long idle limit the kernel stays up between requests; stop ends it
    at its next wait (every wait also checks the stop word)."""
    plan = q.qmccpw_plan(device=0, d_max=65, r_max=8, seed=W.SCRAMBLE_SEED)
    try:
        c = W.Contract(W.ARITH, 64, 100.0, 1.0, 100.0, 0.05, 0.2, 2 ** 12, 4, W.BB)
        q.qmccpw_server_start(plan, precision=1, idle_limit_us=5000000)
        q.qmccpw_wait(plan, q.qmccpw_submit(plan, c), c.R, 60000)
        time.sleep(0.05)
        st = q.qmccpw_server_get_stats(plan)
        assert st["running"] == 1 and st["idle_exits"] == 0
        t0 = time.time()
        q.qmccpw_server_stop(plan)
        assert time.time() - t0 < 2.0
    finally:
        q.qmccpw_free(plan)


def test_construction_mask(q):
    """A MIXED server started for bridge contracts only runs the kernel
    without the PCA product and refuses the other constructions; results as
    alone."""
    plan = q.qmccpw_plan(device=0, d_max=130, r_max=8, seed=W.SCRAMBLE_SEED)
    try:
        cs = [W.Contract(W.ARITH, d, 100.0, 1.0, 100.0, 0.05, 0.2, 3000 + 7 * d, 4, W.BB) for d in (16, 64, 100, 129)]
        alone = [q.qmccpw_greeks(plan, c.type, c.d, c.K, c.T, c.S0, c.r, c.sigma, c.N, c.R, c.construction, 1)
                 for c in cs]
        q.qmccpw_server_start(plan, precision=1, constructions=[W.BB])
        with pytest.raises(q.QmcCpwError) as e:
            q.qmccpw_submit(plan, W.Contract(W.ARITH, 64, 100.0, 1.0, 100.0, 0.05, 0.2, 1024, 4, W.PCA))
        assert e.value.code == q.QMCCPW_ERR_UNSUPPORTED
        got = [q.qmccpw_wait(plan, q.qmccpw_submit(plan, c), c.R, 60000) for c in cs]
        q.qmccpw_server_stop(plan)
        for c, (m, s, p), (m1, s1, p1) in zip(cs, got, alone):
            assert np.array_equal(p, p1), c.label()
    finally:
        q.qmccpw_free(plan)


def test_admission_refuses_a_request_beyond_the_scratch_and_wait_times_out(q):
    """A request whose work-item slots alone pass max_inflight_bytes is refused
    with OOM at submission (nothing is queued); qmccpw_wait on an unfinished
    request returns TIMEOUT and leaves the ticket collectable; requests that
    fit run as usual."""
    plan = q.qmccpw_plan(device=0, d_max=366, r_max=16, seed=W.SCRAMBLE_SEED)
    try:
        q.qmccpw_server_start(plan, precision=q.QMCCPW_MIXED, max_inflight_bytes=8 << 20)
        big = W.Contract(W.ARITH, 64, 100.0, 1.0, 100.0, 0.05, 0.2, 2 ** 26, 16, W.BB)   # 2^18 items: 8 MiB + 512 B
        with pytest.raises(q.QmcCpwError) as e:
            q.qmccpw_submit(plan, big)
        assert e.value.code == q.QMCCPW_ERR_OOM
        long = W.Contract(W.ARITH, 365, 100.0, 1.0, 100.0, 0.05, 0.2, 2 ** 22, 16, W.BB)  # 4 MiB, ~0.1 s of work
        t = q.qmccpw_submit(plan, long)
        with pytest.raises(q.QmcCpwError) as e:
            q.qmccpw_wait(plan, t, long.R, 0)
        assert e.value.code == q.QMCCPW_ERR_TIMEOUT
        mean, se, per = q.qmccpw_wait(plan, t, long.R, 120000)
        assert np.all(np.isfinite(per)) and per.shape == (long.R, 4)
        small = W.Contract(W.BINARY, 16, 100.0, 1.0, 100.0, 0.05, 0.2, 2 ** 12, 4, W.BB)
        m2, s2, p2 = q.qmccpw_wait(plan, q.qmccpw_submit(plan, small), small.R, 60000)
        q.qmccpw_server_stop(plan)
        ref = q.qmccpw_greeks_batch(plan, [long, small], q.QMCCPW_MIXED)
        assert np.array_equal(per, ref[0][2]) and np.array_equal(p2, ref[1][2])
    finally:
        q.qmccpw_free(plan)
