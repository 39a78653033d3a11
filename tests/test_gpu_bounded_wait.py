"""Failure path of the tensor-core kernels' waits, made to run out on purpose
without a fault: a probe kernel waits with the kernels' own bounded poll loop
on an mbarrier that nothing arrives at; the wait must give up within its
limit, the kernel must record the timeout status and exit, and the context
must stay usable."""
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


def test_bounded_wait_gives_up_and_reports_timeout(q):
    t0 = time.perf_counter()
    status = q.qmccpw_selftest_bounded_wait(0, 20000)  # 20 ms limit
    wall = time.perf_counter() - t0
    assert status == q.QMCCPW_ERR_TIMEOUT
    assert wall < 5.0
    # the context is still usable: a normal call right after succeeds
    plan = q.qmccpw_plan(device=0, d_max=65, r_max=4, seed=W.SCRAMBLE_SEED)
    try:
        c = W.Contract(W.ARITH, 64, 100.0, 1.0, 100.0, 0.05, 0.2, 1024, 2, W.PCA)
        m, s, _ = q.qmccpw_greeks(plan, c.type, c.d, c.K, c.T, c.S0, c.r, c.sigma, c.N, c.R, W.PCA,
                                  q.QMCCPW_MIXED_TC_BF16X3)
        assert np.all(np.isfinite(m)) and np.all(np.isfinite(s))
    finally:
        q.qmccpw_free(plan)


def test_bounded_wait_rejects_bad_limits(q):
    with pytest.raises(q.QmcCpwError) as e:
        q.qmccpw_selftest_bounded_wait(0, 0)
    assert e.value.code == q.QMCCPW_ERR_INVALID_ARG
