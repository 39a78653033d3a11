"""Tile autotuner: picks a power-of-two tile per (precision, construction, d),
and the estimator stays at oracle parity with whatever tile is in use."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu
SEED = W.SCRAMBLE_SEED


@pytest.fixture(scope="module")
def q():
    from paper_2209_11337_gb300 import build, qmccpw
    build.build()
    oracle.build()
    return qmccpw


def test_autotune_then_parity(q):
    plan = q.qmccpw_plan(device=0, d_max=366, r_max=8, seed=SEED)
    try:
        sample = [W.Contract(W.ARITH, 16, 100.0, 1.0, 100.0, 0.05, 0.2, 2 ** 12, 4, W.BB),
                  W.Contract(W.BINARY, 200, 100.0, 1.0, 100.0, 0.05, 0.2, 2 ** 12, 4, W.BB),
                  W.Contract(W.LOOKBACK, 64, 100.0, 1.0, 100.0, 0.05, 0.2, 2 ** 12, 4, W.PCA)]
        for prec in (q.QMCCPW_FP64, q.QMCCPW_MIXED):
            q.qmccpw_autotune(plan, sample, prec)
            for c in sample:
                P = q.qmccpw_tuning_get(plan, prec, c.construction, c.d)
                assert P in (32, 64, 128, 256)
        # FP64 with the tuned tiles still matches the oracle at 1e-12
        for c in sample:
            c = W.with_size(c, N=3000, R=3)
            _, _, per = q.qmccpw_greeks(plan, c.type, c.d, c.K, c.T, c.S0, c.r, c.sigma, c.N, c.R,
                                        c.construction, q.QMCCPW_FP64)
            _, _, ref = oracle.greeks(SEED, c.type, c.d, c.K, c.T, c.S0, c.r, c.sigma, c.construction, c.N, c.R)
            scale = np.mean(np.abs(oracle.point_values(SEED, c.type, c.d, c.K, c.T, c.S0, c.r, c.sigma,
                                                       c.construction, 0, 0, 256)), axis=0)
            assert np.all(np.abs(per - ref) <= 1e-12 * np.maximum(np.abs(ref), scale))
    finally:
        q.qmccpw_free(plan)


def test_tuning_set_get_and_reject(q):
    plan = q.qmccpw_plan(device=0, d_max=65, r_max=8, seed=SEED)
    try:
        c = W.Contract(W.ARITH, 64, 100.0, 1.0, 100.0, 0.05, 0.2, 5000, 3, W.BB)
        base = q.qmccpw_greeks(plan, c.type, c.d, c.K, c.T, c.S0, c.r, c.sigma, c.N, c.R, W.BB, q.QMCCPW_MIXED)
        default = q.qmccpw_tuning_get(plan, q.QMCCPW_MIXED, W.BB, 64)
        q.qmccpw_tuning_set(plan, q.QMCCPW_MIXED, W.BB, 64, 64)
        assert q.qmccpw_tuning_get(plan, q.QMCCPW_MIXED, W.BB, 64) == 64
        small = q.qmccpw_greeks(plan, c.type, c.d, c.K, c.T, c.S0, c.r, c.sigma, c.N, c.R, W.BB, q.QMCCPW_MIXED)
        # same points, other tile: the same estimate up to float summation order
        assert np.allclose(small[0], base[0], rtol=1e-6, atol=1e-9)
        q.qmccpw_tuning_set(plan, q.QMCCPW_MIXED, W.BB, 64, 0)
        assert q.qmccpw_tuning_get(plan, q.QMCCPW_MIXED, W.BB, 64) == default
        for bad in (48, 512, 16):
            with pytest.raises(q.QmcCpwError):
                q.qmccpw_tuning_set(plan, q.QMCCPW_MIXED, W.BB, 64, bad)
    finally:
        q.qmccpw_free(plan)
