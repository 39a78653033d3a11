"""Tensor-core PCA (tcgen05, 3-term bf16 / tf32 split) against the oracle and
the FP64 GPU path.

The split product carries the PCA factor to about 2^-17 (bf16: 8 + 8 bits)
or 2^-22 (tf32: 11 + 11 bits) relative, and z likewise; the bars below are
derived from those widths.  Results are stated per Greek by the bench.
"""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu
SEED = W.SCRAMBLE_SEED
SPLIT_EPS = {2: 2.0 ** -16, 3: 2.0 ** -21}  # precision code -> relative width of the 3-term split


@pytest.fixture(scope="module")
def q():
    from paper_2209_11337_gb300 import build, qmccpw
    build.build()
    oracle.build()
    return qmccpw


@pytest.fixture(scope="module")
def plan(q):
    h = q.qmccpw_plan(device=0, d_max=65, r_max=32, seed=SEED)
    yield h
    q.qmccpw_free(h)


@pytest.mark.parametrize("prec", [2, 3])
@pytest.mark.parametrize("typ,d", [(0, 64), (1, 64), (2, 64), (3, 33), (0, 2), (2, 17)])
def test_tc_point_values_against_oracle(q, plan, prec, typ, d):
    k0, count, rep = 1000, 300, 3     # 300 points: three tiles of 128, the last one ragged
    ref = oracle.point_values(SEED, typ, d, 100.0, 1.0, 100.0, 0.05, 0.25, W.PCA, rep, k0, count)
    got = q.qmccpw_point_values(plan, typ, d, 100.0, 1.0, 100.0, 0.05, 0.25, W.PCA, prec, rep, k0, count)
    scale = np.mean(np.abs(ref), axis=0)
    err = np.abs(got - ref) / np.maximum(np.abs(ref), scale)
    eps = SPLIT_EPS[prec]
    # a point's path mixes d terms of relative error ~eps; its values amplify by up to ~1/a
    assert np.median(err) < 50 * eps + 1e-6, (np.median(err, axis=0), np.max(err, axis=0))
    assert np.all(np.isfinite(got))


@pytest.mark.parametrize("prec", [2, 3])
def test_tc_estimator_against_fp64(q, plan, prec):
    cs = [c for c in W.grid_d64(N=2 ** 16, R=8) if c.construction == W.PCA][::3]
    tc = q.qmccpw_greeks_batch(plan, cs, prec)
    f64 = q.qmccpw_greeks_batch(plan, cs, q.QMCCPW_FP64)
    eps = SPLIT_EPS[prec]
    for c, (m, s, p), (m64, s64, p64) in zip(cs, tc, f64):
        scale = np.mean(np.abs(oracle.point_values(SEED, c.type, c.d, c.K, c.T, c.S0, c.r, c.sigma, W.PCA, 0, 0, 512)),
                        axis=0)
        bound = 0.1 * s64 + 20 * eps * scale
        assert np.all(np.abs(m - m64) <= bound), (c.label(), (np.abs(m - m64) / s64).tolist())


def test_tc_repeatable_and_batch_equals_single(q, plan):
    cs = [W.Contract(W.ARITH, 64, 100.0, 1.0, 100.0, 0.05, 0.2, 5000, 3, W.PCA),
          W.Contract(W.LOOKBACK, 40, 95.0, 0.5, 100.0, 0.02, 0.3, 2 ** 12, 2, W.PCA)]
    for prec in (2, 3):
        a = q.qmccpw_greeks_batch(plan, cs, prec)
        b = q.qmccpw_greeks_batch(plan, cs, prec)
        for (m1, _, p1), (m2, _, p2), c in zip(a, b, cs):
            assert np.array_equal(p1, p2)
            m0, _, p0 = q.qmccpw_greeks(plan, c.type, c.d, c.K, c.T, c.S0, c.r, c.sigma, c.N, c.R, W.PCA, prec)
            assert np.array_equal(p0, p1)


def test_tc_precision_runs_bridge_contracts_as_mixed_and_rejects_large_d(q, plan):
    c = W.Contract(W.ARITH, 64, 100.0, 1.0, 100.0, 0.05, 0.2, 1024, 2, W.BB)
    tc = q.qmccpw_greeks(plan, c.type, c.d, c.K, c.T, c.S0, c.r, c.sigma, c.N, c.R, W.BB, 2)
    mixed = q.qmccpw_greeks(plan, c.type, c.d, c.K, c.T, c.S0, c.r, c.sigma, c.N, c.R, W.BB, q.QMCCPW_MIXED)
    assert np.array_equal(tc[2], mixed[2])
    big = q.qmccpw_plan(device=0, d_max=100, r_max=4, seed=SEED)
    try:
        with pytest.raises(q.QmcCpwError) as e:
            q.qmccpw_greeks(big, 0, 100, 100.0, 1.0, 100.0, 0.05, 0.2, 1024, 2, W.PCA, 2)
        assert e.value.code == q.QMCCPW_ERR_UNSUPPORTED
    finally:
        q.qmccpw_free(big)
