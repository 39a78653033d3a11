"""Conditioning on the leading coordinate of the whole path (constructions
BB_LEAD and PCA_LEAD, with a Newton switch point per point) on the GPU
against the oracle.

Bars as in test_gpu_parity: FP64 points and estimates within 1e-12 x
max(|oracle|, mean |per-point value|) (points times max(1, d/64)); MIXED
against FP64 within 0.1 SE per Greek.
"""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu
SEED = W.SCRAMBLE_SEED
RTOL64 = 1e-12


@pytest.fixture(scope="module")
def q():
    from paper_2209_11337_gb300 import build, qmccpw
    build.build()
    oracle.build()
    return qmccpw


@pytest.fixture(scope="module")
def plan(q):
    h = q.qmccpw_plan(device=0, d_max=300, r_max=16, seed=SEED)
    yield h
    q.qmccpw_free(h)


def scale_of(c, count=256):
    pts = oracle.point_values(SEED, c.type, c.d, c.K, c.T, c.S0, c.r, c.sigma, c.construction, 0, 0, count)
    return np.mean(np.abs(pts), axis=0)


@pytest.mark.parametrize("cons", [W.BB_LEAD, W.PCA_LEAD])
@pytest.mark.parametrize("typ,d", [(0, 16), (1, 64), (3, 33), (0, 2), (1, 1), (0, 130), (2, 16), (2, 64), (2, 1),
                                   (2, 130)])
def test_lead_points_fp64_against_oracle(q, plan, cons, typ, d):
    k0, count, rep = 55, 600, 1     # several tiles, the last ragged
    ref = oracle.point_values(SEED, typ, d, 100.0, 1.0, 100.0, 0.05, 0.25, cons, rep, k0, count)
    got = q.qmccpw_point_values(plan, typ, d, 100.0, 1.0, 100.0, 0.05, 0.25, cons, q.QMCCPW_FP64, rep, k0, count)
    scale = np.mean(np.abs(ref), axis=0)
    bound = RTOL64 * max(1.0, d / 64.0) * np.maximum(np.abs(ref), scale)
    assert np.all(np.abs(got - ref) <= bound), np.max(np.abs(got - ref) / np.maximum(np.abs(ref), scale))


@pytest.mark.parametrize("cons", [W.BB_LEAD, W.PCA_LEAD])
@pytest.mark.parametrize("typ,d,N,R", [(0, 16, 2 ** 12, 4), (1, 50, 3000, 3), (2, 40, 3000, 3)])
def test_lead_estimator_fp64_against_oracle(q, plan, cons, typ, d, N, R):
    c = W.Contract(typ, d, 104.0, 0.75, 100.0, 0.03, 0.3, N, R, cons)
    mean, se, per = oracle.greeks(SEED, c.type, c.d, c.K, c.T, c.S0, c.r, c.sigma, cons, N, R)
    m, s, p = q.qmccpw_greeks(plan, c.type, c.d, c.K, c.T, c.S0, c.r, c.sigma, N, R, cons, q.QMCCPW_FP64)
    scale = scale_of(c)
    assert np.all(np.abs(p - per) <= RTOL64 * np.maximum(np.abs(per), scale))
    assert np.all(np.abs(m - mean) <= RTOL64 * np.maximum(np.abs(mean), scale))


def test_lead_mixed_against_fp64(q, plan):
    cs = [W.Contract(t, d, K, 1.0, 100.0, 0.05, 0.2, 2 ** 16, 16, cons)
          for cons in (W.BB_LEAD, W.PCA_LEAD) for t in (W.ARITH, W.BINARY, W.GEOMETRIC, W.LOOKBACK)
          for d, K in ((16, 100.0), (64, 110.0))]
    m32 = q.qmccpw_greeks_batch(plan, cs, q.QMCCPW_MIXED)
    m64 = q.qmccpw_greeks_batch(plan, cs, q.QMCCPW_FP64)
    bad = []
    for c, (a, _, _), (b, s, _) in zip(cs, m32, m64):
        if not np.all(np.abs(a - b) <= 0.1 * s):  # a NaN fails too
            bad.append((c.label(), np.round(np.abs(a - b) / s, 3).tolist()))
    assert not bad, "\n".join(f"{lab}: {err}" for lab, err in bad)


def test_lead_batch_equals_alone(q, plan):
    cs = [W.Contract(W.ARITH, 40, 100.0, 1.0, 100.0, 0.05, 0.2, 3000, 2, W.BB_LEAD),
          W.Contract(W.BINARY, 64, 100.0, 1.0, 100.0, 0.05, 0.2, 2000, 2, W.BB),
          W.Contract(W.GEOMETRIC, 70, 95.0, 0.5, 100.0, 0.02, 0.3, 2500, 3, W.PCA_LEAD),
          W.Contract(W.ARITH, 33, 105.0, 1.0, 100.0, 0.05, 0.25, 1024, 2, W.PCA),
          W.Contract(W.LOOKBACK, 50, 110.0, 1.0, 100.0, 0.05, 0.3, 1500, 2, W.BB_LEAD)]
    for prec in (q.QMCCPW_FP64, q.QMCCPW_MIXED, q.QMCCPW_MIXED_TC_BF16X3):
        batch = q.qmccpw_greeks_batch(plan, cs, prec)
        for c, (_, _, p) in zip(cs, batch):
            _, _, p0 = q.qmccpw_greeks(plan, c.type, c.d, c.K, c.T, c.S0, c.r, c.sigma, c.N, c.R, c.construction, prec)
            assert np.array_equal(p0, p), (prec, c.label())

