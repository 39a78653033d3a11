"""Runs that start at a later Sobol' point (qmccpw_contract.first_point).

The Sobol' sequence extends (Sec. 2.2.2): its first 2^m points are the
2^m-point set and the next 2^m complete the 2^(m+1)-point set, so an
estimate over N1 points can be refined by N2 more without recomputing the
first N1.  Checked three ways:
- FP64, every construction: the per-replicate estimates of a run over points
  F .. F+N-1 against the oracle's per-replicate sums over the same points
  (aligned and unaligned F, a ragged last tile);
- every precision: a run of N1 points from 0 combined with a run of N2 from
  N1 equals the run of N1 + N2 points from 0, replicate by replicate, up to
  the rounding of the combination (the points and their values are the same);
- the serving loop gives the batch call's result bit for bit for such a run,
  and a first_point + N beyond 2^32 is rejected.
"""
from dataclasses import replace

import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def q():
    from paper_2209_11337_gb300 import build, qmccpw
    build.build()
    return qmccpw


@pytest.fixture(scope="module")
def plan(q):
    h = q.qmccpw_plan(device=0, d_max=201, r_max=16, seed=W.SCRAMBLE_SEED)
    yield h
    q.qmccpw_free(h)


def point_scale(c, k0, count=256):
    """Mean |per-point value| of each Greek (the oracle's, points k0 ..): the
    scale of a Greek whose estimate is near 0."""
    pts = oracle.point_values(W.SCRAMBLE_SEED, c.type, c.d, c.K, c.T, c.S0, c.r, c.sigma, c.construction, 0, k0,
                              min(count, c.N))
    return np.mean(np.abs(pts), axis=0)


FP64_CASES = [
    (W.Contract(W.ARITH, 64, 100.0, 1.0, 100.0, 0.05, 0.2, 3000, 4, W.BB), 4096),      # aligned F, ragged N
    (W.Contract(W.BINARY, 17, 105.0, 0.5, 100.0, 0.02, 0.3, 2048, 3, W.PCA), 1000),    # unaligned F
    (W.Contract(W.LOOKBACK, 100, 95.0, 1.0, 100.0, 0.05, 0.25, 777, 2, W.STD), 2 ** 12),
    (W.Contract(W.ARITH, 33, 100.0, 1.0, 100.0, 0.05, 0.2, 1024, 2, W.PCA_LEAD), 517),
    (W.Contract(W.LOOKBACK, 16, 110.0, 1.0, 100.0, 0.05, 0.3, 600, 2, W.BB_LEAD), 2 ** 16),
]


@pytest.mark.parametrize("c,F", FP64_CASES, ids=lambda x: x.label() if hasattr(x, "label") else str(x))
def test_fp64_offset_run_matches_oracle_sums(q, plan, c, F):
    run = replace(c, first_point=F)
    (_, _, per), = q.qmccpw_greeks_batch(plan, [run], q.QMCCPW_FP64)
    sums = oracle.partial_sums(W.SCRAMBLE_SEED, c.type, c.d, c.K, c.T, c.S0, c.r, c.sigma, c.construction,
                               0, c.R, F, c.N)
    ref = sums / c.N
    bound = 1e-12 * np.maximum(np.abs(ref), point_scale(c, F))
    assert np.all(np.abs(per - ref) <= bound), (c.label(), F, per, ref)


SPLIT_CASES = [
    (W.Contract(W.ARITH, 64, 100.0, 1.0, 100.0, 0.05, 0.2, 2 ** 14, 4, W.BB), 2 ** 12, 1),
    (W.Contract(W.BINARY, 200, 100.0, 1.0, 100.0, 0.05, 0.3, 2 ** 13, 4, W.BB), 2 ** 12, 1),
    (W.Contract(W.LOOKBACK, 64, 90.0, 1.0, 100.0, 0.05, 0.1, 2 ** 14, 4, W.PCA), 2 ** 12, 2),
    (W.Contract(W.ARITH, 100, 110.0, 1.0, 100.0, 0.05, 0.3, 2 ** 13, 4, W.PCA), 2 ** 11, 3),
    (W.Contract(W.ARITH, 64, 100.0, 1.0, 100.0, 0.05, 0.2, 2 ** 13, 4, W.BB_LEAD), 3000, 1),
    (W.Contract(W.BINARY, 40, 100.0, 1.0, 100.0, 0.05, 0.2, 2 ** 13, 4, W.STD), 2 ** 12, 0),
]


@pytest.mark.parametrize("c,N1,prec", SPLIT_CASES,
                         ids=lambda x: x.label() if hasattr(x, "label") else str(x))
def test_two_runs_combine_to_the_longer_run(q, plan, c, N1, prec):
    (_, _, whole), = q.qmccpw_greeks_batch(plan, [c], prec)
    (_, _, first), = q.qmccpw_greeks_batch(plan, [replace(c, N=N1)], prec)
    (_, _, rest), = q.qmccpw_greeks_batch(plan, [replace(c, N=c.N - N1, first_point=N1)], prec)
    combined = (N1 * first + (c.N - N1) * rest) / c.N
    bound = 1e-13 * np.maximum(np.abs(whole), point_scale(c, 0))
    assert np.all(np.abs(combined - whole) <= bound), (c.label(), combined, whole)


def test_serving_loop_runs_offsets_like_the_batch_call(q):
    plan = q.qmccpw_plan(device=0, d_max=130, r_max=16, seed=W.SCRAMBLE_SEED)
    try:
        cs = [replace(c, first_point=F) for c, F in
              ((W.Contract(W.ARITH, 100, 100.0, 1.0, 100.0, 0.05, 0.2, 2 ** 13, 4, W.BB), 2 ** 12),
               (W.Contract(W.BINARY, 64, 95.0, 1.0, 100.0, 0.05, 0.3, 5000, 4, W.BB), 3000))]
        ref = q.qmccpw_greeks_batch(plan, cs, q.QMCCPW_MIXED)
        q.qmccpw_server_start(plan, precision=q.QMCCPW_MIXED, constructions=[q.QMCCPW_BB])
        try:
            tickets = [q.qmccpw_submit(plan, c) for c in cs]
            for c, t, (m, s, per) in zip(cs, tickets, ref):
                gm, gs, gper = q.qmccpw_wait(plan, t, c.R, 60000)
                assert np.array_equal(gper, per) and np.array_equal(gm, m), c.label()
        finally:
            q.qmccpw_server_stop(plan)
    finally:
        q.qmccpw_free(plan)


def test_offset_beyond_the_sequence_is_rejected(q, plan):
    c = W.Contract(W.ARITH, 16, 100.0, 1.0, 100.0, 0.05, 0.2, 2 ** 12, 2, W.BB, first_point=2 ** 32 - 2 ** 11)
    with pytest.raises(q.QmcCpwError) as e:
        q.qmccpw_greeks_batch(plan, [c], q.QMCCPW_MIXED)
    assert e.value.code == q.QMCCPW_ERR_INVALID_ARG
