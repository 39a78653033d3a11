"""The standard (forward-increment) construction on the GPU against the oracle.

Bars as in test_gpu_parity: FP64 points and estimates within 1e-12 x
max(|oracle|, mean |per-point value|) (points times max(1, n/64)); MIXED
against FP64 within 0.1 SE per Greek.  Tile sizes are
chosen so that one thread walks a whole path (d = 16) and so that several
threads split a path's dates into blocks (d = 200, 365).
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
    h = q.qmccpw_plan(device=0, d_max=366, r_max=16, seed=SEED)
    yield h
    q.qmccpw_free(h)


def scale_of(c, count=256):
    pts = oracle.point_values(SEED, c.type, c.d, c.K, c.T, c.S0, c.r, c.sigma, W.STD, 0, 0, count)
    return np.mean(np.abs(pts), axis=0)


@pytest.mark.parametrize("typ,d", [(0, 16), (1, 64), (2, 200), (3, 365), (0, 2), (2, 1)])
def test_forward_points_fp64_against_oracle(q, plan, typ, d):
    k0, count, rep = 321, 700, 2       # several tiles, the last ragged
    ref = oracle.point_values(SEED, typ, d, 100.0, 1.0, 100.0, 0.05, 0.25, W.STD, rep, k0, count)
    got = q.qmccpw_point_values(plan, typ, d, 100.0, 1.0, 100.0, 0.05, 0.25, W.STD, q.QMCCPW_FP64, rep, k0, count)
    scale = np.mean(np.abs(ref), axis=0)
    bound = RTOL64 * max(1.0, (d - 1) / 64.0) * np.maximum(np.abs(ref), scale)
    assert np.all(np.abs(got - ref) <= bound), np.max(np.abs(got - ref) / np.maximum(np.abs(ref), scale))


@pytest.mark.parametrize("typ,d,N,R", [(0, 16, 2 ** 12, 4), (2, 100, 3000, 3), (1, 257, 2 ** 11, 2)])
def test_forward_estimator_fp64_against_oracle(q, plan, typ, d, N, R):
    c = W.Contract(typ, d, 105.0, 0.75, 100.0, 0.03, 0.3, N, R, W.STD)
    mean, se, per = oracle.greeks(SEED, c.type, c.d, c.K, c.T, c.S0, c.r, c.sigma, W.STD, N, R)
    m, s, p = q.qmccpw_greeks(plan, c.type, c.d, c.K, c.T, c.S0, c.r, c.sigma, N, R, W.STD, q.QMCCPW_FP64)
    scale = scale_of(c)
    assert np.all(np.abs(p - per) <= RTOL64 * np.maximum(np.abs(per), scale))
    assert np.all(np.abs(m - mean) <= RTOL64 * np.maximum(np.abs(mean), scale))


def test_forward_mixed_against_fp64(q, plan):
    cs = [W.Contract(t, d, K, 1.0, 100.0, 0.05, 0.2, 2 ** 18, 16, W.STD)
          for t in (W.ARITH, W.BINARY, W.LOOKBACK) for d, K in ((64, 100.0), (200, 110.0))]
    m32 = q.qmccpw_greeks_batch(plan, cs, q.QMCCPW_MIXED)
    m64 = q.qmccpw_greeks_batch(plan, cs, q.QMCCPW_FP64)
    for c, (a, _, _), (b, s, _) in zip(cs, m32, m64):
        assert np.all(np.abs(a - b) <= 0.1 * s), (c.label(), (np.abs(a - b) / s).tolist())


def test_forward_in_a_mixed_batch_equals_alone(q, plan):
    cs = [W.Contract(W.ARITH, 64, 100.0, 1.0, 100.0, 0.05, 0.2, 4096, 3, W.STD),
          W.Contract(W.BINARY, 64, 100.0, 1.0, 100.0, 0.05, 0.2, 2000, 2, W.BB),
          W.Contract(W.LOOKBACK, 40, 95.0, 0.5, 100.0, 0.02, 0.3, 3000, 2, W.PCA),
          W.Contract(W.GEOMETRIC, 300, 100.0, 2.0, 100.0, 0.04, 0.25, 1500, 2, W.STD)]
    for prec in (q.QMCCPW_FP64, q.QMCCPW_MIXED, q.QMCCPW_MIXED_TC_BF16X3):
        batch = q.qmccpw_greeks_batch(plan, cs, prec)
        for c, (_, _, p) in zip(cs, batch):
            _, _, p0 = q.qmccpw_greeks(plan, c.type, c.d, c.K, c.T, c.S0, c.r, c.sigma, c.N, c.R, c.construction, prec)
            assert np.array_equal(p0, p), (prec, c.label())
    b = q.Batch(plan, cs, q.QMCCPW_MIXED)
    try:
        assert b.launch_count() == 5  # bridge, standard, PCA grids, the reduction, the statistics
    finally:
        b.free()


def test_forward_geometric_asian_closed_form_on_gpu(q, plan):
    """The whole GPU estimator (FP64) under the standard construction against
    the discretely monitored geometric-Asian closed form (the same pin the
    oracle meets), within 4 SE."""
    import test_oracle_cpw as cpw
    S0, K, r, sig, T, d = 100.0, 100.0, 0.05, 0.2, 1.0, 16
    p, dl, gm = cpw.geometric_asian_call(S0, K, r, sig, T, d)
    vg = cpw.geometric_vega(S0, K, r, sig, T, d)
    m, s, _ = q.qmccpw_greeks(plan, W.GEOMETRIC, d, K, T, S0, r, sig, 2 ** 14, 16, W.STD, q.QMCCPW_FP64)
    for g, ref in enumerate((p, dl, vg, gm)):
        assert abs(m[g] - ref) <= 4.0 * s[g] + 1e-9 * abs(ref), (g, m[g], ref, s[g])
