"""Tensor-core PCA (tcgen05, bf16 / tf32 hi + lo split) against the oracle and
the FP64 GPU path.

The leading product z_hi Ahat_hi is exact (hi parts on fixed grids), so the
split only adds rounding noise of the lo parts: |z - z_hi - z_lo| <= 2^-15
(bf16: |z_lo| <= 2^-6, 8 significant bits) or 2^-21 (tf32: |z_lo| <= 2^-9,
11 bits).  Ahat is one fixed matrix whose rounding no averaging removes: bf16
carries it in three parts (~2^-23), tf32 in two (<= 2^-20).  The per-point
bars below are derived from the z widths; the estimator must show no bias
beyond the float floor the MIXED path has.
"""
import numpy as np
import pytest

import oracle
import point_bounds
import workloads as W

pytestmark = pytest.mark.gpu
SEED = W.SCRAMBLE_SEED


@pytest.fixture(scope="module")
def q():
    from paper_2209_11337_gb300 import build, qmccpw
    build.build()
    oracle.build()
    return qmccpw


@pytest.fixture(scope="module")
def plan(q):
    h = q.qmccpw_plan(device=0, d_max=258, r_max=32, seed=SEED)
    yield h
    q.qmccpw_free(h)


def check_points(q, plan, prec, typ, d, k0, count, rep):
    """Every point and Greek within the bar derived from the split widths and
    the conditional formulas (point_bounds)."""
    ref = oracle.point_values(SEED, typ, d, 100.0, 1.0, 100.0, 0.05, 0.25, W.PCA, rep, k0, count)
    got = q.qmccpw_point_values(plan, typ, d, 100.0, 1.0, 100.0, 0.05, 0.25, W.PCA, prec, rep, k0, count)
    bar = point_bounds.bars(ref, typ, d, 100.0, 1.0, 100.0, 0.05, 0.25, W.PCA, prec)
    err = np.abs(got - ref)
    bad = ~(err <= bar)  # a NaN fails too
    assert not bad.any(), (np.argwhere(bad)[:5].tolist(), got[bad][:5], ref[bad][:5], bar[bad][:5])


@pytest.mark.parametrize("prec", [2, 3])
@pytest.mark.parametrize("typ,d,k0", [(0, 64, 1000), (1, 64, 1000), (2, 64, 1000), (3, 33, 1000), (0, 2, 1000),
                                      (2, 17, 1000), (1, 65, 1000), (0, 64, 2 ** 31 - 150), (1, 40, 2 ** 31 - 7)])
def test_tc_point_values_against_oracle(q, plan, prec, typ, d, k0):
    """300 points: three tiles of 128, the last one ragged; two cases put the
    points across index 2^31 (the Gray code's top bit)."""
    check_points(q, plan, prec, typ, d, k0, 300, 3)


@pytest.mark.parametrize("prec", [2, 3])
@pytest.mark.parametrize("typ,d,k0", [(0, 66, 77), (1, 100, 77), (2, 129, 77), (3, 130, 77), (3, 200, 77),
                                      (0, 257, 77), (2, 257, 77), (1, 150, 2 ** 31 - 60)])
def test_tc_streamed_point_values_against_oracle(q, plan, prec, typ, d, k0):
    """d > 65: Ahat streamed in K-chunks (N = K = 256); tf32 beyond d = 129
    builds Z in two K-halves; two tiles, the second ragged."""
    check_points(q, plan, prec, typ, d, k0, 200, 1)


def greek_scale(c):
    pts = oracle.point_values(SEED, c.type, c.d, c.K, c.T, c.S0, c.r, c.sigma, W.PCA, 0, 0, 1024)
    return np.mean(np.abs(pts), axis=0)


@pytest.mark.parametrize("prec", [2, 3])
def test_tc_estimator_unbiased_against_fp64(q, plan, prec):
    """The PCA contracts of the d=64, N=2^20, R=32 grid against FP64: every
    Greek within 0.1 SE.  Here the RQMC standard error is near 1e-8 relative
    (sigma = 0.1), so the split product must add no bias at that level: a
    tensor-core accumulation bias of ~1 ulp of |W~| per instruction showed
    here as 6-13 SE before the leading product was made exact, and a two-part
    bf16 Ahat (off by up to 2^-15) as up to 11 SE."""
    cs = [c for c in W.grid_d64() if c.construction == W.PCA]
    tc = q.qmccpw_greeks_batch(plan, cs, prec)
    f64 = q.qmccpw_greeks_batch(plan, cs, q.QMCCPW_FP64)
    bad = []
    for c, (m, _, _), (m64, s64, _) in zip(cs, tc, f64):
        err = np.abs(m - m64)
        if not np.all(err <= 0.1 * s64):  # a NaN fails too
            bad.append((c.label(), np.round(err / s64, 3).tolist()))
    assert not bad, bad


@pytest.mark.parametrize("prec", [2, 3])
def test_tc_streamed_estimator_against_fp64(q, plan, prec):
    cs = W.pca_stress(N=2 ** 16, R=8) + [W.Contract(W.GEOMETRIC, 100, 100.0, 1.0, 100.0, 0.05, 0.3, 2 ** 16, 8, W.PCA)]
    tc = q.qmccpw_greeks_batch(plan, cs, prec)
    f64 = q.qmccpw_greeks_batch(plan, cs, q.QMCCPW_FP64)
    for c, (m, _, _), (m64, s64, _) in zip(cs, tc, f64):
        assert np.all(np.abs(m - m64) <= 0.1 * s64), (c.label(), (np.abs(m - m64) / s64).tolist())


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


@pytest.mark.parametrize("prec", [2, 3])
def test_tc_three_segments_batch_equals_single(q, plan, prec):
    """A batch holding bridge, streamed (d > 65) and resident (d <= 65) PCA
    contracts: three launches, each result the same as alone."""
    cs = [W.Contract(W.ARITH, 257, 100.0, 1.0, 100.0, 0.05, 0.2, 3000, 2, W.PCA),
          W.Contract(W.BINARY, 64, 100.0, 1.0, 100.0, 0.05, 0.2, 2000, 3, W.BB),
          W.Contract(W.LOOKBACK, 100, 105.0, 1.0, 100.0, 0.05, 0.3, 1000, 2, W.PCA),
          W.Contract(W.ARITH, 33, 95.0, 0.5, 100.0, 0.02, 0.2, 4096, 2, W.PCA)]
    batch = q.qmccpw_greeks_batch(plan, cs, prec)
    for c, (_, _, p) in zip(cs, batch):
        _, _, p0 = q.qmccpw_greeks(plan, c.type, c.d, c.K, c.T, c.S0, c.r, c.sigma, c.N, c.R, c.construction, prec)
        assert np.array_equal(p0, p)
    b = q.Batch(plan, cs, prec)
    try:
        assert b.launch_count() == 5  # three fused grids, the reduction, the statistics
    finally:
        b.free()


def test_tc_precision_runs_bridge_contracts_as_mixed_and_rejects_large_d(q, plan):
    c = W.Contract(W.ARITH, 64, 100.0, 1.0, 100.0, 0.05, 0.2, 1024, 2, W.BB)
    tc = q.qmccpw_greeks(plan, c.type, c.d, c.K, c.T, c.S0, c.r, c.sigma, c.N, c.R, W.BB, 2)
    mixed = q.qmccpw_greeks(plan, c.type, c.d, c.K, c.T, c.S0, c.r, c.sigma, c.N, c.R, W.BB, q.QMCCPW_MIXED)
    assert np.array_equal(tc[2], mixed[2])
    for prec, d in ((3, 258), (2, 258)):  # both splits: d <= 257
        with pytest.raises(q.QmcCpwError) as e:
            q.qmccpw_greeks(plan, 0, d, 100.0, 1.0, 100.0, 0.05, 0.2, 1024, 2, W.PCA, prec)
        assert e.value.code == q.QMCCPW_ERR_UNSUPPORTED
