"""GPU parity of the basket (several underlying assets, Sec. 6) through the C-ABI.

Bars:
  - FP64 single points: |gpu - oracle| <= 1e-12 * max(|oracle|, mean |value|)
    per Greek, times max(1, m d / 64) (a point sums m d exponentials of
    m-term combinations, and the binary gamma amplifies an error in ln X).
  - FP64 per-replicate estimates, means and standard errors: the same bar
    without the size factor (the per-replicate means average the points).
  - MIXED against FP64 on the same points: |mixed - fp64| <= 0.1 * SE(fp64)
    per Greek; per point within 2e-4 of the Greek's mean magnitude (float
    inverse normal, bridges and exponentials, 1e-7 relative each, through at
    most ~1/a^2 in the binary gamma).
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
    h = q.qmccpw_plan(device=0, d_max=520, r_max=32, seed=SEED)
    yield h
    q.qmccpw_free(h)


def corr_matrix(m, rho, seed):
    rng = np.random.default_rng(seed)
    C = np.full((m, m), rho)
    np.fill_diagonal(C, 1.0)
    if m > 2:
        E = rng.uniform(-0.1, 0.1, (m, m))
        E = 0.5 * (E + E.T)
        np.fill_diagonal(E, 0.0)
        E[0, :] = E[:, 0] = 0.0
        C = C + E
    return C


def basket(typ, d, m, K=100.0, sigma=0.25, seed=0):
    rng = np.random.default_rng(seed + 97 * m + d)
    w = rng.uniform(0.5, 1.5, m)
    return oracle.Basket(typ, d, K * float(np.sum(w)) / m, 1.0, 100.0, 0.05, sigma, w / m,
                         rng.uniform(0.85, 1.15, m), rng.uniform(0.6, 1.6, m), corr_matrix(m, 0.5, seed + m))


def close(gpu, ref, scale, rtol, what):
    bound = rtol * np.maximum(np.abs(ref), scale)
    bad = np.abs(np.asarray(gpu) - np.asarray(ref)) > bound
    assert not bad.any(), (what, np.argwhere(bad)[:5].tolist(), np.asarray(gpu)[bad][:5], np.asarray(ref)[bad][:5])


CASES = [(t, d, m) for t in (0, 1) for d, m in ((1, 1), (1, 3), (2, 2), (16, 1), (16, 3), (64, 4), (30, 8), (8, 5))]


@pytest.mark.parametrize("typ,d,m", CASES)
def test_basket_points_fp64(q, plan, typ, d, m):
    b = basket(typ, d, m)
    rep, k0, count = 3, 7000, 300                  # a ragged tile at an odd offset
    ref = oracle.basket_point_values(SEED, b, rep, k0, count)
    gpu = q.qmccpw_basket_point_values(plan, b, q.QMCCPW_FP64, rep, k0, count)
    close(gpu, ref, np.mean(np.abs(ref), axis=0), RTOL64 * max(1.0, m * d / 64), f"{typ}/{d}/{m}")


@pytest.mark.parametrize("typ,d,m,N", [(0, 16, 3, 1000), (1, 16, 3, 4096), (0, 64, 4, 2048), (1, 8, 8, 777),
                                       (0, 1, 2, 513)])
def test_basket_estimator_fp64(q, plan, typ, d, m, N):
    b = basket(typ, d, m, seed=5)
    R = 4
    rmean, rse, rper = oracle.basket_greeks(SEED, b, N, R)
    mean, se, per = q.qmccpw_basket_greeks(plan, b, N, R, q.QMCCPW_FP64)
    scale = np.mean(np.abs(oracle.basket_point_values(SEED, b, 0, 0, 128)), axis=0)
    close(per, rper, scale, RTOL64, "per replicate")
    close(mean, rmean, scale, RTOL64, "mean")
    close(se, rse, np.maximum(scale * 1e-3, rse), 1e-9, "se")


@pytest.mark.parametrize("typ,cons", [(0, W.BB), (1, W.BB)])
def test_single_asset_basket_equals_the_contract(q, plan, typ, cons):
    """m = 1: the basket kernel (Newton switch point) and the single-asset
    kernel (closed-form switch point) give the same FP64 estimate."""
    b = oracle.Basket(typ, 32, 104.0, 1.0, 100.0, 0.05, 0.3, [1.0], [1.0], [1.0], [[1.0]])
    N, R = 4096, 4
    mean, se, per = q.qmccpw_basket_greeks(plan, b, N, R, q.QMCCPW_FP64)
    cm, cse, cper = q.qmccpw_greeks(plan, typ, 32, 104.0, 1.0, 100.0, 0.05, 0.3, N, R, cons, q.QMCCPW_FP64)
    close(per, cper, np.abs(cm) + 1e-3, 1e-11, "single asset")


@pytest.mark.parametrize("typ,d,m", [(0, 16, 3), (1, 16, 3), (0, 64, 4), (1, 64, 4), (0, 30, 8), (1, 30, 8)])
def test_basket_mixed_within_a_tenth_of_a_standard_error(q, plan, typ, d, m):
    b = basket(typ, d, m, seed=11)
    N, R = 2 ** 15, 16
    m64, se64, _ = q.qmccpw_basket_greeks(plan, b, N, R, q.QMCCPW_FP64)
    m32, _, _ = q.qmccpw_basket_greeks(plan, b, N, R, q.QMCCPW_MIXED)
    err = np.abs(m32 - m64) / se64
    assert np.all(err <= 0.1), (err, m32, m64, se64)


@pytest.mark.parametrize("typ,d,m", [(0, 16, 3), (1, 64, 4), (0, 30, 8)])
def test_basket_mixed_points(q, plan, typ, d, m):
    b = basket(typ, d, m, seed=13)
    p64 = q.qmccpw_basket_point_values(plan, b, q.QMCCPW_FP64, 1, 0, 1000)
    p32 = q.qmccpw_basket_point_values(plan, b, q.QMCCPW_MIXED, 1, 0, 1000)
    scale = np.mean(np.abs(p64), axis=0)
    assert np.all(np.abs(p32 - p64) <= 2e-4 * scale + 1e-12), np.max(np.abs(p32 - p64) / scale, axis=0)


def test_basket_rejects_bad_arguments(q, plan):
    good = basket(0, 8, 2)
    q.qmccpw_basket_greeks(plan, good, 64, 2, q.QMCCPW_FP64)
    bad = [
        (good.replace(corr=np.array([[1.0, -0.3], [-0.3, 1.0]])), q.QMCCPW_ERR_INVALID_ARG),
        (good.replace(corr=np.array([[1.0, 0.3], [0.2, 1.0]])), q.QMCCPW_ERR_INVALID_ARG),
        (good.replace(w=np.array([0.0, 1.0])), q.QMCCPW_ERR_INVALID_ARG),
        (good.replace(d=400), q.QMCCPW_ERR_INVALID_ARG),                       # m d > d_max
        (good.replace(type_=q.QMCCPW_LOOKBACK_FIXED_CALL), q.QMCCPW_ERR_UNSUPPORTED),
    ]
    for b, code in bad:
        with pytest.raises(q.QmcCpwError) as e:
            q.qmccpw_basket_greeks(plan, b, 64, 2, q.QMCCPW_FP64)
        assert e.value.code == code
    with pytest.raises(q.QmcCpwError) as e:
        q.qmccpw_basket_greeks(plan, good, 64, 2, q.QMCCPW_MIXED_TC_BF16X3)
    assert e.value.code == q.QMCCPW_ERR_UNSUPPORTED
