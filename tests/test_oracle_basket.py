"""Pins of the oracle's basket estimator (several underlying assets, Sec. 6).

The basket average X = sum_i w_i mean_j S_i(t_j) of m correlated GBM assets;
the first increment of factor 1 is integrated out and the switch point
X(x*) = K is found by Newton's method.  The pins rebuild the raw path here,
from the definition, with numpy's Cholesky factor and the separately pinned
bridge, and do not use the oracle's closed form or its Newton iteration:

- Cholesky: L L^T = C, lower triangular, equal to numpy's factor.
- m = 1: the basket is the single-asset bridge estimator, point by point
  (an independent code path: closed-form switch point there, Newton here).
- Per point: the value equals a 1-D quadrature over x_1 of the raw
  discounted payoff of the raw basket, its switch point from scipy's brentq.
- Per point: delta, gamma (spot scale S0) and vega (volatility scale sigma)
  equal Richardson finite differences of the value.
- Homogeneity: S0 and K scaled together scale price and vega, keep delta.
- Sobol' layout: z[b*m + k] drives factor k+1's bridge node b, the last m-1
  entries the first increments of factors 2..m.
- Full estimator: plain Monte Carlo of the raw basket payoff agrees.
"""
import math

import numpy as np
import pytest
from scipy import integrate, optimize

import oracle
import test_oracle_cpw as cpw

SEED = 0x220911337


def corr_matrix(m, rho, jitter_seed=0):
    """A positive-definite correlation with positive first row."""
    rng = np.random.default_rng(jitter_seed)
    C = np.full((m, m), rho)
    np.fill_diagonal(C, 1.0)
    if m > 2:
        E = rng.uniform(-0.1, 0.1, (m, m))
        E = 0.5 * (E + E.T)
        np.fill_diagonal(E, 0.0)
        E[0, :] = E[:, 0] = 0.0
        C = C + E
    return C


def random_basket(rng, opt, d, m):
    w = rng.uniform(0.5, 1.5, m)
    a = rng.uniform(0.8, 1.2, m)
    v = rng.uniform(0.6, 1.6, m)
    C = corr_matrix(m, float(rng.uniform(0.2, 0.7)), int(rng.integers(1 << 30)))
    K = float(rng.uniform(80.0, 120.0)) * float(np.sum(w)) / m
    return oracle.Basket(opt, d, K, 1.0, 100.0, 0.05, 0.25, w / m, a, v, C)


def raw_basket(b, z):
    """X(x_1) of the raw basket from z, built here: W = L B with numpy's Cholesky."""
    d, m, n = b.d, b.m, b.d - 1
    dt = b.T / d
    L = np.linalg.cholesky(b.corr)
    Wt = np.zeros((m, d))                          # W~_k at s_0..s_n
    for k in range(m):
        Wt[k] = oracle.bridge(n, dt, np.array([z[bn * m + k] for bn in range(n)]))
    xk = np.concatenate([[0.0], [z[n * m + k - 1] for k in range(1, m)]])
    t = dt * np.arange(1, d + 1)
    sig = b.v * b.sigma
    om = b.r - 0.5 * sig * sig

    def X(x1):
        xs = xk.copy()
        xs[0] = x1
        B = math.sqrt(dt) * xs[:, None] + Wt                  # B_k(t_j), j = 1..d
        W = L @ B
        S = (b.a * b.S0)[:, None] * np.exp(om[:, None] * t[None, :] + sig[:, None] * W)
        return float(np.sum(b.w * S.mean(axis=1)))
    return X


def value_by_quadrature(b, z):
    X = raw_basket(b, z)
    xs = optimize.brentq(lambda x: X(x) - b.K, -80.0, 80.0, xtol=1e-15, rtol=1e-15, maxiter=500)
    disc = math.exp(-b.r * b.T)
    if b.type == 1:
        return disc * 0.5 * math.erfc(xs / math.sqrt(2.0))
    val, _ = integrate.quad(lambda x: (X(x) - b.K) * cpw.pdf(x), xs, max(xs, 0.0) + 40.0,
                            epsabs=1e-14, epsrel=1e-13, limit=200)
    return disc * val


@pytest.mark.parametrize("m", [1, 2, 3, 5, 8])
def test_cholesky_reproduces_the_matrix(oracle_lib, m):
    C = corr_matrix(m, 0.4, m)
    L = oracle_lib.cholesky(C)
    assert np.allclose(np.triu(L, 1), 0.0)
    assert np.allclose(L @ L.T, C, rtol=0, atol=1e-14)
    assert np.allclose(L, np.linalg.cholesky(C), rtol=0, atol=1e-14)


def test_cholesky_rejects_an_indefinite_matrix(oracle_lib):
    with pytest.raises(ValueError):
        oracle_lib.cholesky(np.array([[1.0, 0.9, 0.9], [0.9, 1.0, -0.9], [0.9, -0.9, 1.0]]))


@pytest.mark.parametrize("opt", [0, 1])
@pytest.mark.parametrize("d", [1, 2, 16, 64])
def test_single_asset_basket_is_the_bridge_estimator(oracle_lib, opt, d):
    rng = np.random.default_rng(11 + d + 100 * opt)
    for K, sig in ((90.0, 0.2), (110.0, 0.35)):
        b = oracle.Basket(opt, d, K, 1.0, 100.0, 0.05, sig, [1.0], [1.0], [1.0], [[1.0]])
        z = rng.standard_normal(max(d - 1, 1))[: d - 1]
        ours = oracle_lib.basket_point(b, z)
        ref, _ = oracle_lib.point(opt, d, K, 1.0, 100.0, 0.05, sig, 0, z)
        assert np.allclose(ours, ref, rtol=1e-12, atol=1e-14 * max(1.0, abs(ref[0]))), (ours, ref)


@pytest.mark.parametrize("opt", [0, 1])
@pytest.mark.parametrize("d,m", [(1, 2), (2, 2), (5, 3), (8, 4), (3, 8)])
def test_basket_point_equals_quadrature_over_first_increment(oracle_lib, opt, d, m):
    rng = np.random.default_rng(5 + 7 * d + 31 * m + 1000 * opt)
    for _ in range(3):
        b = random_basket(rng, opt, d, m)
        z = rng.standard_normal(m * d - 1)
        v = oracle_lib.basket_point(b, z)
        q = value_by_quadrature(b, z)
        assert abs(v[0] - q) <= 1e-11 * max(1.0, abs(q)), (v[0], q)


def test_basket_far_out_and_deep_in_the_money(oracle_lib):
    rng = np.random.default_rng(3)
    for K in (20.0, 400.0):
        b = random_basket(rng, 0, 6, 3).replace(K=K)
        z = rng.standard_normal(3 * 6 - 1)
        assert abs(oracle_lib.basket_point(b, z)[0] - value_by_quadrature(b, z)) <= 1e-10 * max(1.0, K)


@pytest.mark.parametrize("opt", [0, 1])
@pytest.mark.parametrize("d,m", [(1, 2), (4, 3), (9, 2)])
def test_basket_greeks_equal_finite_differences(oracle_lib, opt, d, m):
    rng = np.random.default_rng(17 + d + 10 * m + 100 * opt)
    for _ in range(2):
        b = random_basket(rng, opt, d, m)
        z = rng.standard_normal(m * d - 1)
        vals = oracle_lib.basket_point(b, z)
        G_S = lambda s: oracle_lib.basket_point(b.replace(S0=s), z)[0]
        G_v = lambda v: oracle_lib.basket_point(b.replace(sigma=v), z)[0]
        delta = cpw.richardson(G_S, b.S0, 0.1, 1)
        gamma = cpw.richardson(G_S, b.S0, 0.2, 2)
        vega = cpw.richardson(G_v, b.sigma, 2e-4, 1)
        scale = max(1e-3, abs(vals[0]))
        assert abs(vals[1] - delta) <= 1e-8 * max(abs(delta), scale / b.S0), ("delta", vals[1], delta)
        assert abs(vals[2] - vega) <= 1e-7 * max(abs(vega), scale), ("vega", vals[2], vega)
        assert abs(vals[3] - gamma) <= 1e-6 * max(abs(gamma), scale / b.S0 ** 2), ("gamma", vals[3], gamma)


def test_basket_homogeneity_in_spot_and_strike(oracle_lib):
    rng = np.random.default_rng(23)
    b = random_basket(rng, 0, 8, 3)
    z = rng.standard_normal(3 * 8 - 1)
    v1 = oracle_lib.basket_point(b, z)
    lam = 1.7
    v2 = oracle_lib.basket_point(b.replace(S0=lam * b.S0, K=lam * b.K), z)
    assert np.allclose(v2, [lam * v1[0], v1[1], lam * v1[2], v1[3] / lam], rtol=1e-12)


def test_sobol_layout_of_the_basket(oracle_lib):
    """Factor k+1 reads z[b*m + k] for its bridge nodes and z[n*m + k-1] for its
    first increment: with the other assets nearly uncorrelated and weightless,
    only asset 2's own entries move the value."""
    d, m, n = 5, 3, 4
    C = np.array([[1.0, 1e-9, 1e-9], [1e-9, 1.0, 0.0], [1e-9, 0.0, 1.0]])
    b = oracle.Basket(0, d, 60.0, 1.0, 100.0, 0.05, 0.25, [1e-12, 1.0, 1e-12], [1.0, 1.0, 1.0],
                      [1.0, 1.0, 1.0], C)
    rng = np.random.default_rng(2)
    z = rng.standard_normal(m * d - 1)
    base = oracle_lib.basket_point(b, z)[0]
    own = {bn * m + 1 for bn in range(n)} | {n * m + 0}
    for i in range(m * d - 1):
        zz = z.copy()
        zz[i] += 0.5
        moved = abs(oracle_lib.basket_point(b, zz)[0] - base)
        if i in own:
            assert moved > 1e-3, (i, moved)
        else:
            assert moved < 1e-6, (i, moved)


def plain_mc_basket(b, paths, seed):
    """Plain MC of the raw basket call or binary with exact GBM steps."""
    rng = np.random.default_rng(seed)
    d, m = b.d, b.m
    dt = b.T / d
    L = np.linalg.cholesky(b.corr)
    sig = b.v * b.sigma
    om = b.r - 0.5 * sig * sig
    Z = rng.standard_normal((paths, m, d))
    B = np.cumsum(math.sqrt(dt) * Z, axis=2)
    W = np.einsum("ik,pkj->pij", L, B)
    t = dt * np.arange(1, d + 1)
    S = (b.a * b.S0)[None, :, None] * np.exp(om[None, :, None] * t[None, None, :] + sig[None, :, None] * W)
    X = np.sum(b.w[None, :] * S.mean(axis=2), axis=1)
    df = math.exp(-b.r * b.T)
    return df * np.maximum(X - b.K, 0.0) if b.type == 0 else df * (X > b.K)


@pytest.mark.parametrize("opt", [0, 1])
def test_basket_estimator_against_plain_monte_carlo(oracle_lib, opt):
    b = oracle.Basket(opt, 3, 100.0, 1.0, 100.0, 0.05, 0.3, [0.5, 0.3, 0.2], [1.0, 0.9, 1.1], [1.0, 1.3, 0.7],
                      corr_matrix(3, 0.5, 4))
    price = plain_mc_basket(b, 1 << 20, 77 + opt)
    mc, mc_se = price.mean(), price.std() / math.sqrt(len(price))
    mean, se, _ = oracle_lib.basket_greeks(SEED, b, 2 ** 12, 16)
    assert abs(mean[0] - mc) <= 4.0 * math.hypot(mc_se, se[0]), (mean[0], mc, mc_se, se[0])


def test_basket_point_values_follow_the_estimator(oracle_lib):
    b = random_basket(np.random.default_rng(8), 0, 6, 2)
    vals = oracle_lib.basket_point_values(SEED, b, 1, 0, 64)
    mean, _, per = oracle_lib.basket_greeks(SEED, b, 64, 2)
    assert np.allclose(vals.mean(axis=0), per[1], rtol=1e-13, atol=1e-15)


def test_basket_rejects_bad_arguments(oracle_lib):
    good = oracle.Basket(0, 4, 100.0, 1.0, 100.0, 0.05, 0.2, [0.5, 0.5], [1.0, 1.0], [1.0, 1.0],
                         [[1.0, 0.5], [0.5, 1.0]])
    z = np.zeros(7)
    oracle_lib.basket_point(good, z)
    for bad in (good.replace(corr=np.array([[1.0, -0.5], [-0.5, 1.0]])),   # negative correlation to asset 1
                good.replace(corr=np.array([[1.0, 0.5], [0.4, 1.0]])),     # not symmetric
                good.replace(w=np.array([0.0, 1.0])),                       # asset 1 without weight
                good.replace(type_=2)):                                     # no lookback basket
        with pytest.raises(ValueError):
            oracle_lib.basket_point(bad, z)
