"""Pins of the oracle's conditional-pathwise values and of the full estimator.

- Per point: G(theta, z) equals a 1-D quadrature over x_1 of the raw
  discounted payoff (eq. QmcCpwNewTargetDefinition, Sec. 3.3), and delta,
  vega, gamma equal finite differences of G at fixed z (Sec. 4.5).
- d = 1: the conditional value is the Black-Scholes call / cash-or-nothing
  price and Greeks (closed forms typed here from the textbook).
- Full estimator: the discretely monitored geometric-Asian call has a closed
  form; at d = 2 every product's price and Greeks follow from a 2-D
  quadrature; at d = 4 plain Monte Carlo of the raw payoff agrees.
"""
import math

import numpy as np
import pytest
from scipy import integrate, optimize

SEED = 0x220911337
SQ2 = math.sqrt(2.0)


def Phi(x):
    return 0.5 * math.erfc(-x / SQ2)


def pdf(x):
    return math.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)


def functional(opt, S):
    if opt in (0, 1):
        return float(np.mean(S))
    if opt == 2:
        return float(np.max(S))
    return float(np.exp(np.mean(np.log(S))))


def conditional_by_quadrature(opt, K, T, S0, r, sigma, stilde):
    """int e^{-rT} payoff(S(x1)) phi(x1) dx1 with S(t_j) = S~_j exp(omega t1 + sigma sqrt(t1) x1)."""
    d = len(stilde)
    t1 = T / d
    omega = r - 0.5 * sigma * sigma

    def S_of(x):
        return stilde * math.exp(omega * t1 + sigma * math.sqrt(t1) * x)

    f = lambda x: functional(opt, S_of(x)) - K
    lo, hi = -60.0, 60.0
    if f(lo) > 0:
        xs = lo
    elif f(hi) < 0:
        return 0.0
    else:
        xs = optimize.brentq(f, lo, hi, xtol=1e-15, rtol=1e-15, maxiter=500)
    disc = math.exp(-r * T)
    if opt == 1:
        return disc * 0.5 * math.erfc(xs / SQ2)
    val, _ = integrate.quad(lambda x: (functional(opt, S_of(x)) - K) * pdf(x), xs, max(xs, 0.0) + 40.0,
                            epsabs=1e-14, epsrel=1e-13, limit=200)
    return disc * val


CASES = [(opt, d, cons) for opt in (0, 1, 2, 3) for d, cons in ((2, 0), (5, 0), (8, 0), (8, 1), (13, 1), (6, 2))]


@pytest.mark.parametrize("opt,d,cons", CASES)
def test_point_value_equals_quadrature_over_first_gaussian(oracle_lib, opt, d, cons):
    rng = np.random.default_rng(1000 * opt + 10 * d + cons)
    for K in (90.0, 100.0, 112.0):
        z = rng.standard_normal(d - 1)
        vals, st = oracle_lib.point(opt, d, K, 1.0, 100.0, 0.05, 0.25, cons, z)
        ref = conditional_by_quadrature(opt, K, 1.0, 100.0, 0.05, 0.25, st)
        assert abs(vals[0] - ref) <= 1e-11 * max(1.0, abs(ref)), (K, vals[0], ref)


def richardson(f, x, h, order):
    """Central difference of the first (order=1) or second (order=2) derivative, Richardson-extrapolated."""
    def cd(hh):
        if order == 1:
            return (f(x + hh) - f(x - hh)) / (2 * hh)
        return (f(x + hh) - 2 * f(x) + f(x - hh)) / (hh * hh)
    return (4 * cd(h / 2) - cd(h)) / 3


@pytest.mark.parametrize("opt,d,cons", CASES)
def test_point_greeks_equal_finite_differences_of_G(oracle_lib, opt, d, cons):
    rng = np.random.default_rng(7 + 1000 * opt + 10 * d + cons)
    T, r = 1.0, 0.05
    for K, S0, sig in ((95.0, 100.0, 0.2), (104.0, 100.0, 0.3)):
        z = rng.standard_normal(d - 1)
        vals, _ = oracle_lib.point(opt, d, K, T, S0, r, sig, cons, z)
        G_S = lambda s: oracle_lib.point(opt, d, K, T, s, r, sig, cons, z)[0][0]
        G_v = lambda v: oracle_lib.point(opt, d, K, T, S0, r, v, cons, z)[0][0]
        delta = richardson(G_S, S0, 0.1, 1)
        gamma = richardson(G_S, S0, 0.2, 2)
        vega = richardson(G_v, sig, 2e-4, 1)
        scale = max(1e-3, abs(vals[0]))
        assert abs(vals[1] - delta) <= 1e-8 * max(abs(delta), scale / S0), ("delta", vals[1], delta)
        assert abs(vals[2] - vega) <= 1e-7 * max(abs(vega), scale), ("vega", vals[2], vega)
        assert abs(vals[3] - gamma) <= 1e-6 * max(abs(gamma), scale / S0 ** 2), ("gamma", vals[3], gamma)


def bs_call(S0, K, r, sig, T):
    d1 = (math.log(S0 / K) + (r + 0.5 * sig * sig) * T) / (sig * math.sqrt(T))
    d2 = d1 - sig * math.sqrt(T)
    return (S0 * Phi(d1) - K * math.exp(-r * T) * Phi(d2), Phi(d1),
            S0 * pdf(d1) * math.sqrt(T), pdf(d1) / (S0 * sig * math.sqrt(T)))


def bs_digital(S0, K, r, sig, T):
    d1 = (math.log(S0 / K) + (r + 0.5 * sig * sig) * T) / (sig * math.sqrt(T))
    d2 = d1 - sig * math.sqrt(T)
    df = math.exp(-r * T)
    return (df * Phi(d2), df * pdf(d2) / (S0 * sig * math.sqrt(T)),
            -df * pdf(d2) * d1 / sig, -df * pdf(d2) * d1 / (S0 * S0 * sig * sig * T))


@pytest.mark.parametrize("opt", [0, 1, 2, 3])
def test_single_date_reduces_to_black_scholes(oracle_lib, opt):
    for S0, K, r, sig, T in ((100, 100, 0.05, 0.2, 1.0), (100, 80, 0.0, 0.45, 0.25),
                             (90, 120, 0.08, 0.1, 2.0)):
        ref = bs_digital(S0, K, r, sig, T) if opt == 1 else bs_call(S0, K, r, sig, T)
        vals, _ = oracle_lib.point(opt, 1, K, T, S0, r, sig, 0, np.zeros(0))
        for g in range(4):
            assert abs(vals[g] - ref[g]) <= 1e-13 * max(1.0, abs(ref[g])), (g, vals[g], ref[g])
        mean, se, per = oracle_lib.greeks(SEED, opt, 1, K, T, S0, r, sig, 0, 64, 3)
        # every point gives the same value: the replicate spread is rounding only
        assert np.all(se <= 1e-14 * np.maximum(1.0, np.abs(mean)))
        assert np.allclose(mean, ref, rtol=1e-13, atol=1e-15)


def geometric_asian_call(S0, K, r, sig, T, d):
    """Closed form of the discretely monitored geometric-average call (t_j = jT/d, j=1..d)."""
    h = T / d
    tbar = h * (d + 1) / 2.0
    tau = math.sqrt(h * (d + 1) * (2 * d + 1) / (6.0 * d))
    omega = r - 0.5 * sig * sig
    d2 = (math.log(S0 / K) + omega * tbar) / (sig * tau)
    d1 = d2 + sig * tau
    fwd = math.exp(omega * tbar + 0.5 * sig * sig * tau * tau)
    df = math.exp(-r * T)
    price = df * (S0 * fwd * Phi(d1) - K * Phi(d2))
    delta = df * fwd * Phi(d1)
    gamma = df * fwd * pdf(d1) / (S0 * sig * tau)
    return price, delta, gamma


def geometric_vega(S0, K, r, sig, T, d):
    f = lambda v: geometric_asian_call(S0, K, r, v, T, d)[0]
    return richardson(f, sig, 1e-3, 1)


@pytest.mark.parametrize("cons", [0, 1, 2])
@pytest.mark.parametrize("K", [90.0, 100.0, 110.0])
def test_estimator_matches_geometric_asian_closed_form(oracle_lib, cons, K):
    S0, r, sig, T, d = 100.0, 0.05, 0.2, 1.0, 16
    p, dl, gm = geometric_asian_call(S0, K, r, sig, T, d)
    vg = geometric_vega(S0, K, r, sig, T, d)
    mean, se, per = oracle_lib.greeks(SEED, 3, d, K, T, S0, r, sig, cons, 2 ** 13, 16)
    for g, ref in enumerate((p, dl, vg, gm)):
        assert abs(mean[g] - ref) <= 4.0 * se[g] + 1e-9 * abs(ref), (g, mean[g], ref, se[g])
    # the standard error is the sample standard deviation of the replicates over sqrt(R)
    assert np.allclose(se, per.std(axis=0, ddof=1) / math.sqrt(per.shape[0]), rtol=1e-12)
    assert np.allclose(mean, per.mean(axis=0), rtol=1e-13)


def two_date_price(opt, S0, K, r, sig, T):
    """d = 2: double integral over (x1, z) of the raw discounted payoff."""
    h = T / 2.0
    omega = r - 0.5 * sig * sig

    def inner(z):
        st = np.array([S0, S0 * math.exp(omega * h + sig * math.sqrt(h) * z)])
        return conditional_by_quadrature(opt, K, T, S0, r, sig, st)

    pts = [-omega * math.sqrt(h) / sig] if opt == 2 else None
    val, _ = integrate.quad(lambda z: inner(z) * pdf(z), -12.0, 12.0, points=pts,
                            epsabs=1e-13, epsrel=1e-12, limit=400)
    return val


@pytest.mark.slow
@pytest.mark.parametrize("opt", [0, 1, 2])
def test_estimator_two_dates_against_quadrature(oracle_lib, opt):
    S0, K, r, sig, T = 100.0, 100.0, 0.05, 0.25, 1.0
    price = two_date_price(opt, S0, K, r, sig, T)
    f_S = lambda s: two_date_price(opt, s, K, r, sig, T)
    f_v = lambda v: two_date_price(opt, S0, K, r, v, T)
    ref = (price, richardson(f_S, S0, 1.0, 1), richardson(f_v, sig, 2e-3, 1), richardson(f_S, S0, 1.0, 2))
    for cons in (0, 1):
        mean, se, _ = oracle_lib.greeks(SEED, opt, 2, K, T, S0, r, sig, cons, 2 ** 14, 16)
        for g in range(4):
            assert abs(mean[g] - ref[g]) <= 4.0 * se[g] + 2e-7 * max(abs(ref[g]), 1e-3), \
                (cons, g, mean[g], ref[g], se[g])


def plain_mc_raw(opt, S0, K, r, sig, T, d, paths, seed):
    """Plain MC of the raw payoff with exact GBM steps; returns (price, delta) samples.

    Delta of the arithmetic and lookback calls is the classical pathwise
    estimator (Sec. 3.1.2); the binary uses a central bump with common numbers.
    """
    rng = np.random.default_rng(seed)
    h = T / d
    omega = r - 0.5 * sig * sig
    Z = rng.standard_normal((paths, d))
    logS = np.cumsum(omega * h + sig * math.sqrt(h) * Z, axis=1)
    S = S0 * np.exp(logS)
    X = S.mean(axis=1) if opt in (0, 1) else S.max(axis=1)
    df = math.exp(-r * T)
    if opt == 1:
        bump = 1.0
        price = df * (X > K)
        delta = df * ((X * (S0 + bump) / S0 > K).astype(float) - (X * (S0 - bump) / S0 > K)) / (2 * bump)
    else:
        price = df * np.maximum(X - K, 0.0)
        delta = df * (X / S0) * (X > K)
    return price, delta


@pytest.mark.parametrize("opt", [0, 1, 2])
def test_estimator_against_plain_monte_carlo(oracle_lib, opt):
    S0, K, r, sig, T, d = 100.0, 105.0, 0.05, 0.3, 1.0, 4
    price, delta = plain_mc_raw(opt, S0, K, r, sig, T, d, 1 << 21, 99 + opt)
    mc = np.array([price.mean(), delta.mean()])
    mc_se = np.array([price.std() / math.sqrt(len(price)), delta.std() / math.sqrt(len(delta))])
    mean, se, _ = oracle_lib.greeks(SEED, opt, d, K, T, S0, r, sig, 0, 2 ** 12, 16)
    # binary delta by a bump of 1 carries an O(bump^2) bias: allow 1e-4 absolute
    bias = np.array([0.0, 1e-4 if opt == 1 else 0.0])
    assert np.all(np.abs(mean[:2] - mc) <= 4.0 * np.hypot(mc_se, se[:2]) + bias), (mean[:2], mc, mc_se)
