"""Pins of the oracle's conditioning on the leading coordinate (constructions 3
bridge, 4 PCA): the Gaussian integrated out is the leading coordinate of the
full-path construction of the d dates, its switch point found by Newton's
method (the next reduction the paper names in Sec. 6-7).

- Per point: the value equals a 1-D quadrature over that coordinate of the
  raw discounted payoff, with the path's rest and loadings rebuilt here from
  the separately pinned bridge and PCA factors and the switch point found by
  scipy's brentq (not by the oracle's Newton iteration).
- Per point: delta, vega, gamma equal finite differences of the value.
- d = 1: the Black-Scholes call / cash-or-nothing.
- Full estimator: the geometric-Asian closed form, and the same mean as the
  first-increment conditioning (both are unbiased).
- The lookback: its maximum is the upper envelope of the dates' exponentials
  in the leading coordinate; the quadrature integrates the raw maximum
  between every pairwise crossing (found by brute force), and a path built to
  change its leading date several times checks the pieces.
"""
import math

import numpy as np
import pytest
from scipy import integrate, optimize

import oracle
import test_oracle_cpw as cpw

SEED = 0x220911337


def rest_and_loading(cons, d, dt, z):
    """R_j and a_j, j = 1..d: the full-path bridge or PCA with the leading Gaussian 0 / 1."""
    if cons == 3:
        R = oracle.bridge(d, dt, np.concatenate([[0.0], z]))[1:]
        e = np.zeros(d)
        e[0] = 1.0
        a = oracle.bridge(d, dt, e)[1:]
    else:
        A = oracle.pca_matrix(d, dt)
        R = A[:, 1:] @ z
        a = A[:, 0]
    return R, a


def value_by_quadrature(opt, K, T, S0, r, sig, R, a):
    d = len(R)
    t = T / d * np.arange(1, d + 1)
    omega = r - 0.5 * sig * sig

    def X(x):
        S = S0 * np.exp(omega * t + sig * (a * x + R))
        if opt == 2:
            return float(np.max(S))
        return float(np.mean(S)) if opt in (0, 1) else float(np.exp(np.mean(np.log(S))))

    xs = optimize.brentq(lambda x: X(x) - K, -80.0, 80.0, xtol=1e-15, rtol=1e-15, maxiter=500)
    disc = math.exp(-r * T)
    if opt == 1:
        return disc * 0.5 * math.erfc(xs / math.sqrt(2.0))
    # the maximum has kinks where the leading date changes: integrate between
    # them (every pairwise crossing right of x*, found here by brute force)
    pts = [xs]
    if opt == 2:
        ln = np.log(S0) + omega * t + sig * R
        b = sig * a
        for i in range(d):
            for j in range(i + 1, d):
                if b[i] != b[j]:
                    x = (ln[i] - ln[j]) / (b[j] - b[i])
                    if xs < x < max(xs, 0.0) + 40.0:
                        pts.append(x)
    pts = sorted(pts) + [max(xs, 0.0) + 40.0]
    val = 0.0
    for lo, hi in zip(pts[:-1], pts[1:]):
        part, _ = integrate.quad(lambda x: (X(x) - K) * cpw.pdf(x), lo, hi, epsabs=1e-15, epsrel=1e-13, limit=200)
        val += part
    return disc * val


CASES = [(opt, d, cons) for opt in (0, 1, 2, 3) for d, cons in ((2, 3), (5, 3), (16, 3), (2, 4), (7, 4), (16, 4))]


@pytest.mark.parametrize("opt,d,cons", CASES)
def test_lead_value_equals_quadrature_over_the_leading_coordinate(oracle_lib, opt, d, cons):
    rng = np.random.default_rng(11 + 100 * opt + d + 1000 * cons)
    T, r = 1.0, 0.05
    for K, S0, sig in ((95.0, 100.0, 0.2), (110.0, 100.0, 0.35), (100.0, 90.0, 0.15)):
        z = rng.standard_normal(d - 1)
        vals, Rr = oracle_lib.point(opt, d, K, T, S0, r, sig, cons, z)
        R, a = rest_and_loading(cons, d, T / d, z)
        assert np.all(a > 0)  # the average is increasing in the leading coordinate
        assert np.allclose(Rr, R, rtol=0, atol=1e-13)
        ref = value_by_quadrature(opt, K, T, S0, r, sig, R, a)
        assert abs(vals[0] - ref) <= 1e-10 * max(1.0, abs(ref)), (vals[0], ref)


@pytest.mark.parametrize("opt,d,cons", CASES)
def test_lead_greeks_equal_finite_differences(oracle_lib, opt, d, cons):
    rng = np.random.default_rng(5 + 100 * opt + d + 1000 * cons)
    T, r = 1.0, 0.05
    for K, S0, sig in ((97.0, 100.0, 0.25), (104.0, 100.0, 0.3)):
        z = rng.standard_normal(d - 1)
        vals, _ = oracle_lib.point(opt, d, K, T, S0, r, sig, cons, z)
        G_S = lambda s: oracle_lib.point(opt, d, K, T, s, r, sig, cons, z)[0][0]
        G_v = lambda v: oracle_lib.point(opt, d, K, T, S0, r, v, cons, z)[0][0]
        delta = cpw.richardson(G_S, S0, 0.1, 1)
        gamma = cpw.richardson(G_S, S0, 0.2, 2)
        vega = cpw.richardson(G_v, sig, 2e-4, 1)
        scale = max(1e-3, abs(vals[0]))
        assert abs(vals[1] - delta) <= 1e-8 * max(abs(delta), scale / S0), ("delta", vals[1], delta)
        assert abs(vals[2] - vega) <= 1e-7 * max(abs(vega), scale), ("vega", vals[2], vega)
        assert abs(vals[3] - gamma) <= 1e-6 * max(abs(gamma), scale / S0 ** 2), ("gamma", vals[3], gamma)


@pytest.mark.parametrize("cons", [3, 4])
@pytest.mark.parametrize("opt", [0, 1, 2, 3])
def test_lead_single_date_reduces_to_black_scholes(oracle_lib, cons, opt):
    for S0, K, r, sig, T in ((100, 100, 0.05, 0.2, 1.0), (100, 80, 0.0, 0.45, 0.25), (90, 120, 0.08, 0.1, 2.0)):
        ref = cpw.bs_digital(S0, K, r, sig, T) if opt == 1 else cpw.bs_call(S0, K, r, sig, T)
        vals, _ = oracle_lib.point(opt, 1, K, T, S0, r, sig, cons, np.zeros(0))
        for g in range(4):
            assert abs(vals[g] - ref[g]) <= 1e-12 * max(1.0, abs(ref[g])), (g, vals[g], ref[g])


@pytest.mark.parametrize("cons", [3, 4])
def test_lead_lookback_envelope_pieces(oracle_lib, cons):
    """Paths built so the maximum changes its leading date several times
    right of x* (a falling rest of the path, then rising): the value still
    equals the piecewise quadrature, and gamma the slope formula
    K phi(x*) / (S0^2 sigma a_j*) at the date that leads at x*."""
    d, T, r, sig, S0, K = 8, 1.0, 0.03, 0.3, 100.0, 101.0
    rng = np.random.default_rng(23 + cons)
    for _ in range(6):
        z = rng.standard_normal(d - 1) * 2.0
        vals, _ = oracle_lib.point(2, d, K, T, S0, r, sig, cons, z)
        R, a = rest_and_loading(cons, d, T / d, z)
        ref = value_by_quadrature(2, K, T, S0, r, sig, R, a)
        assert abs(vals[0] - ref) <= 1e-10 * max(1.0, abs(ref)), (vals[0], ref)
        t = T / d * np.arange(1, d + 1)
        ln = np.log(S0) + (r - 0.5 * sig * sig) * t + sig * R
        roots = (np.log(K) - ln) / (sig * a)
        j = int(np.argmin(roots))
        xs = roots[j]
        g = math.exp(-r * T) * K * cpw.pdf(xs) / (S0 * S0 * sig * a[j])
        assert abs(vals[3] - g) <= 1e-12 * abs(g), (vals[3], g)


@pytest.mark.parametrize("cons", [3, 4])
@pytest.mark.parametrize("K", [90.0, 100.0, 110.0])
def test_lead_estimator_matches_geometric_asian_closed_form(oracle_lib, cons, K):
    S0, r, sig, T, d = 100.0, 0.05, 0.2, 1.0, 16
    p, dl, gm = cpw.geometric_asian_call(S0, K, r, sig, T, d)
    vg = cpw.geometric_vega(S0, K, r, sig, T, d)
    mean, se, _ = oracle_lib.greeks(SEED, 3, d, K, T, S0, r, sig, cons, 2 ** 12, 16)
    for g, ref in enumerate((p, dl, vg, gm)):
        assert abs(mean[g] - ref) <= 4.0 * se[g] + 1e-9 * abs(ref), (g, mean[g], ref, se[g])


@pytest.mark.parametrize("opt", [0, 1, 2])
def test_lead_and_first_increment_conditioning_agree(oracle_lib, opt):
    """Both conditionings are unbiased estimators of the same Greeks."""
    S0, K, r, sig, T, d = 100.0, 105.0, 0.05, 0.25, 1.0, 16
    m0, s0, _ = oracle_lib.greeks(SEED, opt, d, K, T, S0, r, sig, 0, 2 ** 12, 16)
    for cons in (3, 4):
        m1, s1, _ = oracle_lib.greeks(SEED, opt, d, K, T, S0, r, sig, cons, 2 ** 12, 16)
        assert np.all(np.abs(m1 - m0) <= 4.0 * np.sqrt(s0 ** 2 + s1 ** 2)), (cons, (m1 - m0) / np.sqrt(s0 ** 2 + s1 ** 2))


@pytest.mark.parametrize("n", [1, 2, 3, 16, 64, 257, 366, 1024])
def test_leading_coordinate_loadings_increase_with_the_date(oracle_lib, n):
    """The leading coordinate's loading on the dates of a whole path of n
    dates rises strictly with the date in both forms -- the bridge's terminal
    value (i / sqrt(n) for unit spacing) and the first principal component --
    with gaps far above a rounding.  The lines of the lookback's envelope are
    then ordered by slope as by date, which is what lets the GPU kernels seek
    each next piece among the later dates only."""
    bridge = np.arange(1, n + 1) / math.sqrt(n)
    pca = oracle_lib.pca_matrix(n, 1.0)[:, 0]
    for a in (bridge, pca):
        assert np.all(a > 0)
        if n > 1:
            gaps = np.diff(a)
            assert np.all(gaps > 1e-9 * np.abs(a[1:])), gaps.min()
