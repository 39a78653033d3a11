"""Pins of the oracle's inverse normal and path constructions (CPU only).

Inverse normal: Phi(z) = u checked with Python's own erfc, published quantiles
and scipy's ndtri.  Paths: A A^T = Sigma (eq. WboldTilde), the bridge order of
Sec. 4.4 (terminal value first, then midpoints), and the PCA factor against a
library eigen-decomposition.
"""
import math

import numpy as np
import pytest
from scipy.special import ndtri


def phi_cdf(z: float) -> float:
    return 0.5 * math.erfc(-z / math.sqrt(2.0))


def test_inverse_normal_published_quantiles(oracle_lib):
    # standard table values
    cases = {0.975: 1.959963984540054, 0.95: 1.6448536269514722, 0.5 + 0.3413447460685429: 1.0,
             0.99: 2.3263478740408408, 0.001: -3.090232306167813}
    for u, z in cases.items():
        assert abs(oracle_lib.inv_normal(u)[0] - z) < 4e-15 * max(1.0, abs(z))


def test_inverse_normal_round_trip_and_symmetry(oracle_lib):
    # dyadic u as the estimator uses them, including both extreme points
    ys = np.concatenate([np.arange(0, 2 ** 32, 2 ** 32 // 4099, dtype=np.uint64),
                         np.array([0, 1, 2, 3, 2 ** 31 - 1, 2 ** 31, 2 ** 32 - 2, 2 ** 32 - 1], dtype=np.uint64)])
    u = (ys.astype(np.float64) + 0.5) * 2.0 ** -32
    z = oracle_lib.inv_normal(u)
    for ui, zi in zip(u, z):
        q = min(ui, 1.0 - ui)
        back = phi_cdf(-abs(zi))
        pdf = math.exp(-0.5 * zi * zi) / math.sqrt(2.0 * math.pi)
        # backward error in z: |Phi(z) - q| / phi(z) within about one ulp of z
        assert abs(back - q) / pdf <= 1e-15 * max(1.0, abs(zi)), (ui, zi)
    zr = oracle_lib.inv_normal(1.0 - u)
    assert np.array_equal(zr, -z)
    # library routine
    ref = ndtri(u)
    assert np.max(np.abs(z - ref) / np.maximum(1.0, np.abs(ref))) < 4e-15


def test_inverse_normal_rejects_out_of_range(oracle_lib):
    assert np.isnan(oracle_lib.inv_normal([0.0, 1.0, -0.1, 1.5])).all()


def bridge_matrix(oracle_lib, n, dt):
    cols = []
    for k in range(n):
        e = np.zeros(n)
        e[k] = 1.0
        cols.append(oracle_lib.bridge(n, dt, e)[1:])
    return np.array(cols).T  # A[i-1, k]


def sigma_matrix(n, dt):
    i = np.arange(1, n + 1)
    return dt * np.minimum.outer(i, i).astype(np.float64)


@pytest.mark.parametrize("n", [1, 2, 3, 7, 15, 16, 63, 100, 255, 364])
def test_bridge_covariance(oracle_lib, n):
    dt = 1.0 / (n + 1)
    A = bridge_matrix(oracle_lib, n, dt)
    S = sigma_matrix(n, dt)
    assert np.max(np.abs(A @ A.T - S)) <= 1e-13 * np.max(S)


def test_bridge_order_terminal_then_midpoints(oracle_lib):
    # Sec. 4.4: the first normal fixes the terminal value, the second the
    # midpoint, then the quarter points left to right.
    n, dt = 16, 1.0 / 17
    A = bridge_matrix(oracle_lib, n, dt)
    s = dt * np.arange(1, n + 1)
    assert np.allclose(A[:, 0], s / math.sqrt(s[-1]), rtol=0, atol=1e-15)  # W(s) = s/s_n * W(s_n)
    # column 1 vanishes at the endpoints and peaks at s_8
    col = A[:, 1]
    assert abs(col[-1]) < 1e-15 and np.argmax(col) == 7
    assert np.all(col[7:] >= -1e-15) and np.all(col[:8] >= -1e-15)
    # columns 2 and 3 drive s_4 and s_12 (left before right), and only inside their intervals
    assert np.argmax(A[:, 2]) == 3 and np.all(np.abs(A[8:, 2]) < 1e-15)
    assert np.argmax(A[:, 3]) == 11 and np.all(np.abs(A[:8, 3]) < 1e-15)
    # uneven n: the root interval (0, n) splits at floor(n/2)
    A5 = bridge_matrix(oracle_lib, 5, 0.2)
    assert np.argmax(A5[:, 1]) == 1  # s_2


def forward_matrix(oracle_lib, n, dt):
    cols = []
    for k in range(n):
        e = np.zeros(n)
        e[k] = 1.0
        cols.append(oracle_lib.forward(n, dt, e)[1:])
    return np.array(cols).T


@pytest.mark.parametrize("n", [1, 2, 15, 64, 255])
def test_forward_covariance_and_structure(oracle_lib, n):
    # the standard construction's factor is sqrt(dt) times the lower-triangular
    # matrix of ones: dimension k drives the increment of step k alone
    dt = 1.0 / (n + 1)
    A = forward_matrix(oracle_lib, n, dt)
    assert np.max(np.abs(A @ A.T - sigma_matrix(n, dt))) <= 1e-14 * n * dt
    assert np.allclose(A, math.sqrt(dt) * np.tril(np.ones((n, n))), rtol=0, atol=1e-15)


@pytest.mark.parametrize("n", [1, 2, 15, 63, 255])
def test_pca_factor(oracle_lib, n):
    dt = 1.0 / (n + 1)
    A = oracle_lib.pca_matrix(n, dt)
    S = sigma_matrix(n, dt)
    assert np.max(np.abs(A @ A.T - S)) <= 1e-13 * np.max(S)
    lam = np.sum(A * A, axis=0)
    assert np.all(np.diff(lam) < 0)  # decreasing variance per component
    ref_lam, ref_vec = np.linalg.eigh(S)
    ref_lam, ref_vec = ref_lam[::-1], ref_vec[:, ::-1]
    assert np.allclose(lam, ref_lam, rtol=1e-11, atol=0)
    V = A / np.sqrt(lam)
    for k in range(n):
        sgn = np.sign(ref_vec[0, k])
        assert np.allclose(V[:, k], sgn * ref_vec[:, k], atol=1e-10)
    G = A.T @ A
    assert np.max(np.abs(G - np.diag(np.diag(G)))) < 1e-12 * np.max(lam)


@pytest.mark.parametrize("opt,d,cons", [(0, 16, 0), (1, 9, 1), (2, 33, 0), (3, 5, 1), (0, 12, 2), (2, 7, 2)])
def test_estimator_points_use_the_pinned_pieces(oracle_lib, opt, d, cons):
    # The estimator's point k of replicate r is: scrambled Sobol integers at
    # Gray index g(k), u = (y + 1/2) 2^-32, z = Phi^{-1}(u), then the path and
    # the conditional values.  Rebuild it from the separately pinned pieces.
    seed, rep, k0, count = 0x220911337, 3, 1000, 37
    vals = oracle_lib.point_values(seed, opt, d, 100.0, 1.0, 100.0, 0.05, 0.2, cons, rep, k0, count)
    y = oracle_lib.sobol(seed, rep, d - 1, k0, count, scrambled=True, gray=True)
    for t in range(count):
        z = oracle_lib.inv_normal((y[t].astype(np.float64) + 0.5) * 2.0 ** -32)
        ref, _ = oracle_lib.point(opt, d, 100.0, 1.0, 100.0, 0.05, 0.2, cons, z)
        assert np.array_equal(vals[t], ref)
