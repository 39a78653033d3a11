"""GPU parity: the CUDA path (through the C-ABI) against the CPU oracle.

Bars (written in each test):
  - Sobol' integers after scramble and shift: bit-exact.
  - FP64 per-replicate estimates and means: |gpu - oracle| <=
    1e-12 * max(|oracle|, mean |per-point value|) per Greek (the second term
    guards Greeks whose mean is near zero while its terms are not).
  - FP64 single points: the same bar times max(1, n/64): a point's path sums
    n-term dot products and d exponentials, whose rounding grows with n, and
    the binary gamma amplifies an error in ln X by ~1/a^2.
  - MIXED against FP64 on the same points: |mixed - fp64| <= 0.1 * SE(fp64)
    per Greek.
"""
import math

import numpy as np
import pytest

import oracle
import point_bounds
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
    h = q.qmccpw_plan(device=0, d_max=366, r_max=32, seed=SEED)
    yield h
    q.qmccpw_free(h)


def greek_scale(c, cons, rep=0, count=256):
    pts = oracle.point_values(SEED, c.type, c.d, c.K, c.T, c.S0, c.r, c.sigma, cons, rep, 0, count)
    return np.mean(np.abs(pts), axis=0)


def assert_close64(gpu, ref, scale, what="", rtol=RTOL64):
    gpu, ref = np.asarray(gpu), np.asarray(ref)
    bound = rtol * np.maximum(np.abs(ref), scale)
    bad = np.abs(gpu - ref) > bound
    assert not bad.any(), (what, np.argwhere(bad)[:5].tolist(), gpu[bad][:5], ref[bad][:5])


# ---------------------------------------------------------------------------
@pytest.mark.parametrize("rep,ndims,k0,count", [
    (0, 1, 0, 4096), (3, 63, 0, 1000), (31, 363, 12345, 777), (7, 255, 2 ** 31 - 5, 300),
    (1, 15, 2 ** 32 - 100, 100), (5, 364, 1, 1),
])
def test_sobol_integers_bit_exact(q, plan, rep, ndims, k0, count):
    gpu = q.qmccpw_sobol_points(plan, rep, ndims, k0, count)
    ref = oracle.sobol(SEED, rep, ndims, k0, count, scrambled=True, gray=True)
    assert np.array_equal(gpu, ref)


POINT_CASES = [(t, cons, d) for t in (0, 1, 2, 3) for cons in (W.BB, W.PCA) for d in (1, 2, 16, 64, 100, 365)]


@pytest.mark.parametrize("typ,cons,d", POINT_CASES)
def test_point_values_fp64(q, plan, typ, cons, d):
    c = W.Contract(typ, d, 95.0, 1.5, 100.0, 0.04, 0.25, 0, 0, cons)
    k0, count, rep = 5000, 300, 2
    ref = oracle.point_values(SEED, typ, d, c.K, c.T, c.S0, c.r, c.sigma, cons, rep, k0, count)
    gpu = q.qmccpw_point_values(plan, typ, d, c.K, c.T, c.S0, c.r, c.sigma, cons, q.QMCCPW_FP64, rep, k0, count)
    assert_close64(gpu, ref, np.mean(np.abs(ref), axis=0), f"{typ}/{cons}/{d}", RTOL64 * max(1.0, (d - 1) / 64))


@pytest.mark.parametrize("typ,cons,d", [(t, cons, d) for t in (0, 1, 2, 3) for cons in (W.BB, W.PCA)
                                        for d in (16, 64, 365)])
def test_point_values_mixed_close_to_oracle(q, plan, typ, cons, d):
    """Per point, float path: every point and Greek within the bar derived
    from the float widths (point_bounds); 512 points over tiles of up to 256,
    one tile ragged."""
    k0, count, rep = 77, 512, 1
    ref = oracle.point_values(SEED, typ, d, 105.0, 1.0, 100.0, 0.05, 0.2, cons, rep, k0, count)
    gpu = q.qmccpw_point_values(plan, typ, d, 105.0, 1.0, 100.0, 0.05, 0.2, cons, q.QMCCPW_MIXED, rep, k0, count)
    bar = point_bounds.bars(ref, typ, d, 105.0, 1.0, 100.0, 0.05, 0.2, cons, q.QMCCPW_MIXED)
    bad = ~(np.abs(gpu - ref) <= bar)  # a NaN fails too
    assert not bad.any(), (np.argwhere(bad)[:5].tolist(), gpu[bad][:5], ref[bad][:5], bar[bad][:5])
    # and the point means agree within the mean bar (two-sided)
    assert np.all(np.abs(np.mean(gpu, axis=0) - np.mean(ref, axis=0)) <= np.mean(bar, axis=0))


ESTIMATOR_CASES = [
    W.small_arith(),
    W.Contract(W.BINARY, 16, 100.0, 1.0, 100.0, 0.05, 0.2, 2 ** 14, 8, W.PCA),
    W.Contract(W.LOOKBACK, 9, 90.0, 1.0, 100.0, 0.05, 0.1, 1000, 4, W.BB),          # ragged N
    W.Contract(W.GEOMETRIC, 33, 110.0, 2.0, 100.0, 0.0, 0.3, 2 ** 12 + 37, 2, W.PCA),  # ragged, R = 2
    W.Contract(W.ARITH, 1, 100.0, 1.0, 100.0, 0.05, 0.2, 64, 3, W.BB),               # d = 1
    W.Contract(W.BINARY, 2, 100.0, 0.5, 100.0, 0.05, 0.3, 1, 2, W.BB),                # N = 1
    W.Contract(W.ARITH, 365, 100.0, 1.0, 100.0, 0.05, 0.2, 2 ** 10, 2, W.BB),         # largest d
    W.Contract(W.BINARY, 365, 95.0, 1.5, 100.0, 0.04, 0.25, 2 ** 10, 2, W.PCA),
]


@pytest.mark.parametrize("c", ESTIMATOR_CASES, ids=lambda c: c.label())
def test_estimator_fp64_matches_oracle(q, plan, c):
    mean, se, per = q.qmccpw_greeks(plan, c.type, c.d, c.K, c.T, c.S0, c.r, c.sigma, c.N, c.R,
                                    c.construction, q.QMCCPW_FP64)
    rmean, rse, rper = oracle.greeks(SEED, c.type, c.d, c.K, c.T, c.S0, c.r, c.sigma, c.construction, c.N, c.R)
    scale = greek_scale(c, c.construction, count=min(256, c.N))
    assert_close64(per, rper, scale, "per-replicate")
    assert_close64(mean, rmean, scale, "mean")
    # SE is a difference of nearly equal numbers when it is tiny: compare against the scale
    assert np.all(np.abs(se - rse) <= 1e-9 * np.maximum(rse, 1e-12 * scale)), (se, rse)


@pytest.mark.parametrize("typ", [0, 1, 2, 3])
def test_single_date_gives_black_scholes(q, plan, typ):
    import test_oracle_cpw as ref
    S0, K, r, sig, T = 100.0, 95.0, 0.03, 0.3, 0.75
    exact = ref.bs_digital(S0, K, r, sig, T) if typ == 1 else ref.bs_call(S0, K, r, sig, T)
    for prec in (q.QMCCPW_FP64, q.QMCCPW_MIXED):
        mean, se, _ = q.qmccpw_greeks(plan, typ, 1, K, T, S0, r, sig, 1000, 2, q.QMCCPW_BB, prec)
        tol = 1e-12 if prec == q.QMCCPW_FP64 else 1e-5
        assert np.allclose(mean, exact, rtol=tol, atol=tol * 1e-2), (prec, mean, exact)


def test_repeated_calls_are_bit_identical_and_batch_equals_single(q, plan):
    cs = [W.small_arith(),
          W.Contract(W.LOOKBACK, 64, 90.0, 1.0, 100.0, 0.05, 0.1, 3000, 4, W.PCA),
          W.Contract(W.BINARY, 100, 105.0, 0.5, 100.0, 0.02, 0.4, 2 ** 12, 3, W.BB),
          W.Contract(W.GEOMETRIC, 12, 80.0, 2.0, 100.0, 0.08, 0.5, 777, 2, W.BB)]
    for prec in (q.QMCCPW_FP64, q.QMCCPW_MIXED):
        batch = q.qmccpw_greeks_batch(plan, cs, prec)
        again = q.qmccpw_greeks_batch(plan, cs, prec)
        for c, (m, s, p), (m2, s2, p2) in zip(cs, batch, again):
            assert np.array_equal(p, p2) and np.array_equal(m, m2)
            m1, s1, p1 = q.qmccpw_greeks(plan, c.type, c.d, c.K, c.T, c.S0, c.r, c.sigma, c.N, c.R,
                                         c.construction, prec)
            assert np.array_equal(p, p1) and np.array_equal(m, m1) and np.array_equal(s, s1)


def test_prepared_batch_matches_one_shot(q, plan):
    cs = W.grid_d64(N=2 ** 12, R=4)[:6]
    b = q.Batch(plan, cs, q.QMCCPW_MIXED)
    for _ in range(2):
        b.launch()
    res = b.results()
    one = q.qmccpw_greeks_batch(plan, cs, q.QMCCPW_MIXED)
    for (m, s, p), (m1, s1, p1) in zip(res, one):
        assert np.array_equal(p, p1)
    assert b.launch_count() >= 1
    b.free()


def test_invalid_arguments_are_rejected(q, plan):
    bad = [
        dict(d=367), dict(d=0), dict(R=33), dict(R=1), dict(N=0), dict(N=2 ** 32 + 1), dict(sigma=float("nan")),
        dict(K=-1.0), dict(T=0.0), dict(S0=float("inf")), dict(type=7),
    ]
    base = dict(type=0, d=16, K=100.0, T=1.0, S0=100.0, r=0.05, sigma=0.2, N=256, R=4)
    for override in bad:
        args = dict(base, **override)
        with pytest.raises(q.QmcCpwError) as e:
            q.qmccpw_greeks(plan, args["type"], args["d"], args["K"], args["T"], args["S0"], args["r"],
                            args["sigma"], args["N"], args["R"], q.QMCCPW_BB, q.QMCCPW_FP64)
        assert e.value.code == q.QMCCPW_ERR_INVALID_ARG, override
    with pytest.raises(q.QmcCpwError) as e:
        q.qmccpw_greeks(plan, 0, 300, 100.0, 1.0, 100.0, 0.05, 0.2, 256, 4, q.QMCCPW_PCA, q.QMCCPW_MIXED_TC_TF32X3)
    assert e.value.code == q.QMCCPW_ERR_UNSUPPORTED


# ---------------------------------------------------------------------------
# full size (d = 64, N = 2^20, R = 32), in the launch configuration the bench uses
# ---------------------------------------------------------------------------
FULL = [W.Contract(W.LOOKBACK, 64, 90.0, 1.0, 100.0, 0.05, 0.1, 2 ** 20, 32, W.PCA),
        W.Contract(W.ARITH, 64, 100.0, 1.0, 100.0, 0.05, 0.3, 2 ** 20, 32, W.BB),
        W.Contract(W.BINARY, 64, 110.0, 1.0, 100.0, 0.05, 0.1, 2 ** 20, 32, W.BB)]


@pytest.mark.parametrize("c", FULL, ids=lambda c: c.label())
def test_full_size_sampled_replicates_and_points(q, plan, c):
    grid = W.grid_d64()
    assert c in grid  # the contract is one of the benchmark's
    res = q.qmccpw_greeks_batch(plan, [c], q.QMCCPW_FP64)[0]
    per = res[2]
    scale = greek_scale(c, c.construction)
    reps = [c.R - 1]
    sums = np.vstack([oracle.partial_sums(SEED, c.type, c.d, c.K, c.T, c.S0, c.r, c.sigma, c.construction,
                                          r, 1, 0, c.N) for r in reps])
    assert_close64(per[reps], sums / c.N, scale, "sampled replicates")
    # far points of the last replicate, one by one
    k0 = c.N - 300
    ref = oracle.point_values(SEED, c.type, c.d, c.K, c.T, c.S0, c.r, c.sigma, c.construction, c.R - 1, k0, 300)
    gpu = q.qmccpw_point_values(plan, c.type, c.d, c.K, c.T, c.S0, c.r, c.sigma, c.construction,
                                q.QMCCPW_FP64, c.R - 1, k0, 300)
    assert_close64(gpu, ref, np.mean(np.abs(ref), axis=0), "far points", RTOL64 * max(1.0, (c.d - 1) / 64))
    # statistics: mean and SE of the replicate estimates
    assert np.allclose(res[0], per.mean(axis=0), rtol=1e-13, atol=0)
    assert np.allclose(res[1], per.std(axis=0, ddof=1) / math.sqrt(c.R), rtol=1e-10, atol=0)


def test_mixed_error_against_fp64_in_standard_errors(q, plan):
    """MIXED vs FP64 on the d=64, N=2^20, R=32 grid, per contract and Greek:
    |mixed - fp64| <= 0.1 SE(fp64) for every pair.  The PCA contracts at
    sigma = 0.1 have standard errors near 1e-8 relative, and a path-level
    bias b moves an at-the-money call price by about S0 delta b / price ~
    25 b, so every systematic error of the float path must stay near 1e-10:
    own polynomials for e^x, ln, Phi^{-1} and the normal tail (no hardware
    approximation with a nonzero mean error), float-pair constants wherever a
    float rounding of sigma, omega dt, 1/d or 1/sqrt(2 pi) would act on every
    point the same way."""
    grid = W.grid_d64()
    r64 = q.qmccpw_greeks_batch(plan, grid, q.QMCCPW_FP64)
    r32 = q.qmccpw_greeks_batch(plan, grid, q.QMCCPW_MIXED)
    bad = []
    for c, (m64, se64, _), (m32, _, _) in zip(grid, r64, r32):
        err = np.abs(m32 - m64)
        if not np.all(err <= 0.1 * se64):  # a NaN fails too
            bad.append((c.label(), np.round(err / se64, 3).tolist()))
    assert not bad, bad
