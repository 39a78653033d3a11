"""The serving benchmark's request sizing and pilot reuse on CPU.

A request's N is the smallest power of two in [2^12, 2^22] whose standard
error, the pilot's (N = 2^12) scaled as 1/N, meets the target; the main run
covers only the points beyond the pilot's (first_point = 2^12), and the two
runs combine into the estimate of all N points.  The combination is checked
against the oracle's estimator over the whole point set, replicate by
replicate: the Sobol' sequence extends (Sec. 2.2.2), so the first 2^12 points
of the N are exactly the pilot's.
"""
import importlib.util
import os
import sys

import numpy as np
import pytest

import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_serving_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    sys.modules["bench_serving_under_test"] = mod
    spec.loader.exec_module(mod)
    return mod


@pytest.mark.parametrize("pilot_se,target,expect", [
    (1e-4, 1e-3, 2 ** 12),        # the pilot already meets the target
    (1e-3, 1e-3, 2 ** 12),        # exactly at the target
    (1.5e-3, 1e-3, 2 ** 13),
    (1e-3, 1e-4, 2 ** 16),        # 10x: 2^12 * 16 is the first power of two past 2^12 * 10
    (1e-2, 1e-6, 2 ** 22),        # capped
    (0.0, 1e-5, 2 ** 12),
])
def test_request_size(bench, pilot_se, target, expect):
    assert bench.request_size(pilot_se, target) == expect


@pytest.mark.parametrize("c,n1", [
    (W.Contract(W.ARITH, 16, 100.0, 1.0, 100.0, 0.05, 0.2, 2 ** 11, 4, W.BB), 2 ** 9),
    (W.Contract(W.BINARY, 12, 90.0, 0.5, 100.0, 0.03, 0.3, 3000, 3, W.PCA), 1000),
])
def test_pilot_and_rest_combine_to_the_whole_estimate(bench, oracle_lib, c, n1):
    oracle = oracle_lib
    args = (W.SCRAMBLE_SEED, c.type, c.d, c.K, c.T, c.S0, c.r, c.sigma, c.construction)
    _, _, whole = oracle.greeks(*args, c.N, c.R)
    per1 = oracle.partial_sums(*args, 0, c.R, 0, n1) / n1
    per2 = oracle.partial_sums(*args, 0, c.R, n1, c.N - n1) / (c.N - n1)
    combined = bench.combine_runs(per1, n1, per2, c.N - n1)
    scale = np.abs(whole).max(axis=0)
    assert np.all(np.abs(combined - whole) <= 1e-13 * scale + 1e-300), (combined, whole)
