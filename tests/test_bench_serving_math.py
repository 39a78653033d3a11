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


class StandInServer:
    """The five serving calls of the library, answered on the host: every
    run returns per-replicate estimates whose delta standard error is that of
    the pilot (points 0 .. 2^12-1) scaled as 1/N over the points the request
    has by the end of the run, so the sizing rule's prediction holds exactly.
    It exercises the benchmark's threads, sizing, pilot reuse and accounting;
    the GPU path itself is tested elsewhere."""
    QMCCPW_BB = 0

    def __init__(self):
        import threading
        self.lock = threading.Lock()
        self.runs, self.next, self.point_dates, self.submitted = {}, 0, 0, []

    @staticmethod
    def pilot_se(c):
        return 2e-5 * c.d / 100.0

    def qmccpw_server_start(self, plan, **kw):
        pass

    def qmccpw_submit(self, plan, c):
        with self.lock:
            t = self.next
            self.next += 1
            self.runs[t] = c
            self.point_dates += c.N * c.R * c.d
            self.submitted.append(c)
        return t

    def qmccpw_wait(self, plan, t, R, timeout_ms):
        with self.lock:
            c = self.runs.pop(t)
        e = np.arange(R) - (R - 1) / 2.0
        e = e / e.std(ddof=1)                                # unit sample standard deviation
        per = np.tile(np.array([5.0, 0.5, 20.0, 0.02]), (R, 1))
        if c.first_point == 0:  # the pilot: its own standard error
            per[:, 1] += self.pilot_se(c) * np.sqrt(R) * e
        # the rest adds no spread: the point-weighted combination's SE is the pilot's times 2^12 / N
        se = per.std(axis=0, ddof=1) / np.sqrt(R)
        return per.mean(axis=0), se, per

    def qmccpw_server_get_stats(self, plan):
        return {"point_dates": self.point_dates, "launches": 1, "idle_exits": 0}

    def qmccpw_server_stop(self, plan):
        pass


def test_serving_driver_sizes_reuses_and_counts(bench):
    q = StandInServer()
    rate, window, warm = 400.0, 0.3, 0.1
    out = bench.serve(q, None, 1, rate, window, warmup_s=warm, seed=5)
    reqs = W.arrivals(rate_hz=rate, duration_s=warm + window, seed=5, R=16)
    sizes = [bench.request_size(q.pilot_se(rq.contract), rq.target_se) for rq in reqs]
    in_window = [(rq, n) for rq, n in zip(reqs, sizes) if rq.arrival_s >= warm]
    assert out["requests"] == len(in_window) > 0
    assert out["offered_point_dates_per_s"] == pytest.approx(
        sum(n * rq.contract.R * rq.contract.d for rq, n in in_window) / window)
    assert out["answered_by_pilot"] == pytest.approx(sum(n == 2 ** 12 for _, n in in_window) / len(in_window))
    assert out["delta_se_target_met"] == 1.0
    # every request: a pilot from point 0, and a main run over the points beyond the pilot's when it needs more
    pilots = [c for c in q.submitted if c.first_point == 0]
    mains = [c for c in q.submitted if c.first_point != 0]
    assert len(pilots) == len(reqs) and all(c.N == 2 ** 12 for c in pilots)
    assert sorted(c.first_point + c.N for c in mains) == sorted(n for n in sizes if n > 2 ** 12)
    assert all(c.first_point == 2 ** 12 for c in mains)
    assert out["p50_ms"] is not None and out["p99_ms"] >= out["p50_ms"]
