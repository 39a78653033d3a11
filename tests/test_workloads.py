"""The seeded synthetic inputs follow the configured workloads: the d = 64
benchmark grid, the small case, the d = 256 PCA stress case, the
4096-contract book and the Poisson arrivals of the service (types, sizes and
parameter ranges as configured; the generator itself is SplitMix64, checked
against its published first outputs)."""
import math
from collections import Counter

import numpy as np

import workloads as W


def test_splitmix64_published_outputs():
    # the first outputs of SplitMix64 from state 0 (Steele, Lea & Flood's generator)
    g = W.splitmix64(0)
    assert [next(g) for _ in range(3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_grid_and_small_and_stress_cases():
    grid = W.grid_d64()
    assert len(grid) == 36
    assert {(c.type, c.construction, c.K, c.sigma) for c in grid} == {
        (t, k, K, s) for t in (W.ARITH, W.BINARY, W.LOOKBACK) for k in (W.BB, W.PCA)
        for K in (90.0, 100.0, 110.0) for s in (0.1, 0.3)}
    assert all((c.d, c.N, c.R, c.S0, c.r, c.T) == (64, 2 ** 20, 32, 100.0, 0.05, 1.0) for c in grid)
    s = W.small_arith()
    assert (s.type, s.d, s.N, s.R, s.construction, s.K, s.S0, s.sigma, s.r, s.T) == \
        (W.ARITH, 16, 2 ** 14, 8, W.BB, 100.0, 100.0, 0.2, 0.05, 1.0)
    st = W.pca_stress()
    assert [c.type for c in st] == [W.ARITH, W.BINARY, W.LOOKBACK]
    assert all((c.d, c.N, c.R, c.construction, c.K, c.sigma) == (256, 2 ** 22, 16, W.PCA, 100.0, 0.2) for c in st)


def test_book_follows_its_distributions():
    book = W.book()
    assert len(book) == 4096 and book == W.book()           # seeded: the same book every time
    types = Counter(c.type for c in book)
    assert set(types) == {W.ARITH, W.BINARY, W.LOOKBACK} and min(types.values()) > 1200
    d = np.array([c.d for c in book])
    assert d.min() >= 12 and d.max() <= 365 and abs(d.mean() - 188.5) < 5
    e = Counter(int(math.log2(c.N)) for c in book)
    assert set(e) == set(range(12, 19)) and all(c.N == 2 ** int(math.log2(c.N)) for c in book)
    for name, lo, hi in (("K", 80, 120), ("sigma", 0.1, 0.5), ("T", 0.25, 2.0), ("r", 0.0, 0.08)):
        x = np.array([getattr(c, name) for c in book])
        assert x.min() >= lo and x.max() <= hi, name
        assert abs(x.mean() - (lo + hi) / 2) < 0.03 * (hi - lo), name
    assert all(c.S0 == 100.0 and c.R == 16 and c.construction == W.BB for c in book)


def test_arrivals_are_poisson_at_the_rate():
    reqs = W.arrivals(rate_hz=2000.0, duration_s=2.0, seed=5)
    t = np.array([rq.arrival_s for rq in reqs])
    assert np.all(np.diff(t) > 0) and t[-1] < 2.0
    assert abs(len(reqs) - 4000) < 4 * math.sqrt(4000)     # Poisson count within 4 standard deviations
    gaps = np.diff(t)
    assert abs(gaps.mean() - 1 / 2000.0) < 0.05 / 2000.0
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.1           # exponential gaps: coefficient of variation 1
    assert {rq.target_se for rq in reqs} == {1e-3, 1e-4, 1e-5}
    assert all(rq.contract.N == 2 ** 12 and rq.contract.R == 16 for rq in reqs)
