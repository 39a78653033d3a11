"""Seeded synthetic workloads for QMC-CPW Greeks.

Holds only input descriptions (contract and market parameters, point and
replicate counts, arrival times) drawn from fixed seeds; none of the method's
arithmetic.  Both the CUDA path (bench, GPU tests) and the CPU oracle (tests)
take their inputs from here.

The paper's experiments (Sec. 5) are synthetic: S(0)=100, sigma=0.2, r=0.1,
T=1, K in {90, 100, 110}, d in {64, 256}, 2^12..2^19 paths.  The workloads
below restate them at the sizes the GB300 build is measured on.
"""
from __future__ import annotations

from dataclasses import dataclass, replace
from typing import List

ARITH, BINARY, LOOKBACK, GEOMETRIC = 0, 1, 2, 3
BB, PCA, STD, BB_LEAD, PCA_LEAD = 0, 1, 2, 3, 4
FP64, MIXED, MIXED_TC_BF16X3, MIXED_TC_TF32X3 = 0, 1, 2, 3
TYPE_NAMES = {ARITH: "arith", BINARY: "binary", LOOKBACK: "lookback", GEOMETRIC: "geometric"}
CONS_NAMES = {BB: "bb", PCA: "pca", STD: "std", BB_LEAD: "bblead", PCA_LEAD: "pcalead"}

#: key of the random linear scrambles and digital shifts
SCRAMBLE_SEED = 0x220911337


@dataclass(frozen=True)
class Contract:
    type: int
    d: int
    K: float
    T: float
    S0: float
    r: float
    sigma: float
    N: int
    R: int
    construction: int = BB
    first_replicate: int = 0  # replicates first_replicate .. first_replicate + R - 1 of the randomisation
    first_point: int = 0      # Sobol' points first_point .. first_point + N - 1 of each replicate

    def label(self) -> str:
        return (f"{TYPE_NAMES[self.type]}-{CONS_NAMES[self.construction]}-d{self.d}-K{self.K:g}"
                f"-s{self.sigma:g}-N{self.N}-R{self.R}" + (f"@{self.first_replicate}" if self.first_replicate else "")
                + (f"+{self.first_point}" if self.first_point else ""))


def splitmix64(state: int):
    """SplitMix64 stream (Steele, Lea & Flood 2014) as a Python generator of 64-bit ints."""
    mask = (1 << 64) - 1
    while True:
        state = (state + 0x9E3779B97F4A7C15) & mask
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & mask
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & mask
        yield z ^ (z >> 31)


def _uniform(gen) -> float:
    return (next(gen) >> 11) * 2.0 ** -53


def small_arith() -> Contract:
    """Arithmetic-Asian call, d=16, bridge, N=2^14, R=8 (the small case)."""
    return Contract(ARITH, 16, 100.0, 1.0, 100.0, 0.05, 0.2, 2 ** 14, 8, BB)


def grid_d64(N: int = 2 ** 20, R: int = 32) -> List[Contract]:
    """{arith, binary, lookback} x {bridge, PCA} x K in {90,100,110} x sigma in {0.1,0.3}, d=64."""
    out = []
    for typ in (ARITH, BINARY, LOOKBACK):
        for cons in (BB, PCA):
            for K in (90.0, 100.0, 110.0):
                for sig in (0.1, 0.3):
                    out.append(Contract(typ, 64, K, 1.0, 100.0, 0.05, sig, N, R, cons))
    return out


def pca_stress(N: int = 2 ** 22, R: int = 16) -> List[Contract]:
    """PCA, d=256, the three products at S0=K=100, sigma=0.2, r=0.05, T=1."""
    return [Contract(t, 256, 100.0, 1.0, 100.0, 0.05, 0.2, N, R, PCA) for t in (ARITH, BINARY, LOOKBACK)]


def book(count: int = 4096, seed: int = 4, R: int = 16, construction: int = BB) -> List[Contract]:
    """Batched book: type ~ U{3}, d ~ U{12..365}, K ~ U(80,120), S0=100, sigma ~ U(0.1,0.5),
    T ~ U(0.25,2), r ~ U(0,0.08), N = 2^e with e ~ U{12..18}."""
    g = splitmix64(seed)
    out = []
    for _ in range(count):
        typ = next(g) % 3
        d = 12 + next(g) % (365 - 12 + 1)
        K = 80.0 + 40.0 * _uniform(g)
        sig = 0.1 + 0.4 * _uniform(g)
        T = 0.25 + 1.75 * _uniform(g)
        r = 0.08 * _uniform(g)
        e = 12 + next(g) % 7
        out.append(Contract(int(typ), int(d), K, T, 100.0, r, sig, 2 ** int(e), R, construction))
    return out


@dataclass(frozen=True)
class Request:
    arrival_s: float
    contract: Contract
    target_se: float


def arrivals(rate_hz: float = 2000.0, duration_s: float = 10.0, seed: int = 5, R: int = 16) -> List[Request]:
    """Poisson arrivals of book-like contracts, each with a target delta standard error
    drawn from {1e-3, 1e-4, 1e-5}; N is left at 2^12 for the caller to size."""
    import math

    g = splitmix64(seed)
    t = 0.0
    out = []
    while True:
        t += -math.log(1.0 - _uniform(g)) / rate_hz
        if t >= duration_s:
            break
        typ = next(g) % 3
        d = 12 + next(g) % (365 - 12 + 1)
        K = 80.0 + 40.0 * _uniform(g)
        sig = 0.1 + 0.4 * _uniform(g)
        T = 0.25 + 1.75 * _uniform(g)
        r = 0.08 * _uniform(g)
        tgt = (1e-3, 1e-4, 1e-5)[next(g) % 3]
        out.append(Request(t, Contract(int(typ), int(d), K, T, 100.0, r, sig, 2 ** 12, R, BB), tgt))
    return out


def with_size(c: Contract, N: int = None, R: int = None) -> Contract:
    return replace(c, N=c.N if N is None else N, R=c.R if R is None else R)


@dataclass(frozen=True)
class BasketSpec:
    """A basket of m assets (Sec. 6's multi-asset extension): type on the
    basket average, d dates, strike K, maturity T, spot scale S0, rate r,
    volatility scale sigma; per asset the weight w, relative spot a and
    relative volatility v; corr the m x m correlation (rows as tuples)."""
    type: int
    d: int
    K: float
    T: float
    S0: float
    r: float
    sigma: float
    w: tuple
    a: tuple
    v: tuple
    corr: tuple

    @property
    def m(self) -> int:
        return len(self.w)


def basket_d64(type_: int = ARITH, m: int = 4, K: float = 100.0) -> BasketSpec:
    """The measured basket: m = 4 equally weighted assets, d = 64, spots
    100 x (1, 0.95, 1.05, 1.1), volatilities 0.25 x (1, 0.8, 1.2, 1.4),
    pairwise correlation 0.5 (first m of each list)."""
    a = (1.0, 0.95, 1.05, 1.1, 0.9, 1.0, 1.2, 0.85)[:m]
    v = (1.0, 0.8, 1.2, 1.4, 0.9, 1.1, 0.7, 1.3)[:m]
    corr = tuple(tuple(1.0 if i == k else 0.5 for k in range(m)) for i in range(m))
    return BasketSpec(type_, 64, K, 1.0, 100.0, 0.05, 0.25, tuple([1.0 / m] * m), a, v, corr)
