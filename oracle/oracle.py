"""ctypes wrapper around the plain C oracle (``qmccpw_oracle.c``).

TEST INFRASTRUCTURE ONLY.  ``build()`` compiles the C file with gcc into
``oracle/_build/liboracle.so`` (OpenMP over replicates, ``-ffp-contract=off``
so x86 and Arm round alike).  Every function below returns numpy arrays and
raises ``ValueError`` when the C side rejects its arguments.
"""
from __future__ import annotations

import contextlib
import ctypes
import os
import subprocess
import threading

import numpy as np

__all__ = [
    "ARITH", "BINARY", "LOOKBACK", "GEOMETRIC", "BB", "PCA", "STD", "forward",
    "build", "lib", "primitive_polys", "direction_numbers", "scramble",
    "sobol", "inv_normal", "bridge", "pca_matrix", "point", "point_values",
    "greeks", "partial_sums", "using_library", "compile_source", "Basket", "cholesky",
    "basket_point", "basket_point_values", "basket_greeks",
]

ARITH, BINARY, LOOKBACK, GEOMETRIC = 0, 1, 2, 3
BB, PCA, STD = 0, 1, 2

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qmccpw_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None


def compile_source(src: str, out_path: str) -> str:
    """gcc-compile an oracle source file into a shared library at ``out_path``."""
    tmp = out_path + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-I", _HERE, "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out_path)
    return out_path


def build(force: bool = False) -> str:
    """Compile the oracle (idempotent unless ``force``); returns the .so path."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and \
            os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(_SRC),
                                               os.path.getmtime(os.path.join(_HERE, "qmccpw_oracle.h"))):
        return _LIB_PATH
    return compile_source(_SRC, _LIB_PATH)


def _load(path: str) -> ctypes.CDLL:
    L = ctypes.CDLL(path)
    u32p = ctypes.POINTER(ctypes.c_uint32)
    dp = ctypes.POINTER(ctypes.c_double)
    i, u32, u64, d = ctypes.c_int, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double
    L.oracle_primitive_polys.argtypes = [i, u32p]
    L.oracle_direction_numbers.argtypes = [i, u32p]
    L.oracle_scramble.argtypes = [u64, u32, u32, u32p, u32p]
    L.oracle_scramble.restype = None
    L.oracle_sobol.argtypes = [u64, u32, i, u64, u64, i, i, u32p]
    L.oracle_inv_normal.argtypes = [d]
    L.oracle_inv_normal.restype = d
    L.oracle_bridge.argtypes = [i, d, dp, dp]
    L.oracle_pca_matrix.argtypes = [i, d, dp]
    L.oracle_forward.argtypes = [i, d, dp, dp]
    L.oracle_point.argtypes = [i, i, d, d, d, d, d, i, dp, dp, dp]
    L.oracle_point_values.argtypes = [u64, i, i, d, d, d, d, d, i, u32, u64, u64, dp]
    L.oracle_greeks.argtypes = [u64, i, i, d, d, d, d, d, i, u64, i, i, dp, dp, dp]
    L.oracle_partial_sums.argtypes = [u64, i, i, d, d, d, d, d, i, u32, i, u64, u64, i, dp]
    L.oracle_cholesky.argtypes = [i, dp, dp]
    L.oracle_basket_point.argtypes = [i, i, i, d, d, d, d, d, dp, dp, dp, dp, dp, dp]
    L.oracle_basket_point_values.argtypes = [u64, i, i, i, d, d, d, d, d, dp, dp, dp, dp, u32, u64, u64, dp]
    L.oracle_basket_greeks.argtypes = [u64, i, i, i, d, d, d, d, d, dp, dp, dp, dp, u64, i, i, dp, dp, dp]
    return L


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            _lib = _load(build())
        return _lib


@contextlib.contextmanager
def using_library(path: str):
    """Route every wrapper below through another build of the oracle for the
    duration of the block (the tests compile copies with planted mistakes and
    check that the pins reject them)."""
    global _lib
    lib()
    with _lock:
        saved = _lib
        _lib = _load(path)
    try:
        yield
    finally:
        with _lock:
            _lib = saved


def _u32(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))


def _f64(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _check(rc, what):
    if rc != 0:
        raise ValueError(f"oracle rejected arguments of {what}")


def primitive_polys(count: int) -> np.ndarray:
    out = np.zeros(max(count, 1), dtype=np.uint32)
    _check(lib().oracle_primitive_polys(count, _u32(out)), "primitive_polys")
    return out[:count]


def direction_numbers(ndims: int) -> np.ndarray:
    out = np.zeros((max(ndims, 1), 32), dtype=np.uint32)
    _check(lib().oracle_direction_numbers(ndims, _u32(out)), "direction_numbers")
    return out[:ndims]


def scramble(seed: int, r: int, j: int):
    rows = np.zeros(32, dtype=np.uint32)
    shift = np.zeros(1, dtype=np.uint32)
    lib().oracle_scramble(seed, r, j, _u32(rows), _u32(shift))
    return rows, int(shift[0])


def sobol(seed: int, r: int, ndims: int, k0: int, count: int, scrambled: bool = True,
          gray: bool = True) -> np.ndarray:
    out = np.zeros((count, ndims), dtype=np.uint32)
    _check(lib().oracle_sobol(seed, r, ndims, k0, count, int(scrambled), int(gray), _u32(out)), "sobol")
    return out


def inv_normal(u) -> np.ndarray:
    u = np.atleast_1d(np.asarray(u, dtype=np.float64))
    f = lib().oracle_inv_normal
    return np.array([f(float(x)) for x in u])


def bridge(n: int, dt: float, z) -> np.ndarray:
    z = np.ascontiguousarray(z, dtype=np.float64)
    W = np.zeros(n + 1)
    zz = z if n > 0 else np.zeros(1)
    _check(lib().oracle_bridge(n, dt, _f64(zz), _f64(W)), "bridge")
    return W


def forward(n: int, dt: float, z) -> np.ndarray:
    """Standard construction: W~(s_i) = W~(s_{i-1}) + sqrt(dt) z_i."""
    z = np.ascontiguousarray(z, dtype=np.float64)
    W = np.zeros(n + 1)
    zz = z if n > 0 else np.zeros(1)
    _check(lib().oracle_forward(n, dt, _f64(zz), _f64(W)), "forward")
    return W


def pca_matrix(n: int, dt: float) -> np.ndarray:
    A = np.zeros((max(n, 1), max(n, 1)))
    _check(lib().oracle_pca_matrix(n, dt, _f64(A)), "pca_matrix")
    return A[:n, :n]


def point(opt: int, d: int, K: float, T: float, S0: float, r: float, sigma: float,
          construction: int, z):
    """Values (price, delta, vega, gamma) and the separated path S~ of one point."""
    z = np.ascontiguousarray(z if d > 1 else np.zeros(1), dtype=np.float64)
    out = np.zeros(4)
    st = np.zeros(d)
    _check(lib().oracle_point(opt, d, K, T, S0, r, sigma, construction, _f64(z), _f64(out), _f64(st)),
           "point")
    return out, st


def point_values(seed: int, opt: int, d: int, K: float, T: float, S0: float, r: float,
                 sigma: float, construction: int, rep: int, k0: int, count: int) -> np.ndarray:
    out = np.zeros((count, 4))
    _check(lib().oracle_point_values(seed, opt, d, K, T, S0, r, sigma, construction, rep, k0, count,
                                     _f64(out)), "point_values")
    return out


def greeks(seed: int, opt: int, d: int, K: float, T: float, S0: float, r: float, sigma: float,
           construction: int, N: int, R: int, threads: int = 0):
    """Full estimator: (mean[4], se[4], per_replicate[R,4])."""
    per = np.zeros((R, 4))
    mean = np.zeros(4)
    se = np.zeros(4)
    _check(lib().oracle_greeks(seed, opt, d, K, T, S0, r, sigma, construction, N, R, threads,
                               _f64(per), _f64(mean), _f64(se)), "greeks")
    return mean, se, per


def partial_sums(seed: int, opt: int, d: int, K: float, T: float, S0: float, r: float,
                 sigma: float, construction: int, r0: int, nrep: int, k0: int, count: int,
                 threads: int = 0) -> np.ndarray:
    """Per-replicate SUMS over points k0..k0+count-1 of replicates r0..r0+nrep-1."""
    out = np.zeros((nrep, 4))
    _check(lib().oracle_partial_sums(seed, opt, d, K, T, S0, r, sigma, construction, r0, nrep, k0,
                                     count, threads, _f64(out)), "partial_sums")
    return out


# ---------------------------------------------------------------------------
# basket of m assets (Sec. 6's multi-asset extension; see qmccpw_oracle.h)
# ---------------------------------------------------------------------------
class Basket:
    """A basket contract: type (ARITH or BINARY on the basket average), d
    dates, strike K, maturity T, spot scale S0, rate r, volatility scale
    sigma, and per asset the weight w, relative spot a, relative volatility
    v, plus the correlation matrix corr (m x m)."""

    def __init__(self, type_, d, K, T, S0, r, sigma, w, a, v, corr):
        self.type, self.d, self.K, self.T, self.S0, self.r, self.sigma = type_, d, K, T, S0, r, sigma
        self.w = np.ascontiguousarray(w, dtype=np.float64)
        self.a = np.ascontiguousarray(a, dtype=np.float64)
        self.v = np.ascontiguousarray(v, dtype=np.float64)
        self.corr = np.ascontiguousarray(corr, dtype=np.float64)
        self.m = len(self.w)

    def replace(self, **kw):
        args = dict(type_=self.type, d=self.d, K=self.K, T=self.T, S0=self.S0, r=self.r, sigma=self.sigma,
                    w=self.w, a=self.a, v=self.v, corr=self.corr)
        args.update(kw)
        return Basket(**args)

    def _args(self):
        return (self.type, self.d, self.m, self.K, self.T, self.S0, self.r, self.sigma,
                _f64(self.w), _f64(self.a), _f64(self.v), _f64(self.corr))


def cholesky(C) -> np.ndarray:
    C = np.ascontiguousarray(C, dtype=np.float64)
    m = C.shape[0]
    L = np.zeros((m, m))
    _check(lib().oracle_cholesky(m, _f64(C), _f64(L)), "cholesky")
    return L


def basket_point(b: Basket, z) -> np.ndarray:
    """Values (price, delta, vega, gamma) of one point from its m d - 1 normals."""
    z = np.ascontiguousarray(z if b.m * b.d > 1 else np.zeros(1), dtype=np.float64)
    out = np.zeros(4)
    _check(lib().oracle_basket_point(*b._args(), _f64(z), _f64(out)), "basket_point")
    return out


def basket_point_values(seed: int, b: Basket, rep: int, k0: int, count: int) -> np.ndarray:
    out = np.zeros((count, 4))
    _check(lib().oracle_basket_point_values(seed, *b._args(), rep, k0, count, _f64(out)), "basket_point_values")
    return out


def basket_greeks(seed: int, b: Basket, N: int, R: int, threads: int = 0):
    """Full estimator of a basket: (mean[4], se[4], per_replicate[R,4])."""
    per = np.zeros((R, 4))
    mean = np.zeros(4)
    se = np.zeros(4)
    _check(lib().oracle_basket_greeks(seed, *b._args(), N, R, threads, _f64(per), _f64(mean), _f64(se)),
           "basket_greeks")
    return mean, se, per
