"""The float inverse normal and exponential of the MIXED path, on the host.

The kernels evaluate Phi^{-1} and e^x in float from fitted polynomials
(csrc/invnorm_coeffs.h, written by csrc/gen_invnorm.py).  These tests
(1) regenerate the coefficients and check that the committed header is what
the generator writes, and (2) restate the kernels' float evaluation order in
numpy (float32 roundings, an FMA as one rounding of the exact double value;
the hardware log2 replaced by a correctly rounded one) and compare with
scipy's double ndtri and numpy's exp:
- the largest relative error stays within a few float ulps, and
- the error has no smooth part: its mean over narrow bins of the argument is
  near zero.  A smooth error of Phi^{-1} is the same for every point and does
  not average out over points; the earlier coefficients (each rounded to float
  on its own) left one of up to ~8e-8 and biased the PCA estimates of the
  d = 64 grid by up to 0.8 standard errors against FP64.
"""
import os
import re
import sys

import numpy as np
import pytest

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2209_11337_gb300", "csrc")
f32 = np.float32


def header():
    text = open(os.path.join(CSRC, "invnorm_coeffs.h")).read()

    def scalar(name):
        return float(re.search(rf"#define {name} ([-+0-9.e]+)f", text).group(1))

    def array(name):
        body = re.search(rf"#define {name} \{{([^}}]*)\}}", text).group(1)
        return np.array([float(x.strip().rstrip("f")) for x in body.split(",")])

    return {"W0": scalar("QMC_INVN_W0"), "SC": scalar("QMC_INVN_SHIFT_C"), "ST": scalar("QMC_INVN_SHIFT_T"),
            "C0_HI": scalar("QMC_INVN_C0_HI"), "C0_LO": scalar("QMC_INVN_C0_LO"),
            "CENTRAL": array("QMC_INVN_CENTRAL"), "TAIL": array("QMC_INVN_TAIL"), "EXP2": array("QMC_EXP2_POLY")}


def fma32(a, b, c):
    return f32(np.float64(a) * np.float64(b) + np.float64(c))


def horner32(coef, t):
    acc = np.full_like(t, f32(coef[-1]))
    for c in coef[-2::-1]:
        acc = fma32(acc, t, f32(c))
    return acc


def inv_normal32(y, h):
    """The kernels' float Phi^{-1} of u = (y + 1/2) 2^-32 (scalar form)."""
    y = y.astype(np.uint64)
    upper = y >= 2 ** 31
    lo = np.where(upper, (2 ** 32 - 1) - y, y)
    q = f32((lo.astype(np.float64) + 0.5) * 2.0 ** -32)           # one rounding, as the kernel's two FMAs
    x = fma32(f32(-2.0), q, f32(1.0))
    q4 = f32(np.float64(f32(4.0)) * q)
    a = fma32(-q4, q, q4)
    w = f32(np.float64(f32(-0.693147181)) * np.float64(f32(np.log2(a.astype(np.float64)))))
    central = w < f32(h["W0"])
    t_c = f32(np.float64(w) - np.float64(f32(h["SC"])))
    p_c = f32(np.float64(fma32(horner32(h["CENTRAL"], t_c), t_c, f32(h["C0_LO"]))) + np.float64(f32(h["C0_HI"])))
    s = f32(np.sqrt(np.float64(w)))
    t_t = f32(np.float64(s) - np.float64(f32(h["ST"])))
    p_t = horner32(h["TAIL"], t_t)
    p = np.where(central, p_c, p_t)
    z = f32(-np.float64(x) * np.float64(p))
    return np.where(upper, -z, z), (y.astype(np.float64) + 0.5) * 2.0 ** -32, w


def ex32(x, h):
    """The kernels' float e^x: 2^k 2^f, k from the low bits of x log2 e + 1.5 2^23."""
    x = f32(x)
    r = fma32(x, f32(1.44269502), f32(12582912.0))
    kf = f32(np.float64(r) - 12582912.0)
    f = fma32(x, f32(1.92596299e-8), fma32(x, f32(1.44269502), -kf))
    p = horner32(h["EXP2"], f)
    return np.ldexp(p.astype(np.float64), kf.astype(np.int64)).astype(np.float32)


def binned_mean(arg, err, bins):
    edges = np.quantile(arg, np.linspace(0.0, 1.0, bins + 1))
    idx = np.clip(np.searchsorted(edges, arg, side="right") - 1, 0, bins - 1)
    sums = np.bincount(idx, weights=err, minlength=bins)
    counts = np.bincount(idx, minlength=bins)
    return sums / np.maximum(counts, 1)


def test_header_is_what_the_generator_writes():
    pytest.importorskip("mpmath")
    sys.path.insert(0, CSRC)
    try:
        import gen_invnorm as g
    finally:
        sys.path.remove(CSRC)
    h = header()
    c = g.fit(0.0, g.W0, g.DEG_C, "w", g.SHIFT_C, pair_c0=True)
    t = g.fit(np.sqrt(g.W0), np.sqrt(g.W_MAX), g.DEG_T, "s", g.SHIFT_T)
    e, _, _ = g.fit_exp2()
    assert f32(c[0]) == f32(h["C0_HI"]) and f32(c[1]) == f32(h["C0_LO"])
    assert np.array_equal(f32(c[2:]), f32(h["CENTRAL"]))
    assert np.array_equal(f32(t), f32(h["TAIL"]))
    assert np.array_equal(f32(e), f32(h["EXP2"]))


def test_float_inverse_normal_error_is_small_and_has_no_smooth_part():
    from scipy.special import ndtri
    h = header()
    rng = np.random.default_rng(20250911)
    y = rng.integers(0, 2 ** 32, size=2_000_000, dtype=np.uint64)
    z, u, w = inv_normal32(y, h)
    ref = ndtri(u)
    # relative to max(|z|, 1): near z = 0 the float q = min(u, 1 - u) (ulp 2^-25
    # at 1/2) bounds the absolute error of 1 - 2q, hence of z, at ~1e-7
    err = (z.astype(np.float64) - ref) / np.maximum(np.abs(ref), 1.0)
    assert np.max(np.abs(err)) < 2.5e-7, np.max(np.abs(err))
    # the smooth part, signed with z: the mean of err * sign(z) over 40 bins of
    # w (each ~50000 draws, rounding noise ~3e-10)
    smooth = binned_mean(w.astype(np.float64), err * np.sign(ref), 40)
    assert np.max(np.abs(smooth)) < 1.5e-8, np.max(np.abs(smooth))


def test_float_exponential_error_is_small_and_has_no_smooth_part():
    h = header()
    rng = np.random.default_rng(7)
    x = f32(rng.uniform(-6.0, 6.0, size=2_000_000))
    got = ex32(x, h).astype(np.float64)
    ref = np.exp(x.astype(np.float64))
    rel = got / ref - 1.0
    assert np.max(np.abs(rel)) < 1.5e-7, np.max(np.abs(rel))
    frac = x.astype(np.float64) * np.log2(np.e)
    frac = frac - np.round(frac)                 # the reduced argument f in [-1/2, 1/2]
    smooth = binned_mean(frac, rel, 40)
    assert np.max(np.abs(smooth)) < 1.5e-8, np.max(np.abs(smooth))
