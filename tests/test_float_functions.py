"""The float functions of the MIXED path, on the host.

The kernels evaluate e^x, -ln a, Phi^{-1} and the normal tail in float from
this project's own polynomials (csrc/float_coeffs.h, written by
csrc/gen_float_coeffs.py) with IEEE adds and fused multiply-adds only (plus
rcp.approx refined by a Newton step, restated here as the correctly rounded
reciprocal).  These tests (1) regenerate the coefficients and check that the
committed header is what the generator writes, and (2) restate the kernels'
float evaluation order in numpy (float32 roundings, an FMA as one rounding of
the exact double value) and compare with scipy's double ndtri, numpy's exp
and log and mpmath's erfc:
- the largest relative error stays within a few float ulps, and
- the error has no smooth part: its mean over narrow bins of the argument,
  and its projections that move an estimate (E[z dz], E[(z^3 - 3z) dz] for
  the inverse normal; the mean over a drifting path's exponents for e^x),
  are near zero.  A smooth error is the same for every point and does not
  average out over points; on the d = 64 benchmark grid (standard errors near
  1e-8 relative) the hardware lg2.approx inside the earlier inverse normal
  (E[z dz] = -2e-8) and an exponential whose linear coefficient was a rounded
  ln 2 (-8e-10 on drifting paths) each moved estimates by several tenths of a
  standard error.
"""
import os
import re
import sys

import numpy as np
import pytest

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2209_11337_gb300", "csrc")
f32 = np.float32
f64 = np.float64


def header():
    text = open(os.path.join(CSRC, "float_coeffs.h")).read()

    def scalar(name):
        return f32(float(re.search(rf"#define {name} ([-+0-9.e]+)f", text).group(1)))

    def array(name):
        body = re.search(rf"#define {name} \{{([^}}]*)\}}", text).group(1)
        return np.array([f32(float(x.strip().rstrip("f"))) for x in body.split(",")], dtype=np.float32)

    names = ["INVN_W0", "INVN_SHIFT_C", "INVN_SHIFT_T", "INVN_C0_HI", "INVN_C0_LO", "INVN_T0_HI", "INVN_T0_LO",
             "NTAIL_KAPPA", "NTAIL_YMAX", "NTAIL_SHIFT", "NTAIL_C0_HI", "NTAIL_C0_LO", "NTAIL_C1_HI", "NTAIL_C1_LO"]
    h = {n: scalar("QMC_" + n) for n in names}
    for n in ("EXP_POLY", "LN_POLY", "INVN_CENTRAL", "INVN_TAIL", "NTAIL_POLY"):
        h[n] = array("QMC_" + n)
    return h


def fma32(a, b, c):
    return f32(f64(a) * f64(b) + f64(c))


def horner32(coef, t, acc=None):
    acc = np.full_like(t, f32(coef[-1])) if acc is None else acc
    for c in coef[-2::-1]:
        acc = fma32(acc, t, f32(c))
    return acc


MAGIC = f32(12582912.0)
LOG2E = f32(1.44269502)
LN2_HI = f32(0.693147182464599609375)
LN2_LO = f32(-1.904654290e-09)


def exp32(x, h, xl=None):
    """fx::exp_f, or fx::exp_ff with a low part xl."""
    x = f32(x)
    m = fma32(x, LOG2E, MAGIC)
    nk = f32(f64(MAGIC) - f64(m))
    if xl is None:
        r = fma32(nk, LN2_HI, x)
        q = horner32(h["EXP_POLY"][1:], r)  # (1 + r q(r))(1 + delta), delta = -k lo
        delta = f32(f64(nk) * f64(LN2_LO))
        small = fma32(delta, f32(f64(q) * f64(r)), delta)
        p = f32(1.0 + f64(fma32(q, r, small)))
        return np.ldexp(p.astype(f64), (-nk).astype(np.int64)).astype(np.float32)
    else:
        P = f32(f64(nk) * f64(LN2_HI))
        perr = fma32(nk, LN2_HI, -P)
        r0 = f32(f64(x) + f64(P))
        small = f32(f64(fma32(nk, LN2_LO, f32(xl))) + f64(perr))
        r = f32(f64(r0) + f64(small))
    p = horner32(h["EXP_POLY"], r)
    return np.ldexp(p.astype(f64), (-nk).astype(np.int64)).astype(np.float32)


def neg_ln32(a, h):
    """fx::neg_ln2 on float a > 0."""
    a = f32(a)
    bits = a.view(np.uint32).astype(np.int64)
    e = (bits - 0x3F3504F3) >> 23
    m = ((bits - (e << 23)) & 0xFFFFFFFF).astype(np.uint32).view(np.float32)
    ef = f32(e.astype(f64))
    num = f32(f64(m) - 1.0)
    den = f32(f64(m) + 1.0)
    f = f32(f64(num) * f64(f32(1.0 / den.astype(f64))))
    t = f32(f64(f) * f64(f))
    p = horner32(-h["LN_POLY"], t)
    nlnm = fma32(f, p, f32(f64(ef) * f64(-LN2_LO)))
    return fma32(ef, -LN2_HI, nlnm)


def inv_normal32(y, h):
    """Arith<float>::inv_normal2 of u = (y + 1/2) 2^-32: (z, u, w)."""
    y = y.astype(np.uint64)
    upper = y >= 2 ** 31
    lo = np.where(upper, (2 ** 32 - 1) - y, y)
    q = f32((lo.astype(f64) + 0.5) * 2.0 ** -32)  # one rounding, as the kernel's two FMAs
    nq = -q
    xm = fma32(f32(-2.0), nq, f32(-1.0))
    q4 = f32(-4.0 * f64(nq))
    a = fma32(q4, nq, q4)
    w = neg_ln32(a, h)
    central = w < h["INVN_W0"]
    tc = f32(f64(w) - f64(h["INVN_SHIFT_C"]))
    pc = f32(f64(fma32(horner32(h["INVN_CENTRAL"], tc), tc, h["INVN_C0_LO"])) + f64(h["INVN_C0_HI"]))
    s = f32(np.sqrt(np.maximum(w, 0).astype(f64)))
    tt = f32(f64(s) - f64(h["INVN_SHIFT_T"]))
    pt = f32(f64(fma32(horner32(h["INVN_TAIL"], tt), tt, h["INVN_T0_LO"])) + f64(h["INVN_T0_HI"]))
    p = np.where(central, pc, pt)
    z = f32(f64(xm) * f64(p))
    return np.where(upper, -z, z), (y.astype(f64) + 0.5) * 2.0 ** -32, w


def ntail32(yh, h, yl=None):
    """fx::ntail: Phi(-y) for float y >= 0 (low part yl)."""
    yh = f32(yh)
    yl = np.zeros_like(yh) if yl is None else f32(yl)
    y = np.minimum(yh, h["NTAIL_YMAX"])
    sh = f32(f64(yh) * f64(yh))
    sl = f32(f64(fma32(yh, yh, -sh)) + f64(f32(f64(f32(2.0 * f64(yh))) * f64(yl))))
    gauss = np.where(yh <= h["NTAIL_YMAX"], exp32(f32(-0.5 * f64(sh)), h, f32(-0.5 * f64(sl))), f32(0))
    t = f32(1.0 / f64(fma32(h["NTAIL_KAPPA"], y, f32(1.0))))
    u = f32(f64(t) - f64(h["NTAIL_SHIFT"]))
    p = horner32(h["NTAIL_POLY"], u)
    p = f32(f64(fma32(p, u, h["NTAIL_C1_LO"])) + f64(h["NTAIL_C1_HI"]))
    p = f32(f64(fma32(p, u, h["NTAIL_C0_LO"])) + f64(h["NTAIL_C0_HI"]))
    return f32(f64(gauss) * f64(f32(f64(t) * f64(p)))), gauss


def binned_mean(arg, err, bins):
    edges = np.quantile(arg, np.linspace(0.0, 1.0, bins + 1))
    idx = np.clip(np.searchsorted(edges, arg, side="right") - 1, 0, bins - 1)
    sums = np.bincount(idx, weights=err, minlength=bins)
    counts = np.bincount(idx, minlength=bins)
    return sums / np.maximum(counts, 1)


def test_header_is_what_the_generator_writes(tmp_path):
    pytest.importorskip("mpmath")
    sys.path.insert(0, CSRC)
    try:
        import gen_float_coeffs as g
    finally:
        sys.path.remove(CSRC)
    h = header()
    ce, _ = g.fit_exp()
    cl, _ = g.fit_ln()
    cc, _, _ = g.fit_invn_central()
    ct, _, _ = g.fit_invn_tail()
    cn, _, _ = g.fit_ntail()
    assert np.array_equal(f32(ce), h["EXP_POLY"]) and np.array_equal(f32(cl), h["LN_POLY"])
    assert g.split(cc[0]) == (float(h["INVN_C0_HI"]), float(h["INVN_C0_LO"]))
    assert np.array_equal(f32(cc[1:]), h["INVN_CENTRAL"])
    assert g.split(ct[0]) == (float(h["INVN_T0_HI"]), float(h["INVN_T0_LO"]))
    assert np.array_equal(f32(ct[1:]), h["INVN_TAIL"])
    assert g.split(cn[0]) == (float(h["NTAIL_C0_HI"]), float(h["NTAIL_C0_LO"]))
    assert g.split(cn[1]) == (float(h["NTAIL_C1_HI"]), float(h["NTAIL_C1_LO"]))
    assert np.array_equal(f32(cn[2:]), h["NTAIL_POLY"])
    assert f32(g.KAPPA) == g.KAPPA  # the tail's variable is exact in float


def test_exponential_has_no_smooth_error_on_drifting_paths():
    h = header()
    rng = np.random.default_rng(7)
    # every reduced argument
    x = f32(rng.uniform(-80.0, 80.0, size=2_000_000))
    rel = exp32(x, h).astype(f64) / np.exp(x.astype(f64)) - 1.0
    assert np.max(np.abs(rel)) < 1.5e-7, np.max(np.abs(rel))
    frac = x.astype(f64) / np.log(2.0)
    frac = frac - np.round(frac)
    assert np.max(np.abs(binned_mean(frac, rel, 40))) < 3e-10
    # exponents of a path with drift (sigma 0.1 and 0.3, d = 64): mean relative error
    n = 4_000_000
    s = rng.integers(1, 64, n) / 64.0
    W = rng.normal(0.0, 1.0, n) * np.sqrt(s)
    for sig in (0.1, 0.3):
        lx = f32(sig * W + (0.05 - sig * sig / 2) * s)
        rel = exp32(lx, h).astype(f64) / np.exp(lx.astype(f64)) - 1.0
        assert abs(rel.mean()) < 1.5e-11, (sig, rel.mean())  # noise ~2e-11 / 2


def test_exponential_has_no_bias_for_any_k():
    # per k of the reduction the mean relative error over the arguments that
    # share it: dropping the -k ln2_lo remainder below half an ulp of the
    # reduced argument biased e^x by up to 5.6e-9 at x near 1.8 (k = 3), which
    # the leading-coordinate switch point turned into a 0.4 SE bias
    h = header()
    rng = np.random.default_rng(17)
    worst = 0.0
    for k in range(-20, 21):
        x = f32(k * np.log(2.0) + rng.uniform(-0.34, 0.34, size=400_000))
        rel = exp32(x, h).astype(f64) / np.exp(x.astype(f64)) - 1.0
        worst = max(worst, abs(rel.mean()))
    assert worst < 3e-10, worst  # noise per k ~3e-11
    # the leading-coordinate exponents: ln(S0/d) + small terms, S0 = 100, d = 16
    x = f32(np.log(100.0 / 16.0) + 0.05 * rng.standard_normal(2_000_000))
    rel = exp32(x, h).astype(f64) / np.exp(x.astype(f64)) - 1.0
    assert abs(rel.mean()) < 3e-10, rel.mean()


def test_float_float_exponential_has_no_smooth_error_for_any_k():
    # the Gaussian factor of the conditional step, e^{-y^2/2}: per k of the
    # reduction (|k| up to 125) the mean relative error over the arguments
    # that share it (the low part of the float-float argument varies there)
    h = header()
    rng = np.random.default_rng(5)
    yy = rng.uniform(0.0, 13.0, size=4_000_000)
    yh = f32(yy)
    yl = f32(yy - yh.astype(f64))
    sh = f32(f64(yh) * f64(yh))
    sl = f32(f64(fma32(yh, yh, -sh)) + f64(f32(f64(f32(2.0 * f64(yh))) * f64(yl))))
    xh, xl = f32(-0.5 * f64(sh)), f32(-0.5 * f64(sl))
    got = exp32(xh, h, xl).astype(f64)
    ref = np.exp(-0.5 * (yh.astype(f64) + yl.astype(f64)) ** 2)
    rel = got / ref - 1.0
    ok = ref > 1e-36
    assert np.max(np.abs(rel[ok])) < 2.5e-7
    k = np.round(xh.astype(f64) / np.log(2.0)).astype(int)
    worst = 0.0
    for kk in np.unique(k[ok]):
        sel = ok & (k == kk)
        if sel.sum() > 20000:
            worst = max(worst, abs(rel[sel].mean()))
    assert worst < 3e-9, worst  # noise per k ~1e-9 / 3


def test_negative_log_has_no_smooth_error():
    h = header()
    rng = np.random.default_rng(11)
    a = f32(np.exp(-rng.uniform(0.0, 22.0, size=2_000_000)))
    a = a[a > 0]
    got = neg_ln32(a, h).astype(f64)
    ref = -np.log(a.astype(f64))
    err = got - ref
    assert np.max(np.abs(err) / np.maximum(ref, 1.0)) < 2.5e-7
    # where the inverse normal uses it (a = 4q(1 - q), w = -ln a < 6.25): the
    # error is the rounding of w (ulp <= 2^-21, noise per bin ~2e-10)
    q = f32(rng.uniform(0.0, 0.5, size=8_000_000))
    a = fma32(f32(4.0) * q, -q, f32(4.0) * q)
    w = neg_ln32(a, h).astype(f64)
    ref = -np.log(a.astype(f64))
    keep = ref < 6.25
    assert np.max(np.abs(binned_mean(ref[keep], (w - ref)[keep], 20))) < 1e-9


def test_float_inverse_normal_error_is_small_and_has_no_smooth_part():
    from scipy.special import ndtri
    h = header()
    rng = np.random.default_rng(20250911)
    y = rng.integers(0, 2 ** 32, size=4_000_000, dtype=np.uint64)
    z, u, w = inv_normal32(y, h)
    ref = ndtri(u)
    dz = z.astype(f64) - ref
    # relative to max(|z|, 1): near z = 0 the float q = min(u, 1 - u) (ulp 2^-25
    # at 1/2) bounds the absolute error of 1 - 2q, hence of z, at ~1e-7
    err = dz / np.maximum(np.abs(ref), 1.0)
    assert np.max(np.abs(err)) < 2.5e-7, np.max(np.abs(err))
    # the smooth part, signed with z: the mean of err * sign(z) over 40 bins of w
    # (each ~100000 draws, rounding noise ~2e-10)
    smooth = binned_mean(w.astype(f64), err * np.sign(ref), 40)
    assert np.max(np.abs(smooth)) < 1.2e-9, np.max(np.abs(smooth))
    # the projections that act on an estimate: a rescaling of z (E[z dz], the
    # volatility of every path) and the next odd Hermite moment; noise ~3e-11
    assert abs(np.mean(ref * dz)) < 2e-10, np.mean(ref * dz)
    assert abs(np.mean((ref ** 3 - 3 * ref) * dz)) < 6e-10, np.mean((ref ** 3 - 3 * ref) * dz)


def test_normal_tail_matches_erfc_with_no_smooth_error():
    mp = pytest.importorskip("mpmath")
    from scipy.special import erfc
    h = header()
    rng = np.random.default_rng(3)
    y = f32(rng.uniform(0.0, 12.5, size=4_000_000))
    got, _ = ntail32(y, h)
    ref = 0.5 * erfc(y.astype(f64) / np.sqrt(2.0))
    rel = got.astype(f64) / ref - 1.0
    assert np.max(np.abs(rel)) < 5e-7, np.max(np.abs(rel))
    # 40 bins of 1e5 draws: rounding noise ~2.4e-10 per bin
    assert np.max(np.abs(binned_mean(y.astype(f64), rel, 40))) < 1e-9
    # spot values against mpmath (scipy's erfc has its own last-digit errors)
    for yy in (0.0, 0.5, 1.0, 2.5, 5.0, 8.0, 12.0):
        t, _ = ntail32(np.array([yy], dtype=np.float32), h)
        exact = float(mp.erfc(mp.mpf(yy) / mp.sqrt(2)) / 2)
        assert abs(float(t[0]) / exact - 1.0) < 3e-7, (yy, float(t[0]), exact)
    # beyond the range: zero; and the float-float low part enters the Gaussian
    # factor e^{-y^2/2} (the Mills-ratio factor takes y's float part: the
    # dropped part is a zero-mean rounding remainder), d/dy = -y T there
    t, g = ntail32(np.array([13.5], dtype=np.float32), h)
    assert t[0] == 0 and g[0] == 0
    yh = np.array([1.25], dtype=np.float32)
    t0, _ = ntail32(yh, h)
    t1, _ = ntail32(yh, h, np.array([1e-6], dtype=np.float32))
    d = (float(t1[0]) - float(t0[0])) / 1e-6
    assert abs(d / (-1.25 * float(t0[0])) - 1.0) < 0.05
