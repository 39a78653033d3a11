"""Fit the float polynomials of the MIXED path and write float_coeffs.h.

Every function the float path evaluates per date or per point is this
project's own polynomial, fitted here (relative least squares on Chebyshev
nodes, references from mpmath at 40 digits) and evaluated on the device with
IEEE float additions and fused multiply-adds only, so its error is the
rounding of those operations (zero-mean) plus the fit's own smooth error.  A
smooth error is the same for every point and does not average out: the
estimators of the d = 64 benchmark grid have standard errors of 1e-8
relative, and a path-level bias d moves an at-the-money call price by about
S0 delta d / price ~ 25 d, so the fits keep their smooth error near 1e-10.
Two rules serve that: coefficients are rounded to float one at a time,
lowest order first, the remaining ones refitted after each rounding; and
where a low-order coefficient's rounding cannot be absorbed (the constant
term at the centre of the interval, the linear term near it) it is kept as a
float pair, or made exact by the choice of variable.

1. e^r, |r| <= ln2/2 (the reduction r = x - k ln2 with ln2 as a float pair):
   degree 8 with c0 = c1 = 1 exact (a rounded ln2 as the linear coefficient
   of 2^f would leave an error linear in f, -1.7e-8 f, that biases paths with
   a drift).
2. ln m for m in [sqrt(1/2), sqrt(2)): ln m = f P(f^2), f = (m-1)/(m+1),
   P of degree 4 with P(0) = 2 exact (the atanh series).
3. The inverse normal in the two-branch form of Giles ("Approximating the
   erfinv function", GPU Computing Gems Jade, 2011): with x = 1 - 2q and
   w = -ln(4q(1-q)), Phi^{-1}(q) = -x p(w) for w < W0 and -x p_t(sqrt w)
   beyond (sqrt(2) folded in); p of degree 12 in (w - W0/2), p_t of degree
   11 in (sqrt w - its midpoint), constant terms as float pairs.
4. The upper normal tail T(y) = Phi(-y), y in [0, YMAX]: T(y) = e^{-y^2/2}
   t g(t) with t = 1/(1 + KAPPA y), g(t) = M(y)(1 + KAPPA y)/sqrt(2 pi), M the
   Mills ratio; g of degree 13 in (t - its midpoint), constant and linear
   terms as float pairs; KAPPA exact in float.

    python paper_2209_11337_gb300/csrc/gen_float_coeffs.py    # rewrites float_coeffs.h
"""
import os

import mpmath as mp
import numpy as np

mp.mp.dps = 40
f32 = np.float32

EXP_R = float(mp.log(2) / 2) + 1e-4      # reduced argument range (the rounding of k x log2 e adds < 1e-5)
DEG_EXP = 8
DEG_LN = 4
LN_F = float((mp.sqrt(2) - 1) / (mp.sqrt(2) + 1))   # largest |f|
W0 = 6.25                                # central / tail switch of the inverse normal, in w
W_MAX = float(-mp.log(4 * mp.mpf(2) ** -33 * (1 - mp.mpf(2) ** -33)))  # smallest q = 2^-33
DEG_C, DEG_T = 12, 11
KAPPA = 0.40625                          # 13/32: exact in float
YMAX = 13.0                              # beyond, e^{-y^2/2} underflows float
DEG_N = 13


def chebyshev(lo, hi, n=500):
    k = np.arange(n)
    return 0.5 * (lo + hi) + 0.5 * (hi - lo) * np.cos(np.pi * (k + 0.5) / n)


def fit_float(v, y, deg, shift=0.0, fixed=(), pairs=0):
    """Relative least squares of y on (v - shift)^k, k <= deg.  `fixed`: given
    leading coefficients (exact in float); the rest rounded to float one at a
    time, lowest order first, refitting the others after each; coefficients
    of order < `pairs` are kept as float pairs (returned as hi + lo doubles)."""
    X = np.vander(v - shift, deg + 1, increasing=True) / y[:, None]
    out = [float(c) for c in fixed]
    for i in range(len(out), deg + 1):
        rhs = np.ones_like(y) - (X[:, :i] @ np.array(out) if out else 0.0)
        coef, *_ = np.linalg.lstsq(X[:, i:], rhs, rcond=None)
        c = coef[0]
        if i < pairs:
            hi = float(f32(c))
            out.append(hi + float(f32(c - hi)))
        else:
            out.append(float(f32(c)))
    return np.array(out)


def split(c):
    hi = float(f32(c))
    return hi, float(f32(c - hi))


def peval(c, x):
    acc = np.zeros_like(x) + c[-1]
    for ci in c[-2::-1]:
        acc = acc * x + ci
    return acc


def max_rel(c, lo, hi, shift, ref_fn, n=3001):
    xs = np.linspace(lo, hi, n)
    ref = np.array([float(ref_fn(x)) for x in xs])
    return float(np.max(np.abs(peval(c, xs - shift) / ref - 1)))


# ---- targets ------------------------------------------------------------------
def target_w(w):
    """sqrt(2) erfinv(x)/x as a function of w = -ln(1 - x^2)."""
    w = mp.mpf(w)
    if w == 0:
        return mp.sqrt(2) * mp.sqrt(mp.pi) / 2
    x = mp.sqrt(1 - mp.exp(-w))
    return mp.sqrt(2) * mp.erfinv(x) / x


def ln_over_f(t):
    """ln(m)/f as a function of t = f^2, f = (m-1)/(m+1): 2 atanh(f)/f."""
    t = mp.mpf(t)
    return 2 * mp.atanh(mp.sqrt(t)) / mp.sqrt(t) if t > 0 else mp.mpf(2)


def g_of_t(t):
    t = mp.mpf(t)
    y = (1 / t - 1) / KAPPA
    mills = mp.erfc(y / mp.sqrt(2)) / 2 / (mp.exp(-y * y / 2) / mp.sqrt(2 * mp.pi))
    return mills * (1 + KAPPA * y) / mp.sqrt(2 * mp.pi)


# ---- fits -------------------------------------------------------------------
def fit_exp():
    r = chebyshev(-EXP_R, EXP_R, 300)
    y = np.array([float(mp.exp(mp.mpf(x))) for x in r])
    c = fit_float(r, y, DEG_EXP, fixed=(1.0, 1.0))
    return c, max_rel(c, -EXP_R, EXP_R, 0.0, lambda x: mp.exp(mp.mpf(x)))


def fit_ln():
    t = chebyshev(0.0, LN_F ** 2, 200)
    y = np.array([float(ln_over_f(x)) for x in t])
    c = fit_float(t, y, DEG_LN, fixed=(2.0,))
    return c, max_rel(c, 0.0, LN_F ** 2, 0.0, ln_over_f)


def fit_invn_central():
    shift = W0 / 2
    v = chebyshev(0.0, W0)
    y = np.array([float(target_w(x)) for x in v])
    c = fit_float(v, y, DEG_C, shift, pairs=1)
    return c, shift, max_rel(c, 0.0, W0, shift, target_w)


def fit_invn_tail():
    lo, hi = np.sqrt(W0), np.sqrt(W_MAX)
    shift = float(f32(0.5 * (lo + hi)))
    s = chebyshev(lo, hi, 400)
    y = np.array([float(target_w(x * x)) for x in s])
    c = fit_float(s, y, DEG_T, shift, pairs=1)
    return c, shift, max_rel(c, lo, hi, shift, lambda x: target_w(mp.mpf(x) ** 2))


def fit_ntail():
    tmin = 1.0 / (1.0 + KAPPA * YMAX)
    shift = float(f32(0.5 * (tmin + 1.0)))
    t = chebyshev(tmin, 1.0, 400)
    y = np.array([float(g_of_t(x)) for x in t])
    c = fit_float(t, y, DEG_N, shift, pairs=2)
    return c, shift, max_rel(c, tmin, 1.0, shift, g_of_t)


def fmt(xs):
    return "{" + ", ".join(f"{float(f32(x)):.9e}f" for x in xs) + "}"


def main():
    ce, ee = fit_exp()
    cl, el = fit_ln()
    cc, sc, ec = fit_invn_central()
    ct, st, et = fit_invn_tail()
    cn, sn, en = fit_ntail()
    c0h, c0l = split(cc[0])
    t0h, t0l = split(ct[0])
    n0h, n0l = split(cn[0])
    n1h, n1l = split(cn[1])
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "float_coeffs.h")
    with open(out, "w") as f:
        f.write("// Generated by gen_float_coeffs.py (do not edit): polynomials of the MIXED float path.\n")
        f.write("// Largest relative error of each fit with its float coefficients in exact arithmetic:\n")
        f.write(f"//   e^r, |r| <= {EXP_R:.6f}, degree {DEG_EXP}: {ee:.2e}\n")
        f.write(f"//   ln(m)/f in f^2, degree {DEG_LN}: {el:.2e}\n")
        f.write(f"//   inverse normal, central w in [0, {W0}], degree {DEG_C} in (w - {sc}): {ec:.2e}\n")
        f.write(f"//   inverse normal, tail sqrt(w) in [{np.sqrt(W0):.4f}, {np.sqrt(W_MAX):.4f}], degree {DEG_T}"
                f" in (s - {st:.9g}): {et:.2e}\n")
        f.write(f"//   normal tail g(t), t = 1/(1 + {KAPPA} y), y in [0, {YMAX}], degree {DEG_N} in (t - {sn:.9g}): {en:.2e}\n")
        f.write("#pragma once\n")
        f.write("#define QMC_EXP_POLY " + fmt(ce) + "  /* c0 .. c8 */\n")
        f.write("#define QMC_LN_POLY " + fmt(cl) + "  /* in f^2, c0 = 2 */\n")
        f.write(f"#define QMC_INVN_W0 {W0}f\n#define QMC_INVN_SHIFT_C {sc}f\n#define QMC_INVN_SHIFT_T {st:.9e}f\n")
        f.write(f"#define QMC_INVN_C0_HI {c0h:.9e}f\n#define QMC_INVN_C0_LO {c0l:.9e}f\n")
        f.write("#define QMC_INVN_CENTRAL " + fmt(cc[1:]) + "  /* c1 .. */\n")
        f.write(f"#define QMC_INVN_T0_HI {t0h:.9e}f\n#define QMC_INVN_T0_LO {t0l:.9e}f\n")
        f.write("#define QMC_INVN_TAIL " + fmt(ct[1:]) + "  /* c1 .. */\n")
        f.write(f"#define QMC_NTAIL_KAPPA {KAPPA}f\n#define QMC_NTAIL_YMAX {YMAX}f\n#define QMC_NTAIL_SHIFT {sn:.9e}f\n")
        f.write(f"#define QMC_NTAIL_C0_HI {n0h:.9e}f\n#define QMC_NTAIL_C0_LO {n0l:.9e}f\n")
        f.write(f"#define QMC_NTAIL_C1_HI {n1h:.9e}f\n#define QMC_NTAIL_C1_LO {n1l:.9e}f\n")
        f.write("#define QMC_NTAIL_POLY " + fmt(cn[2:]) + "  /* c2 .. */\n")
    print(f"exp {ee:.2e} ln {el:.2e} central {ec:.2e} tail {et:.2e} ntail {en:.2e} -> {out}")


if __name__ == "__main__":
    main()
