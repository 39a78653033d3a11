"""Fit the float polynomials used by the MIXED fused kernel.

1. Inverse normal.

Method (Giles, "Approximating the erfinv function", GPU Computing Gems Jade,
2011): with x = 1 - 2q (q = min(u, 1-u)) and w = -ln(1 - x^2) = -ln(4q(1-q)),
erfinv(x)/x is a smooth function of w on [0, W0] and of s = sqrt(w) beyond,
and Phi^{-1}(q) = -sqrt(2) erfinv(x).  The polynomials here are this
project's own least-squares fits (Chebyshev nodes, relative weighting, 80-digit
reference from mpmath) in a shifted monomial form for Horner evaluation in
float, with the sqrt(2) folded in.

The coefficients are rounded to float one at a time, lowest order first,
the remaining ones refitted after each rounding, so the roundings do not add
up to a smooth error of the polynomial; the central constant term is kept as
a float pair (hi + lo) and added last.  A smooth error of Phi^{-1} is the same
for every point and does not average out over points: with independently
rounded coefficients it biased the tensor-core PCA estimates of the d = 64
benchmark grid by up to 0.8 standard errors against FP64, where an exactly
rounded Phi^{-1} left 0.4.

2. 2^f on [-1/2, 1/2] for the path exponentials e^x = 2^k 2^f (k the
   nearest integer to x log2 e): a degree-6 relative least-squares fit,
   rounded the same way.

    python paper_2209_11337_gb300/csrc/gen_invnorm.py    # rewrites invnorm_coeffs.h
"""
import os

import mpmath as mp
import numpy as np

mp.mp.dps = 80
W0 = 6.25                               # central / tail switch in w
W_MAX = float(-mp.log(4 * mp.mpf(2) ** -33 * (1 - mp.mpf(2) ** -33)))  # smallest q = 2^-33
DEG_C, DEG_T = 10, 9
SHIFT_C = 3.0                            # central polynomial in (w - SHIFT_C)
SHIFT_T = 3.25                           # tail polynomial in (s - SHIFT_T)
DEG_E = 6


def target_w(w):
    """sqrt(2) erfinv(x)/x as a function of w = -ln(1 - x^2)."""
    w = mp.mpf(w)
    if w == 0:
        return mp.sqrt(2) * mp.sqrt(mp.pi) / 2
    x = mp.sqrt(1 - mp.exp(-w))
    return mp.sqrt(2) * mp.erfinv(x) / x


def fit_float(v, y, deg, shift, pair_c0=False):
    """Relative least squares of y on (v - shift)^k, k <= deg, the coefficients
    rounded to float lowest order first with the rest refitted; with pair_c0
    the constant term comes back as a float pair (hi, lo) ahead of c1..c_deg."""
    X = np.vander(v - shift, deg + 1, increasing=True) / y[:, None]
    fixed = []
    for i in range(deg + 1):
        rhs = np.ones_like(y) - (X[:, :i] @ np.array(fixed) if fixed else 0.0)
        coef, *_ = np.linalg.lstsq(X[:, i:], rhs, rcond=None)
        fixed.append(coef[0] if (pair_c0 and i == 0) else float(np.float32(coef[0])))
    if pair_c0:
        hi = float(np.float32(fixed[0]))
        return np.array([hi, float(np.float32(fixed[0] - hi))] + fixed[1:])
    return np.array(fixed)


def chebyshev(lo, hi, n=400):
    k = np.arange(n)
    return 0.5 * (lo + hi) + 0.5 * (hi - lo) * np.cos(np.pi * (k + 0.5) / n)


def fit(lo, hi, deg, var, shift, pair_c0=False):
    v = chebyshev(lo, hi)
    w = v if var == "w" else v * v
    y = np.array([float(target_w(wi)) for wi in w])
    return fit_float(v, y, deg, shift, pair_c0)


def horner32(coef, xs):
    acc = np.float32(coef[-1])
    for c in coef[-2::-1]:
        acc = np.float32(np.float64(acc) * xs + np.float32(c))  # one rounding, as an FMA
    return acc


def horner32_pair(coef, xs):
    """c0 = coef[0] + coef[1] (a float pair), c1.. = coef[2:]: the kernel's order."""
    q = horner32(coef[2:], xs)
    return np.float32(np.float32(np.float64(q) * xs + np.float32(coef[1])) + np.float32(coef[0]))


def check(coef, lo, hi, var, shift, pair_c0=False):
    v = np.linspace(lo, hi, 20001)[::40]
    w = v if var == "w" else v * v
    ref = np.array([float(target_w(wi)) for wi in w])
    xs = (v - shift).astype(np.float32)
    approx = (horner32_pair(coef, xs) if pair_c0 else horner32(coef, xs)).astype(np.float64)
    rel = approx / ref - 1
    return float(np.max(np.abs(rel))), float(np.mean(rel))


def fit_exp2():
    f = chebyshev(-0.5, 0.5, 200)
    y = np.array([float(mp.power(2, mp.mpf(x))) for x in f])
    coef = fit_float(f, y, DEG_E, 0.0)
    fs = np.linspace(-0.5, 0.5, 4001)[::4]
    ref = np.array([float(mp.power(2, mp.mpf(x))) for x in fs])
    rel = horner32(coef, fs.astype(np.float32)).astype(np.float64) / ref - 1
    return coef, float(np.max(np.abs(rel))), float(np.mean(rel))


def main():
    e, ee, me = fit_exp2()
    c = fit(0.0, W0, DEG_C, "w", SHIFT_C, pair_c0=True)
    t = fit(np.sqrt(W0), np.sqrt(W_MAX), DEG_T, "s", SHIFT_T)
    ec, mc = check(c, 0.0, W0, "w", SHIFT_C, pair_c0=True)
    et, mt = check(t, np.sqrt(W0), np.sqrt(W_MAX), "s", SHIFT_T)
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "invnorm_coeffs.h")
    with open(out, "w") as f:
        f.write("// Generated by gen_invnorm.py (do not edit): float inverse-normal polynomials.\n")
        f.write(f"// central: w in [0, {W0}], poly in (w - {SHIFT_C}), degree {DEG_C}, constant term a float pair;"
                f" max rel err {ec:.2e}, mean {mc:.1e} (float Horner)\n")
        f.write(f"// tail: s = sqrt(w) in [{np.sqrt(W0):.4f}, {np.sqrt(W_MAX):.4f}], poly in (s - {SHIFT_T}),"
                f" degree {DEG_T}; max rel err {et:.2e}, mean {mt:.1e}\n#pragma once\n")
        f.write(f"#define QMC_INVN_W0 {W0}f\n#define QMC_INVN_SHIFT_C {SHIFT_C}f\n#define QMC_INVN_SHIFT_T {SHIFT_T}f\n")
        f.write(f"#define QMC_INVN_C0_HI {c[0]:.9e}f\n#define QMC_INVN_C0_LO {c[1]:.9e}f\n")
        f.write("#define QMC_INVN_CENTRAL {" + ", ".join(f"{x:.9e}f" for x in c[2:]) + "}  /* c1 .. */\n")
        f.write("#define QMC_INVN_TAIL {" + ", ".join(f"{x:.9e}f" for x in t) + "}\n")
        f.write(f"// 2^f on [-1/2, 1/2], degree {DEG_E}, max rel err {ee:.2e}, mean {me:.1e} (float Horner)\n")
        f.write("#define QMC_EXP2_POLY {" + ", ".join(f"{x:.9e}f" for x in e) + "}\n")
    print("central", ec, mc, "tail", et, mt, "exp2", ee, me, "->", out)


if __name__ == "__main__":
    main()
