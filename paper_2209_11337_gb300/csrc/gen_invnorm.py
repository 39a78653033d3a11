"""Fit the float polynomials used by the MIXED fused kernel.

1. Inverse normal.

Method (Giles, "Approximating the erfinv function", GPU Computing Gems Jade,
2011): with x = 1 - 2q (q = min(u, 1-u)) and w = -ln(1 - x^2) = -ln(4q(1-q)),
erfinv(x)/x is a smooth function of w on [0, W0] and of s = sqrt(w) beyond,
and Phi^{-1}(q) = -sqrt(2) erfinv(x).  The polynomials here are this
project's own least-squares fits (Chebyshev nodes, relative weighting, 80-digit
reference from mpmath), rebased to a shifted monomial form for Horner
evaluation in float, with the sqrt(2) folded in.

2. 2^f on [-1/2, 1/2] for the path exponentials e^x = 2^k 2^f (k the
   nearest integer to x log2 e): a degree-6 relative least-squares fit.

    python paper_2209_11337_gb300/csrc/gen_invnorm.py    # rewrites invnorm_coeffs.h
"""
import os

import mpmath as mp
import numpy as np

mp.mp.dps = 80
W0 = 6.25                               # central / tail switch in w
W_MAX = float(-mp.log(4 * mp.mpf(2) ** -33 * (1 - mp.mpf(2) ** -33)))  # smallest q = 2^-33
DEG_C, DEG_T = 9, 9
SHIFT_C = 3.0                            # central polynomial in (w - SHIFT_C)
SHIFT_T = 3.25                           # tail polynomial in (s - SHIFT_T)


def target_w(w):
    """sqrt(2) erfinv(x)/x as a function of w = -ln(1 - x^2)."""
    w = mp.mpf(w)
    if w == 0:
        return mp.sqrt(2) * mp.sqrt(mp.pi) / 2
    x = mp.sqrt(1 - mp.exp(-w))
    return mp.sqrt(2) * mp.erfinv(x) / x


def fit(lo, hi, deg, var, shift):
    # Chebyshev nodes on the fitting variable, many more than the degree
    k = np.arange(400)
    t = np.cos(np.pi * (k + 0.5) / 400)
    v = 0.5 * (lo + hi) + 0.5 * (hi - lo) * t
    w = v if var == "w" else v * v
    y = np.array([float(target_w(wi)) for wi in w])
    X = np.vander(v - shift, deg + 1, increasing=True)
    coef, *_ = np.linalg.lstsq(X / y[:, None], np.ones_like(y), rcond=None)  # relative least squares
    return coef


def horner32(coef, xs):
    acc = np.float32(coef[-1])
    for c in coef[-2::-1]:
        acc = np.float32(np.float32(acc) * xs + np.float32(c))
    return acc


def check(coef, lo, hi, var, shift):
    v = np.linspace(lo, hi, 20001)
    w = v if var == "w" else v * v
    ref = np.array([float(target_w(wi)) for wi in w[::40]])
    approx = horner32(coef, (v[::40] - shift).astype(np.float32)).astype(np.float64)
    return float(np.max(np.abs(approx / ref - 1)))


DEG_E = 6


def fit_exp2():
    k = np.arange(200)
    f = 0.5 * np.cos(np.pi * (k + 0.5) / 200)
    y = np.array([float(mp.power(2, mp.mpf(x))) for x in f])
    X = np.vander(f, DEG_E + 1, increasing=True)
    coef, *_ = np.linalg.lstsq(X / y[:, None], np.ones_like(y), rcond=None)
    fs = np.linspace(-0.5, 0.5, 4001)
    ref = np.array([float(mp.power(2, mp.mpf(x))) for x in fs[::4]])
    approx = horner32(coef, fs[::4].astype(np.float32)).astype(np.float64)
    return coef, float(np.max(np.abs(approx / ref - 1)))


def main():
    e, ee = fit_exp2()
    c = fit(0.0, W0, DEG_C, "w", SHIFT_C)
    t = fit(np.sqrt(W0), np.sqrt(W_MAX), DEG_T, "s", SHIFT_T)
    ec = check(c, 0.0, W0, "w", SHIFT_C)
    et = check(t, np.sqrt(W0), np.sqrt(W_MAX), "s", SHIFT_T)
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "invnorm_coeffs.h")
    with open(out, "w") as f:
        f.write("// Generated by gen_invnorm.py (do not edit): float inverse-normal polynomials.\n")
        f.write(f"// central: w in [0, {W0}], poly in (w - {SHIFT_C}), max rel err {ec:.2e} (float Horner)\n")
        f.write(f"// tail: s = sqrt(w) in [{np.sqrt(W0):.4f}, {np.sqrt(W_MAX):.4f}], poly in (s - {SHIFT_T}),"
                f" max rel err {et:.2e}\n#pragma once\n")
        f.write(f"#define QMC_INVN_W0 {W0}f\n#define QMC_INVN_SHIFT_C {SHIFT_C}f\n#define QMC_INVN_SHIFT_T {SHIFT_T}f\n")
        f.write("#define QMC_INVN_CENTRAL {" + ", ".join(f"{x:.9e}f" for x in c) + "}\n")
        f.write("#define QMC_INVN_TAIL {" + ", ".join(f"{x:.9e}f" for x in t) + "}\n")
        f.write(f"// 2^f on [-1/2, 1/2], degree {DEG_E}, max rel err {ee:.2e} (float Horner)\n")
        f.write("#define QMC_EXP2_POLY {" + ", ".join(f"{x:.9e}f" for x in e) + "}\n")
    print("central max rel err", ec, "tail max rel err", et, "exp2 max rel err", ee, "->", out)


if __name__ == "__main__":
    main()
