"""Per-point error bounds of the float paths against the FP64 oracle (a test
helper, no GPU).

A point's float values differ from the FP64 ones through (1) the error of
ln X (X the path functional: the average or the maximum of S~/S0) and (2) the
float-float conditional step's own rounding.  (1) is bounded from the widths
of every float step:

  z          float inverse normal: |dz| <= 2.5e-7 max(|z|, 1), |z| < 6.4
             (u >= 2^-33); tensor cores add the lo-part rounding of the hi/lo
             split, 2^-15 (bf16: lo below 2^-6 with 8 significant bits) or
             2^-21 (tf32: below 2^-9 with 11 bits)
  w_i        the unit-spacing path, sum_k A_ik z_k: |dw_i| <= L1 |dz|max plus a
             float dot product's rounding (n ulps of sum |A_ik z_k|) plus, on
             tensor cores, Ahat's part rounding (bf16 three parts: 2^-23
             max|Ahat|; tf32 two: 2^-20 max|Ahat|) times sum |z_k|;
             L1 = max_i sum_k |A_ik| of the construction's factor
  ln S~_i    sigma sqrt(dt) |dw_i| + the exponential (2e-7)
  ln X       the largest ln S~_i error plus the float sum of d terms (d ulps)

and each Greek's sensitivity to ln X follows from the conditional formulas
(Sec. 3.3.2, 4.5), written with the point's own FP64 values, so no path
quantity is needed (G price, D delta, V vega, M gamma; a = sigma sqrt(t_1),
phi(psi) recovered from M or D):
  call (arithmetic, lookback, geometric):
    dG/dlnX = G + K e^{-rT} Phi-bar(psi) <= G + K e^{-rT}
    dD/dlnX = D + M S0                   (D1 S0 X phi(psi - a) = K e^{-rT} phi(psi))
    dM/dlnX = M |psi| / a
    dV/dlnX <= (M S0^2 a (|D/X|max / a + |psi| sqrt(t_1) / a)) + V
               + S0 Xmax |D/X|max (the error of D = dX/dsigma itself), with
               |D/X| <= 6 sqrt(T) + sigma T and X <= e^{6 sigma sqrt(T)} (paths
               within six standard deviations)
  binary:
    dG/dlnX = D S0
    dD/dlnX = D |psi| / a
    dM/dlnX = |d/dpsi (D (psi/a - 1)/S0)| / a
    dV/dlnX <= (|V| |psi| + D S0 a (1/sigma + |D/X|max / a)) / a
The bar per point and Greek is that sensitivity times the ln X bound, plus
1e-6 max(|value|, scale) for the conditional step (float Phi-bar and the
density: relative 3e-7; the float-float combinations: far below), scale the
mean |value| of the points tested.  A date of one point off by O(1) in w (a
wrong tensor-memory column or operand row) moves ln X by about
sigma sqrt(dt) |w| / d, far above these bars.
"""
import math

import numpy as np

import oracle
import workloads as W

EPS_INVN = 2.5e-7 * 6.4      # float inverse normal, absolute, at the largest |z|
ULP = 2.0 ** -24
SPLIT_Z = {W.MIXED: 0.0, W.MIXED_TC_BF16X3: 2.0 ** -15, W.MIXED_TC_TF32X3: 2.0 ** -21}
SPLIT_A = {W.MIXED: 0.0, W.MIXED_TC_BF16X3: 2.0 ** -23, W.MIXED_TC_TF32X3: 2.0 ** -20}


def factor(cons: int, n: int) -> np.ndarray:
    """The construction's factor for unit spacing: W~ = A z."""
    if n == 0:
        return np.zeros((0, 0))
    if cons == W.PCA:
        return oracle.pca_matrix(n, 1.0)
    eye = np.eye(n)
    fn = oracle.bridge if cons == W.BB else oracle.forward
    return np.column_stack([fn(n, 1.0, eye[k])[1:] for k in range(n)])  # W~(s_1..s_n), W~(s_0) = 0


def ln_x_bound(cons: int, d: int, T: float, sigma: float, precision: int) -> float:
    n = d - 1
    if n == 0:
        return 4e-7
    A = factor(cons, n)
    l1 = float(np.max(np.sum(np.abs(A), axis=1)))
    amax = float(np.max(np.abs(A)))
    dz = EPS_INVN + SPLIT_Z[precision]
    dw = l1 * dz + n * ULP * 6.4 * l1 + n * 6.4 * SPLIT_A[precision] * amax
    return sigma * math.sqrt(T / d) * dw + 2e-7 + (d + 2) * ULP


def bars(values: np.ndarray, typ: int, d: int, K: float, T: float, S0: float, r: float, sigma: float,
         cons: int, precision: int) -> np.ndarray:
    """Per-point, per-Greek bound on |float - FP64| (values: the FP64 points, n x 4)."""
    G, D, V, M = (values[:, g] for g in range(4))
    t1 = T / d
    a = sigma * math.sqrt(t1)
    disc = math.exp(-r * T)
    dx = 6.0 * math.sqrt(T) + sigma * T  # |D/X| for paths within six standard deviations
    if typ == W.BINARY:
        phi = np.abs(D) * S0 * a / disc
    else:
        phi = np.abs(M) * S0 * S0 * a / (disc * K)
    psi = np.sqrt(np.maximum(0.0, -2.0 * np.log(np.clip(phi * math.sqrt(2 * math.pi), 1e-300, 1.0))))
    if typ == W.BINARY:
        s = np.stack([np.abs(D) * S0,
                      np.abs(D) * psi / a,
                      (np.abs(V) * psi + np.abs(D) * S0 * a * (1.0 / sigma + dx / a)) / a,
                      np.abs(D) * (psi * np.abs(psi / a - 1.0) + 1.0 / a) / (S0 * a)], axis=1)
    else:
        s = np.stack([np.abs(G) + disc * K,
                      np.abs(D) + np.abs(M) * S0,
                      np.abs(M) * S0 * S0 * a * (dx / a + psi * math.sqrt(t1) / a) + np.abs(V)
                      + S0 * math.exp(6.0 * sigma * math.sqrt(T)) * dx,
                      np.abs(M) * psi / a], axis=1)
    eps = ln_x_bound(cons, d, T, sigma, precision)
    scale = np.mean(np.abs(values), axis=0)
    return s * eps + 1e-6 * np.maximum(np.abs(values), scale)
