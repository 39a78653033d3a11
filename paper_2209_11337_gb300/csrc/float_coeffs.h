// Generated by gen_float_coeffs.py (do not edit): polynomials of the MIXED float path.
// Largest relative error of each fit with its float coefficients in exact arithmetic:
//   e^r, |r| <= 0.346674, degree 8: 9.68e-12
//   ln(m)/f in f^2, degree 4: 2.93e-11
//   inverse normal, central w in [0, 6.25], degree 12 in (w - 3.125): 6.45e-10
//   inverse normal, tail sqrt(w) in [2.5000, 4.6355], degree 11 in (s - 3.567734): 8.35e-10
//   normal tail g(t), t = 1/(1 + 0.40625 y), y in [0, 13.0], degree 13 in (t - 0.579602003): 4.58e-11
#pragma once
#define QMC_EXP_POLY {1.000000000e+00f, 1.000000000e+00f, 5.000000000e-01f, 1.666666716e-01f, 4.166667163e-02f, 8.333196864e-03f, 1.388773671e-03f, 1.995424391e-04f, 2.546113319e-05f}  /* c0 .. c8 */
#define QMC_LN_POLY {2.000000000e+00f, 6.666666269e-01f, 4.000084996e-01f, 2.851014137e-01f, 2.402921170e-01f}  /* in f^2, c0 = 2 */
#define QMC_INVN_W0 6.25f
#define QMC_INVN_SHIFT_C 3.125f
#define QMC_INVN_SHIFT_T 3.567734003e+00f
#define QMC_INVN_C0_HI 2.338620663e+00f
#define QMC_INVN_C0_LO 4.685584543e-08f
#define QMC_INVN_CENTRAL {3.396349549e-01f, -8.532895707e-03f, -1.047498197e-03f, 2.640782623e-04f, -1.964501462e-05f, -1.929631708e-06f, 6.035394335e-07f, -4.133504206e-08f, -6.691615262e-09f, 1.500286895e-09f, 6.982438065e-12f, -1.895752132e-11f}  /* c1 .. */
#define QMC_INVN_T0_HI 4.813605785e+00f
#define QMC_INVN_T0_LO -5.272720571e-08f
#define QMC_INVN_TAIL {1.425224066e+00f, 4.080932122e-03f, -2.539101988e-03f, 1.260712859e-03f, -7.434281288e-04f, 4.669105983e-04f, -2.593540121e-04f, 1.129342854e-04f, -1.737377897e-05f, -1.955930020e-05f, 9.781919289e-06f}  /* c1 .. */
#define QMC_NTAIL_KAPPA 0.40625f
#define QMC_NTAIL_YMAX 13.0f
#define QMC_NTAIL_SHIFT 5.796020031e-01f
#define QMC_NTAIL_C0_HI 3.150736392e-01f
#define QMC_NTAIL_C0_LO 5.832194172e-10f
#define QMC_NTAIL_C1_HI 3.779495656e-01f
#define QMC_NTAIL_C1_LO -4.368732487e-09f
#define QMC_NTAIL_POLY {1.880797744e-01f, -7.136301696e-02f, -8.585448563e-02f, 5.339292064e-02f, 3.333422914e-02f, -5.205040425e-02f, 7.519405801e-03f, 3.529731184e-02f, -3.289426491e-02f, -4.346681759e-03f, 2.638891712e-02f, -1.262066979e-02f}  /* c2 .. */
