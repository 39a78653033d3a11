// Generated by gen_invnorm.py (do not edit): float inverse-normal polynomials.
// central: w in [0, 6.25], poly in (w - 3.0), max rel err 1.76e-07 (float Horner)
// tail: s = sqrt(w) in [2.5000, 4.6355], poly in (s - 3.25), max rel err 9.05e-08
#pragma once
#define QMC_INVN_W0 6.25f
#define QMC_INVN_SHIFT_C 3.0f
#define QMC_INVN_SHIFT_T 3.25f
#define QMC_INVN_CENTRAL {2.296035303e+00f, 3.417169974e-01f, -8.115864477e-03f, -1.182613189e-03f, 2.766207622e-04f, -1.792970698e-05f, -2.699825612e-06f, 6.252942986e-07f, -4.162018171e-09f, -7.202387477e-09f}
#define QMC_INVN_TAIL {4.361272918e+00f, 1.421650378e+00f, 7.592531650e-03f, -5.296074360e-03f, 3.544517404e-03f, -2.438567572e-03f, 1.314214131e-03f, -3.878564037e-04f, 8.778505019e-06f, 1.698554924e-05f}
// 2^f on [-1/2, 1/2], degree 6, max rel err 8.73e-08 (float Horner)
#define QMC_EXP2_POLY {1.000000001e+00f, 6.931472056e-01f, 2.402264661e-01f, 5.550328998e-02f, 9.618519534e-03f, 1.339986036e-03f, 1.533757682e-04f}
