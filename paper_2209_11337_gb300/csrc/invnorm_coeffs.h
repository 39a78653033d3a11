// Generated by gen_invnorm.py (do not edit): float inverse-normal polynomials.
// central: w in [0, 6.25], poly in (w - 3.0), degree 10, constant term a float pair; max rel err 1.11e-07, mean 1.1e-09 (float Horner)
// tail: s = sqrt(w) in [2.5000, 4.6355], poly in (s - 3.25), degree 9; max rel err 8.27e-08, mean -4.1e-09
#pragma once
#define QMC_INVN_W0 6.25f
#define QMC_INVN_SHIFT_C 3.0f
#define QMC_INVN_SHIFT_T 3.25f
#define QMC_INVN_C0_HI 2.296035051e+00f
#define QMC_INVN_C0_LO 8.209132574e-08f
#define QMC_INVN_CENTRAL {3.417170048e-01f, -8.115011267e-03f, -1.182568609e-03f, 2.759317285e-04f, -1.796644392e-05f, -2.504350505e-06f, 6.330791962e-07f, -2.690105738e-08f, -7.682931624e-09f, 9.305930471e-10f}  /* c1 .. */
#define QMC_INVN_TAIL {4.361272812e+00f, 1.421650290e+00f, 7.594018243e-03f, -5.295349285e-03f, 3.538578749e-03f, -2.439438133e-03f, 1.323711011e-03f, -3.894915571e-04f, 3.335269639e-06f, 1.935372711e-05f}
// 2^f on [-1/2, 1/2], degree 6, max rel err 6.11e-08, mean 1.2e-09 (float Horner)
#define QMC_EXP2_POLY {1.000000000e+00f, 6.931471825e-01f, 2.402264476e-01f, 5.550359190e-02f, 9.618841112e-03f, 1.339113689e-03f, 1.523800602e-04f}
