/*
 * Plain FP64 CPU oracle for the QMC conditional-pathwise (QMC-CPW) Greeks
 * estimator of Bilokon, Kucherenko & Williams, "Quasi-Monte Carlo methods for
 * calculating derivatives sensitivities on the GPU" (arXiv 2209.11337).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link or
 * call this file: only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark use it.  It shares no code, header, table or constant
 * generator with the CUDA library; both sides are written independently from
 * the paper and from the published definitions they cite.
 *
 * Conventions (all functions):
 *   - d monitoring dates t_j = j*T/d, j = 1..d; n = d-1 sampled Gaussians
 *     (the first Gaussian x_1 is integrated out in closed form, Sec. 3.3.1).
 *   - option type: 0 arithmetic-Asian call, 1 binary-Asian (pays 1 if the
 *     arithmetic average exceeds K), 2 fixed-strike lookback call,
 *     3 geometric-Asian call (test-only product with a closed form).
 *   - construction: 0 Brownian bridge, 1 PCA, 2 standard (forward increments),
 *     all with x_1 (the first Brownian increment) integrated out; 3 and 4:
 *     the leading coordinate of the full-path bridge (3) or PCA (4) of the d
 *     dates integrated out instead, its switch point x* found by Newton's
 *     method (no lookback).  For 3 and 4, oracle_point's stilde (if given)
 *     receives the rest of the path R_j, j = 1..d.
 *   - value order of every 4-vector: price, delta, vega, gamma.
 *   - every int-returning function returns 0 on success, -1 on bad arguments.
 */
#ifndef QMCCPW_ORACLE_H
#define QMCCPW_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* The first `count` primitive polynomials over GF(2), in increasing
 * (degree, integer value) order; bit i of out[k] is the coefficient of x^i
 * (Sec. 2.2.2, eq. SobolPrimitivePolynomial). */
int oracle_primitive_polys(int count, uint32_t *out);

/* Unscrambled direction numbers: v[j*32 + (i-1)] = m_i << (32-i) for Sobol
 * dimension j (0-based), i = 1..32 (Sec. 2.2.2, eq. SobolRecurrenceRelation). */
int oracle_direction_numbers(int ndims, uint32_t *v);

/* Random linear scramble of replicate r, dimension j: rows[i-1] is the row
 * mask of output digit i of the lower-triangular unit-diagonal GF(2) matrix
 * L, *shift is the digital shift e (Sec. 2.2.3 randomisation). */
void oracle_scramble(uint64_t seed, uint32_t r, uint32_t j, uint32_t rows[32], uint32_t *shift);

/* 32-bit Sobol integers of points k0..k0+count-1 (index g(k) = k^(k>>1) if
 * gray, else k), dimensions 0..ndims-1, row-major out[(k-k0)*ndims + j].
 * scrambled != 0 applies replicate r's L and e. */
int oracle_sobol(uint64_t seed, uint32_t r, int ndims, uint64_t k0, uint64_t count,
                 int scrambled, int gray, uint32_t *out);

/* Inverse standard normal distribution function: the z with Phi(z) = u. */
double oracle_inv_normal(double u);

/* Brownian bridge: W[0..n] at s_i = i*dt from z[0..n-1] (z[0] drives s_n). */
int oracle_bridge(int n, double dt, const double *z, double *W);

/* Standard construction (Sec. 4.1-4.2 listing): W~(s_i) = W~(s_{i-1}) + sqrt(dt) z[i-1]. */
int oracle_forward(int n, double dt, const double *z, double *W);

/* PCA factor A (n x n, row-major) of Sigma_ik = dt*min(i,k): A = V diag(sqrt(lambda)). */
int oracle_pca_matrix(int n, double dt, double *A);

/* One point: the four conditional-pathwise values from the n normals z.
 * If stilde != NULL it receives the separated path S~(t_1..t_d). */
int oracle_point(int type, int d, double K, double T, double S0, double r, double sigma,
                 int construction, const double *z, double out[4], double *stilde);

/* Per-point values of points k0..k0+count-1 of replicate rep (out[count*4]). */
int oracle_point_values(uint64_t seed, int type, int d, double K, double T, double S0,
                        double r, double sigma, int construction, uint32_t rep,
                        uint64_t k0, uint64_t count, double *out);

/* The full estimator: per_rep[R*4] per-replicate means, mean[4] over replicates,
 * se[4] = standard error of that mean.  threads <= 0: OpenMP default. */
int oracle_greeks(uint64_t seed, int type, int d, double K, double T, double S0, double r,
                  double sigma, int construction, uint64_t N, int R, int threads,
                  double *per_rep, double *mean, double *se);

/* Same estimator restricted to replicates r0..r0+nrep-1 and points k0..k0+count-1:
 * sums[nrep*4] are the plain per-replicate SUMS (not means) over those points. */
int oracle_partial_sums(uint64_t seed, int type, int d, double K, double T, double S0,
                        double r, double sigma, int construction, uint32_t r0, int nrep,
                        uint64_t k0, uint64_t count, int threads, double *sums);

/* Basket of m <= 8 assets (Sec. 6's multi-asset extension): types 0
 * (arithmetic-Asian call on the basket average) and 1 (binary on it), bridge
 * per factor, the first increment of factor 1 integrated out, switch point
 * by Newton's method.  w[m] weights (w[0] > 0, others >= 0), a[m] relative
 * spots (S_i(0) = a_i S0), v[m] relative volatilities (sigma_i = v_i sigma),
 * corr[m*m] the correlation matrix (row-major, symmetric positive definite,
 * unit diagonal, corr[0][i] > 0).  Delta and gamma are with respect to the
 * spot scale S0, vega to the volatility scale sigma.  z holds m*d-1 normals:
 * z[b*m + k] drives bridge node b (0..d-2) of factor k+1 (k = 0..m-1), and
 * z[(d-1)*m + k-1] the first increment of factor k+1 (k = 1..m-1). */
int oracle_cholesky(int m, const double *C, double *L);
int oracle_basket_point(int type, int d, int m, double K, double T, double S0, double r, double sigma,
                        const double *w, const double *a, const double *v, const double *corr,
                        const double *z, double out[4]);
int oracle_basket_point_values(uint64_t seed, int type, int d, int m, double K, double T, double S0,
                               double r, double sigma, const double *w, const double *a, const double *v,
                               const double *corr, uint32_t rep, uint64_t k0, uint64_t count, double *out);
int oracle_basket_greeks(uint64_t seed, int type, int d, int m, double K, double T, double S0, double r,
                         double sigma, const double *w, const double *a, const double *v, const double *corr,
                         uint64_t N, int R, int threads, double *per_rep, double *mean, double *se);

#ifdef __cplusplus
}
#endif
#endif
