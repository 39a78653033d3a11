/*
 * Plain FP64 CPU oracle for QMC-CPW Greeks (arXiv 2209.11337).
 *
 * TEST INFRASTRUCTURE ONLY: used by tests/, the smoke check and the CPU
 * baseline of bench.py.  Written for readability, not speed: every step is
 * the definition from the paper (section / equation named beside it) or from
 * the published algorithm it cites, computed in double precision, point by
 * point, with no blocking or reordering.  Where the paper is silent or
 * ambiguous the reading taken is stated at that step.
 *
 * Compile with -ffp-contract=off so that x86 and Arm builds round alike.
 */
#include "qmccpw_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define MAX_DIMS 4096

/* ------------------------------------------------------------------------ */
/* SplitMix64 (Steele, Lea & Flood, OOPSLA 2014), used counter-style: the    */
/* value for counter c under key s is the (c+1)-th output of the generator   */
/* whose state starts at s.                                                   */
/* ------------------------------------------------------------------------ */
static uint64_t splitmix64_at(uint64_t key, uint64_t counter)
{
    uint64_t z = key + (counter + 1u) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* Key of the stream that draws the initial direction integers m_1..m_q. */
static const uint64_t DIRECTION_KEY = 0x2209113370D1CE5Dull;

/* ------------------------------------------------------------------------ */
/* Sec. 2.2.2: primitive polynomials.  A polynomial of degree q with         */
/* constant term 1 is primitive iff the smallest p with P | x^p + 1 is       */
/* 2^q - 1, i.e. iff x has multiplicative order 2^q - 1 modulo P.  The order  */
/* is found by brute force: multiply by x until the residue returns to 1.   */
/* ------------------------------------------------------------------------ */
static int poly_degree(uint32_t p)
{
    int q = -1;
    while (p) { p >>= 1; ++q; }
    return q;
}

static int is_primitive(uint32_t p)
{
    int q = poly_degree(p);
    if (q < 1 || !(p & 1u)) return 0;
    uint32_t period = (1u << q) - 1u;
    uint32_t residue = 1u; /* the polynomial "1" */
    for (uint32_t e = 1; e <= period; ++e) {
        residue <<= 1;                    /* times x */
        if (residue & (1u << q)) residue ^= p; /* reduce modulo P */
        if (residue == 1u) return e == period;
    }
    return 0;
}

int oracle_primitive_polys(int count, uint32_t *out)
{
    if (count < 0 || (count > 0 && !out)) return -1;
    int found = 0;
    for (uint32_t p = 2; found < count; ++p) {
        if (p >= (1u << 20)) return -1;
        if (is_primitive(p)) out[found++] = p;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Sec. 2.2.2: direction numbers.  Dimension 0 has generator matrix I       */
/* (van der Corput).  Dimension j >= 1 uses the j-th primitive polynomial    */
/* x^q + c_1 x^{q-1} + ... + c_{q-1} x + 1, initial m_1..m_q odd with        */
/* m_i < 2^i (drawn from SplitMix64 under DIRECTION_KEY, counter (j<<8)|i),  */
/* and the recurrence                                                         */
/*   m_i = 2c_1 m_{i-1} ^ 4c_2 m_{i-2} ^ ... ^ 2^{q-1}c_{q-1} m_{i-q+1}       */
/*         ^ 2^q m_{i-q} ^ m_{i-q}.                                           */
/* The direction number g_i = m_i / 2^i is stored as the 32-bit integer      */
/* m_i << (32 - i) (binary point before bit 31).                              */
/* The paper names no table of initial values (Sec. 2.2.2, last paragraph); */
/* this seeded choice is the reading used on both sides.                     */
/* ------------------------------------------------------------------------ */
int oracle_direction_numbers(int ndims, uint32_t *v)
{
    if (ndims < 0 || ndims > MAX_DIMS || (ndims > 0 && !v)) return -1;
    if (ndims == 0) return 0;
    uint32_t *polys = NULL;
    if (ndims > 1) {
        polys = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(ndims - 1));
        if (!polys || oracle_primitive_polys(ndims - 1, polys) != 0) { free(polys); return -1; }
    }
    for (int j = 0; j < ndims; ++j) {
        uint64_t m[33]; /* m[1..32] */
        if (j == 0) {
            for (int i = 1; i <= 32; ++i) m[i] = 1u;
        } else {
            uint32_t p = polys[j - 1];
            int q = poly_degree(p);
            for (int i = 1; i <= q && i <= 32; ++i) {
                uint64_t draw = splitmix64_at(DIRECTION_KEY, ((uint64_t)j << 8) | (uint64_t)i) >> 32;
                m[i] = (draw & ((1ull << i) - 1u)) | 1u;
            }
            for (int i = q + 1; i <= 32; ++i) {
                uint64_t mi = 0;
                for (int k = 1; k <= q - 1; ++k) {
                    uint64_t ck = (p >> (q - k)) & 1u; /* coefficient of x^{q-k} */
                    if (ck) mi ^= (m[i - k] << k);
                }
                mi ^= (m[i - q] << q);
                mi ^= m[i - q];
                m[i] = mi;
            }
        }
        for (int i = 1; i <= 32; ++i) v[j * 32 + (i - 1)] = (uint32_t)(m[i] << (32 - i));
    }
    free(polys);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Sec. 2.2.3 randomisation, read as a random linear scramble plus digital   */
/* shift: y' = L y + e over GF(2) on the 32 binary digits of a coordinate,   */
/* L lower triangular with unit diagonal (digit i of the output depends on   */
/* input digits 1..i, digit 1 being the 1/2 digit).  Row i of L has bits for  */
/* digits k < i drawn from SplitMix64 under the caller's seed, counter       */
/* (r<<32)|(j<<8)|(i-1); e uses counter (r<<32)|(j<<8)|32.  Digit i lives in */
/* bit 32-i of the word.                                                      */
/* ------------------------------------------------------------------------ */
void oracle_scramble(uint64_t seed, uint32_t r, uint32_t j, uint32_t rows[32], uint32_t *shift)
{
    uint64_t base = ((uint64_t)r << 32) | ((uint64_t)j << 8);
    for (int i = 1; i <= 32; ++i) {
        uint32_t diag = 1u << (32 - i);
        uint32_t above = (i >= 2) ? (0xFFFFFFFFu << (33 - i)) : 0u;
        uint32_t draw = (uint32_t)(splitmix64_at(seed, base | (uint64_t)(i - 1)) >> 32);
        rows[i - 1] = (draw & above) | diag;
    }
    *shift = (uint32_t)(splitmix64_at(seed, base | 32u) >> 32);
}

static int parity32(uint32_t x)
{
    int p = 0;
    while (x) { p ^= 1; x &= x - 1u; }
    return p;
}

/* y = G a(k) mod 2 (eq. GeneratorMatrixExpression) as the XOR of the        */
/* direction numbers selected by the set bits of the index.                  */
static uint32_t sobol_unscrambled(const uint32_t *vdim, uint64_t index)
{
    uint32_t y = 0;
    for (int b = 0; b < 32; ++b)
        if ((index >> b) & 1u) y ^= vdim[b];
    return y;
}

/* Apply L (matrix-vector product over GF(2)) and the shift e. */
static uint32_t scramble_apply(const uint32_t rows[32], uint32_t shift, uint32_t y)
{
    uint32_t out = 0;
    for (int i = 1; i <= 32; ++i)
        if (parity32(rows[i - 1] & y)) out |= 1u << (32 - i);
    return out ^ shift;
}

int oracle_sobol(uint64_t seed, uint32_t r, int ndims, uint64_t k0, uint64_t count,
                 int scrambled, int gray, uint32_t *out)
{
    if (ndims < 1 || ndims > MAX_DIMS || !out) return -1;
    if (k0 + count > (1ull << 32) || k0 + count < k0) return -1;
    uint32_t *v = (uint32_t *)malloc(sizeof(uint32_t) * 32u * (size_t)ndims);
    uint32_t *rows = (uint32_t *)malloc(sizeof(uint32_t) * 32u * (size_t)ndims);
    uint32_t *shift = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)ndims);
    if (!v || !rows || !shift || oracle_direction_numbers(ndims, v) != 0) {
        free(v); free(rows); free(shift); return -1;
    }
    for (int j = 0; j < ndims; ++j) oracle_scramble(seed, r, (uint32_t)j, rows + 32 * j, shift + j);
    for (uint64_t t = 0; t < count; ++t) {
        uint64_t k = k0 + t;
        uint64_t index = gray ? (k ^ (k >> 1)) : k;
        for (int j = 0; j < ndims; ++j) {
            uint32_t y = sobol_unscrambled(v + 32 * j, index);
            if (scrambled) y = scramble_apply(rows + 32 * j, shift[j], y);
            out[t * (uint64_t)ndims + (uint64_t)j] = y;
        }
    }
    free(v); free(rows); free(shift);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Normal distribution.  Phi(z) = erfc(-z/sqrt2)/2, the complementary form   */
/* keeps relative accuracy in the lower tail.                                 */
/* ------------------------------------------------------------------------ */
static const double INV_SQRT2 = 0.70710678118654752440;
static const double INV_SQRT2PI = 0.39894228040143267794;

static double norm_cdf(double z) { return 0.5 * erfc(-z * INV_SQRT2); }
static double norm_sf(double z) { return 0.5 * erfc(z * INV_SQRT2); } /* 1 - Phi(z) */
static double norm_pdf(double z) { return INV_SQRT2PI * exp(-0.5 * z * z); }

/* Inverse normal: z with Phi(z) = u.  Start from Abramowitz & Stegun         */
/* 26.2.23 (absolute error < 4.5e-4) on the lower half q = min(u, 1-u), then */
/* refine with Halley's method on f(z) = Phi(z) - q until the step is below  */
/* one part in 1e16.  For u > 1/2 the result is -z(1-u); 1-u is exact for the */
/* dyadic u used here.                                                         */
double oracle_inv_normal(double u)
{
    if (!(u > 0.0 && u < 1.0)) return NAN;
    double q = (u <= 0.5) ? u : 1.0 - u;
    double t = sqrt(-2.0 * log(q));
    double z = -(t - (2.515517 + 0.802853 * t + 0.010328 * t * t) /
                     (1.0 + 1.432788 * t + 0.189269 * t * t + 0.001308 * t * t * t));
    for (int it = 0; it < 50; ++it) {
        double e = (norm_cdf(z) - q) / norm_pdf(z);
        double step = e / (1.0 + 0.5 * z * e);
        z -= step;
        if (fabs(step) <= 1e-16 * fmax(1.0, fabs(z))) break;
    }
    return (u <= 0.5) ? z : -z;
}

/* ------------------------------------------------------------------------ */
/* Sec. 4.4 Brownian bridge for the n values W~(s_1..s_n), s_i = i*dt, with  */
/* W~(s_0) = 0.  z[0] sets the terminal value W~(s_n) = sqrt(s_n) z[0]; then */
/* intervals (l, r) are refined breadth first, left to right within a level: */
/* m = floor((l+r)/2) gets the conditional mean of its endpoints plus the    */
/* conditional standard deviation times the next z (Glasserman, Sec. 3.1).   */
/* The paper's listing assumes 2^m steps on a unit horizon and walks each     */
/* level right to left; this general form is the reading used on both sides. */
/* ------------------------------------------------------------------------ */
int oracle_bridge(int n, double dt, const double *z, double *W)
{
    if (n < 0 || !(dt > 0.0) || !W || (n > 0 && !z)) return -1;
    W[0] = 0.0;
    if (n == 0) return 0;
    int *ql = (int *)malloc(sizeof(int) * (size_t)(2 * n + 2));
    int *qr = (int *)malloc(sizeof(int) * (size_t)(2 * n + 2));
    if (!ql || !qr) { free(ql); free(qr); return -1; }
    int next = 0;
    W[n] = sqrt(n * dt) * z[next++];
    int head = 0, tail = 0;
    ql[tail] = 0; qr[tail] = n; ++tail;
    while (head < tail) {
        int l = ql[head], r = qr[head]; ++head;
        if (r - l < 2) continue;
        int m = (l + r) / 2;
        double sl = l * dt, sm = m * dt, sr = r * dt;
        double mean = ((sr - sm) * W[l] + (sm - sl) * W[r]) / (sr - sl);
        double sd = sqrt((sm - sl) * (sr - sm) / (sr - sl));
        W[m] = mean + sd * z[next++];
        ql[tail] = l; qr[tail] = m; ++tail;
        ql[tail] = m; qr[tail] = r; ++tail;
    }
    free(ql); free(qr);
    return (next == n) ? 0 : -1;
}

/* ------------------------------------------------------------------------ */
/* Standard construction: the path the paper's simulation listing builds     */
/* (Sec. 4.1-4.2), one independent increment per step,                       */
/*   W~(s_i) = W~(s_{i-1}) + sqrt(dt) z_i,  i = 1..n,  W~(s_0) = 0,            */
/* so Sobol' dimension i drives the increment of step i.                      */
/* ------------------------------------------------------------------------ */
int oracle_forward(int n, double dt, const double *z, double *W)
{
    if (n < 0 || !(dt > 0.0) || !W || (n > 0 && !z)) return -1;
    const double h = sqrt(dt);
    W[0] = 0.0;
    for (int i = 1; i <= n; ++i) W[i] = W[i - 1] + h * z[i - 1];
    return 0;
}

/* ------------------------------------------------------------------------ */
/* PCA construction (named as future work in Sec. 6 / 7): W~ = A z with      */
/* A A^T = Sigma, Sigma_ik = dt*min(i,k) (eq. WboldTilde with equal steps).   */
/* For this matrix the eigenpairs are known in closed form:                   */
/*   lambda_k = dt / (4 sin^2((2k-1) pi / (2(2n+1)))),                        */
/*   v_k(i)   = 2/sqrt(2n+1) * sin((2k-1) i pi / (2n+1)),  k, i = 1..n,       */
/* in decreasing lambda; A(i,k) = v_k(i) sqrt(lambda_k), so Sobol dimension k  */
/* drives principal component k.                                              */
/* ------------------------------------------------------------------------ */
int oracle_pca_matrix(int n, double dt, double *A)
{
    if (n < 0 || !(dt > 0.0) || (n > 0 && !A)) return -1;
    const double pi = 3.14159265358979323846;
    for (int k = 1; k <= n; ++k) {
        double s = sin((2.0 * k - 1.0) * pi / (2.0 * (2.0 * n + 1.0)));
        double lambda = dt / (4.0 * s * s);
        for (int i = 1; i <= n; ++i) {
            double vki = 2.0 / sqrt(2.0 * n + 1.0) * sin((2.0 * k - 1.0) * i * pi / (2.0 * n + 1.0));
            A[(size_t)(i - 1) * (size_t)n + (size_t)(k - 1)] = vki * sqrt(lambda);
        }
    }
    return 0;
}

static int pca_apply(int n, const double *A, const double *z, double *W)
{
    W[0] = 0.0;
    for (int i = 1; i <= n; ++i) {
        double acc = 0.0;
        for (int k = 0; k < n; ++k) acc += A[(size_t)(i - 1) * (size_t)n + (size_t)k] * z[k];
        W[i] = acc;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.3.1-3.3.2 and Sec. 4.5: separated path and conditional Greeks.     */
/*   S~(t_j) = S0 exp(omega (t_j - t_1) + sigma W~(t_j - t_1)), j = 1..d,     */
/*   omega = r - sigma^2/2, t_1 = T/d, a = sigma sqrt(t_1),                   */
/*   psi = (ln K - ln X - omega t_1) / a  (the switch point in x_1),          */
/* with X the path functional (arithmetic mean, maximum or geometric mean of */
/* S~) and D = dX/dsigma at fixed z.                                          */
/* ------------------------------------------------------------------------ */
typedef struct {
    int type, d;
    double K, T, S0, r, sigma;
} contract_t;

static int check_contract(const contract_t *c, int construction)
{
    if (c->type < 0 || c->type > 3) return -1;
    if (c->d < 1 || c->d > MAX_DIMS) return -1;
    if (!(c->K > 0.0) || !(c->T > 0.0) || !(c->S0 > 0.0) || !(c->sigma > 0.0)) return -1;
    if (!isfinite(c->K) || !isfinite(c->T) || !isfinite(c->S0) || !isfinite(c->sigma) || !isfinite(c->r)) return -1;
    if (construction < 0 || construction > 4) return -1;
    return 0;
}

/* Values from the path W~(s_0..s_n), s_i = i t_1 (the date t_{i+1}). */
static void greeks_from_path(const contract_t *c, const double *W, double out[4], double *stilde)
{
    const int d = c->d, n = d - 1;
    const double t1 = c->T / d;
    const double omega = c->r - 0.5 * c->sigma * c->sigma;
    const double a = c->sigma * sqrt(t1);

    double X, D;
    if (c->type == 0 || c->type == 1) {           /* arithmetic mean of S~ */
        double sum = 0.0, dsum = 0.0;
        for (int i = 0; i <= n; ++i) {
            double s = i * t1;
            double St = c->S0 * exp(omega * s + c->sigma * W[i]);
            if (stilde) stilde[i] = St;
            sum += St;
            dsum += St * (W[i] - c->sigma * s);
        }
        X = sum / d;
        D = dsum / d;
    } else if (c->type == 2) {                    /* maximum of S~, lowest index on ties */
        double best = -1.0, dbest = 0.0;
        for (int i = 0; i <= n; ++i) {
            double s = i * t1;
            double St = c->S0 * exp(omega * s + c->sigma * W[i]);
            if (stilde) stilde[i] = St;
            if (St > best) { best = St; dbest = St * (W[i] - c->sigma * s); }
        }
        X = best;
        D = dbest;
    } else {                                      /* geometric mean of S~ */
        double lsum = 0.0, wsum = 0.0;
        for (int i = 0; i <= n; ++i) {
            double s = i * t1;
            double St = c->S0 * exp(omega * s + c->sigma * W[i]);
            if (stilde) stilde[i] = St;
            lsum += omega * s + c->sigma * W[i];
            wsum += W[i] - c->sigma * s;
        }
        X = c->S0 * exp(lsum / d);
        D = X * wsum / d;
    }

    const double psi = (log(c->K) - log(X) - omega * t1) / a;
    const double disc = exp(-c->r * c->T);
    const double disc1 = exp(c->r * (t1 - c->T));
    const double pdf = norm_pdf(psi);
    if (c->type == 1) {
        /* binary Asian, eq. GAnalyticalSolution and Sec. 4.5.1 */
        out[0] = disc * norm_sf(psi);
        out[1] = disc * pdf / (c->S0 * a);
        out[2] = disc * pdf * (D / (a * X) + psi / c->sigma - sqrt(t1));
        out[3] = disc * pdf / (c->S0 * c->S0 * a) * (psi / a - 1.0);
    } else {
        /* calls on X: Sec. 4.5.2 (arithmetic), Sec. 4.5.3 (lookback, read     */
        /* without the 1/d in front of the argmax term: dX/dsigma of a maximum */
        /* is the derivative of the maximising term alone), and the same form  */
        /* for the geometric mean.                                              */
        const double sf_shift = norm_sf(psi - a);
        out[0] = disc1 * X * sf_shift - disc * c->K * norm_sf(psi);
        out[1] = disc1 * (X / c->S0) * sf_shift;
        out[2] = disc1 * sf_shift * D + disc * c->K * pdf * sqrt(t1);
        out[3] = disc * c->K * pdf / (c->S0 * c->S0 * a);
    }
}

/* ------------------------------------------------------------------------ */
/* Conditioning on the leading coordinate of the full-path construction     */
/* (constructions 3: bridge, 4: PCA; the next reduction the paper names in  */
/* Sec. 6-7, GPCA-style).  The whole path W(t_1..t_d), t_j = j dt, is built */
/* from d Gaussians by the bridge or PCA of d dates; W(t_j) = a_j x + R_j    */
/* with x the leading Gaussian (bridge: the terminal value; PCA: the first   */
/* component), a_j > 0 its loading, R_j the rest built from the n = d-1      */
/* sampled Gaussians.  With c_j = (S0/d) exp(omega t_j + sigma R_j) and     */
/* b_j = sigma a_j the average is X(x) = sum_j c_j exp(b_j x), increasing    */
/* in x; the payoff switches at the root x* of X(x*) = K, found by Newton's  */
/* method on ln X(x) - ln K (convex and increasing, so the iteration        */
/* converges from any start), and integrating x out gives, with             */
/* E[e^{b x}; x > x*] = e^{b^2/2} Phi(b - x*):                                */
/*   call:   e^{-rT} [ sum_j c_j e^{b_j^2/2} Phi(b_j - x*) - K Phi(-x*) ]      */
/*   binary: e^{-rT} Phi(-x*)                                                */
/* and the pathwise Greeks by differentiating these at fixed R (the terms  */
/* from moving x* cancel in the call price, since X(x*) = K).  The          */
/* geometric mean is log-linear in x: X(x) = G e^{b x}, b = sigma mean(a),  */
/* and x* is explicit.  The lookback maximum M(x) = max_j c_j e^{b_j x}     */
/* (c_j = S0 exp(omega t_j + sigma R_j), no 1/d) is the upper envelope of    */
/* the lines ln c_j + b_j x: increasing (every b_j > 0), so x* = min_j of    */
/* the lines' own roots (ln K - ln c_j)/b_j, and right of x* the envelope   */
/* is a run of pieces [u, v], each one line j, the next line the first of   */
/* steeper slope to overtake it; each piece contributes                      */
/*   c_j e^{b_j^2/2} [Phi(b_j - u) - Phi(b_j - v)]                            */
/* (e^{bx} phi(x) = e^{b^2/2} phi(x - b)), the price less K Phi(-x*); delta   */
/* is that sum over S0, vega the same pieces with the derivative of each     */
/* line, gamma = e^{-rT} K phi(x*) / (S0^2 b_j*) from moving x*.              */
/* ------------------------------------------------------------------------ */
static double phi_bar(double y) { return norm_sf(y); }  /* P(x > y) */

/* R_j and a_j, j = 1..d (index j-1), from the n = d-1 sampled z. */
static int lead_path(const contract_t *c, int construction, const double *A, const double *z, double *R, double *a)
{
    const int d = c->d;
    const double dt = c->T / d;
    if (construction == 3) {
        double *zz = (double *)calloc((size_t)d + 1, sizeof(double));
        double *W = (double *)malloc(sizeof(double) * ((size_t)d + 1));
        if (!zz || !W) { free(zz); free(W); return -1; }
        for (int k = 1; k < d; ++k) zz[k] = z[k - 1];       /* the leading Gaussian set to 0 */
        int rc = oracle_bridge(d, dt, zz, W);
        for (int j = 1; j <= d && rc == 0; ++j) R[j - 1] = W[j];
        for (int k = 0; k < d; ++k) zz[k] = 0.0;
        zz[0] = 1.0;                                          /* the loading of the leading one */
        if (rc == 0) rc = oracle_bridge(d, dt, zz, W);
        for (int j = 1; j <= d && rc == 0; ++j) a[j - 1] = W[j];
        free(zz); free(W);
        return rc;
    }
    for (int j = 0; j < d; ++j) {
        double acc = 0.0;
        for (int k = 1; k < d; ++k) acc += A[(size_t)j * (size_t)d + (size_t)k] * z[k - 1];
        R[j] = acc;
        a[j] = A[(size_t)j * (size_t)d];
    }
    return 0;
}

/* The lookback under leading-coordinate conditioning: the envelope pieces
 * right of the switch point, walked from its active line. */
static void lead_lookback_values(const contract_t *c, const double *R, const double *a, double out[4])
{
    const int d = c->d;
    const double dt = c->T / d, sig = c->sigma, K = c->K, S0 = c->S0;
    const double omega = c->r - 0.5 * sig * sig;
    const double disc = exp(-c->r * c->T);
    double xs = INFINITY;
    int cur = -1;
    for (int j = 0; j < d; ++j) {                   /* x* and its line: the smallest root, steeper on ties */
        const double lc = log(S0) + omega * (j + 1) * dt + sig * R[j];
        const double root = (log(K) - lc) / (sig * a[j]);
        if (cur < 0 || root < xs || (root == xs && a[j] > a[cur])) {
            xs = root;
            cur = j;
        }
    }
    double price = 0.0, vega = 0.0;
    double u = xs;
    while (1) {
        const double lc_cur = log(S0) + omega * (cur + 1) * dt + sig * R[cur];
        const double b = sig * a[cur];
        /* the first steeper line to overtake the current one */
        double v = INFINITY;
        int next = -1;
        for (int j = 0; j < d; ++j) {
            if (!(a[j] > a[cur])) continue;
            const double lc = log(S0) + omega * (j + 1) * dt + sig * R[j];
            double xj = (lc_cur - lc) / (sig * a[j] - b);
            if (xj < u) xj = u;                     /* already level with it at u */
            if (xj < v || (xj == v && next >= 0 && a[j] > a[next])) {
                v = xj;
                next = j;
            }
        }
        const double ch = exp(lc_cur + 0.5 * b * b);  /* c_j e^{b^2/2} */
        const double mass = phi_bar(u - b) - (isinf(v) ? 0.0 : phi_bar(v - b));
        const double dens = norm_pdf(u - b) - (isinf(v) ? 0.0 : norm_pdf(v - b));
        const double t = (cur + 1) * dt;
        price += ch * mass;
        vega += ch * ((R[cur] - sig * t + a[cur] * b) * mass + a[cur] * dens);
        if (next < 0) break;
        u = v;
        cur = next;
    }
    /* the line active at x* again, for gamma */
    double b_star = INFINITY, xs2 = INFINITY;
    for (int j = 0; j < d; ++j) {
        const double lc = log(S0) + omega * (j + 1) * dt + sig * R[j];
        const double root = (log(K) - lc) / (sig * a[j]);
        if (root < xs2 || (root == xs2 && sig * a[j] > b_star)) {
            xs2 = root;
            b_star = sig * a[j];
        }
    }
    out[0] = disc * (price - K * phi_bar(xs));
    out[1] = disc * price / S0;
    out[2] = disc * vega;
    out[3] = disc * K * norm_pdf(xs) / (S0 * S0 * b_star);
}

static void lead_values(const contract_t *c, const double *R, const double *a, double out[4])
{
    const int d = c->d;
    const double dt = c->T / d, sig = c->sigma, K = c->K, S0 = c->S0;
    const double omega = c->r - 0.5 * sig * sig;
    const double disc = exp(-c->r * c->T);
    if (c->type == 3) {                              /* geometric: log-linear in x */
        double lmean = 0.0, amean = 0.0, bmean = 0.0;
        for (int j = 0; j < d; ++j) {
            const double t = (j + 1) * dt;
            lmean += omega * t + sig * R[j];
            amean += a[j];
            bmean += R[j] - sig * t;
        }
        lmean /= d; amean /= d; bmean /= d;
        const double G = S0 * exp(lmean), b = sig * amean;
        const double xs = (log(K) - log(G)) / b;
        const double eb = G * exp(0.5 * b * b);
        out[0] = disc * (eb * phi_bar(xs - b) - K * phi_bar(xs));
        out[1] = disc * eb * phi_bar(xs - b) / S0;
        out[2] = disc * eb * ((amean * b + bmean) * phi_bar(xs - b) + amean * norm_pdf(xs - b));
        out[3] = disc * norm_pdf(xs) * K / (S0 * S0 * b);
        return;
    }
    if (c->type == 2) {
        lead_lookback_values(c, R, a, out);
        return;
    }
    /* log c_j and b_j; Newton on g(x) = ln X(x) - ln K from x = 0 */
    double *lc = (double *)malloc(sizeof(double) * (size_t)d);
    double *b = (double *)malloc(sizeof(double) * (size_t)d);
    if (!lc || !b) { free(lc); free(b); for (int g = 0; g < 4; ++g) out[g] = NAN; return; }
    for (int j = 0; j < d; ++j) {
        const double t = (j + 1) * dt;
        lc[j] = log(S0 / d) + omega * t + sig * R[j];
        b[j] = sig * a[j];
    }
    double x = 0.0;
    for (int it = 0; it < 200; ++it) {
        double m = -INFINITY;
        for (int j = 0; j < d; ++j) m = fmax(m, lc[j] + b[j] * x);
        double s0 = 0.0, s1 = 0.0;
        for (int j = 0; j < d; ++j) {
            const double e = exp(lc[j] + b[j] * x - m);
            s0 += e;
            s1 += b[j] * e;
        }
        const double g = m + log(s0) - log(K);
        const double step = g / (s1 / s0);
        x -= step;
        if (fabs(step) <= 1e-15 * (1.0 + fabs(x))) break;
    }
    double X1 = 0.0, X2 = 0.0, F0 = 0.0, V = 0.0, B = 0.0;
    for (int j = 0; j < d; ++j) {
        const double t = (j + 1) * dt;
        const double e = exp(lc[j] + b[j] * x);               /* c_j e^{b_j x*} */
        const double eh = exp(lc[j] + 0.5 * b[j] * b[j]);      /* c_j e^{b_j^2/2} */
        X1 += b[j] * e;
        X2 += b[j] * b[j] * e;
        F0 += eh * phi_bar(x - b[j]);
        V += eh * ((sig * a[j] * a[j] + R[j] - sig * t) * phi_bar(x - b[j]) + a[j] * norm_pdf(x - b[j]));
        B += e * (a[j] * x + R[j] - sig * t);
    }
    const double pdf = norm_pdf(x);
    if (c->type == 0) {
        out[0] = disc * (F0 - K * phi_bar(x));
        out[1] = disc * F0 / S0;
        out[2] = disc * V;
        out[3] = disc * pdf * K * K / (S0 * S0 * X1);
    } else {
        out[0] = disc * phi_bar(x);
        out[1] = disc * pdf * K / (S0 * X1);
        out[2] = disc * pdf * B / X1;
        out[3] = disc * K * pdf * (x * K - 2.0 * X1 + K * X2 / X1) / ((S0 * X1) * (S0 * X1));
    }
    free(lc); free(b);
}

static int build_path(const contract_t *c, int construction, const double *A, const double *z, double *W)
{
    const int n = c->d - 1;
    const double t1 = c->T / c->d;
    if (construction == 0) return oracle_bridge(n, t1, z, W);
    if (construction == 2) return oracle_forward(n, t1, z, W);
    return pca_apply(n, A, z, W);
}

int oracle_point(int type, int d, double K, double T, double S0, double r, double sigma,
                 int construction, const double *z, double out[4], double *stilde)
{
    contract_t c = {type, d, K, T, S0, r, sigma};
    if (check_contract(&c, construction) != 0 || !out || (d > 1 && !z)) return -1;
    const int n = d - 1;
    if (construction >= 3) {
        /* stilde (if given) receives R_j, j = 1..d; the loadings a_j are not returned */
        double *R = (double *)malloc(sizeof(double) * (size_t)d);
        double *a = (double *)malloc(sizeof(double) * (size_t)d);
        double *A = NULL;
        int rc = (R && a) ? 0 : -1;
        if (rc == 0 && construction == 4) {
            A = (double *)malloc(sizeof(double) * (size_t)d * (size_t)d);
            rc = (A && oracle_pca_matrix(d, T / d, A) == 0) ? 0 : -1;
        }
        if (rc == 0) rc = lead_path(&c, construction, A, z, R, a);
        if (rc == 0) {
            lead_values(&c, R, a, out);
            if (stilde) for (int j = 0; j < d; ++j) stilde[j] = R[j];
        }
        free(R); free(a); free(A);
        return rc;
    }
    double *W = (double *)malloc(sizeof(double) * (size_t)(n + 1));
    double *A = NULL;
    if (!W) return -1;
    if (construction == 1 && n > 0) {
        A = (double *)malloc(sizeof(double) * (size_t)n * (size_t)n);
        if (!A || oracle_pca_matrix(n, T / d, A) != 0) { free(W); free(A); return -1; }
    }
    int rc = build_path(&c, construction, A, z, W);
    if (rc == 0) greeks_from_path(&c, W, out, stilde);
    free(W); free(A);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* The estimator: per replicate r, points k = 0..N-1 at Sobol index          */
/* g(k) = k ^ (k >> 1), uniform u = (y + 1/2) 2^-32 of the scrambled integer */
/* y, z = Phi^{-1}(u) per dimension, path, values; the replicate estimate is */
/* the mean over its points (Neumaier-compensated sum), the final estimate   */
/* the mean over replicates, and the error the standard error of that mean,  */
/* sqrt(sum (C_r - C)^2 / (R (R-1))).  Sec. 5 defines the spread of single  */
/* runs with 1/L; the standard error of the mean is reported instead.        */
/* ------------------------------------------------------------------------ */
typedef struct { double s, c; } neumaier_t;

static void neumaier_add(neumaier_t *acc, double x)
{
    double t = acc->s + x;
    if (fabs(acc->s) >= fabs(x)) acc->c += (acc->s - t) + x;
    else acc->c += (x - t) + acc->s;
    acc->s = t;
}

static double neumaier_value(const neumaier_t *acc) { return acc->s + acc->c; }

typedef struct {
    contract_t c;
    int construction;
    uint64_t seed;
    uint32_t *v;      /* n x 32 direction numbers */
    double *A;        /* PCA factor, n x n */
} problem_t;

static int problem_init(problem_t *p, uint64_t seed, const contract_t *c, int construction)
{
    memset(p, 0, sizeof(*p));
    p->c = *c;
    p->construction = construction;
    p->seed = seed;
    const int n = c->d - 1;
    if (n == 0 && construction != 4) return 0;
    if (n == 0) {
        p->A = (double *)malloc(sizeof(double));
        return (p->A && oracle_pca_matrix(1, c->T, p->A) == 0) ? 0 : -1;
    }
    p->v = (uint32_t *)malloc(sizeof(uint32_t) * 32u * (size_t)n);
    if (!p->v || oracle_direction_numbers(n, p->v) != 0) return -1;
    if (construction == 1) {
        p->A = (double *)malloc(sizeof(double) * (size_t)n * (size_t)n);
        if (!p->A || oracle_pca_matrix(n, c->T / c->d, p->A) != 0) return -1;
    }
    if (construction == 4) {  /* the full-path factor, d x d */
        p->A = (double *)malloc(sizeof(double) * (size_t)c->d * (size_t)c->d);
        if (!p->A || oracle_pca_matrix(c->d, c->T / c->d, p->A) != 0) return -1;
    }
    return 0;
}

static void problem_free(problem_t *p) { free(p->v); free(p->A); }

/* Sums over points k0..k0+count-1 of replicate rep. */
static int replicate_sums(const problem_t *p, uint32_t rep, uint64_t k0, uint64_t count,
                          double sums[4], double *per_point)
{
    const int n = p->c.d - 1;
    uint32_t *rows = NULL, *shift = NULL;
    double *z = (double *)malloc(sizeof(double) * (size_t)(n + 1));
    double *W = (double *)malloc(sizeof(double) * (size_t)(n + 2));
    double *a = (double *)malloc(sizeof(double) * (size_t)(n + 2));
    int rc = 0;
    if (!z || !W || !a) rc = -1;
    if (rc == 0 && n > 0) {
        rows = (uint32_t *)malloc(sizeof(uint32_t) * 32u * (size_t)n);
        shift = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n);
        if (!rows || !shift) rc = -1;
        else for (int j = 0; j < n; ++j) oracle_scramble(p->seed, rep, (uint32_t)j, rows + 32 * j, shift + j);
    }
    neumaier_t acc[4] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
    for (uint64_t t = 0; rc == 0 && t < count; ++t) {
        uint64_t k = k0 + t;
        uint64_t index = k ^ (k >> 1);
        for (int j = 0; j < n; ++j) {
            uint32_t y = scramble_apply(rows + 32 * j, shift[j], sobol_unscrambled(p->v + 32 * j, index));
            double u = ((double)y + 0.5) * 0x1p-32;
            z[j] = oracle_inv_normal(u);
        }
        double val[4];
        if (p->construction >= 3) {
            rc = lead_path(&p->c, p->construction, p->A, z, W, a);
            if (rc != 0) break;
            lead_values(&p->c, W, a, val);
        } else {
            rc = build_path(&p->c, p->construction, p->A, z, W);
            if (rc != 0) break;
            greeks_from_path(&p->c, W, val, NULL);
        }
        for (int g = 0; g < 4; ++g) neumaier_add(&acc[g], val[g]);
        if (per_point) for (int g = 0; g < 4; ++g) per_point[t * 4 + (uint64_t)g] = val[g];
    }
    for (int g = 0; g < 4; ++g) sums[g] = neumaier_value(&acc[g]);
    free(z); free(W); free(a); free(rows); free(shift);
    return rc;
}

int oracle_point_values(uint64_t seed, int type, int d, double K, double T, double S0,
                        double r, double sigma, int construction, uint32_t rep,
                        uint64_t k0, uint64_t count, double *out)
{
    contract_t c = {type, d, K, T, S0, r, sigma};
    if (check_contract(&c, construction) != 0 || !out) return -1;
    if (k0 + count > (1ull << 32) || k0 + count < k0) return -1;
    problem_t p;
    int rc = problem_init(&p, seed, &c, construction);
    double sums[4];
    if (rc == 0) rc = replicate_sums(&p, rep, k0, count, sums, out);
    problem_free(&p);
    return rc;
}

int oracle_partial_sums(uint64_t seed, int type, int d, double K, double T, double S0,
                        double r, double sigma, int construction, uint32_t r0, int nrep,
                        uint64_t k0, uint64_t count, int threads, double *sums)
{
    contract_t c = {type, d, K, T, S0, r, sigma};
    if (check_contract(&c, construction) != 0 || nrep < 1 || !sums) return -1;
    if (k0 + count > (1ull << 32) || k0 + count < k0) return -1;
    problem_t p;
    int rc = problem_init(&p, seed, &c, construction);
    if (rc != 0) { problem_free(&p); return rc; }
    int bad = 0;
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
#endif
    for (int i = 0; i < nrep; ++i) {
        if (replicate_sums(&p, r0 + (uint32_t)i, k0, count, sums + 4 * i, NULL) != 0) bad |= 1;
    }
    (void)threads;
    problem_free(&p);
    return bad ? -1 : 0;
}

/* Mean over the R replicate estimates (rows of 4) and the standard error of
 * that mean, sqrt(sum (C_r - C)^2 / (R (R-1))), both sums compensated. */
static void replicate_mean_se(const double *per_rep, int R, double *mean, double *se)
{
    for (int g = 0; g < 4; ++g) {
        neumaier_t acc = {0, 0};
        for (int i = 0; i < R; ++i) neumaier_add(&acc, per_rep[4 * i + g]);
        double m = neumaier_value(&acc) / R;
        neumaier_t dev = {0, 0};
        for (int i = 0; i < R; ++i) {
            double e = per_rep[4 * i + g] - m;
            neumaier_add(&dev, e * e);
        }
        mean[g] = m;
        se[g] = sqrt(neumaier_value(&dev) / ((double)R * (double)(R - 1)));
    }
}

int oracle_greeks(uint64_t seed, int type, int d, double K, double T, double S0, double r,
                  double sigma, int construction, uint64_t N, int R, int threads,
                  double *per_rep, double *mean, double *se)
{
    if (N < 1 || N > (1ull << 32) || R < 2 || !per_rep || !mean || !se) return -1;
    int rc = oracle_partial_sums(seed, type, d, K, T, S0, r, sigma, construction, 0u, R, 0u, N,
                                 threads, per_rep);
    if (rc != 0) return rc;
    for (int i = 0; i < R * 4; ++i) per_rep[i] /= (double)N;
    replicate_mean_se(per_rep, R, mean, se);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Basket of m assets (Sec. 6: the same simulation with several underlying   */
/* assets, the path and the payoff formulas redefined).                       */
/*   S_i(t) = a_i S0 exp(omega_i t + sigma_i W_i(t)), sigma_i = v_i sigma,    */
/*   omega_i = r - sigma_i^2/2, W = L B with L the lower Cholesky factor of   */
/*   the correlation matrix (L_11 = 1) and B m independent Brownian motions;  */
/*   the basket average X = sum_i w_i (1/d) sum_j S_i(t_j).                   */
/* The first increment of factor 1, B_1(t_1) = sqrt(t_1) x_1, is integrated  */
/* out as in Sec. 3.3.1: each factor k is B_k(t_j) = sqrt(t_1) x_k +         */
/* W~_k(t_j - t_1) with W~_k built by the bridge from its own n = d-1         */
/* normals, so W_i(t_j) = L_i1 sqrt(t_1) x_1 + R_ij with                     */
/*   R_ij = sum_k L_ik W~_k(t_j - t_1) + sum_{k>=2} L_ik sqrt(t_1) x_k,        */
/* and X(x_1) = sum_i C_i e^{b_i x_1}, b_i = sigma_i L_i1 sqrt(t_1),          */
/*   C_i = (w_i a_i S0 / d) sum_j exp(omega_i t_j + sigma_i R_ij).            */
/* With every correlation to asset 1 positive, all b_i > 0: X is increasing */
/* in x_1 from 0, and the switch point x* of X(x*) = K is found by Newton's  */
/* method on ln X - ln K (convex, increasing).  Integrating x_1 out         */
/* (E[e^{b x}; x > x*] = e^{b^2/2} Phi-bar(x* - b)):                          */
/*   call:   e^{-rT} [ sum_i C_i e^{b_i^2/2} Phi-bar(x* - b_i) - K Phi-bar(x*) ] */
/*   binary: e^{-rT} Phi-bar(x*)                                             */
/* Greeks at fixed z: delta and gamma with respect to the spot scale S0 (all */
/* spots move together), vega with respect to the volatility scale sigma     */
/* (all volatilities move together); with D_i = (w_i a_i S0/d) sum_j         */
/* exp(omega_i t_j + sigma_i R_ij) (R_ij - sigma_i t_j), X' = sum_i C_i b_i    */
/* e^{b_i x*}, X'' = sum_i C_i b_i^2 e^{b_i x*}:                              */
/*   call delta  e^{-rT} sum_i (C_i/S0) e^{b_i^2/2} Phi-bar(x* - b_i)          */
/*   call gamma  e^{-rT} K^2 phi(x*) / (S0^2 X')                              */
/*   call vega   e^{-rT} sum_i v_i e^{b_i^2/2} [D_i Phi-bar(x* - b_i)          */
/*               + C_i L_i1 sqrt(t_1) (b_i Phi-bar(x* - b_i) + phi(x* - b_i))] */
/*   binary delta e^{-rT} phi(x*) K / (S0 X')                                 */
/*   binary gamma e^{-rT} K phi(x*) (x* K - 2 X' + K X''/X') / (S0 X')^2      */
/*   binary vega  e^{-rT} phi(x*) sum_i v_i e^{b_i x*} [D_i + C_i L_i1 sqrt(t_1) x*] / X' */
/* (the terms from moving x* cancel in the call price since X(x*) = K).      */
/* Sobol' dimensions: b m + (k-1) drives bridge node b (0..n-1) of factor k  */
/* (1..m); n m + (k-2) drives x_k, k = 2..m: m d - 1 in all.  With m = 1 this */
/* is the single-asset bridge estimator point by point.                       */
/* ------------------------------------------------------------------------ */
#define ORACLE_ASSETS_MAX 8

typedef struct {
    int type, d, m;
    double K, T, S0, r, sigma;
    double w[ORACLE_ASSETS_MAX], a[ORACLE_ASSETS_MAX], v[ORACLE_ASSETS_MAX];
    double L[ORACLE_ASSETS_MAX * ORACLE_ASSETS_MAX];
} basket_t;

/* Cholesky factor of a symmetric positive definite m x m matrix (row-major):
 * L lower triangular with C = L L^T, by the Cholesky-Banachiewicz order.  */
int oracle_cholesky(int m, const double *C, double *L)
{
    if (m < 1 || m > ORACLE_ASSETS_MAX || !C || !L) return -1;
    for (int i = 0; i < m * m; ++i) L[i] = 0.0;
    for (int i = 0; i < m; ++i) {
        for (int j = 0; j <= i; ++j) {
            double s = C[i * m + j];
            for (int k = 0; k < j; ++k) s -= L[i * m + k] * L[j * m + k];
            if (i == j) {
                if (!(s > 0.0)) return -1;
                L[i * m + i] = sqrt(s);
            } else {
                L[i * m + j] = s / L[j * m + j];
            }
        }
    }
    return 0;
}

static int basket_init(basket_t *b, int type, int d, int m, double K, double T, double S0, double r,
                       double sigma, const double *w, const double *a, const double *v, const double *corr)
{
    memset(b, 0, sizeof(*b));
    if (type != 0 && type != 1) return -1;
    if (m < 1 || m > ORACLE_ASSETS_MAX || d < 1 || (int64_t)m * d > MAX_DIMS) return -1;
    if (!w || !a || !v || !corr) return -1;
    if (!(K > 0.0) || !(T > 0.0) || !(S0 > 0.0) || !(sigma > 0.0)) return -1;
    if (!isfinite(K) || !isfinite(T) || !isfinite(S0) || !isfinite(sigma) || !isfinite(r)) return -1;
    if (!(w[0] > 0.0)) return -1;
    for (int i = 0; i < m; ++i) {
        if (!(w[i] >= 0.0) || !(a[i] > 0.0) || !(v[i] > 0.0)) return -1;
        if (!isfinite(w[i]) || !isfinite(a[i]) || !isfinite(v[i])) return -1;
        if (!(corr[i] > 0.0) || corr[i * m + i] != 1.0) return -1;  /* positive correlation to asset 1, unit diagonal */
        for (int k = 0; k < m; ++k)
            if (corr[i * m + k] != corr[k * m + i] || !(fabs(corr[i * m + k]) <= 1.0)) return -1;
    }
    b->type = type; b->d = d; b->m = m;
    b->K = K; b->T = T; b->S0 = S0; b->r = r; b->sigma = sigma;
    for (int i = 0; i < m; ++i) { b->w[i] = w[i]; b->a[i] = a[i]; b->v[i] = v[i]; }
    double L[ORACLE_ASSETS_MAX * ORACLE_ASSETS_MAX];
    if (oracle_cholesky(m, corr, L) != 0) return -1;
    for (int i = 0; i < m; ++i)
        for (int k = 0; k < m; ++k) b->L[i * ORACLE_ASSETS_MAX + k] = L[i * m + k];
    return 0;
}

/* The four values of one point from its m d - 1 normals z. */
static int basket_values(const basket_t *b, const double *z, double out[4])
{
    const int d = b->d, m = b->m, n = d - 1;
    const double dt = b->T / d, t1 = dt, st1 = sqrt(t1);
    double *Wt = (double *)malloc(sizeof(double) * (size_t)m * (size_t)(n + 1));
    double *zk = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    if (!Wt || !zk) { free(Wt); free(zk); return -1; }
    for (int k = 0; k < m; ++k) {            /* factor k+1: W~ over s_0..s_n */
        for (int bnode = 0; bnode < n; ++bnode) zk[bnode] = z[bnode * m + k];
        if (oracle_bridge(n, dt, zk, Wt + (size_t)k * (n + 1)) != 0) { free(Wt); free(zk); return -1; }
    }
    double C[ORACLE_ASSETS_MAX], D[ORACLE_ASSETS_MAX], bb[ORACLE_ASSETS_MAX], sig[ORACLE_ASSETS_MAX];
    for (int i = 0; i < m; ++i) {
        const double *Li = b->L + i * ORACLE_ASSETS_MAX;
        sig[i] = b->v[i] * b->sigma;
        const double om = b->r - 0.5 * sig[i] * sig[i];
        double first = 0.0;                  /* sum_{k>=2} L_ik sqrt(t_1) x_k */
        for (int k = 1; k < m; ++k) first += Li[k] * st1 * z[n * m + (k - 1)];
        double sc = 0.0, sd = 0.0;
        for (int j = 1; j <= d; ++j) {
            const double tj = j * dt;
            double R = first;
            for (int k = 0; k < m; ++k) R += Li[k] * Wt[(size_t)k * (n + 1) + (j - 1)];
            const double e = exp(om * tj + sig[i] * R);
            sc += e;
            sd += e * (R - sig[i] * tj);
        }
        const double f = b->w[i] * b->a[i] * b->S0 / d;
        C[i] = f * sc;
        D[i] = f * sd;
        bb[i] = sig[i] * Li[0] * st1;
    }
    free(Wt); free(zk);
    /* Newton on ln X(x) - ln K from x = 0 (log-sum-exp with its largest term factored out) */
    double x = 0.0;
    for (int it = 0; it < 200; ++it) {
        double mx = -INFINITY;
        for (int i = 0; i < m; ++i) if (C[i] > 0.0) mx = fmax(mx, log(C[i]) + bb[i] * x);
        double s0 = 0.0, s1 = 0.0;
        for (int i = 0; i < m; ++i) {
            if (!(C[i] > 0.0)) continue;
            const double e = exp(log(C[i]) + bb[i] * x - mx);
            s0 += e;
            s1 += bb[i] * e;
        }
        const double step = (mx + log(s0) - log(b->K)) / (s1 / s0);
        x -= step;
        if (fabs(step) <= 1e-15 * (1.0 + fabs(x))) break;
    }
    const double disc = exp(-b->r * b->T), pdf = norm_pdf(x), K = b->K, S0 = b->S0;
    double F0 = 0.0, X1 = 0.0, X2 = 0.0, V = 0.0, B = 0.0;
    for (int i = 0; i < m; ++i) {
        const double l1 = b->L[i * ORACLE_ASSETS_MAX] * st1;    /* L_i1 sqrt(t_1) */
        const double e = C[i] * exp(bb[i] * x);                   /* C_i e^{b_i x*} */
        const double eh = C[i] * exp(0.5 * bb[i] * bb[i]);        /* C_i e^{b_i^2/2} */
        const double sfb = phi_bar(x - bb[i]);
        F0 += eh * sfb;
        X1 += bb[i] * e;
        X2 += bb[i] * bb[i] * e;
        V += b->v[i] * exp(0.5 * bb[i] * bb[i]) * (D[i] * sfb + C[i] * l1 * (bb[i] * sfb + norm_pdf(x - bb[i])));
        B += b->v[i] * exp(bb[i] * x) * (D[i] + C[i] * l1 * x);
    }
    if (b->type == 0) {
        out[0] = disc * (F0 - K * phi_bar(x));
        out[1] = disc * F0 / S0;
        out[2] = disc * V;
        out[3] = disc * K * K * pdf / (S0 * S0 * X1);
    } else {
        out[0] = disc * phi_bar(x);
        out[1] = disc * pdf * K / (S0 * X1);
        out[2] = disc * pdf * B / X1;
        const double sx = S0 * X1;
        out[3] = disc * K * pdf * (K * x - 2.0 * X1 + K * X2 / X1) / (sx * sx);
    }
    return 0;
}

int oracle_basket_point(int type, int d, int m, double K, double T, double S0, double r, double sigma,
                        const double *w, const double *a, const double *v, const double *corr,
                        const double *z, double out[4])
{
    basket_t b;
    if (basket_init(&b, type, d, m, K, T, S0, r, sigma, w, a, v, corr) != 0 || !out) return -1;
    if (m * d > 1 && !z) return -1;
    return basket_values(&b, z, out);
}

/* Sums over points k0..k0+count-1 of replicate rep (per_point optional). */
static int basket_replicate_sums(const basket_t *b, uint64_t seed, const uint32_t *v, uint32_t rep,
                                 uint64_t k0, uint64_t count, double sums[4], double *per_point)
{
    const int nd = b->m * b->d - 1;
    uint32_t *rows = NULL, *shift = NULL;
    double *z = (double *)malloc(sizeof(double) * (size_t)(nd + 1));
    int rc = z ? 0 : -1;
    if (rc == 0 && nd > 0) {
        rows = (uint32_t *)malloc(sizeof(uint32_t) * 32u * (size_t)nd);
        shift = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)nd);
        if (!rows || !shift) rc = -1;
        else for (int j = 0; j < nd; ++j) oracle_scramble(seed, rep, (uint32_t)j, rows + 32 * j, shift + j);
    }
    neumaier_t acc[4] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
    for (uint64_t t = 0; rc == 0 && t < count; ++t) {
        const uint64_t k = k0 + t, index = k ^ (k >> 1);
        for (int j = 0; j < nd; ++j) {
            const uint32_t y = scramble_apply(rows + 32 * j, shift[j], sobol_unscrambled(v + 32 * j, index));
            z[j] = oracle_inv_normal(((double)y + 0.5) * 0x1p-32);
        }
        double val[4];
        rc = basket_values(b, z, val);
        if (rc != 0) break;
        for (int g = 0; g < 4; ++g) neumaier_add(&acc[g], val[g]);
        if (per_point) for (int g = 0; g < 4; ++g) per_point[t * 4 + (uint64_t)g] = val[g];
    }
    for (int g = 0; g < 4; ++g) sums[g] = neumaier_value(&acc[g]);
    free(z); free(rows); free(shift);
    return rc;
}

int oracle_basket_point_values(uint64_t seed, int type, int d, int m, double K, double T, double S0,
                               double r, double sigma, const double *w, const double *a, const double *v,
                               const double *corr, uint32_t rep, uint64_t k0, uint64_t count, double *out)
{
    basket_t b;
    if (basket_init(&b, type, d, m, K, T, S0, r, sigma, w, a, v, corr) != 0 || !out) return -1;
    if (k0 + count > (1ull << 32) || k0 + count < k0) return -1;
    const int nd = m * d - 1;
    uint32_t *dirs = (uint32_t *)malloc(sizeof(uint32_t) * 32u * (size_t)(nd > 0 ? nd : 1));
    if (!dirs || oracle_direction_numbers(nd, dirs) != 0) { free(dirs); return -1; }
    double sums[4];
    const int rc = basket_replicate_sums(&b, seed, dirs, rep, k0, count, sums, out);
    free(dirs);
    return rc;
}

int oracle_basket_greeks(uint64_t seed, int type, int d, int m, double K, double T, double S0, double r,
                         double sigma, const double *w, const double *a, const double *v, const double *corr,
                         uint64_t N, int R, int threads, double *per_rep, double *mean, double *se)
{
    basket_t b;
    if (basket_init(&b, type, d, m, K, T, S0, r, sigma, w, a, v, corr) != 0) return -1;
    if (N < 1 || N > (1ull << 32) || R < 2 || !per_rep || !mean || !se) return -1;
    const int nd = m * d - 1;
    uint32_t *dirs = (uint32_t *)malloc(sizeof(uint32_t) * 32u * (size_t)(nd > 0 ? nd : 1));
    if (!dirs || oracle_direction_numbers(nd, dirs) != 0) { free(dirs); return -1; }
    int bad = 0;
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
#endif
    for (int i = 0; i < R; ++i)
        if (basket_replicate_sums(&b, seed, dirs, (uint32_t)i, 0u, N, per_rep + 4 * i, NULL) != 0) bad |= 1;
    (void)threads;
    free(dirs);
    if (bad) return -1;
    for (int i = 0; i < R * 4; ++i) per_rep[i] /= (double)N;
    replicate_mean_se(per_rep, R, mean, se);
    return 0;
}
