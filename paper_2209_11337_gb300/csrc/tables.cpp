// Host-side tables of the QMC-CPW path: Sobol' direction integers (Sec. 2.2.2),
// random linear scrambles with digital shifts (Sec. 2.2.3), the breadth-first
// Brownian bridge schedule (Sec. 4.4) and the PCA factor of the Brownian
// covariance (eq. WboldTilde).  All are built once per plan / per d and
// uploaded; none is touched on the hot path.
#include <cmath>
#include <cstring>
#include <stdexcept>

#include "qmccpw_internal.h"

namespace qmccpw {

uint64_t splitmix64_at(uint64_t key, uint64_t counter) {
    uint64_t z = key + (counter + 1u) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

namespace {

int degree_of(uint32_t p) { return 31 - __builtin_clz(p); }

// a*b mod P over GF(2), P of degree q.
uint32_t gf2_mulmod(uint32_t a, uint32_t b, uint32_t P, int q) {
    uint32_t acc = 0;
    const uint32_t top = 1u << q;
    while (b) {
        if (b & 1u) acc ^= a;
        b >>= 1;
        a <<= 1;
        if (a & top) a ^= P;
    }
    return acc;
}

// x^e mod P by square-and-multiply.
uint32_t gf2_pow_x(uint64_t e, uint32_t P, int q) {
    uint32_t base = 2u;
    if (base & (1u << q)) base ^= P;  // q == 1: x == 1 mod (x+1)
    uint32_t acc = 1u;
    while (e) {
        if (e & 1u) acc = gf2_mulmod(acc, base, P, q);
        base = gf2_mulmod(base, base, P, q);
        e >>= 1;
    }
    return acc;
}

// Primitive iff the multiplicative order of x modulo P is exactly 2^q - 1:
// x^(2^q-1) = 1 and x^((2^q-1)/p) != 1 for each prime p dividing 2^q - 1.
bool primitive(uint32_t P) {
    if (!(P & 1u)) return false;
    const int q = degree_of(P);
    if (q < 1) return false;
    const uint64_t order = (1ull << q) - 1u;
    if (gf2_pow_x(order, P, q) != 1u) return false;
    uint64_t rest = order;
    for (uint64_t f = 2; f * f <= rest; ++f) {
        if (rest % f) continue;
        while (rest % f == 0) rest /= f;
        if (gf2_pow_x(order / f, P, q) == 1u) return false;
    }
    if (rest > 1 && gf2_pow_x(order / rest, P, q) == 1u) return false;
    return true;
}

}  // namespace

std::vector<uint32_t> direction_integers(int ndims) {
    std::vector<uint32_t> v(static_cast<size_t>(ndims) * 32u, 0u);
    uint32_t P = 2;  // candidate polynomial, enumerated upward
    for (int j = 0; j < ndims; ++j) {
        uint32_t *vj = v.data() + 32 * j;
        if (j == 0) {  // generator matrix I: van der Corput
            for (int b = 0; b < 32; ++b) vj[b] = 1u << (31 - b);
            continue;
        }
        do { ++P; } while (!primitive(P));
        const int q = degree_of(P);
        // initial direction integers from odd m_i < 2^i
        for (int i = 1; i <= q && i <= 32; ++i) {
            const uint64_t draw = splitmix64_at(kDirectionKey, (static_cast<uint64_t>(j) << 8) | i) >> 32;
            const uint32_t m = static_cast<uint32_t>((draw & ((1ull << i) - 1u)) | 1u);
            vj[i - 1] = m << (32 - i);
        }
        // recurrence on direction integers: v_i = v_{i-q} ^ (v_{i-q} >> q) ^ sum_k c_k v_{i-k}
        for (int i = q + 1; i <= 32; ++i) {
            uint32_t x = vj[i - q - 1] ^ (vj[i - q - 1] >> q);
            for (int k = 1; k < q; ++k)
                if ((P >> (q - k)) & 1u) x ^= vj[i - k - 1];
            vj[i - 1] = x;
        }
    }
    return v;
}

void scrambled_table(uint64_t seed, uint32_t rep, const std::vector<uint32_t> &v, int ndims,
                     int jstride, uint32_t *table_bj, uint32_t *shift) {
    for (int j = 0; j < ndims; ++j) {
        const uint64_t base = (static_cast<uint64_t>(rep) << 32) | (static_cast<uint64_t>(j) << 8);
        // columns of L: column of digit c (bit 32-c) holds the digits i >= c whose row has digit c
        uint32_t col[33];
        for (int c = 1; c <= 32; ++c) col[c] = 1u << (32 - c);  // unit diagonal
        for (int i = 2; i <= 32; ++i) {
            const uint32_t row = static_cast<uint32_t>(splitmix64_at(seed, base | static_cast<uint64_t>(i - 1)) >> 32)
                                 & (0xFFFFFFFFu << (33 - i));  // digits 1..i-1
            for (int c = 1; c < i; ++c)
                if (row & (1u << (32 - c))) col[c] |= 1u << (32 - i);
        }
        for (int b = 0; b < 32; ++b) {
            const uint32_t x = v[32 * j + b];
            uint32_t y = 0;
            for (int c = 1; c <= 32; ++c)
                if (x & (1u << (32 - c))) y ^= col[c];
            table_bj[static_cast<size_t>(b) * jstride + j] = y;
        }
        shift[j] = static_cast<uint32_t>(splitmix64_at(seed, base | 32u) >> 32);
    }
}

BridgePlan bridge_plan(int n, double dt) {
    BridgePlan bp;
    bp.n = n;
    if (n <= 0) {
        bp.level_start = {0};
        return bp;
    }
    // the fourth field of a step carries the bits of float(m), the date index
    // as a float, so kernels form s_m = m dt without a conversion
    auto fbits = [](int m) {
        const float f = static_cast<float>(m);
        int32_t b;
        std::memcpy(&b, &f, sizeof(b));
        return b;
    };
    // level 0: the terminal value from W(0) = 0
    bp.steps.push_back({n, 0, 0, fbits(n)});
    bp.w.insert(bp.w.end(), {0.0, 0.0, std::sqrt(n * dt)});
    bp.level_start = {0, 1};
    std::vector<std::pair<int, int>> level = {{0, n}};
    while (true) {
        std::vector<std::pair<int, int>> next;
        for (auto [l, r] : level) {
            if (r - l < 2) continue;
            const int m = (l + r) / 2;
            const double den = static_cast<double>(r - l);
            bp.steps.push_back({m, l, r, fbits(m)});
            bp.w.insert(bp.w.end(), {(r - m) / den, (m - l) / den, std::sqrt(dt * (m - l) * (r - m) / den)});
            next.push_back({l, m});
            next.push_back({m, r});
        }
        if (static_cast<int>(bp.steps.size()) == bp.level_start.back()) break;
        bp.level_start.push_back(static_cast<int32_t>(bp.steps.size()));
        level.swap(next);
    }
    if (static_cast<int>(bp.steps.size()) != n) throw std::logic_error("bridge schedule size");
    return bp;
}

std::vector<double> pca_factor(int n, double dt) {
    // Sigma = dt*min(i,k): eigenvalues dt/(4 sin^2(theta_k/2)), eigenvectors
    // sin(i theta_k) with theta_k = (2k-1) pi/(2n+1), normalised by 2/sqrt(2n+1).
    std::vector<double> A(static_cast<size_t>(n) * n);
    const double pi = 3.14159265358979323846;
    const double norm = 2.0 / std::sqrt(2.0 * n + 1.0);
    for (int k = 1; k <= n; ++k) {
        const double theta = (2.0 * k - 1.0) * pi / (2.0 * n + 1.0);
        const double s = std::sin(0.5 * theta);
        const double root_lambda = std::sqrt(dt) / (2.0 * s);
        for (int i = 1; i <= n; ++i)
            A[static_cast<size_t>(i - 1) * n + (k - 1)] = norm * std::sin(i * theta) * root_lambda;
    }
    return A;
}

void contract_constants(ContractDev &c) {
    c.dt = c.T / c.d;
    c.a = c.sigma * std::sqrt(c.dt);
    c.omega = c.r - 0.5 * c.sigma * c.sigma;
    c.psi0 = std::log(c.K / c.S0) - c.omega * c.dt;
    c.disc = std::exp(-c.r * c.T);
    c.ln_lead_c0 = std::log(c.S0 / c.d);
    c.ln_S0 = std::log(c.S0);
    c.ln_K = std::log(c.K);
    c.disc1 = std::exp(c.r * (c.dt - c.T));
    c.sqrt_t1 = std::sqrt(c.dt);
    c.inv_a = 1.0 / c.a;
    c.disc1_S0 = c.disc1 * c.S0;
    c.disc_K = c.disc * c.K;
    c.k_bin_delta = c.disc / (c.S0 * c.a);
    c.k_bin_gamma = c.disc / (c.S0 * c.S0 * c.a);
    c.k_call_gamma = c.disc * c.K / (c.S0 * c.S0 * c.a);
    c.inv_sigma = 1.0 / c.sigma;
    c.inv_d = 1.0 / c.d;
    const double inv_sqrt_2pi = 0.398942280401432677939946059934;  // 1/sqrt(2 pi)
    const double n = c.d - 1;
    const double s1 = 0.5 * n * (n + 1.0);  // sum of the date indices after t_1
    split_ff(c.sigma * c.sqrt_t1, c.ff_sig_sdt);
    split_ff(c.omega * c.dt, c.ff_om_dt);
    split_ff(c.sqrt_t1, c.ff_sqrt_t1);
    split_ff(-c.sigma * c.dt, c.ff_nsig_dt);
    split_ff(c.inv_d, c.ff_inv_d);
    split_ff(c.sqrt_t1 * c.inv_d, c.ff_sdt_d);
    split_ff(-c.sigma * c.dt * c.inv_d, c.ff_nsigdt_d);
    split_ff(c.sigma * c.sqrt_t1 * c.inv_d, c.ff_sig_sdt_d);
    split_ff(c.omega * c.dt * s1 * c.inv_d, c.ff_geo_l0);
    split_ff(-c.sigma * c.dt * s1 * c.inv_d, c.ff_geo_d0);
    split_ff(c.psi0, c.ff_psi0);
    split_ff(c.inv_a, c.ff_inv_a);
    split_ff(c.inv_sigma, c.ff_inv_sigma);
    split_ff(c.a, c.ff_a);
    split_ff(c.disc1_S0, c.ff_disc1_S0);
    split_ff(c.disc_K, c.ff_disc_K);
    split_ff(c.disc1, c.ff_disc1);
    split_ff(c.disc, c.ff_disc);
    split_ff(c.disc_K * c.sqrt_t1 * inv_sqrt_2pi, c.ff_kv_call);
    split_ff(c.k_call_gamma * inv_sqrt_2pi, c.ff_kg_call);
    split_ff(c.k_bin_delta * inv_sqrt_2pi, c.ff_kd_bin);
    split_ff(c.k_bin_gamma * inv_sqrt_2pi, c.ff_kg_bin);
    split_ff(c.disc * inv_sqrt_2pi, c.ff_kphi);
    split_ff(c.sigma, c.ff_sig);
    split_ff(c.ln_lead_c0, c.ff_lnS0d);
    split_ff(c.ln_K, c.ff_lnK);
}

// Cholesky factor by columns (the Cholesky-Crout order): column k's
// diagonal from the entries left of it, then the entries below it.
bool cholesky_lower(int m, const double *C, double *L) {
    for (int i = 0; i < m * m; ++i) L[i] = 0.0;
    for (int k = 0; k < m; ++k) {
        double diag = C[k * m + k];
        for (int q = 0; q < k; ++q) diag -= L[k * m + q] * L[k * m + q];
        if (!(diag > 0.0)) return false;
        const double lkk = std::sqrt(diag);
        L[k * m + k] = lkk;
        for (int i = k + 1; i < m; ++i) {
            double s = C[i * m + k];
            for (int q = 0; q < k; ++q) s -= L[i * m + q] * L[k * m + q];
            L[i * m + k] = s / lkk;
        }
    }
    return true;
}

}  // namespace qmccpw
