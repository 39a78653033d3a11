// Device code shared by the CUDA-core kernel (kernels.cu) and the
// tensor-core PCA kernel (pca_tc.cu): precision traits, the inverse normal,
// the path accumulator, the conditional step and the tile reduction.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "float_coeffs.h"
#include "qmccpw_internal.h"

namespace qmccpw {
namespace {

// ---------------------------------------------------------------------------
// precision traits
// ---------------------------------------------------------------------------
template <typename T> struct Arith;

template <> struct Arith<double> {
    // z = Phi^{-1}(u), u = (y + 1/2) 2^-32, evaluated on the lower half
    // q = min(u, 1-u) (exact in double) and reflected.
    __device__ static double inv_normal(uint32_t y) {
        const bool upper = y >= 0x80000000u;
        const uint32_t lo = upper ? ~y : y;
        const double q = fma(static_cast<double>(lo), 0x1p-32, 0x1p-33);
        const double z = normcdfinv(q);
        return upper ? -z : z;
    }
    __device__ static double ex(double x) { return exp(x); }
};

// ---------------------------------------------------------------------------
// float functions of the MIXED path: this project's own polynomials
// (float_coeffs.h, fitted by gen_float_coeffs.py), evaluated with IEEE float
// adds and fused multiply-adds, plus reciprocals from rcp.approx refined by
// one Newton step.  The hardware approximations (lg2/ex2.approx, and the
// library's expf/erfcf built on them) carry error patterns of a few 1e-8
// with a nonzero mean over any range of arguments; such an error is the same
// for every point and does not average out, while a rounding error of an
// IEEE operation on a continuously varying value has mean zero.
// ---------------------------------------------------------------------------
// Packed two-lane FP32 arithmetic (one instruction for two elements): the
// polynomial chains below run on pairs of independent elements, with the
// same operations in the same order as the one-element forms, so a pair
// gives bit for bit the two single results.
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }

// Exact float of an integer below 2^23 without a conversion instruction
// (conversions share the slow FP64 pipe on this GPU): place it in the
// mantissa of 2^23 and subtract 2^23.
__device__ __forceinline__ float small_uint_to_float(uint32_t x) {
    return __uint_as_float(0x4B000000u | x) - 8388608.0f;
}

namespace fx {
constexpr float kMagic = 12582912.0f;              // 1.5 2^23: x + kMagic holds rint(x) in its low mantissa bits
constexpr float kLog2e = 1.44269502f;              // only picks k: any nearby value is exact enough
constexpr float kLn2Hi = 0.693147182464599609375f; // ln 2 = kLn2Hi + kLn2Lo to ~2^-48
constexpr float kLn2Lo = -1.904654290e-09f;

// 1/x to ~0.5 ulp for positive normal x: rcp.approx and one Newton step
__device__ __forceinline__ float rcp_nr(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return fmaf(r, fmaf(-x, r, 1.0f), r);
}
__device__ __forceinline__ float2 rcp_nr2(float2 x) {
    // scalar asm operands (an output bound to a float2 member lost one lane)
    float rx, ry;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rx) : "f"(x.x));
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(ry) : "f"(x.y));
    const float2 r = make_float2(rx, ry);
    return fma2(r, fma2(make_float2(-x.x, -x.y), r, f2(1.0f)), r);
}

// e^x for |x| <= 86: 2^k e^r, k the nearest integer to x log2 e, r = x - k ln2
// with ln2 = hi + lo: r1 = x - k hi is exact (a multiple of 2^-24 below 1/2
// in magnitude), e^r = (1 + r1 q(r1))(1 + delta) with the degree-8
// polynomial 1 + r q(r) (c0 = c1 = 1 exact) and delta = -k lo, i.e.
// 1 + [r1 q + delta (1 + r1 q)]: the small bracket term meets the unrounded
// product r1 q in the last FMA.  Added to r1 instead, delta sits below half
// an ulp of the float r1 for most arguments and is dropped the same way for
// every x of that k (e^x near x = 1.8, k = 3, came out 5.6e-9 low on
// average); added to the rounded result, the same.  2^k goes to the exponent
// field (k in the low bits of the magic sum, shifted out of its high bits).
__device__ __forceinline__ float exp_f(float x) {
    constexpr float c[] = QMC_EXP_POLY;
    const float m = fmaf(x, kLog2e, kMagic);
    const float nk = kMagic - m;  // -k, exact
    const float r = fmaf(nk, kLn2Hi, x);
    float q = c[8];
#pragma unroll
    for (int i = 7; i >= 1; --i) q = fmaf(q, r, c[i]);
    const float delta = nk * kLn2Lo;
    const float p = 1.0f + fmaf(q, r, fmaf(delta, q * r, delta));
    return __uint_as_float(__float_as_uint(p) + (__float_as_uint(m) << 23));
}
__device__ __forceinline__ float2 exp_f2(float2 x) {
    constexpr float c[] = QMC_EXP_POLY;
    const float2 m = fma2(x, f2(kLog2e), f2(kMagic));
    const float2 nk = fma2(m, f2(-1.0f), f2(kMagic));  // -k, exact
    const float2 r = fma2(nk, f2(kLn2Hi), x);
    float2 q = f2(c[8]);
#pragma unroll
    for (int i = 7; i >= 1; --i) q = fma2(q, r, f2(c[i]));
    const float2 delta = mul2(nk, f2(kLn2Lo));
    const float2 p = add2(f2(1.0f), fma2(q, r, fma2(delta, mul2(q, r), delta)));
    return make_float2(__uint_as_float(__float_as_uint(p.x) + (__float_as_uint(m.x) << 23)),
                       __uint_as_float(__float_as_uint(p.y) + (__float_as_uint(m.y) << 23)));
}

// e^{xh + xl} for a float-float argument (|xl| <= ulp(xh)/2, -86 <= xh <=
// 0).  For large |xh| the float xh lies on a grid coarser than the reduced
// argument's, so a reduction rounded on its own would err by the same amount
// for every xh with the same k; here k ln2 is split exactly (its product
// error by an FMA), xh - P is exact (Sterbenz), and all the small parts,
// with xl among them, meet the exact difference in one final rounding.
__device__ __forceinline__ float exp_ff(float xh, float xl) {
    constexpr float c[] = QMC_EXP_POLY;
    const float m = fmaf(xh, kLog2e, kMagic);
    const float nk = kMagic - m;
    const float P = nk * kLn2Hi;                       // -k ln2 (hi part), rounded
    const float Perr = fmaf(nk, kLn2Hi, -P);           // its rounding error, exact
    const float r0 = xh + P;                           // exact: xh and -P within a factor 2 (or k = 0)
    const float small = fmaf(nk, kLn2Lo, xl) + Perr;   // -k ln2 (lo part) + xl + Perr
    const float r = r0 + small;
    float p = c[8];
#pragma unroll
    for (int i = 7; i >= 0; --i) p = fmaf(p, r, c[i]);
    return __uint_as_float(__float_as_uint(p) + (__float_as_uint(m) << 23));
}

// -ln a for positive normal floats a (two at a time): a = 2^e m, m in
// [sqrt(1/2), sqrt 2) by integer operations on the bits, ln m = f P(f^2)
// with f = (m - 1)/(m + 1) (the atanh series; m - 1 is exact), e ln2 with
// ln2 as a float pair.  P's coefficients enter negated, so the packed chain
// forms -ln m without a negated operand.
__device__ __forceinline__ float2 neg_ln2(float2 a) {
    constexpr float c[] = QMC_LN_POLY;
    constexpr int n = sizeof(c) / sizeof(c[0]);
    // e + 127 = floor(log2(a / sqrt(1/2))) + 127 from the bits of a (a normal,
    // 0 < a < 2^127): unsigned adds and logical shifts only (an arithmetic
    // shift of the signed difference gave one lane of the pair unshifted)
    const uint32_t bx = __float_as_uint(a.x), by = __float_as_uint(a.y);
    const uint32_t ebx = (bx + (0x3F800000u - 0x3F3504F3u)) >> 23;
    const uint32_t eby = (by + (0x3F800000u - 0x3F3504F3u)) >> 23;
    // m = a 2^-e in [sqrt(1/2), sqrt 2): the exponent field less e
    const float2 m = make_float2(__uint_as_float(bx - (ebx << 23) + (127u << 23)),
                                 __uint_as_float(by - (eby << 23) + (127u << 23)));
    // e as a float through the magic constant (1.5 2^23 + e - kMagic): no conversion instruction
    const float2 ef = add2(make_float2(__uint_as_float(0x4B400000u - 127u + ebx),
                                       __uint_as_float(0x4B400000u - 127u + eby)), f2(-kMagic));
    const float2 num = add2(m, f2(-1.0f));
    const float2 den = add2(m, f2(1.0f));
    const float2 f = mul2(num, rcp_nr2(den));
    const float2 t = mul2(f, f);
    float2 p = f2(-c[n - 1]);
#pragma unroll
    for (int i = n - 2; i >= 0; --i) p = fma2(p, t, f2(-c[i]));
    // -ln m - e ln2_lo in one rounding (the unrounded product f P meets the
    // small term: added to a rounded -ln m, a term below half its ulp would be
    // lost the same way for every a with that e), then - e ln2_hi
    const float2 nlnm = fma2(f, p, mul2(ef, f2(-kLn2Lo)));
    return fma2(ef, f2(-kLn2Hi), nlnm);  // -(e ln2 + ln m)
}

// Upper normal tail T(y) = Phi(-y) for 0 <= y <= YMAX (float-float y:
// y^2 / 2 enters the exponential to float-float accuracy):
// T = e^{-y^2/2} t g(t), t = 1/(1 + KAPPA y), g fitted (the Mills ratio times
// (1 + KAPPA y)/sqrt(2 pi)), its constant and linear terms as float pairs.
// Beyond YMAX the tail is 0 (below 1e-38).  Also returns e^{-y^2/2}.
__device__ __forceinline__ float ntail(float yh, float yl, float &gauss) {
    constexpr float c[] = QMC_NTAIL_POLY;
    constexpr int n = sizeof(c) / sizeof(c[0]);
    const float y = fminf(yh, QMC_NTAIL_YMAX);
    // y^2 as a float-float (Dekker product), halved exactly
    const float sh = yh * yh;
    const float sl = fmaf(yh, yh, -sh) + 2.0f * yh * yl;
    gauss = yh <= QMC_NTAIL_YMAX ? exp_ff(-0.5f * sh, -0.5f * sl) : 0.0f;
    const float t = rcp_nr(fmaf(QMC_NTAIL_KAPPA, y, 1.0f));
    const float u = t - QMC_NTAIL_SHIFT;
    float p = c[n - 1];
#pragma unroll
    for (int i = n - 2; i >= 0; --i) p = fmaf(p, u, c[i]);
    p = fmaf(p, u, QMC_NTAIL_C1_LO) + QMC_NTAIL_C1_HI;
    p = fmaf(p, u, QMC_NTAIL_C0_LO) + QMC_NTAIL_C0_HI;
    return gauss * (t * p);
}
}  // namespace fx

template <> struct Arith<float> {
    // q = (lo + 1/2) 2^-32 <= 1/2 from lo = a 2^23 + b (one rounding), the
    // reflection sign of the upper half; shared by the one- and two-element
    // forms.  With B = 2^23 + b (b placed in the mantissa of 2^23),
    // B 2^-32 - (2^-9 - 2^-33) = (2b + 1) 2^-33 exactly (2b + 1 < 2^24), so one
    // FMA gives the low part and one more q.
    static constexpr float kQLow = -(0x1p-9f - 0x1p-33f);  // exact: 24 significant bits
    // -q for two draws, the floating-point steps in packed form (the
    // negated constants give exactly -q; the packed form then needs no
    // negated operands below)
    __device__ static __forceinline__ float2 neg_q_of2(uint32_t y0, uint32_t y1, uint32_t &s0, uint32_t &s1) {
        const uint32_t lo0 = y0 ^ static_cast<uint32_t>(static_cast<int32_t>(y0) >> 31);
        const uint32_t lo1 = y1 ^ static_cast<uint32_t>(static_cast<int32_t>(y1) >> 31);
        s0 = y0 & 0x80000000u;
        s1 = y1 & 0x80000000u;
        const float2 fa = add2(make_float2(__uint_as_float(0x4B000000u | (lo0 >> 23)),
                                           __uint_as_float(0x4B000000u | (lo1 >> 23))), f2(-8388608.0f));
        const float2 fb = make_float2(__uint_as_float(0x4B000000u | (lo0 & 0x007FFFFFu)),
                                      __uint_as_float(0x4B000000u | (lo1 & 0x007FFFFFu)));
        return fma2(fa, f2(-0x1p-9f), fma2(fb, f2(-0x1p-32f), f2(-kQLow)));
    }
    // the tail polynomial of one draw in s = sqrt(w) (0.1% of draws)
    __device__ static __forceinline__ float tail(float w) {
        constexpr float c[] = QMC_INVN_TAIL;
        constexpr int n = sizeof(c) / sizeof(c[0]);
        const float t = sqrtf(w) - QMC_INVN_SHIFT_T;
        float p = c[n - 1];
#pragma unroll
        for (int i = n - 2; i >= 0; --i) p = fmaf(p, t, c[i]);
        return fmaf(p, t, QMC_INVN_T0_LO) + QMC_INVN_T0_HI;
    }
    __device__ static __forceinline__ float central(float w) {
        constexpr float c[] = QMC_INVN_CENTRAL;
        constexpr int n = sizeof(c) / sizeof(c[0]);
        const float t = w - QMC_INVN_SHIFT_C;
        float p = c[n - 1];
#pragma unroll
        for (int i = n - 2; i >= 0; --i) p = fmaf(p, t, c[i]);
        return fmaf(p, t, QMC_INVN_C0_LO) + QMC_INVN_C0_HI;
    }
    // z = Phi^{-1}(u), u = (y + 1/2) 2^-32, for two draws: w = -ln(4q(1-q))
    // by the own logarithm, the central branch (99.9% of draws) in packed
    // form; a pair with a tail draw takes the one-element branches
    __device__ static float2 inv_normal2(uint32_t y0, uint32_t y1) {
        uint32_t s0, s1;
        const float2 nq = neg_q_of2(y0, y1, s0, s1);
        const float2 xm = fma2(f2(-2.0f), nq, f2(-1.0f));  // 2q - 1 = -x
        const float2 q4 = mul2(f2(-4.0f), nq);
        const float2 a = fma2(q4, nq, q4);                 // 4q(1 - q), one rounding
        const float2 w = fx::neg_ln2(a);
        float2 p;
        if (w.x < QMC_INVN_W0 && w.y < QMC_INVN_W0) {
            constexpr float c[] = QMC_INVN_CENTRAL;
            constexpr int n = sizeof(c) / sizeof(c[0]);
            const float2 t = add2(w, f2(-QMC_INVN_SHIFT_C));
            p = f2(c[n - 1]);
#pragma unroll
            for (int i = n - 2; i >= 0; --i) p = fma2(p, t, f2(c[i]));
            p = add2(fma2(p, t, f2(QMC_INVN_C0_LO)), f2(QMC_INVN_C0_HI));
        } else {
            p.x = w.x < QMC_INVN_W0 ? central(w.x) : tail(w.x);
            p.y = w.y < QMC_INVN_W0 ? central(w.y) : tail(w.y);
        }
        const float2 z = mul2(xm, p);
        return make_float2(__uint_as_float(__float_as_uint(z.x) ^ s0), __uint_as_float(__float_as_uint(z.y) ^ s1));
    }
    // The central branch of a pair alone (the results of inv_normal2 for a
    // pair without a tail draw); returns whether the pair has a tail draw, in
    // which case the caller redoes it with inv_normal2 (0.2% of pairs).  The
    // Sobol' runs call it with the redo deferred to the end of the run: a
    // test and branch per pair split the unrolled run into one basic block
    // per pair, so the compiler could not interleave the polynomial chains
    // of consecutive pairs (14% of the bridge kernel's time at d = 64).
    __device__ static __forceinline__ bool inv_normal2_central(uint32_t y0, uint32_t y1, float2 &z) {
        constexpr float c[] = QMC_INVN_CENTRAL;
        constexpr int n = sizeof(c) / sizeof(c[0]);
        uint32_t s0, s1;
        const float2 nq = neg_q_of2(y0, y1, s0, s1);
        const float2 xm = fma2(f2(-2.0f), nq, f2(-1.0f));
        const float2 q4 = mul2(f2(-4.0f), nq);
        const float2 w = fx::neg_ln2(fma2(q4, nq, q4));
        const float2 t = add2(w, f2(-QMC_INVN_SHIFT_C));
        float2 p = f2(c[n - 1]);
#pragma unroll
        for (int i = n - 2; i >= 0; --i) p = fma2(p, t, f2(c[i]));
        p = add2(fma2(p, t, f2(QMC_INVN_C0_LO)), f2(QMC_INVN_C0_HI));
        const float2 zz = mul2(xm, p);
        z = make_float2(__uint_as_float(__float_as_uint(zz.x) ^ s0), __uint_as_float(__float_as_uint(zz.y) ^ s1));
        return fmaxf(w.x, w.y) >= QMC_INVN_W0;
    }
    // one draw: the pair form's second lane duplicated (the same operations)
    __device__ static float inv_normal(uint32_t y) { return inv_normal2(y, y).x; }
    __device__ static float ex(float x) { return fx::exp_f(x); }
    __device__ static float2 ex2(float2 x) { return fx::exp_f2(x); }
};

// ---------------------------------------------------------------------------
// per-thread path accumulator (Sec. 4.5: S~_A or S~_max and the vega sum,
// formed on the fly)
// ---------------------------------------------------------------------------
template <typename T> struct PathAcc {
    T x;       // sum of S~/S0 (arith, binary), max S~/S0 (lookback), sum of log(S~/S0) (geometric)
    T dsum;    // sum of S~/S0 (W - sigma s) (arith, binary), at the max (lookback), sum of (W - sigma s) (geometric)
    int32_t m; // lookback: date index of the max (lowest on ties)

    __device__ void init(int type, bool has_first_date) {
        // date t_1 (s = 0, W~ = 0): S~/S0 = 1, log = 0, no vega term
        if (type == QMCCPW_LOOKBACK_FIXED_CALL) {
            x = has_first_date ? T(1) : T(-1);
            dsum = T(0);
            m = has_first_date ? 0 : 0x7fffffff;
        } else {
            x = (type == QMCCPW_GEOMETRIC_ASIAN_CALL || !has_first_date) ? T(0) : T(1);
            dsum = T(0);
            m = 0;
        }
    }

    // node: date index after t_1 (ties of the lookback maximum); s = node * dt
    template <int TYPE>
    __device__ __forceinline__ void add(int32_t node, T W, T omega, T sigma, T s) {
        const T lx = fma(sigma, W, omega * s);
        const T wv = fma(-sigma, s, W);
        if constexpr (TYPE == QMCCPW_GEOMETRIC_ASIAN_CALL) {
            x += lx;
            dsum += wv;
        } else {
            take<TYPE>(node, Arith<T>::ex(lx), wv);
        }
    }

    template <int TYPE>
    __device__ __forceinline__ void take(int32_t node, T e, T wv) {
        if constexpr (TYPE == QMCCPW_LOOKBACK_FIXED_CALL) {
            if (e > x || (e == x && node < m)) {
                x = e;
                dsum = e * wv;
                m = node;
            }
        } else {
            x += e;
            dsum = fma(e, wv, dsum);
        }
    }

    __device__ void merge(int type, const PathAcc &o) {
        if (type == QMCCPW_LOOKBACK_FIXED_CALL) {
            if (o.x > x || (o.x == x && o.m < m)) {
                x = o.x;
                dsum = o.dsum;
                m = o.m;
            }
        } else {
            x += o.x;
            dsum += o.dsum;
        }
    }
};


// The float path works on the path of unit spacing w = W~ / sqrt(dt) (the
// bridge, PCA and standard factors for dt = 1, no rescaling per element) and
// takes every constant that scales it as a float pair: the exponent
// omega s + sigma W~ = (sigma sqrt(dt)) w + (omega dt) node.  A float sigma
// alone (0.1 is 0.1 + 1.5e-9) would act as a shifted volatility on every
// path, and a float omega as a shifted drift.
struct PathConst {
    float a_hi, a_lo;  // sigma sqrt(dt)
    float b_hi, b_lo;  // omega dt
    __device__ explicit PathConst(const ContractDev &c)
        : a_hi(c.ff_sig_sdt[0]), a_lo(c.ff_sig_sdt[1]), b_hi(c.ff_om_dt[0]), b_lo(c.ff_om_dt[1]) {}
    __device__ PathConst() : a_hi(0.0f), a_lo(0.0f), b_hi(0.0f), b_lo(0.0f) {}
    // the exponent at a date: the small terms first, each FMA one rounding
    __device__ __forceinline__ float lx(float node, float w) const {
        return fmaf(w, a_hi, fmaf(node, b_hi, fmaf(w, a_lo, node * b_lo)));
    }
    __device__ __forceinline__ float2 lx2(float2 node, float2 w) const {
        return fma2(w, f2(a_hi), fma2(node, f2(b_hi), fma2(w, f2(a_lo), mul2(node, f2(b_lo)))));
    }
};

// Float accumulator of a point's path sums.  Arithmetic and binary: x =
// sum_j e_j (e_j = S~_j / S0), yw = sum_j e_j w_j, yn = sum_j e_j node_j, so
// that D = dX/dsigma = sqrt(dt) yw - sigma dt yn is formed once per point
// with its constants in float-float.  Lookback: x = max_j e_j, yw and m the
// w and the date index there (lowest on ties).  Geometric: x = sum_j w_j
// (the date indices sum to a constant).
template <> struct PathAcc<float> {
    float x, yw, yn;
    int32_t m;

    __device__ void init(int type, bool has_first_date) {
        // date t_1 (node 0, w = 0): e = 1, no vega term
        yw = 0.0f;
        yn = 0.0f;
        if (type == QMCCPW_LOOKBACK_FIXED_CALL) {
            x = has_first_date ? 1.0f : -1.0f;
            m = has_first_date ? 0 : 0x7fffffff;
        } else {
            x = (type == QMCCPW_GEOMETRIC_ASIAN_CALL || !has_first_date) ? 0.0f : 1.0f;
            m = 0;
        }
    }

    template <int TYPE>
    __device__ __forceinline__ void take(int32_t node, float nf, float e, float w) {
        if constexpr (TYPE == QMCCPW_LOOKBACK_FIXED_CALL) {
            if (e > x || (e == x && node < m)) {
                x = e;
                yw = w;
                m = node;
            }
        } else {
            x += e;
            yw = fmaf(e, w, yw);
            yn = fmaf(e, nf, yn);
        }
    }

    // one date: node = its index after t_1, w the unit-spacing path there
    template <int TYPE>
    __device__ __forceinline__ void add(int32_t node, float w, const PathConst &k) {
        if constexpr (TYPE == QMCCPW_GEOMETRIC_ASIAN_CALL) {
            x += w;
        } else {
            const float nf = small_uint_to_float(static_cast<uint32_t>(node));
            take<TYPE>(node, nf, fx::exp_f(k.lx(nf, w)), w);
        }
    }

    // two dates (node0 before node1): exponents and exponentials in packed
    // form, the sums in date order (equal to two calls of add)
    // (nf0, nf1: the dates as floats, when the caller has them; else formed here)
    template <int TYPE>
    __device__ __forceinline__ void add2(int32_t node0, int32_t node1, float w0, float w1, const PathConst &k,
                                         float nf0 = -1.0f, float nf1 = -1.0f) {
        if constexpr (TYPE == QMCCPW_GEOMETRIC_ASIAN_CALL) {
            x += w0;
            x += w1;
        } else {
            const float2 nf = nf0 >= 0.0f ? make_float2(nf0, nf1)
                                          : make_float2(small_uint_to_float(static_cast<uint32_t>(node0)),
                                                        small_uint_to_float(static_cast<uint32_t>(node1)));
            const float2 e = fx::exp_f2(k.lx2(nf, make_float2(w0, w1)));
            take<TYPE>(node0, nf.x, e.x, w0);
            take<TYPE>(node1, nf.y, e.y, w1);
        }
    }

    __device__ void merge(int type, const PathAcc &o) {
        if (type == QMCCPW_LOOKBACK_FIXED_CALL) {
            if (o.x > x || (o.x == x && o.m < m)) {
                x = o.x;
                yw = o.yw;
                m = o.m;
            }
        } else {
            x += o.x;
            yw += o.yw;
            yn += o.yn;
        }
    }
};

// ---------------------------------------------------------------------------
// conditional step: values of one point from X^ = X/S0 and D^ = D/S0
// ---------------------------------------------------------------------------
__device__ __forceinline__ double sf64(double x) { return 0.5 * erfc(x * 0.70710678118654752440); }
__device__ __forceinline__ double pdf64(double x) { return 0.39894228040143267794 * exp(-0.5 * x * x); }

__device__ void values_fp64(const ContractDev &c, double xhat, double dhat, double v[4]) {
    const double psi = (c.psi0 - log(xhat)) * c.inv_a;
    const double pdf = pdf64(psi);
    if (c.type == QMCCPW_BINARY_ASIAN) {
        v[0] = c.disc * sf64(psi);
        v[1] = c.disc * pdf / (c.S0 * c.a);
        v[2] = c.disc * pdf * (dhat / (c.a * xhat) + psi / c.sigma - c.sqrt_t1);
        v[3] = c.disc * pdf / (c.S0 * c.S0 * c.a) * (psi / c.a - 1.0);
    } else {
        const double sfs = sf64(psi - c.a);
        v[0] = c.disc1 * c.S0 * xhat * sfs - c.disc * c.K * sf64(psi);
        v[1] = c.disc1 * xhat * sfs;
        v[2] = c.disc1 * sfs * c.S0 * dhat + c.disc * c.K * pdf * c.sqrt_t1;
        v[3] = c.disc * c.K * pdf / (c.S0 * c.S0 * c.a);
    }
}

// ---------------------------------------------------------------------------
// float-float arithmetic (a value is hi + lo, |lo| <= ulp(hi)/2): Dekker
// products through FMA and Knuth's TwoSum, on the FP32 pipe, which on GB300
// runs 64x the FP64 rate
// ---------------------------------------------------------------------------
struct ff {
    float hi, lo;
};

__device__ __forceinline__ ff ff_fast_two_sum(float a, float b) {  // |a| >= |b|
    const float s = a + b;
    return {s, b - (s - a)};
}

__device__ __forceinline__ ff ff_two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}

__device__ __forceinline__ ff ff_mul(ff a, float b) {
    const float p = a.hi * b;
    const float e = fmaf(a.hi, b, -p);
    return ff_fast_two_sum(p, fmaf(a.lo, b, e));
}

__device__ __forceinline__ ff ff_add(ff a, ff b) {
    const ff s = ff_two_sum(a.hi, b.hi);
    return ff_fast_two_sum(s.hi, s.lo + (a.lo + b.lo));
}

__device__ __forceinline__ ff ff_neg(ff a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ ff ff_of(const float (&c)[2]) { return {c[0], c[1]}; }
__device__ __forceinline__ double ff_to_double(ff a) { return static_cast<double>(a.hi) + static_cast<double>(a.lo); }

// 1/x to ~1 ulp for positive normal x: the SFU approximation and one Newton
// step (IEEE division expands to a longer sequence)
__device__ __forceinline__ float rcp_f32(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r * fmaf(-x, r, 2.0f);
}

__device__ __forceinline__ ff ff_mul_ff(ff a, ff b) {
    const float p = a.hi * b.hi;
    const float e = fmaf(a.hi, b.hi, -p);
    return ff_fast_two_sum(p, fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e)));
}

// ln x in float-float for a positive normal float x, absolute error < 1e-9
// (60x below the float rounding of x itself):
// x = 2^e m, m in [1/sqrt2, sqrt2), ln m = 2 atanh f with f = (m-1)/(m+1)
// formed in float-float (|f| <= 0.172); 2f is carried in float-float and the
// rest of the series, 2f^3 (1/3 + f^2/5 + ... + f^8/11) <= 3.4e-3, in float
// from f's leading part (truncation < 2e-11, rounding and the dropped low
// part of f < 1e-9); e ln2 with a 2-part ln2 whose leading part has 16
// trailing zero bits, so e times it is exact.
__device__ __forceinline__ ff ln_ff(float x) {
    const uint32_t b = __float_as_uint(x);
    uint32_t eb = (b >> 23) & 0xFFu;
    float m = __uint_as_float((b & 0x007FFFFFu) | 0x3F800000u);
    if (m > 1.41421356f) {
        m *= 0.5f;
        eb += 1u;
    }
    const float num = m - 1.0f;                  // exact
    const ff den = ff_two_sum(m, 1.0f);          // m + 1, exact
    const float inv = rcp_f32(den.hi);
    const float q1 = num * inv;
    const float r = fmaf(-q1, den.hi, num) - q1 * den.lo;  // the remainder corrects q1's rounding
    const ff f = ff_fast_two_sum(q1, r * inv);
    const float f2 = f.hi * f.hi;
    float t = fmaf(f2, 1.0f / 11.0f, 1.0f / 9.0f);
    t = fmaf(t, f2, 1.0f / 7.0f);
    t = fmaf(t, f2, 1.0f / 5.0f);
    t = fmaf(t, f2, 1.0f / 3.0f);
    const ff lnm = ff_add(ff{2.0f * f.hi, 2.0f * f.lo}, ff{2.0f * f.hi * f2 * t, 0.0f});
    const float e = small_uint_to_float(eb) - 127.0f;  // exponent without a conversion instruction
    const ff eln2 = ff_fast_two_sum(e * 0.693145751953125f, e * 1.42860676533018e-06f);
    return ff_add(eln2, lnm);
}

// Mixed precision: the switch point psi and every combination with the
// contract constants in float-float (about 44 significant bits, on the FP32
// pipe: on this GPU a warp's FP64 instruction holds its sub-partition's FP64
// unit ~64x longer than an FP32 one).  The normal tails come from the own
// T(y) (fx::ntail): relative accuracy for every y, so Phi-bar near 1 is kept
// as the float-float 1 - T (a float Phi-bar there rounds to 1 and drops a
// one-signed tail), and e^{-psi^2/2} from the float-float psi^2.  The price of
// a call is a difference of two terms of size ~K; both are formed in
// float-float, and 1/sqrt(2 pi) sits in the float-float constants.
__device__ void values_mixed(const ContractDev &c, float xhat, float dhat, ff v[4]) {
    const ff psi = ff_mul_ff(ff_add(ff_of(c.ff_psi0), ff_neg(ln_ff(xhat))), ff_of(c.ff_inv_a));
    float g2;  // e^{-psi^2/2}
    const bool up2 = psi.hi >= 0.0f;
    const float T2 = fx::ntail(up2 ? psi.hi : -psi.hi, up2 ? psi.lo : -psi.lo, g2);
    const ff sf2 = up2 ? ff{T2, 0.0f} : ff_two_sum(1.0f, -T2);  // Phi-bar(psi)
    if (c.type == QMCCPW_BINARY_ASIAN) {
        v[0] = ff_mul_ff(ff_of(c.ff_disc), sf2);
        v[1] = ff_mul(ff_of(c.ff_kd_bin), g2);
        // D/(a X) + psi/sigma - sqrt(t1), then times e^{-rT} phi(psi)
        ff br = ff_mul(ff_of(c.ff_inv_a), dhat * fx::rcp_nr(xhat));
        br = ff_add(br, ff_mul_ff(psi, ff_of(c.ff_inv_sigma)));
        br = ff_add(br, ff_neg(ff_of(c.ff_sqrt_t1)));
        v[2] = ff_mul_ff(ff_mul(ff_of(c.ff_kphi), g2), br);
        // e^{-rT} phi(psi) / (S0^2 a) (psi/a - 1)
        const ff g = ff_add(ff_mul_ff(psi, ff_of(c.ff_inv_a)), ff{-1.0f, 0.0f});
        v[3] = ff_mul_ff(ff_mul(ff_of(c.ff_kg_bin), g2), g);
    } else {
        const ff psi1 = ff_add(psi, ff_neg(ff_of(c.ff_a)));  // psi - a
        const bool up1 = psi1.hi >= 0.0f;
        float g1;
        const float T1 = fx::ntail(up1 ? psi1.hi : -psi1.hi, up1 ? psi1.lo : -psi1.lo, g1);
        const ff sf1 = up1 ? ff{T1, 0.0f} : ff_two_sum(1.0f, -T1);  // Phi-bar(psi - a)
        const ff cx = ff_mul(ff_of(c.ff_disc1_S0), xhat);
        v[0] = ff_add(ff_mul_ff(cx, sf1), ff_neg(ff_mul_ff(ff_of(c.ff_disc_K), sf2)));
        v[1] = ff_mul_ff(ff_mul(ff_of(c.ff_disc1), xhat), sf1);
        v[2] = ff_add(ff_mul(ff_mul_ff(ff_of(c.ff_disc1_S0), sf1), dhat), ff_mul(ff_of(c.ff_kv_call), g2));
        v[3] = ff_mul(ff_of(c.ff_kg_call), g2);
    }
}

// ---------------------------------------------------------------------------
// conditioning on the leading coordinate of the whole path (constructions
// BB_LEAD, PCA_LEAD; the next reduction Sec. 6-7 name): the path of the d
// dates is W(t_j) = a_j x + R_j, x the leading Gaussian, so the average is
// X(x) = sum_j c_j e^{b_j x} with c_j = (S0/d) e^{omega t_j + sigma R_j},
// b_j = sigma a_j > 0.  The switch point x* solves X(x*) = K: Newton's method
// on ln X(x) - ln K, convex and increasing in x, converges from x = 0.  Then
// with E[e^{bx}; x > x*] = e^{b^2/2} Phi(b - x*) the conditional values are
// closed forms: call e^{-rT}[sum_j c_j e^{b_j^2/2} Phi(b_j - x*) - K Phi(-x*)],
// binary e^{-rT} Phi(-x*), and their derivatives at fixed R.  The geometric
// mean is log-linear in x, so its x* is explicit.  R[1..d] is the rest of the
// path (unit spacing of the tables already scaled), a from the contract's
// loading table times sqrt(dt).
// ---------------------------------------------------------------------------
template <typename T> struct LeadMath;
template <> struct LeadMath<double> {
    __device__ static double ex(double x) { return exp(x); }
    __device__ static double ln(double x) { return log(x); }
    __device__ static double sf(double x) { return 0.5 * erfc(x * 0.70710678118654752440); }
    __device__ static double pdf(double x) { return 0.39894228040143267794 * exp(-0.5 * x * x); }
    static constexpr double tol = 1e-15;
    static constexpr int iters = 200;
};
template <> struct LeadMath<float> {
    __device__ static float ex(float x) { return Arith<float>::ex(x); }
    __device__ static float ln(float x) { return logf(x); }
    __device__ static float sf(float x) { return 0.5f * erfcf(x * 0.707106781f); }
    __device__ static float pdf(float x) { return 0.398942280f * expf(-0.5f * x * x); }
    static constexpr float tol = 2e-7f;
    static constexpr int iters = 24;
};

template <typename T>
__device__ __forceinline__ T lead_loading(const ContractDev &c, int j) {  // a_{j+1}, 0-based j (double)
    return __ldg(c.lead_a64 + j) * c.sqrt_t1;
}

// values of one point: out = price, delta, vega, gamma (before the tile sum);
// the float path returns them as float pairs: the conditioning on the leading
// coordinate leaves the per-point values so close together that rounding each
// to one float would round them all the same way (a bias of up to half an
// ulp, above the standard error)
template <typename T> struct LeadOut { using type = double; };
template <> struct LeadOut<float> { using type = ff; };
__device__ __forceinline__ ff split_to_ff(double x) {
    const float hi = static_cast<float>(x);
    return ff{hi, static_cast<float>(x - static_cast<double>(hi))};
}
template <typename T>
__device__ void lead_values(const ContractDev &c, const T *R, typename LeadOut<T>::type out[4]);

// FP64: the formulas as they stand
// The lookback: its maximum max_j c_j e^{b_j x} (c_j = S0 e^{omega t_j +
// sigma R_j}) is the upper envelope of the lines ln c_j + b_j x, all
// increasing, so x* is the smallest of the lines' own roots; right of it the
// envelope is a run of pieces [u, v], one date each, the next date the first
// steeper line to overtake the current one, and each piece contributes its
// closed-form integral c_j e^{b^2/2} [Phi-bar(u - b) - Phi-bar(v - b)] (and
// the matching vega term); gamma comes from moving x* along the line active
// there.  In double for both precisions (R converted from float): the roots
// and crossings are compared as fractions by cross-multiplication, so a
// point takes one division for x* and one per piece boundary.
template <typename T>
__device__ void lead_lookback(const ContractDev &c, const T *R, double out[4]) {
    const int d = c.d;
    const double sig = c.sigma, omega = c.omega, dt = c.dt, lnK = c.ln_K;
    auto lc_of = [&](int j) { return c.ln_S0 + omega * ((j + 1) * dt) + sig * static_cast<double>(R[j + 1]); };
    // x* = min_j (ln K - lc_j) / b_j, ties to the steeper line
    double num = 0.0, den = 1.0;
    int cur = -1;
    for (int j = 0; j < d; ++j) {
        const double nj = lnK - lc_of(j), bj = sig * lead_loading<double>(c, j);
        if (cur < 0 || nj * den < num * bj || (nj * den == num * bj && bj > den)) {
            num = nj;
            den = bj;
            cur = j;
        }
    }
    const double xs = num / den, b_star = den;
    double price = 0.0, vega = 0.0, u = xs;
    // with loadings increasing in the date, the steeper lines are the later dates'
    const bool later_only = c.lead_increasing != 0;
    for (int piece = 0; piece < d; ++piece) {
        const double lcc = lc_of(cur), bc = sig * lead_loading<double>(c, cur);
        // the first steeper line to overtake: smallest (lcc - lc_j) / (b_j - bc) >= u
        double vn = 0.0, vd = 0.0;  // the crossing as a fraction, vd > 0 once found
        int next = -1;
        for (int j = later_only ? cur + 1 : 0; j < d; ++j) {
            const double bj = sig * lead_loading<double>(c, j);
            if (!(bj > bc)) continue;
            double nj = lcc - lc_of(j);
            const double dj = bj - bc;
            if (nj < u * dj) nj = u * dj;  // level with it at u already
            if (next < 0 || nj * vd < vn * dj || (nj * vd == vn * dj && bj > sig * lead_loading<double>(c, next))) {
                vn = nj;
                vd = dj;
                next = j;
            }
        }
        const double ch = exp(lcc + 0.5 * bc * bc);
        const double a = lead_loading<double>(c, cur);
        const double t = (cur + 1) * dt;
        const double su = 0.5 * erfc((u - bc) * 0.70710678118654752440);
        const double pu = 0.39894228040143267794 * exp(-0.5 * (u - bc) * (u - bc));
        double mass = su, dens = pu;
        double v = 0.0;
        if (next >= 0) {
            v = vn / vd;
            mass -= 0.5 * erfc((v - bc) * 0.70710678118654752440);
            dens -= 0.39894228040143267794 * exp(-0.5 * (v - bc) * (v - bc));
        }
        price += ch * mass;
        vega += ch * ((static_cast<double>(R[cur + 1]) - sig * t + a * bc) * mass + a * dens);
        if (next < 0) break;
        u = v;
        cur = next;
    }
    const double disc = c.disc, S0 = c.S0, K = c.K;
    out[0] = disc * (price - K * 0.5 * erfc(xs * 0.70710678118654752440));
    out[1] = disc * price / S0;
    out[2] = disc * vega;
    out[3] = disc * K * 0.39894228040143267794 * exp(-0.5 * xs * xs) / (S0 * S0 * b_star);
}

template <>
__device__ void lead_values<double>(const ContractDev &c, const double *R, double out[4]) {
    if (c.type == QMCCPW_LOOKBACK_FIXED_CALL) {
        lead_lookback<double>(c, R, out);
        return;
    }
    using M = LeadMath<double>;
    const int d = c.d;
    const double dt = c.dt, sig = c.sigma, omega = c.omega, K = c.K, S0 = c.S0, disc = c.disc;
    if (c.type == QMCCPW_GEOMETRIC_ASIAN_CALL) {
        double lmean = 0, amean = 0, bmean = 0;
        for (int j = 0; j < d; ++j) {
            const double t = (j + 1) * dt, Rj = R[j + 1];
            lmean += omega * t + sig * Rj;
            amean += lead_loading<double>(c, j);
            bmean += Rj - sig * t;
        }
        lmean *= c.inv_d;
        amean *= c.inv_d;
        bmean *= c.inv_d;
        const double b = sig * amean;
        const double xs = (c.psi0 + c.omega * c.dt - lmean) / b;  // (ln(K/S0) - lmean) / b, G = S0 e^{lmean}
        const double eb = S0 * exp(lmean + 0.5 * b * b);
        out[0] = disc * (eb * M::sf(xs - b) - K * M::sf(xs));
        out[1] = disc * eb * M::sf(xs - b) / S0;
        out[2] = disc * eb * ((amean * b + bmean) * M::sf(xs - b) + amean * M::pdf(xs - b));
        out[3] = disc * M::pdf(xs) * K / (S0 * S0 * b);
        return;
    }
    // Newton on g(x) = ln X(x) - ln K from x = 0; stop on a step below the
    // tolerance or (from the third step) one that no longer shrinks
    double x = 0, last = 1e300;
    for (int it = 0; it < M::iters; ++it) {
        double s0 = 0, s1 = 0;
        for (int j = 0; j < d; ++j) {
            const double b = sig * lead_loading<double>(c, j);
            const double e = exp(c.ln_lead_c0 + omega * ((j + 1) * dt) + sig * R[j + 1] + b * x);
            s0 += e;
            s1 += b * e;
        }
        const double step = (log(s0) - c.ln_K) * (s0 / s1);
        x -= step;
        const double mag = fabs(step);
        if (mag <= M::tol * (1.0 + fabs(x)) || (it >= 2 && mag >= last)) break;
        last = mag;
    }
    double X1 = 0, X2 = 0, F0 = 0, V = 0, B = 0;
    const double pdf = M::pdf(x);
    for (int j = 0; j < d; ++j) {
        const double t = (j + 1) * dt, a = lead_loading<double>(c, j), b = sig * a, Rj = R[j + 1];
        const double lc = c.ln_lead_c0 + omega * t + sig * Rj;
        const double e = exp(lc + b * x);               // c_j e^{b_j x*}
        const double eh = exp(lc + 0.5 * b * b);        // c_j e^{b_j^2/2}
        const double sfj = M::sf(x - b);
        X1 += b * e;
        X2 += b * b * e;
        F0 += eh * sfj;
        V += eh * (sig * a * a + Rj - sig * t) * sfj + a * e * pdf;  // e^{b^2/2} phi(x*-b) = e^{b x*} phi(x*)
        B += e * (a * x + Rj - sig * t);
    }
    if (c.type == QMCCPW_ARITH_ASIAN_CALL) {
        out[0] = disc * (F0 - K * M::sf(x));
        out[1] = disc * F0 / S0;
        out[2] = disc * V;
        out[3] = disc * pdf * K * K / (S0 * S0 * X1);
    } else {
        out[0] = disc * M::sf(x);
        out[1] = disc * pdf * K / (S0 * X1);
        out[2] = disc * pdf * B / X1;
        out[3] = disc * K * pdf * (x * K - 2.0 * X1 + K * X2 / X1) / ((S0 * X1) * (S0 * X1));
    }
}

// Mixed: two places where float would bias every point the same way are
// moved out of float.
// (1) The switch point: X(x) = (S0/d) sum_j e^{omega t_j + sigma R_j + b_j x};
//     the constant ln(S0/(d K)) of g(x) = ln X(x) - ln K enters as a
//     float-float pair (its float rounding alone would shift x* by ~1e-7/b),
//     the sum is accumulated and its logarithm taken in float-float.
// (2) The call price F0 - K Phi(-x*) is a difference of two nearly equal
//     terms.  With K = sum_j e_j (e_j = c_j e^{b_j x*}) and the Mills ratio
//     M(y) = Phi(-y)/phi(y), each term is c_j e^{b_j^2/2} Phi(b_j - x*) -
//     e_j Phi(-x*) = e_j phi(x*) [M(x* - b_j) - M(x*)], and the bracket is the
//     power series sum_k m_k b_j^k with m_k = (-1)^k M^(k)(x*)/k! >= 0 (M is
//     completely monotone), so it sums positive terms.  M(x*) and the m_k come
//     from the recurrence M' = xM - 1, M^(k+1) = x M^(k) + k M^(k-1) in double,
//     once per point.  The residual X(x*) - K of the float switch point is
//     added back at first order.
constexpr int kMillsTerms = 20;

// The loading of date j+1 times sqrt(dt) as a float pair (the table holds
// the unit-spacing loading as float pairs: the PCA's first column is no float).
__device__ __forceinline__ ff lead_loading_ff(const ContractDev &c, int j) {
    const float2 a = __ldg(reinterpret_cast<const float2 *>(c.lead_a32) + j);
    return ff_mul_ff(ff{a.x, a.y}, ff_of(c.ff_sqrt_t1));
}

template <>
__device__ void lead_values<float>(const ContractDev &c, const float *R, ff out[4]) {
    if (c.type == QMCCPW_LOOKBACK_FIXED_CALL) {
        double o[4];
        lead_lookback<float>(c, R, o);
        for (int g = 0; g < 4; ++g) out[g] = split_to_ff(o[g]);
        return;
    }
    const int d = c.d;
    const double K = c.K, S0 = c.S0, disc = c.disc;
    const float sh = c.ff_sig[0], sl = c.ff_sig[1];
    if (c.type == QMCCPW_GEOMETRIC_ASIAN_CALL) {
        // log-linear in x: a float sum of the path, the rest per point in double
        // (the sums of t_j and of the loadings are the contract's constants)
        float sumR = 0.0f;
        for (int j = 0; j < d; ++j) sumR += R[j + 1];
        const double st = c.dt * 0.5 * d * (d + 1.0);  // sum of t_j
        const double lm = (c.sigma * sumR + c.omega * st) * c.inv_d;
        const double am = c.lead_amean;
        const double bm = (sumR - c.sigma * st) * c.inv_d;
        double o[4];
        const double b = c.sigma * am;
        const double xs = (c.psi0 + c.omega * c.dt - lm) / b;
        const double eb = S0 * exp(lm + 0.5 * b * b);
        const double sfb = 0.5 * erfc((xs - b) * 0.70710678118654752440), sfx = 0.5 * erfc(xs * 0.70710678118654752440);
        const double pb = 0.39894228040143267794 * exp(-0.5 * (xs - b) * (xs - b));
        const double px = 0.39894228040143267794 * exp(-0.5 * xs * xs);
        o[0] = disc * (eb * sfb - K * sfx);
        o[1] = disc * eb * sfb / S0;
        o[2] = disc * eb * ((am * b + bm) * sfb + am * pb);
        o[3] = disc * px * K / (S0 * S0 * b);
        for (int g = 0; g < 4; ++g) out[g] = split_to_ff(o[g]);
        return;
    }
    // the exponent of c_j e^{b_j x}: ln(S0/d) + omega t_j + sigma R_j + b_j x
    // with b_j x = a_j (sigma sqrt(dt) x), every constant a float pair, the
    // small terms first (a float sigma, omega or loading would bias every point)
    auto expo = [&](int j, const ff &ys) {
        const float2 a = __ldg(reinterpret_cast<const float2 *>(c.lead_a32) + j);
        const float nf = small_uint_to_float(static_cast<uint32_t>(j + 1)), Rj = R[j + 1];
        float t = fmaf(a.y, ys.hi, c.ff_lnS0d[1]);
        t = fmaf(a.x, ys.lo, t);
        t = fmaf(Rj, sl, t);
        t = fmaf(nf, c.ff_om_dt[1], t);
        t = fmaf(nf, c.ff_om_dt[0], t);
        t = fmaf(Rj, sh, t);
        t = fmaf(a.x, ys.hi, t);
        return t + c.ff_lnS0d[0];
    };
    // (1) switch point: Newton on ln X(x) - ln K in float to its rounding
    // floor, then one step with the sum and g in float-float
    float x = 0, last = 1e30f;
    for (int it = 0; it <= LeadMath<float>::iters; ++it) {
        const bool polish = it == LeadMath<float>::iters;
        const ff ys = ff_mul(ff_of(c.ff_sig_sdt), x);
        ff s0{0.0f, 0.0f};
        float s1 = 0;
        for (int j = 0; j < d; ++j) {
            const float e = fx::exp_f(expo(j, ys));
            const float2 a = __ldg(reinterpret_cast<const float2 *>(c.lead_a32) + j);
            if (polish) s0 = ff_add(s0, ff{e, 0.0f});
            else s0.hi += e;
            s1 = fmaf(a.x, e, s1);  // sum a_j e_j: the derivative's scale, times sigma sqrt(dt) below
        }
        float gv;
        if (polish) {
            const ff g = ff_add(ff_add(ln_ff(s0.hi), ff{s0.lo / s0.hi, 0.0f}), ff_neg(ff_of(c.ff_lnK)));
            gv = g.hi + g.lo;
        } else {
            gv = logf(s0.hi) - (c.ff_lnK[0] + c.ff_lnK[1]);
        }
        const float step = gv * (s0.hi / (s1 * (c.ff_sig_sdt[0] + c.ff_sig_sdt[1])));
        x -= step;
        if (polish) break;
        const float mag = fabsf(step);
        if (mag <= LeadMath<float>::tol * (1.0f + fabsf(x)) || (it >= 2 && mag >= last)) it = LeadMath<float>::iters - 1;
        last = mag;
    }
    // (2) the Mills ratio at x* and its series coefficients, in double
    // (the loop is unrolled: k and 1/k! are constants, so the FP64 pipe,
    // 1/64 of the FP32 rate, sees no division or conversion here)
    const double xd = x;
    const double pdf = 0.39894228040143267794 * exp(-0.5 * xd * xd);
    const double Mx = 0.5 * erfc(xd * 0.70710678118654752440) / pdf;
    float mk[kMillsTerms];
    {
        double m_prev = Mx, m_cur = xd * Mx - 1.0;  // M, M'
        double inv_fact = 1.0;
#pragma unroll
        for (int k = 1; k <= kMillsTerms; ++k) {
            inv_fact *= 1.0 / static_cast<double>(k);
            const double m = m_cur * inv_fact;  // (-1)^k m_k
            mk[k - 1] = static_cast<float>((k & 1) ? -m : m);
            const double m_next = xd * m_cur + static_cast<double>(k) * m_prev;
            m_prev = m_cur;
            m_cur = m_next;
        }
    }
    const ff ys = ff_mul(ff_of(c.ff_sig_sdt), x);
    float X1 = 0, X2 = 0, SP = 0, SA = 0, V1 = 0, B = 0;
    ff Xs{0.0f, 0.0f}, W0{0.0f, 0.0f};
    for (int j = 0; j < d; ++j) {
        const ff as = lead_loading_ff(c, j);                  // a_j sqrt(dt)
        const ff b = ff_mul_ff(as, ff{sh, sl});               // b_j = sigma a_j sqrt(dt)
        const ff bb = ff_mul_ff(b, b);
        const float nf = small_uint_to_float(static_cast<uint32_t>(j + 1)), Rj = R[j + 1];
        const ff nst = ff_mul(ff_of(c.ff_nsig_dt), nf);        // -sigma t_j
        const ff Cw = ff_add(ff_mul_ff(b, as), nst);          // sigma a_j^2 dt - sigma t_j
        const ff Cb = ff_add(ff_mul(as, x), nst);             // a_j x* - sigma t_j
        const float e = fx::exp_f(expo(j, ys));               // c_j e^{b_j x*}
        float Q = mk[kMillsTerms - 1];
#pragma unroll
        for (int k = kMillsTerms - 2; k >= 0; --k) Q = fmaf(Q, b.hi, mk[k]);
        const float P = fmaf(Q, b.hi, Q * b.lo);              // M(x* - b) - M(x*) = b Q(b)
        // e_j w_j and e_j B_j (w_j = R_j + sigma a_j^2 - sigma t_j, B_j = R_j + a_j x*
        // - sigma t_j) and the weighted sums: each product with a pair's low part
        // meets the unrounded product of its high part in one FMA (added to an
        // already rounded sum it would sit below half an ulp and be dropped the
        // same way at every point: X1 came out 7.8e-9 low, 0.11 SE of a PCA-lead delta)
        const float ew = fmaf(e, Rj, fmaf(e, Cw.hi, e * Cw.lo));
        const float eb = fmaf(e, Rj, fmaf(e, Cb.hi, e * Cb.lo));
        Xs = ff_add(Xs, ff{e, 0.0f});
        X1 += fmaf(b.hi, e, b.lo * e);
        X2 += fmaf(bb.hi, e, bb.lo * e);
        SP = fmaf(e, P, SP);                       // sum e_j [M(x*-b_j) - M(x*)]
        SA += fmaf(as.hi, e, as.lo * e);
        V1 = fmaf(ew, P, V1);
        W0 = ff_add(W0, ff{ew, 0.0f});             // sum e_j w_j: signs mixed, kept in float-float
        B += eb;
    }
    // X(x*) - K of the float switch point
    const double resid = (static_cast<double>(Xs.hi) + Xs.lo) - K;
    const double sfx = Mx * pdf;  // Phi(-x*)
    if (c.type == QMCCPW_ARITH_ASIAN_CALL) {
        out[0] = split_to_ff(disc * (pdf * SP + resid * sfx));
        out[1] = split_to_ff(disc * (pdf * SP + (K + resid) * sfx) / S0);
        out[2] = split_to_ff(disc * pdf * (Mx * (static_cast<double>(W0.hi) + W0.lo) + V1 + SA));
        out[3] = split_to_ff(disc * pdf * K * K / (S0 * S0 * X1));
    } else {
        out[0] = split_to_ff(disc * sfx);
        out[1] = split_to_ff(disc * pdf * K / (S0 * X1));
        out[2] = split_to_ff(disc * pdf * B / X1);
        out[3] = split_to_ff(disc * K * pdf * (xd * K - 2.0 * X1 + K * X2 / X1) / ((S0 * X1) * (S0 * X1)));
    }
}

// ---------------------------------------------------------------------------
// Sobol' integers of one dimension over a run of consecutive points
// ---------------------------------------------------------------------------
// y XORed with the direction integers of the set bits of g: the point whose
// Gray code differs from y's by g.  From the digital shift and g(k0) it is
// point k0.  For a tile starting at k_t, a multiple of a power of two above
// every in-tile offset b, g(k_t + b) = g(k_t) ^ g(b) (the bits of k_t and b,
// and of their halves, do not overlap), so a run at offset b starts from the
// tile's first point by the few bits of g(b).
__device__ __forceinline__ uint32_t sobol_from_gray(const uint32_t *__restrict__ tab, int jstride, int j, uint32_t y,
                                                    uint32_t g) {
    while (g) {
        y ^= __ldg(tab + (__ffs(g) - 1) * jstride + j);
        g &= g - 1u;
    }
    return y;
}

// the same for two dimensions (one walk over the set bits of g, two loads per bit)
__device__ __forceinline__ void sobol_from_gray_pair(const uint32_t *__restrict__ tab, int jstride, int ja, int jb,
                                                     uint32_t ya0, uint32_t yb0, uint32_t g, uint32_t &ya,
                                                     uint32_t &yb) {
    ya = ya0;
    yb = yb0;
    while (g) {
        const uint32_t *row = tab + (__ffs(g) - 1) * jstride;
        ya ^= __ldg(row + ja);
        yb ^= __ldg(row + jb);
        g &= g - 1u;
    }
}

// First point k0 of a dimension (or two): from the digital shift by the set
// bits of g(k0).
__device__ __forceinline__ uint32_t sobol_first(const uint32_t *__restrict__ tab, int jstride, int j,
                                                uint32_t shift, uint32_t k0) {
    return sobol_from_gray(tab, jstride, j, shift, k0 ^ (k0 >> 1));
}

__device__ __forceinline__ void sobol_first_pair(const uint32_t *__restrict__ tab, int jstride, int ja, int jb,
                                                 uint32_t shift_a, uint32_t shift_b, uint32_t k0, uint32_t &ya,
                                                 uint32_t &yb) {
    sobol_from_gray_pair(tab, jstride, ja, jb, shift_a, shift_b, k0 ^ (k0 >> 1), ya, yb);
}

__host__ __device__ constexpr int ctz_const(int s) {
    int b = 0;
    while (!(s & 1)) {
        s >>= 1;
        ++b;
    }
    return b;
}

// A run of 2^LG consecutive points whose first index k0 is a multiple of
// 2^LG: point s of the run steps by direction integer ctz(s) < LG, the same
// for every such run, so those LG integers are loaded once and the run is
// unrolled (no index arithmetic or load per point).
template <int LG, typename Emit>
__device__ __forceinline__ void sobol_run(const uint32_t *__restrict__ tab, int jstride, int j, uint32_t y,
                                          Emit &&emit) {
    uint32_t v[LG > 0 ? LG : 1];
#pragma unroll
    for (int b = 0; b < LG; ++b) v[b] = __ldg(tab + b * jstride + j);
    emit(0, y);
#pragma unroll
    for (int s = 1; s < (1 << LG); ++s) {
        y ^= v[ctz_const(s)];
        emit(s, y);
    }
}

// Sobol' integers y(k0), ..., y(k0 + len - 1) of dimension j in Gray-code
// order (x(g(k+1)) = x(g(k)) xor v_ctz(k+1)), handed to emit(s, y).  A full
// aligned run of 4..64 points takes the unrolled form above.
template <typename Emit>
__device__ __forceinline__ void sobol_points(const uint32_t *__restrict__ tab, int jstride, int j, uint32_t y,
                                             uint32_t k0, int len, int chunk_log2, Emit &&emit) {
    // y: the point k0 (sobol_first, or the tile's first point and sobol_from_gray)
    if (len == (1 << chunk_log2) && (k0 & (static_cast<uint32_t>(len) - 1u)) == 0u) {
        switch (chunk_log2) {
            case 2: sobol_run<2>(tab, jstride, j, y, emit); return;
            case 3: sobol_run<3>(tab, jstride, j, y, emit); return;
            case 4: sobol_run<4>(tab, jstride, j, y, emit); return;
            case 5: sobol_run<5>(tab, jstride, j, y, emit); return;
            case 6: sobol_run<6>(tab, jstride, j, y, emit); return;
            default: break;
        }
    }
    emit(0, y);
    for (int s = 1; s < len; ++s) {
        y ^= __ldg(tab + (__ffs(k0 + s) - 1) * jstride + j);
        emit(s, y);
    }
}

// The points of a run handed out in consecutive pairs for the float paths,
// which evaluate the inverse normal two draws at a time.  A full aligned run
// (first index a multiple of 2^LG) has the inverse normal's tail test taken
// out of the unrolled body: emit2(s, z) receives the central
// values of points s, s+1 and a bit per pair records a tail draw; after the
// run each recorded pair (rare) is rebuilt from the run's first point by the
// bits of its Gray index and its exact values emitted again.
template <int LG, typename Emit2>
__device__ __forceinline__ void sobol_run_deferred(const uint32_t *__restrict__ tab, int jstride, int j, uint32_t y,
                                                   Emit2 &&emit2) {
    static_assert(LG >= 1 && LG <= 6, "runs of 2..64 points");
    uint32_t v[LG];
#pragma unroll
    for (int b = 0; b < LG; ++b) v[b] = __ldg(tab + b * jstride + j);
    const uint32_t y_first = y;
    uint32_t redo = 0;
#pragma unroll
    for (int s = 0; s < (1 << LG); s += 2) {
        if (s > 0) y ^= v[ctz_const(s)];
        const uint32_t y1 = y ^ v[0];
        float2 z;
        if (Arith<float>::inv_normal2_central(y, y1, z)) redo |= 1u << (s >> 1);
        emit2(s, z);
        y = y1;
    }
    while (redo) {
        const int s = 2 * (__ffs(redo) - 1);
        redo &= redo - 1u;
        const uint32_t g = static_cast<uint32_t>(s) ^ (static_cast<uint32_t>(s) >> 1);
        uint32_t ys = y_first;
#pragma unroll
        for (int b = 0; b < LG; ++b)
            if ((g >> b) & 1u) ys ^= v[b];
        emit2(s, Arith<float>::inv_normal2(ys, ys ^ v[0]));
    }
}

template <typename Emit1, typename Emit2>
__device__ __forceinline__ void sobol_point_deferred(const uint32_t *__restrict__ tab, int jstride, int j,
                                                     uint32_t y, uint32_t k0, int len, int chunk_log2,
                                                     Emit1 &&emit1, Emit2 &&emit2) {
    // y: the point k0 (sobol_first, or the tile's first point and sobol_from_gray)
    if (len == (1 << chunk_log2) && (k0 & (static_cast<uint32_t>(len) - 1u)) == 0u) {
        switch (chunk_log2) {
            case 2: sobol_run_deferred<2>(tab, jstride, j, y, emit2); return;
            case 3: sobol_run_deferred<3>(tab, jstride, j, y, emit2); return;
            case 4: sobol_run_deferred<4>(tab, jstride, j, y, emit2); return;
            case 5: sobol_run_deferred<5>(tab, jstride, j, y, emit2); return;
            case 6: sobol_run_deferred<6>(tab, jstride, j, y, emit2); return;
            default: break;
        }
    }
    int s = 0;
    for (; s + 1 < len; s += 2) {
        if (s > 0) y ^= __ldg(tab + (__ffs(k0 + s) - 1) * jstride + j);
        const uint32_t y1 = y ^ __ldg(tab + (__ffs(k0 + s + 1) - 1) * jstride + j);
        emit2(s, Arith<float>::inv_normal2(y, y1));
        y = y1;
    }
    if (s < len) {
        if (s > 0) y ^= __ldg(tab + (__ffs(k0 + s) - 1) * jstride + j);
        emit1(s, y);
    }
}

__device__ __forceinline__ int find_contract(const uint64_t *__restrict__ base, int count, uint64_t item) {
    int lo = 0, hi = count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(base + mid) <= item) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// The next work item of the dynamic schedule (CTAs take items as they finish
// one; an item's result never depends on which CTA ran it), decoded once by
// thread 0 and handed to the CTA through shared memory: contract, replicate
// and its tiles [tile, tile_end).  `stop` ends the loop for every thread.
// Starts and ends with a barrier, so every thread may read `w` from one call
// to the next (the item's fields need not be held in registers).
struct WorkItem {
    uint64_t item, tile, tile_end;
    int32_t ci;
    uint32_t rep;
};

// Tiles [tile, tile_end) of item `it` (0-based within its replicate) of c.
__device__ __forceinline__ void item_tiles(const ContractDev &c, uint64_t it, uint64_t &tile, uint64_t &tile_end) {
    tile = it * static_cast<uint64_t>(c.tpi);
    tile_end = min(tile + static_cast<uint64_t>(c.tpi), static_cast<uint64_t>(c.tiles));
}

__device__ __forceinline__ void next_work(const LaunchParams &p, WorkItem &w, bool stop = false) {
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint64_t item = stop ? p.item_end : p.item_begin + atomicAdd(p.work_counter, 1ull);
        w.item = item;
        if (item < p.item_end) {
            const int ci = find_contract(p.item_base, p.count, item);
            const ContractDev &c = p.contracts[ci];
            const uint64_t local = item - c.item_base;
            const uint64_t items = static_cast<uint64_t>(c.items);
            const uint64_t r = local / items;
            w.ci = ci;
            w.rep = static_cast<uint32_t>(r) + static_cast<uint32_t>(c.rep_first) + p.rep_offset;
            item_tiles(c, local - r * items, w.tile, w.tile_end);
        }
    }
    __syncthreads();
}

// Partial accumulators of a point live in several threads; they are staged
// in shared memory as slot-major arrays and merged by one thread per point in
// slot order (a fixed order, so the result does not depend on scheduling).
// Staging needs kStageBytes per (slot, point) entry, at most 4 * kThreads
// entries.
constexpr int kStageBytes = 20;

__device__ __forceinline__ void stage_partial(void *base, int P, int slot, int point, const PathAcc<double> &a) {
    double *rx = reinterpret_cast<double *>(base);
    double *rd = rx + kThreads * 4;
    int32_t *rm = reinterpret_cast<int32_t *>(rd + kThreads * 4);
    rx[slot * P + point] = a.x;
    rd[slot * P + point] = a.dsum;
    rm[slot * P + point] = a.m;
}

__device__ __forceinline__ void merge_partials(const void *base, int P, int slots, int point, int type, PathAcc<double> &a) {
    const double *rx = reinterpret_cast<const double *>(base);
    const double *rd = rx + kThreads * 4;
    const int32_t *rm = reinterpret_cast<const int32_t *>(rd + kThreads * 4);
    a.x = rx[point];
    a.dsum = rd[point];
    a.m = rm[point];
    for (int s = 1; s < slots; ++s) {
        PathAcc<double> o;
        o.x = rx[s * P + point];
        o.dsum = rd[s * P + point];
        o.m = rm[s * P + point];
        a.merge(type, o);
    }
}

// (float: `cap` entries per array, at least slots x P)
__device__ __forceinline__ void stage_partial(void *base, int P, int slot, int point, const PathAcc<float> &a,
                                              int cap = kThreads * 4) {
    float *rx = reinterpret_cast<float *>(base);
    float *rw = rx + cap;
    float *rn = rw + cap;
    int32_t *rm = reinterpret_cast<int32_t *>(rn + cap);
    rx[slot * P + point] = a.x;
    rw[slot * P + point] = a.yw;
    rn[slot * P + point] = a.yn;
    rm[slot * P + point] = a.m;
}

__device__ __forceinline__ void merge_partials(const void *base, int P, int slots, int point, int type, PathAcc<float> &a,
                                               int cap = kThreads * 4) {
    const float *rx = reinterpret_cast<const float *>(base);
    const float *rw = rx + cap;
    const float *rn = rw + cap;
    const int32_t *rm = reinterpret_cast<const int32_t *>(rn + cap);
    a.x = rx[point];
    a.yw = rw[point];
    a.yn = rn[point];
    a.m = rm[point];
    for (int s = 1; s < slots; ++s) {
        PathAcc<float> o;
        o.x = rx[s * P + point];
        o.yw = rw[s * P + point];
        o.yn = rn[s * P + point];
        o.m = rm[s * P + point];
        a.merge(type, o);
    }
}

// X^ = X/S0 and D^ = D/S0 of a point from its merged accumulator (double:
// the accumulator holds D itself; float: see PathAcc<float>, with the
// constants 1/d, sqrt(dt)/d, -sigma dt/d as float pairs)
__device__ __forceinline__ void finish_functional(const ContractDev &c, const PathAcc<double> &acc, double &xhat,
                                                  double &dhat) {
    if (c.type == QMCCPW_LOOKBACK_FIXED_CALL) {
        xhat = acc.x;
        dhat = acc.dsum;
    } else if (c.type == QMCCPW_GEOMETRIC_ASIAN_CALL) {
        xhat = exp(acc.x * c.inv_d);
        dhat = xhat * acc.dsum * c.inv_d;
    } else {
        xhat = acc.x * c.inv_d;
        dhat = acc.dsum * c.inv_d;
    }
}

// omega, sigma and the date spacing of the double path
__device__ __forceinline__ void market_of(const ContractDev &c, double &omega, double &sigma, double &dt) {
    omega = c.omega;
    sigma = c.sigma;
    dt = c.dt;
}

// a w + b n with a, b float pairs: the small terms first
__device__ __forceinline__ float lin2(const float (&a)[2], float w, const float (&b)[2], float n) {
    return fmaf(w, a[0], fmaf(n, b[0], fmaf(w, a[1], n * b[1])));
}

__device__ __forceinline__ void finish_functional(const ContractDev &c, const PathAcc<float> &acc, float &xhat,
                                                  float &dhat) {
    if (c.type == QMCCPW_LOOKBACK_FIXED_CALL) {
        // D^ = e* (sqrt(dt) w* - sigma dt node*)
        xhat = acc.x;
        dhat = acc.x * lin2(c.ff_sqrt_t1, acc.yw, c.ff_nsig_dt, small_uint_to_float(static_cast<uint32_t>(acc.m)));
    } else if (c.type == QMCCPW_GEOMETRIC_ASIAN_CALL) {
        // mean log = (sigma sqrt(dt) sum w + omega dt sum node)/d, the second a constant
        xhat = fx::exp_f(fmaf(acc.x, c.ff_sig_sdt_d[0], fmaf(acc.x, c.ff_sig_sdt_d[1], c.ff_geo_l0[1])) + c.ff_geo_l0[0]);
        dhat = xhat * (fmaf(acc.x, c.ff_sdt_d[0], fmaf(acc.x, c.ff_sdt_d[1], c.ff_geo_d0[1])) + c.ff_geo_d0[0]);
    } else {
        xhat = fmaf(acc.x, c.ff_inv_d[0], acc.x * c.ff_inv_d[1]);
        dhat = lin2(c.ff_sdt_d, acc.yw, c.ff_nsigdt_d, acc.yn);
    }
}

// Tile sum of the 4 values of every thread (zero for threads without a
// point): the kThreads x 4 values go through shared memory; warp g < 4 sums
// Greek g (each lane kThreads/32 consecutive threads, then a shuffle tree),
// a fixed order, and lane 0 of warp g hands it to sink(g, sum).  `smem`
// needs 4 * kThreads doubles; the caller's shared memory must be free on
// entry.  Ends with a barrier.
template <typename Sink>
__device__ __forceinline__ void tile_reduce(const double (&v)[4], unsigned char *smem, Sink &&sink) {
    __syncthreads();
    double *vals = reinterpret_cast<double *>(smem);
#pragma unroll
    for (int g = 0; g < 4; ++g) vals[g * kThreads + threadIdx.x] = v[g];
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp < 4) {
        const double *col = vals + warp * kThreads + lane * (kThreads / 32);
        double s = 0.0;
#pragma unroll
        for (int i = 0; i < kThreads / 32; ++i) s += col[i];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
        if (lane == 0) sink(warp, s);
    }
    __syncthreads();
}

// The same tile sum for float-float values: TwoSum-based adds on the FP32
// pipe; the sink receives the float-float sum.  `smem` needs 8 * kThreads
// floats.
template <typename Sink>
__device__ __forceinline__ void tile_reduce(const ff (&v)[4], unsigned char *smem, Sink &&sink) {
    __syncthreads();
    float *vals = reinterpret_cast<float *>(smem);
    if (threadIdx.x < kThreads) {  // larger blocks: the values live in the first kThreads threads
#pragma unroll
        for (int g = 0; g < 4; ++g) {
            vals[(2 * g) * kThreads + threadIdx.x] = v[g].hi;
            vals[(2 * g + 1) * kThreads + threadIdx.x] = v[g].lo;
        }
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp < 4) {
        const float *hi = vals + (2 * warp) * kThreads + lane * (kThreads / 32);
        const float *lo = vals + (2 * warp + 1) * kThreads + lane * (kThreads / 32);
        ff s = {0.0f, 0.0f};
#pragma unroll
        for (int i = 0; i < kThreads / 32; ++i) s = ff_add(s, ff{hi[i], lo[i]});
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const ff o = {__shfl_down_sync(0xffffffffu, s.hi, off), __shfl_down_sync(0xffffffffu, s.lo, off)};
            s = ff_add(s, o);
        }
        if (lane == 0) sink(warp, s);
    }
    __syncthreads();
}

// One tile's sums written to out[0..3] (the tile is the whole work item).
__device__ __forceinline__ void tile_sum(double *out, const double (&v)[4], unsigned char *smem) {
    tile_reduce(v, smem, [&](int g, double s) { out[g] = s; });
}
__device__ __forceinline__ void tile_sum(double *out, const ff (&v)[4], unsigned char *smem) {
    tile_reduce(v, smem, [&](int g, ff s) { out[g] = ff_to_double(s); });
}

// The sums of a work item's tiles, in tile order, in `acc` (shared memory,
// 8 doubles), owned per Greek g by lane 0 of warp g (the thread that adds the
// tile sums into it and flushes it): zero it before the first item
// (item_acc_clear), add each tile (tile_acc), write the item's slot and
// restart (item_flush) after its last tile.  Double values: a Neumaier sum
// and its compensation per Greek.  Float-float values (the float kernels):
// the float-float sum itself (about 48 bits over at most 16 tiles), kept on
// the FP32 pipe and converted to double once per item -- a double operation
// holds its sub-partition's FP64 unit for dozens of cycles, and a chain of
// them per tile, in the one lane the tile's last barrier waits for, stalled
// the whole CTA.
__device__ __forceinline__ bool item_acc_owner() { return (threadIdx.x & 31) == 0 && threadIdx.x < 128; }
__device__ __forceinline__ void item_acc_clear(double *acc) {
    if (item_acc_owner()) acc[threadIdx.x >> 5] = acc[4 + (threadIdx.x >> 5)] = 0.0;
}
__device__ __forceinline__ void tile_acc(double *acc, const double (&v)[4], unsigned char *smem) {
    tile_reduce(v, smem, [&](int g, double x) {
        const double s = acc[g], t = s + x;
        acc[4 + g] += fabs(s) >= fabs(x) ? (s - t) + x : (x - t) + s;
        acc[g] = t;
    });
}
__device__ __forceinline__ void tile_acc(double *acc, const ff (&v)[4], unsigned char *smem) {
    float *a = reinterpret_cast<float *>(acc);  // (hi, lo) of Greek g at 2g, 2g + 1
    tile_reduce(v, smem, [&](int g, ff x) {
        const ff t = ff_add(ff{a[2 * g], a[2 * g + 1]}, x);
        a[2 * g] = t.hi;
        a[2 * g + 1] = t.lo;
    });
}
template <typename V>
__device__ __forceinline__ void item_flush(double *out, double *acc) {
    if (item_acc_owner()) {
        const int g = threadIdx.x >> 5;
        if constexpr (std::is_same<V, double>::value) {
            out[g] = acc[g] + acc[4 + g];
            acc[g] = acc[4 + g] = 0.0;
        } else {
            float *a = reinterpret_cast<float *>(acc);
            out[g] = ff_to_double(ff{a[2 * g], a[2 * g + 1]});
            a[2 * g] = a[2 * g + 1] = 0.0f;
        }
    }
}
// The value type of a kernel's per-point results: double, or float-float for the float kernels.
template <typename T> using PointValue = typename std::conditional<sizeof(T) == 8, double, ff>::type;

}  // namespace
}  // namespace qmccpw
