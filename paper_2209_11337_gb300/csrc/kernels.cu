// Fused QMC-CPW kernel for sm_103a and its reduction kernels.
//
// One CTA processes one work item = (contract, replicate, tile of P points),
// in three phases that never leave the SM:
//   1. Sobol' + inverse normal (Sec. 2.2, Sec. 4.1): threads own (dimension,
//      chunk of consecutive points); the first point of a chunk is built
//      from the set bits of its Gray index, the rest by one XOR each
//      (g(k) ^ g(k-1) = 2^ctz(k)).  z lands in a shared-memory tile whose row
//      is one point; for the bridge, dimension j is stored at the date it
//      drives so the bridge can overwrite it in place.
//   2. Path construction and running sums (Sec. 3.3.1, 4.4): bridge levels
//      are processed breadth first, the nodes of a level spread over the
//      G = 256/P threads of a point (a barrier between levels); PCA rows are
//      independent dot products.  Each new W~(s_m) immediately contributes
//      S~/S0 = exp(omega s_m + sigma W~) to the path functional X and to
//      D = dX/dsigma; nothing per date is kept.
//   3. Conditional step (Sec. 3.3.2, 4.5): per point the switch point
//      psi = (ln(K/S0) - omega t_1 - ln X^)/a in double precision, then
//      price, delta, vega, gamma; a warp-shuffle + shared-memory tree sums the
//      tile into 4 doubles written to a per-item slot (no atomics, so the
//      result does not depend on scheduling).
// A second kernel sums each replicate's tile slots in tile order with
// compensated (Neumaier) arithmetic; a third forms mean and standard error
// over replicates.
#include <cuda_runtime.h>

#include <cstdint>

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

template <> struct Arith<float> {
    __device__ static float inv_normal(uint32_t y) {
        const bool upper = y >= 0x80000000u;
        const uint32_t lo = upper ? ~y : y;
        const float q = fmaf(__uint2float_rn(lo), 0x1p-32f, 0x1p-33f);
        const float z = normcdfinvf(q);
        return upper ? -z : z;
    }
    __device__ static float ex(float x) { return expf(x); }
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

    template <int TYPE>
    __device__ __forceinline__ void add(int32_t node, T W, T omega, T sigma, T dt) {
        const T s = static_cast<T>(node) * dt;
        const T lx = omega * s + sigma * W;
        const T wv = W - sigma * s;
        if constexpr (TYPE == QMCCPW_GEOMETRIC_ASIAN_CALL) {
            x += lx;
            dsum += wv;
        } else {
            const T e = Arith<T>::ex(lx);
            if constexpr (TYPE == QMCCPW_LOOKBACK_FIXED_CALL) {
                if (e > x || (e == x && node < m)) {
                    x = e;
                    dsum = e * wv;
                    m = node;
                }
            } else {
                x += e;
                dsum += e * wv;
            }
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

// Mixed precision: the switch point psi in double; the normal tail and
// density in float; the combination with the contract constants in double.
// The price of a call is the difference of two terms of size ~K: float
// constants there would bias every point by ~2^-24 K, which no averaging
// removes.  Beyond |psi| = 12 the float density and tail underflow, so
// those (rare) points take the double formulas.
__device__ void values_mixed(const ContractDev &c, float xhat, float dhat, double v[4]) {
    const double psi = (c.psi0 - log(static_cast<double>(xhat))) * c.inv_a;
    if (fabs(psi) > 12.0) {
        values_fp64(c, static_cast<double>(xhat), static_cast<double>(dhat), v);
        return;
    }
    const float p = static_cast<float>(psi);
    const float pdf = 0.398942280f * expf(-0.5f * p * p);
    if (c.type == QMCCPW_BINARY_ASIAN) {
        const double sf = 0.5f * erfcf(p * 0.707106781f);
        const double pd = pdf;
        v[0] = c.disc * sf;
        v[1] = c.k_bin_delta * pd;
        v[2] = c.disc * pd * (static_cast<double>(dhat / xhat) * c.inv_a + psi * c.inv_sigma - c.sqrt_t1);
        v[3] = c.k_bin_gamma * pd * (psi * c.inv_a - 1.0);
    } else {
        const float a = static_cast<float>(c.a);
        const double sfs = 0.5f * erfcf((p - a) * 0.707106781f);
        const double sf = 0.5f * erfcf(p * 0.707106781f);
        const double xh = xhat;
        v[0] = c.disc1_S0 * xh * sfs - c.disc_K * sf;
        v[1] = c.disc1 * xh * sfs;
        v[2] = c.disc1_S0 * sfs * static_cast<double>(dhat) + c.disc_K * c.sqrt_t1 * static_cast<double>(pdf);
        v[3] = c.k_call_gamma * static_cast<double>(pdf);
    }
}

// ---------------------------------------------------------------------------
// Sobol' integers of one dimension over a run of consecutive points
// ---------------------------------------------------------------------------
// First point k0: XOR of the direction integers of the set bits of g(k0),
// starting from the digital shift.
__device__ __forceinline__ uint32_t sobol_first(const uint32_t *__restrict__ tab, int jstride, int j,
                                                uint32_t shift, uint32_t k0) {
    uint32_t g = k0 ^ (k0 >> 1);
    uint32_t y = shift;
    while (g) {
        const int b = __ffs(g) - 1;
        y ^= __ldg(tab + b * jstride + j);
        g &= g - 1u;
    }
    return y;
}

// ---------------------------------------------------------------------------
// the fused kernel
// ---------------------------------------------------------------------------
__device__ __forceinline__ int find_contract(const uint64_t *__restrict__ base, int count, uint64_t item) {
    int lo = 0, hi = count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(base + mid) <= item) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Bridge (Sec. 4.4): levels breadth first; within a level the nodes of a
// point are spread over its G threads; W~ overwrites z in the point's row.
template <typename T, int TYPE>
__device__ void bridge_phase(const ContractDev &c, T *zw, int stride, PathAcc<T> &acc) {
    const int P = 1 << c.tile_log2;
    const int pt = threadIdx.x & (P - 1);
    const int grp = threadIdx.x >> c.tile_log2;
    const int G = c.groups;
    T *row = zw + pt * stride;
    const T omega = static_cast<T>(c.omega), sigma = static_cast<T>(c.sigma), dt = static_cast<T>(c.dt);
    for (int lvl = 0; lvl < c.n_levels; ++lvl) {
        const int b_end = __ldg(c.level_start + lvl + 1);
        for (int b = __ldg(c.level_start + lvl) + grp; b < b_end; b += G) {
            const int4 st = __ldg(reinterpret_cast<const int4 *>(c.steps) + b);
            const T Wl = row[st.y], Wr = row[st.z], z = row[st.x];
            T Wm;
            if constexpr (sizeof(T) == 8) {
                const double *w = c.w64 + 3 * b;
                Wm = __ldg(w) * Wl + __ldg(w + 1) * Wr + __ldg(w + 2) * z;
            } else {
                // hi + lo coefficients: the low parts first, then the high parts
                const float4 h = __ldg(reinterpret_cast<const float4 *>(c.w32) + 2 * b);
                const float4 g = __ldg(reinterpret_cast<const float4 *>(c.w32) + 2 * b + 1);
                float lo = h.y * Wl;
                lo = fmaf(h.w, Wr, lo);
                lo = fmaf(g.y, z, lo);
                Wm = fmaf(h.x, Wl, fmaf(h.z, Wr, fmaf(g.x, z, lo)));
            }
            row[st.x] = Wm;
            acc.template add<TYPE>(st.x, Wm, omega, sigma, dt);
        }
        if (G > 1) __syncthreads();
    }
}

// PCA, plain form (double precision, and tiles of fewer than 32 points): the
// G threads of a point take every G-th row of A.
template <typename T, int TYPE>
__device__ void pca_rows_phase(const ContractDev &c, const T *zw, int stride, PathAcc<T> &acc) {
    const int P = 1 << c.tile_log2;
    const int pt = threadIdx.x & (P - 1);
    const int grp = threadIdx.x >> c.tile_log2;
    const T *row = zw + pt * stride;
    const T omega = static_cast<T>(c.omega), sigma = static_cast<T>(c.sigma), dt = static_cast<T>(c.dt);
    const int n = c.n;
    for (int i = 1 + grp; i <= n; i += c.groups) {
        T Wi = T(0);
        if constexpr (sizeof(T) == 8) {
            const double *Ai = c.pca64 + static_cast<size_t>(i - 1) * n;
            for (int k = 0; k < n; ++k) Wi += __ldg(Ai + k) * row[k + 1];
        } else {
            const int n_pad = (n + 15) & ~15;
            for (int k = 0; k < n; ++k) Wi = fmaf(__ldg(c.pcaT32 + static_cast<size_t>(k) * n_pad + (i - 1)), row[k + 1], Wi);
        }
        acc.template add<TYPE>(i, Wi, omega, sigma, dt);
    }
}

// PCA as a register-blocked product W = Z A^T on the FP32 pipe: a thread owns
// PB points (lanes are consecutive points, so the z loads are conflict free)
// and 16 rows of A^T (the same for the whole warp, so each float4 of A^T is
// one broadcast load).  Per k: PB shared loads, 4 uniform loads, 16 PB FMAs.
template <int PB, int TYPE>
__device__ void pca_gemm_phase(const ContractDev &c, const float *zw, int stride, PathAcc<float> (&acc)[PB],
                               int &slot, int &slots, int (&pts)[PB]) {
    const int P = 1 << c.tile_log2;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int groups = P / (32 * PB);
    slots = (kThreads / 32) / groups;
    const int g = warp % groups;
    slot = warp / groups;
    const int n = c.n, n4 = ((n + 15) & ~15) >> 2;
    const float omega = static_cast<float>(c.omega), sigma = static_cast<float>(c.sigma), dt = static_cast<float>(c.dt);
    const float *zr[PB];
#pragma unroll
    for (int j = 0; j < PB; ++j) {
        pts[j] = g * 32 * PB + lane + 32 * j;
        zr[j] = zw + pts[j] * stride + 1;
        acc[j].init(TYPE, slot == 0);
    }
    const float4 *AT = reinterpret_cast<const float4 *>(c.pcaT32);
    for (int rb = slot; rb * 16 < n; rb += slots) {
        float w[PB][16];
#pragma unroll
        for (int j = 0; j < PB; ++j)
#pragma unroll
            for (int r = 0; r < 16; ++r) w[j][r] = 0.0f;
        const float4 *a = AT + 4 * rb;
        for (int k = 0; k < n; ++k, a += n4) {
            const float4 a0 = __ldg(a), a1 = __ldg(a + 1), a2 = __ldg(a + 2), a3 = __ldg(a + 3);
            const float av[16] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w,
                                  a2.x, a2.y, a2.z, a2.w, a3.x, a3.y, a3.z, a3.w};
#pragma unroll
            for (int j = 0; j < PB; ++j) {
                const float z = zr[j][k];
#pragma unroll
                for (int r = 0; r < 16; ++r) w[j][r] = fmaf(av[r], z, w[j][r]);
            }
        }
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            const int i = rb * 16 + r + 1;
            if (i <= n) {
#pragma unroll
                for (int j = 0; j < PB; ++j) acc[j].template add<TYPE>(i, w[j][r], omega, sigma, dt);
            }
        }
    }
}

// Partial accumulators of a point live in several threads; they are staged
// in shared memory as slot-major arrays and merged by one thread per point in
// slot order (a fixed order, so the result does not depend on scheduling).
template <typename T>
__device__ __forceinline__ void stage_partial(void *base, int P, int slot, int point, const PathAcc<T> &a) {
    T *rx = reinterpret_cast<T *>(base);
    T *rd = rx + kThreads * 4;
    int32_t *rm = reinterpret_cast<int32_t *>(rd + kThreads * 4);
    rx[slot * P + point] = a.x;
    rd[slot * P + point] = a.dsum;
    rm[slot * P + point] = a.m;
}

template <typename T>
__device__ __forceinline__ void merge_partials(const void *base, int P, int slots, int point, int type, PathAcc<T> &a) {
    const T *rx = reinterpret_cast<const T *>(base);
    const T *rd = rx + kThreads * 4;
    const int32_t *rm = reinterpret_cast<const int32_t *>(rd + kThreads * 4);
    a.x = rx[point];
    a.dsum = rd[point];
    a.m = rm[point];
    for (int s = 1; s < slots; ++s) {
        PathAcc<T> o;
        o.x = rx[s * P + point];
        o.dsum = rd[s * P + point];
        o.m = rm[s * P + point];
        a.merge(type, o);
    }
}

// Phase 2 for one product type: returns, for threads t < P, the merged
// accumulator of point t in `acc` (other threads' acc is unspecified).
template <typename T, int CONS, int TYPE>
__device__ void path_phase(const ContractDev &c, T *zw, int stride, PathAcc<T> &acc) {
    const int P = 1 << c.tile_log2;
    if constexpr (CONS == QMCCPW_BB) {
        acc.init(TYPE, threadIdx.x < P);
        bridge_phase<T, TYPE>(c, zw, stride, acc);
        if (c.groups == 1) return;
        __syncthreads();
        stage_partial<T>(zw, P, threadIdx.x >> c.tile_log2, threadIdx.x & (P - 1), acc);
        __syncthreads();
        if (threadIdx.x < P) merge_partials<T>(zw, P, c.groups, threadIdx.x, TYPE, acc);
        return;
    } else {
    if constexpr (sizeof(T) == 4) {
        if (P >= 32) {
            int slot = 0, slots = 1;
            if (P >= 128) {
                PathAcc<float> a4[4];
                int pts[4];
                pca_gemm_phase<4, TYPE>(c, zw, stride, a4, slot, slots, pts);
                __syncthreads();
#pragma unroll
                for (int j = 0; j < 4; ++j) stage_partial<float>(zw, P, slot, pts[j], a4[j]);
            } else if (P == 64) {
                PathAcc<float> a2[2];
                int pts[2];
                pca_gemm_phase<2, TYPE>(c, zw, stride, a2, slot, slots, pts);
                __syncthreads();
#pragma unroll
                for (int j = 0; j < 2; ++j) stage_partial<float>(zw, P, slot, pts[j], a2[j]);
            } else {
                PathAcc<float> a1[1];
                int pts[1];
                pca_gemm_phase<1, TYPE>(c, zw, stride, a1, slot, slots, pts);
                __syncthreads();
                stage_partial<float>(zw, P, slot, pts[0], a1[0]);
            }
            __syncthreads();
            if (threadIdx.x < P) merge_partials<float>(zw, P, slots, threadIdx.x, TYPE, acc);
            return;
        }
    }
    acc.init(TYPE, threadIdx.x < P);
    pca_rows_phase<T, TYPE>(c, zw, stride, acc);
    if (c.groups == 1) return;
    __syncthreads();
    stage_partial<T>(zw, P, threadIdx.x >> c.tile_log2, threadIdx.x & (P - 1), acc);
    __syncthreads();
    if (threadIdx.x < P) merge_partials<T>(zw, P, c.groups, threadIdx.x, TYPE, acc);
    }
}

// CONS is the construction of every contract this launch covers (the host
// launches one grid per construction over that construction's items).
template <typename T, int CONS>
__global__ void __launch_bounds__(kThreads) fused_kernel(const __grid_constant__ LaunchParams p) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double warp_part[kThreads / 32][4];

    for (uint64_t item = p.item_begin + blockIdx.x; item < p.item_end; item += gridDim.x) {
        const int ci = find_contract(p.item_base, p.count, item);
        const ContractDev &c = p.contracts[ci];
        const int P = 1 << c.tile_log2;
        const int n = c.n;
        const int stride = c.row_stride;
        const uint64_t local = item - c.item_base;
        const uint32_t rep = static_cast<uint32_t>(local / static_cast<uint64_t>(c.tiles)) + p.rep_offset;
        const uint64_t tile = local % static_cast<uint64_t>(c.tiles);
        T *zw = reinterpret_cast<T *>(smem);

        // ---- phase 1: Sobol' + inverse normal -> zw[point][slot]
        if (n > 0) {
            const uint32_t *tab = p.sobol_table + static_cast<size_t>(rep) * 32u * p.jstride;
            const uint32_t *shf = p.sobol_shift + static_cast<size_t>(rep) * p.jstride;
            const int chunk = 1 << c.chunk_log2;
            const int work = (P >> c.chunk_log2) * n;
            for (int it = threadIdx.x; it < work; it += kThreads) {
                const int j = it % n;
                const int ch = it / n;
                const int slot = (CONS == QMCCPW_BB) ? __ldg(&c.steps[j].m) : j + 1;
                T *dst = zw + static_cast<size_t>(ch * chunk) * stride + slot;
                // points at or past N (ragged last tile) are never generated: their
                // index could pass 2^32; they are zero-filled and left out of the sums
                const uint64_t first_local = tile * P + static_cast<uint64_t>(ch) * chunk;
                const int len = first_local >= c.N ? 0 : static_cast<int>(min(static_cast<uint64_t>(chunk), c.N - first_local));
                if (len > 0) {
                    const uint32_t k0 = static_cast<uint32_t>(p.point_k0 + first_local);
                    uint32_t y = sobol_first(tab, p.jstride, j, __ldg(shf + j), k0);
                    dst[0] = Arith<T>::inv_normal(y);
                    for (int s = 1; s < len; ++s) {
                        y ^= __ldg(tab + (__ffs(k0 + s) - 1) * p.jstride + j);
                        dst[s * stride] = Arith<T>::inv_normal(y);
                    }
                }
                for (int s = len; s < chunk; ++s) dst[s * stride] = T(0);
            }
        }
        for (int pt = threadIdx.x; pt < P; pt += kThreads) zw[pt * stride] = T(0);
        __syncthreads();

        // ---- phase 2: path construction and running sums, merged per point
        PathAcc<T> acc;
        switch (c.type) {
            case QMCCPW_ARITH_ASIAN_CALL: path_phase<T, CONS, QMCCPW_ARITH_ASIAN_CALL>(c, zw, stride, acc); break;
            case QMCCPW_BINARY_ASIAN: path_phase<T, CONS, QMCCPW_BINARY_ASIAN>(c, zw, stride, acc); break;
            case QMCCPW_LOOKBACK_FIXED_CALL: path_phase<T, CONS, QMCCPW_LOOKBACK_FIXED_CALL>(c, zw, stride, acc); break;
            default: path_phase<T, CONS, QMCCPW_GEOMETRIC_ASIAN_CALL>(c, zw, stride, acc); break;
        }
        const int pt = threadIdx.x;

        // ---- phase 3: conditional values of the point, tile sum
        double v[4] = {0.0, 0.0, 0.0, 0.0};
        const uint64_t local_point = tile * P + pt;
        if (pt < P && local_point < c.N) {
            T xhat, dhat;
            if (c.type == QMCCPW_LOOKBACK_FIXED_CALL) {
                xhat = acc.x;
                dhat = acc.dsum;
            } else if (c.type == QMCCPW_GEOMETRIC_ASIAN_CALL) {
                const T inv_d = T(1) / static_cast<T>(c.d);
                xhat = Arith<T>::ex(acc.x * inv_d);
                dhat = xhat * acc.dsum * inv_d;
            } else {
                const T inv_d = T(1) / static_cast<T>(c.d);
                xhat = acc.x * inv_d;
                dhat = acc.dsum * inv_d;
            }
            if constexpr (sizeof(T) == 8) values_fp64(c, xhat, dhat, v);
            else values_mixed(c, xhat, dhat, v);
            if (p.point_out) {
                double *o = p.point_out + local_point * 4;
                o[0] = v[0]; o[1] = v[1]; o[2] = v[2]; o[3] = v[3];
            }
        }
        // block sum: warp shuffle tree, then the 8 warp partials in order
#pragma unroll
        for (int g = 0; g < 4; ++g) {
            double s = v[g];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
            if ((threadIdx.x & 31) == 0) warp_part[threadIdx.x >> 5][g] = s;
        }
        __syncthreads();
        if (threadIdx.x < 4) {
            double s = 0.0;
            for (int w = 0; w < kThreads / 32; ++w) s += warp_part[w][threadIdx.x];
            p.tile_sums[item * 4 + threadIdx.x] = s;
        }
        __syncthreads();  // smem and warp_part are reused by the next item
    }
}

// ---------------------------------------------------------------------------
// per-replicate compensated reduction of the tile slots, then statistics
// ---------------------------------------------------------------------------
struct Neumaier {
    double s, c;
    __device__ void add(double x) {
        const double t = s + x;
        if (fabs(s) >= fabs(x)) c += (s - t) + x;
        else c += (x - t) + s;
        s = t;
    }
    __device__ void add(const Neumaier &o) {
        add(o.s);
        c += o.c;
    }
    __device__ double value() const { return s + c; }
};

__global__ void __launch_bounds__(256) reduce_kernel(const ContractDev *__restrict__ contracts,
                                                     const uint64_t *__restrict__ rep_owner,
                                                     const double *__restrict__ tile_sums,
                                                     double *__restrict__ per_rep) {
    __shared__ Neumaier part[256][4];
    const uint64_t slot = blockIdx.x;  // global replicate slot
    const ContractDev &c = contracts[rep_owner[slot]];
    const uint64_t r = slot - c.rep_base;
    const uint64_t first = c.item_base + r * static_cast<uint64_t>(c.tiles);
    Neumaier acc[4] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
    for (uint64_t t = threadIdx.x; t < static_cast<uint64_t>(c.tiles); t += blockDim.x)
        for (int g = 0; g < 4; ++g) acc[g].add(tile_sums[(first + t) * 4 + g]);
    for (int g = 0; g < 4; ++g) part[threadIdx.x][g] = acc[g];
    __syncthreads();
    for (int half = 128; half > 0; half >>= 1) {
        if (threadIdx.x < half)
            for (int g = 0; g < 4; ++g) part[threadIdx.x][g].add(part[threadIdx.x + half][g]);
        __syncthreads();
    }
    if (threadIdx.x < 4) per_rep[slot * 4 + threadIdx.x] = part[0][threadIdx.x].value() / static_cast<double>(c.N);
}

__global__ void stats_kernel(const ContractDev *__restrict__ contracts, int count,
                             const double *__restrict__ per_rep, double *__restrict__ stats) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= count * 4) return;
    const int ci = t >> 2, g = t & 3;
    const ContractDev &c = contracts[ci];
    Neumaier s = {0, 0};
    for (int r = 0; r < c.R; ++r) s.add(per_rep[(c.rep_base + r) * 4 + g]);
    const double mean = s.value() / c.R;
    Neumaier dev = {0, 0};
    for (int r = 0; r < c.R; ++r) {
        const double e = per_rep[(c.rep_base + r) * 4 + g] - mean;
        dev.add(e * e);
    }
    stats[ci * 8 + g] = mean;
    stats[ci * 8 + 4 + g] = sqrt(dev.value() / (static_cast<double>(c.R) * (c.R - 1)));
}

// ---------------------------------------------------------------------------
// plan set-up: scrambled direction-integer tables (Sec. 2.2.3) and the
// Sobol' diagnostic dump
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t splitmix64_dev(uint64_t key, uint64_t counter) {
    uint64_t z = key + (counter + 1u) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// One thread per (replicate, dimension): rows of L (digit i depends on
// digits 1..i) from SplitMix64, then every direction integer v becomes L v,
// and the shift e is stored beside them.
__global__ void scramble_kernel(uint64_t seed, const uint32_t *__restrict__ v, int ndims, int jstride,
                                int reps, uint32_t *__restrict__ table, uint32_t *__restrict__ shift) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ndims * reps) return;
    const int j = t % ndims;
    const uint32_t r = static_cast<uint32_t>(t / ndims);
    const uint64_t base = (static_cast<uint64_t>(r) << 32) | (static_cast<uint64_t>(j) << 8);
    uint32_t rows[32];
#pragma unroll
    for (int i = 1; i <= 32; ++i) {
        const uint32_t draw = static_cast<uint32_t>(splitmix64_dev(seed, base | static_cast<uint64_t>(i - 1)) >> 32);
        const uint32_t below = (i >= 2) ? (0xFFFFFFFFu << (33 - i)) : 0u;
        rows[i - 1] = (draw & below) | (1u << (32 - i));
    }
    uint32_t *tr = table + static_cast<size_t>(r) * 32u * jstride;
    for (int b = 0; b < 32; ++b) {
        const uint32_t x = v[32 * j + b];
        uint32_t y = 0;
#pragma unroll
        for (int i = 1; i <= 32; ++i) y |= static_cast<uint32_t>(__popc(rows[i - 1] & x) & 1) << (32 - i);
        tr[b * jstride + j] = y;
    }
    shift[static_cast<size_t>(r) * jstride + j] = static_cast<uint32_t>(splitmix64_dev(seed, base | 32u) >> 32);
}

// Same generation code as phase 1: one thread per (dimension, run of 16
// consecutive points).
__global__ void sobol_dump_kernel(const uint32_t *__restrict__ tab, const uint32_t *__restrict__ shf, int jstride,
                                  int ndims, uint64_t k0, uint64_t count, uint32_t *__restrict__ out) {
    constexpr int kRun = 16;
    const uint64_t t = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x;
    const uint64_t runs = (count + kRun - 1) / kRun;
    if (t >= runs * ndims) return;
    const int j = static_cast<int>(t % ndims);
    const uint64_t run = t / ndims;
    const uint32_t first = static_cast<uint32_t>(k0 + run * kRun);
    uint32_t y = sobol_first(tab, jstride, j, __ldg(shf + j), first);
    for (int s = 0; s < kRun; ++s) {
        const uint64_t idx = run * kRun + s;
        if (idx >= count) break;
        if (s) y ^= __ldg(tab + (__ffs(first + s) - 1) * jstride + j);
        out[idx * ndims + j] = y;
    }
}

}  // namespace

size_t fused_smem_bytes(int precision, int n, int tile_log2) {
    const size_t elem = (precision == QMCCPW_FP64) ? 8 : 4;
    const int stride = (n + 1) | 1;
    const size_t zw = static_cast<size_t>(1u << tile_log2) * stride * elem;
    // staging of partial accumulators: up to 4 * kThreads (slot, point) entries of (x, dsum, m)
    const size_t red = 4 * kThreads * (2 * elem + sizeof(int32_t));
    return ((zw > red ? zw : red) + 15) & ~size_t(15);
}

template <typename T>
static cudaError_t set_limit_all(int bytes) {
    cudaError_t e = cudaFuncSetAttribute(fused_kernel<T, QMCCPW_BB>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(fused_kernel<T, QMCCPW_PCA>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

int fused_set_smem_limit(int precision, size_t bytes) {
    const int b = static_cast<int>(bytes);
    return static_cast<int>(precision == QMCCPW_FP64 ? set_limit_all<double>(b) : set_limit_all<float>(b));
}

int fused_occupancy(int precision, int construction, size_t smem_bytes, int *blocks_per_sm) {
    cudaError_t e;
    if (precision == QMCCPW_FP64)
        e = construction == QMCCPW_BB
                ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fused_kernel<double, QMCCPW_BB>, kThreads, smem_bytes)
                : cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fused_kernel<double, QMCCPW_PCA>, kThreads, smem_bytes);
    else
        e = construction == QMCCPW_BB
                ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fused_kernel<float, QMCCPW_BB>, kThreads, smem_bytes)
                : cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fused_kernel<float, QMCCPW_PCA>, kThreads, smem_bytes);
    return static_cast<int>(e);
}

int launch_fused(const LaunchParams &p, int precision, int construction, size_t smem_bytes, int grid, void *stream) {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (precision == QMCCPW_FP64) {
        if (construction == QMCCPW_BB) fused_kernel<double, QMCCPW_BB><<<grid, kThreads, smem_bytes, s>>>(p);
        else fused_kernel<double, QMCCPW_PCA><<<grid, kThreads, smem_bytes, s>>>(p);
    } else {
        if (construction == QMCCPW_BB) fused_kernel<float, QMCCPW_BB><<<grid, kThreads, smem_bytes, s>>>(p);
        else fused_kernel<float, QMCCPW_PCA><<<grid, kThreads, smem_bytes, s>>>(p);
    }
    return static_cast<int>(cudaGetLastError());
}

int launch_reduce(const ContractDev *contracts, int32_t count, const double *tile_sums, double *per_rep,
                  double *stats, uint64_t total_reps, const uint64_t *rep_owner, void *stream) {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    reduce_kernel<<<static_cast<unsigned>(total_reps), 256, 0, s>>>(contracts, rep_owner, tile_sums, per_rep);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return static_cast<int>(e);
    stats_kernel<<<(count * 4 + 127) / 128, 128, 0, s>>>(contracts, count, per_rep, stats);
    return static_cast<int>(cudaGetLastError());
}

int launch_scramble(uint64_t seed, const uint32_t *v, int ndims, int jstride, int reps, uint32_t *table,
                    uint32_t *shift, void *stream) {
    const int total = ndims * reps;
    scramble_kernel<<<(total + 127) / 128, 128, 0, static_cast<cudaStream_t>(stream)>>>(seed, v, ndims, jstride,
                                                                                         reps, table, shift);
    return static_cast<int>(cudaGetLastError());
}

int launch_sobol_dump(const uint32_t *table, const uint32_t *shift, int jstride, int ndims, uint64_t k0,
                      uint64_t count, uint32_t *out, void *stream) {
    const uint64_t runs = (count + 15) / 16;
    const uint64_t total = runs * static_cast<uint64_t>(ndims);
    sobol_dump_kernel<<<static_cast<unsigned>((total + 127) / 128), 128, 0, static_cast<cudaStream_t>(stream)>>>(
        table, shift, jstride, ndims, k0, count, out);
    return static_cast<int>(cudaGetLastError());
}

}  // namespace qmccpw
