// Basket of m correlated GBM assets (Sec. 6: options on several underlying
// assets, the path simulation and the payoff formulas redefined).
//
// One CTA processes one work item = (replicate, tile of P points):
//   1. Sobol' + inverse normal (as the single-asset kernel): dimension
//      b*m + k drives bridge node b of factor k, dimension n*m + k-1 the first
//      increment x_k of factor k >= 1; z lands in the point's row at the slot
//      of the date its node fills, factor-interleaved: slot 1 + (t-1)*m + k
//      holds factor k at date index t (t = 1..n), slot 0 is the zero of
//      W~(s_0), slot 1 + n*m + k-1 the first increment x_k.
//   2. Each factor's bridge (Sec. 4.4, unit spacing), level by level in
//      place; the (node, factor) pairs of a level are spread over the G
//      threads of a point.
//   3. Per asset i and date j the unit-spacing combination
//      u_i(j) = sum_k L_ik (w~_k(j-1) + [k >= 1] x_k), the exponential
//      e = exp((sigma_i sqrt(dt)) u + (omega_i dt) j) and the sums
//      X_i = sum_j e, Yw_i = sum_j e u, Yn_i = sum_j e j (the G threads of a
//      point take alternate dates), merged per point in a fixed order.
//   4. Per point: C_i = f_i X_i, D_i = f_i (sqrt(dt) Yw_i - sigma_i dt Yn_i)
//      (f_i = w_i a_i S0 / d), the switch point x* of sum_i C_i e^{b_i x} = K
//      by Newton's method on ln X - ln K, price and Greeks in closed form, in
//      double; then the tile sum into the item's slot.
// FP64: every step in double.  MIXED: steps 1-3 in float (the library's own
// inverse normal and exponential, the factor L and the per-asset constants as
// float pairs, the sums in float), step 4 in double.
#include <cuda_runtime.h>

#include <cstdint>

#include "qmccpw_device.cuh"
#include "qmccpw_internal.h"

namespace qmccpw {
namespace {

constexpr int kMaxM = QMCCPW_ASSETS_MAX;

// slot of factor k's value at date index t (t = 0: the zero slot)
__device__ __forceinline__ int bslot(int m, int t, int k) { return t == 0 ? 0 : 1 + (t - 1) * m + k; }

// ---- phase 1 -------------------------------------------------------------------
template <typename T>
__device__ void basket_sobol(const BasketParams &p, uint32_t rep, uint64_t tile, T *zw) {
    const BasketDev &b = p.b;
    const int P = 1 << b.tile_log2;
    const int nd = b.m * b.d - 1;
    const int stride = b.row_stride;
    const uint32_t *tab = p.sobol_table + static_cast<size_t>(rep) * 32u * p.jstride;
    const uint32_t *shf = p.sobol_shift + static_cast<size_t>(rep) * p.jstride;
    const int chunk = 1 << b.chunk_log2;
    const int nchunks = P >> b.chunk_log2;
    const bool by_warp = nd >= 32;
    const int step = by_warp ? kThreads / 32 : kThreads;
    const int first = by_warp ? (threadIdx.x >> 5) : threadIdx.x;
    const int work = by_warp ? nchunks * ((nd + 31) >> 5) : nchunks * nd;
    for (int it = first; it < work; it += step) {
        int j, ch;
        if (by_warp) {
            const int per = (nd + 31) >> 5;
            ch = it / per;
            j = (it - ch * per) * 32 + (threadIdx.x & 31);
            if (j >= nd) continue;
        } else {
            j = it % nd;
            ch = it / nd;
        }
        T *dst = zw + static_cast<size_t>(ch * chunk) * stride + __ldg(b.slot_of_dim + j);
        const uint64_t first_local = tile * P + static_cast<uint64_t>(ch) * chunk;
        const int len = first_local >= b.N ? 0 : static_cast<int>(min(static_cast<uint64_t>(chunk), b.N - first_local));
        if (len > 0) {
            const uint32_t k0 = static_cast<uint32_t>(p.point_k0 + first_local);
            const uint32_t y0 = sobol_first(tab, p.jstride, j, __ldg(shf + j), k0);
            if constexpr (sizeof(T) == 4) {
                sobol_point_deferred(
                    tab, p.jstride, j, y0, k0, len, b.chunk_log2,
                    [&](int s, uint32_t y) { dst[s * stride] = Arith<float>::inv_normal(y); },
                    [&](int s, float2 z) {
                        dst[s * stride] = z.x;
                        dst[(s + 1) * stride] = z.y;
                    });
            } else {
                sobol_points(tab, p.jstride, j, y0, k0, len, b.chunk_log2,
                             [&](int s, uint32_t y) { dst[s * stride] = Arith<double>::inv_normal(y); });
            }
        }
        for (int s = len; s < chunk; ++s) dst[s * stride] = T(0);
    }
    for (int pt = threadIdx.x; pt < P; pt += kThreads) zw[pt * stride] = T(0);
}

// ---- phase 2: the m bridges, unit spacing, in place ----------------------------
template <typename T>
__device__ void basket_bridges(const BasketDev &b, T *zw) {
    const int P = 1 << b.tile_log2, G = b.groups, m = b.m;
    T *row = zw + (threadIdx.x & (P - 1)) * b.row_stride;
    const int g = threadIdx.x >> b.tile_log2;
    for (int lvl = 0; lvl < b.n_levels; ++lvl) {
        const int b0 = __ldg(b.level_start + lvl), b1 = __ldg(b.level_start + lvl + 1);
        const int items = (b1 - b0) * m;
        for (int it = g; it < items; it += G) {
            const int node = b0 + it / m, k = it - (it / m) * m;
            const int4 st = __ldg(reinterpret_cast<const int4 *>(b.steps) + node);
            const int sm = bslot(m, st.x, k);
            const T Wl = row[bslot(m, st.y, k)], Wr = row[bslot(m, st.z, k)], z = row[sm];
            if constexpr (sizeof(T) == 8) {
                const double *w = b.w64 + 3 * node;
                row[sm] = __ldg(w) * Wl + __ldg(w + 1) * Wr + __ldg(w + 2) * z;
            } else {
                const float4 h = __ldg(reinterpret_cast<const float4 *>(b.w32) + 2 * node);
                const float4 q = __ldg(reinterpret_cast<const float4 *>(b.w32) + 2 * node + 1);
                float lo = h.y * Wl;
                lo = fmaf(h.w, Wr, lo);
                lo = fmaf(q.y, z, lo);
                row[sm] = fmaf(h.x, Wl, fmaf(h.z, Wr, fmaf(q.x, z, lo)));
            }
        }
        if (G > 1) __syncthreads();
    }
}

// ---- phase 3: per-asset sums over this thread's dates --------------------------
// FP64 form.
template <int M>
__device__ void basket_sums(const BasketDev &b, const double *row, int g, double (&X)[M], double (&Yw)[M],
                            double (&Yn)[M]) {
    const int n = b.n;
    double F[M];
#pragma unroll
    for (int i = 0; i < M; ++i) {
        double s = 0.0;
#pragma unroll
        for (int k = 1; k <= i; ++k) s += b.L[i * kMaxM + k] * row[1 + n * M + k - 1];
        F[i] = s;
        X[i] = Yw[i] = Yn[i] = 0.0;
    }
    for (int j = 1 + g; j <= b.d; j += b.groups) {
        double w[M];
#pragma unroll
        for (int k = 0; k < M; ++k) w[k] = j == 1 ? 0.0 : row[1 + (j - 2) * M + k];
        const double jf = static_cast<double>(j);
#pragma unroll
        for (int i = 0; i < M; ++i) {
            double u = F[i];
#pragma unroll
            for (int k = 0; k <= i; ++k) u += b.L[i * kMaxM + k] * w[k];
            const double e = exp(b.sig_sdt[i] * u + b.om_dt[i] * jf);
            X[i] += e;
            Yw[i] += e * u;
            Yn[i] += e * jf;
        }
    }
}

// Float form: the constants as pairs (hi + lo: a float sigma, omega, or
// factor entry would perturb every path the same way), the small terms first.
template <int M>
__device__ void basket_sums(const BasketDev &b, const float *row, int g, float (&X)[M], float (&Yw)[M],
                            float (&Yn)[M]) {
    const int n = b.n;
    float F[M];
#pragma unroll
    for (int i = 0; i < M; ++i) {
        float lo = 0.0f, hi = 0.0f;
#pragma unroll
        for (int k = 1; k <= i; ++k) {
            const float x = row[1 + n * M + k - 1];
            lo = fmaf(b.Lf[i * kMaxM + k][1], x, lo);
            hi = fmaf(b.Lf[i * kMaxM + k][0], x, hi);
        }
        F[i] = hi + lo;
        X[i] = Yw[i] = Yn[i] = 0.0f;
    }
    for (int j = 1 + g; j <= b.d; j += b.groups) {
        float w[M];
#pragma unroll
        for (int k = 0; k < M; ++k) w[k] = j == 1 ? 0.0f : row[1 + (j - 2) * M + k];
        const float jf = small_uint_to_float(static_cast<uint32_t>(j));
#pragma unroll
        for (int i = 0; i < M; ++i) {
            float lo = 0.0f, hi = F[i];
#pragma unroll
            for (int k = 0; k <= i; ++k) {
                lo = fmaf(b.Lf[i * kMaxM + k][1], w[k], lo);
                hi = fmaf(b.Lf[i * kMaxM + k][0], w[k], hi);
            }
            const float u = hi + lo;
            const float x = fmaf(u, b.ff_sig_sdt[i][0],
                                 fmaf(jf, b.ff_om_dt[i][0], fmaf(u, b.ff_sig_sdt[i][1], jf * b.ff_om_dt[i][1])));
            const float e = fx::exp_f(x);
            X[i] += e;
            Yw[i] = fmaf(e, u, Yw[i]);
            Yn[i] = fmaf(e, jf, Yn[i]);
        }
    }
}

// ---- phase 4: the values of one point from its per-asset sums (double) ---------
__device__ __forceinline__ double sf(double x) { return 0.5 * erfc(x * 0.70710678118654752440); }

__device__ void basket_point_values(const BasketDev &b, const double *C, const double *D, double v[4]) {
    const int m = b.m;
    // Newton on ln X(x) - ln K from x = 0: convex and increasing, so after the
    // first step the iterates approach the root from the right, monotonically
    double x = 0.0, last = 1e300;
    for (int it = 0; it < 100; ++it) {
        double s0 = 0.0, s1 = 0.0;
        for (int i = 0; i < m; ++i) {
            const double e = C[i] * exp(b.bcoef[i] * x);
            s0 += e;
            s1 += b.bcoef[i] * e;
        }
        const double step = (log(s0) - b.ln_K) * (s0 / s1);
        x -= step;
        const double mag = fabs(step);
        if (mag <= 1e-15 * (1.0 + fabs(x)) || (it >= 2 && mag >= last)) break;
        last = mag;
    }
    const double pdf = 0.39894228040143267794 * exp(-0.5 * x * x);
    double F0 = 0.0, X1 = 0.0, X2 = 0.0, V = 0.0, B = 0.0;
    for (int i = 0; i < m; ++i) {
        const double bi = b.bcoef[i], ebx = exp(bi * x), e = C[i] * ebx;
        X1 += bi * e;
        X2 += bi * bi * e;
        if (b.type == QMCCPW_ARITH_ASIAN_CALL) {
            // C_i e^{b^2/2} phi(x - b) = phi(x) C_i e^{b x}
            const double sfb = sf(x - bi), eh = C[i] * b.ehalf[i];
            F0 += eh * sfb;
            V += b.v[i] * (b.ehalf[i] * sfb * (D[i] + C[i] * b.l1[i] * bi) + b.l1[i] * pdf * e);
        } else {
            B += b.v[i] * ebx * (D[i] + C[i] * b.l1[i] * x);
        }
    }
    const double K = b.K, S0 = b.S0, disc = b.disc;
    if (b.type == QMCCPW_ARITH_ASIAN_CALL) {
        v[0] = disc * (F0 - K * sf(x));
        v[1] = disc * F0 / S0;
        v[2] = disc * V;
        v[3] = disc * K * K * pdf / (S0 * S0 * X1);
    } else {
        v[0] = disc * sf(x);
        v[1] = disc * pdf * K / (S0 * X1);
        v[2] = disc * pdf * B / X1;
        v[3] = disc * K * pdf * (x * K - 2.0 * X1 + K * X2 / X1) / ((S0 * X1) * (S0 * X1));
    }
}

template <typename T, int M>
__device__ void basket_item_m(const BasketParams &p, uint64_t tile, T *zw, double v[4]) {
    const BasketDev &b = p.b;
    const int P = 1 << b.tile_log2;
    const int pt = threadIdx.x & (P - 1), g = threadIdx.x >> b.tile_log2, G = b.groups;
    T X[M], Yw[M], Yn[M];
    basket_sums<M>(b, zw + pt * b.row_stride, g, X, Yw, Yn);
    __syncthreads();  // the rows are read; their space takes the partial sums
    T *part = zw + (static_cast<size_t>(g) * P + pt) * (3 * M);
#pragma unroll
    for (int i = 0; i < M; ++i) {
        part[3 * i] = X[i];
        part[3 * i + 1] = Yw[i];
        part[3 * i + 2] = Yn[i];
    }
    __syncthreads();
    for (int q = 0; q < 4; ++q) v[q] = 0.0;
    const uint64_t local = tile * P + pt;
    if (threadIdx.x < P && local < b.N) {
        double C[M], D[M];
#pragma unroll
        for (int i = 0; i < M; ++i) {
            double x = 0.0, yw = 0.0, yn = 0.0;
            for (int h = 0; h < G; ++h) {  // the G threads' partial sums in thread order
                const T *o = zw + (static_cast<size_t>(h) * P + pt) * (3 * M) + 3 * i;
                x += static_cast<double>(o[0]);
                yw += static_cast<double>(o[1]);
                yn += static_cast<double>(o[2]);
            }
            C[i] = b.f[i] * x;
            D[i] = b.f[i] * (b.sqrt_dt * yw - b.sig_dt[i] * yn);
        }
        basket_point_values(b, C, D, v);
        if (p.point_out)
            for (int q = 0; q < 4; ++q) p.point_out[local * 4 + q] = v[q];
    }
}

template <typename T>
__global__ void __launch_bounds__(kThreads, 2) basket_kernel(const __grid_constant__ BasketParams p) {
    extern __shared__ __align__(16) unsigned char smem[];
    T *zw = reinterpret_cast<T *>(smem);
    const BasketDev &b = p.b;
    for (uint64_t item = blockIdx.x; item < p.items; item += gridDim.x) {
        const uint64_t rep_local = item / b.tiles;
        const uint64_t tile = item - rep_local * b.tiles;
        const uint32_t rep = static_cast<uint32_t>(rep_local) + p.rep_offset;
        basket_sobol<T>(p, rep, tile, zw);
        __syncthreads();
        basket_bridges<T>(b, zw);
        __syncthreads();
        double v[4];
        switch (b.m) {
            case 1: basket_item_m<T, 1>(p, tile, zw, v); break;
            case 2: basket_item_m<T, 2>(p, tile, zw, v); break;
            case 3: basket_item_m<T, 3>(p, tile, zw, v); break;
            case 4: basket_item_m<T, 4>(p, tile, zw, v); break;
            case 5: basket_item_m<T, 5>(p, tile, zw, v); break;
            case 6: basket_item_m<T, 6>(p, tile, zw, v); break;
            case 7: basket_item_m<T, 7>(p, tile, zw, v); break;
            default: basket_item_m<T, 8>(p, tile, zw, v); break;
        }
        tile_sum(p.tile_sums + item * 4, v, smem);  // ends with a barrier: the tile is free again
    }
}

}  // namespace

int launch_basket(const BasketParams &p, int precision, size_t smem_bytes, int grid, void *stream) {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (precision == QMCCPW_FP64) basket_kernel<double><<<grid, kThreads, smem_bytes, s>>>(p);
    else basket_kernel<float><<<grid, kThreads, smem_bytes, s>>>(p);
    return static_cast<int>(cudaGetLastError());
}

int basket_prepare(size_t optin_bytes) {
    cudaError_t e = cudaFuncSetAttribute(basket_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(optin_bytes));
    if (e != cudaSuccess) return static_cast<int>(e);
    return static_cast<int>(cudaFuncSetAttribute(basket_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 static_cast<int>(optin_bytes)));
}

int basket_occupancy(int precision, size_t smem_bytes, int *blocks_per_sm) {
    const void *f = precision == QMCCPW_FP64 ? reinterpret_cast<const void *>(basket_kernel<double>)
                                              : reinterpret_cast<const void *>(basket_kernel<float>);
    return static_cast<int>(cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, f, kThreads, smem_bytes));
}

}  // namespace qmccpw
