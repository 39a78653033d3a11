// Device code of one work item of the fused QMC-CPW pipeline, shared by the
// one-launch-per-batch kernel (kernels.cu) and the persistent serving kernel
// (serve.cu), and the per-replicate reduction both use.
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
//      psi = (ln(K/S0) - omega t_1 - ln X^)/a, then price, delta, vega,
//      gamma; a warp-shuffle + shared-memory tree sums the tile into 4
//      doubles, added (compensated, in tile order) to the work item's total,
//      which goes to the item's slot after its last tile (no atomics, so the
//      result does not depend on scheduling).
// The replicate estimate is the compensated (Neumaier) sum of its item
// slots in a fixed order, divided by N (reduce_replicate); mean and standard
// error over replicates follow (replicate_stats).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "qmccpw_device.cuh"
#include "qmccpw_internal.h"

namespace qmccpw {
namespace {

// ---------------------------------------------------------------------------
// path phases
// ---------------------------------------------------------------------------
// small non-negative int as T (float: without a conversion instruction)
template <typename T> __device__ __forceinline__ T small_int_to(int i);
template <> __device__ __forceinline__ double small_int_to<double>(int i) { return static_cast<double>(i); }

// The contract fields a bridge node reads, copied to registers once per
// phase (a store to the row could otherwise make the compiler read them again
// from the contract in global memory at every node).
struct BridgeTables {
    const int4 *steps;
    const double *w64;
    const float4 *w32;
    double sqrt_t1;
    float sdt_hi, sdt_lo;
    __device__ explicit BridgeTables(const ContractDev &c)
        : steps(reinterpret_cast<const int4 *>(c.steps)), w64(c.w64), w32(reinterpret_cast<const float4 *>(c.w32)),
          sqrt_t1(c.sqrt_t1), sdt_hi(c.ff_sqrt_t1[0]), sdt_lo(c.ff_sqrt_t1[1]) {}
};

// Node b of a bridge schedule in a point's row: W~ at its date from its
// endpoints and z (unit-spacing weights, z scaled by sqrt(dt)), written in
// place of z.
// Float: SCALED gives W~ (z scaled by sqrt(dt)); otherwise the path of unit
// spacing w = W~ / sqrt(dt) that the float accumulator takes.
template <typename T, bool SCALED = true>
__device__ __forceinline__ T bridge_node(const BridgeTables &t, T *row, int b, int4 &st) {
    st = __ldg(t.steps + b);
    const T Wl = row[st.y], Wr = row[st.z];
    T z = row[st.x];
    T Wm;
    if constexpr (sizeof(T) == 8) {
        const double *w = t.w64 + 3 * b;
        Wm = __ldg(w) * Wl + __ldg(w + 1) * Wr + __ldg(w + 2) * (t.sqrt_t1 * z);
    } else {
        if constexpr (SCALED) z = fmaf(z, t.sdt_hi, z * t.sdt_lo);  // z sqrt(dt): the tables hold unit-spacing weights
        // hi + lo coefficients: the low parts first, then the high parts
        const float4 h = __ldg(t.w32 + 2 * b);
        const float4 g = __ldg(t.w32 + 2 * b + 1);
        float lo = h.y * Wl;
        lo = fmaf(h.w, Wr, lo);
        lo = fmaf(g.y, z, lo);
        Wm = fmaf(h.x, Wl, fmaf(h.z, Wr, fmaf(g.x, z, lo)));
    }
    row[st.x] = Wm;
    return Wm;
}

// The whole bridge of the leading-coordinate construction, levels breadth
// first, W~ left in the rows (no running sums: the values need the whole
// path first).
template <typename T>
__device__ void bridge_store(const ContractDev &c, T *zw, int stride) {
    const int P = 1 << c.tile_log2;
    T *row = zw + (threadIdx.x & (P - 1)) * stride;
    const int grp = threadIdx.x >> c.tile_log2;
    const BridgeTables t(c);
    const int32_t *level_start = c.level_start;
    const int n_levels = c.n_levels, G = c.groups;
    for (int lvl = 0; lvl < n_levels; ++lvl) {
        const int b_end = __ldg(level_start + lvl + 1);
        for (int b = __ldg(level_start + lvl) + grp; b < b_end; b += G) {
            int4 st;
            bridge_node<T>(t, row, b, st);
        }
        if (G > 1) __syncthreads();
    }
}

// The rest of the PCA path of the leading-coordinate construction: R_i =
// sqrt(dt) sum_k Ahat[i][k] z_k over the d components (z_1 = 0 in slot 1),
// into the second row.  FP64: the G threads of a point take every G-th date.
// Float: they take blocks of 8 consecutive dates, each k step reading the
// block's 8 entries of row k of A^T (hi and lo parts) as float4 pairs; the
// factor is carried as hi + lo because its float rounding would be one fixed
// perturbation of the covariance of the rest, which the conditioning on the
// leading component makes the dominant error.  Each date's sum runs over k
// in order.
template <typename T>
__device__ void lead_pca_store(const ContractDev &c, const T *zw, T *rbuf, int stride) {
    const int P = 1 << c.tile_log2;
    const int pt = threadIdx.x & (P - 1);
    const int grp = threadIdx.x >> c.tile_log2;
    const int G = c.groups;
    const int nd = c.d;  // whole-path dimension
    const T *row = zw + pt * stride;
    T *out = rbuf + pt * stride;
    if constexpr (sizeof(T) == 8) {
        for (int i = 1 + grp; i <= nd; i += G) {
            T w = T(0);
            const double *Ai = c.pca64 + static_cast<size_t>(i - 1) * nd;
            for (int k = 2; k <= nd; ++k) w = fma(__ldg(Ai + k - 1), row[k], w);
            out[i] = w * c.sqrt_t1;
        }
    } else {
        const int n_pad = (nd + 15) & ~15;  // A^T rows padded with zeros to a multiple of 16
        const float4 *AT = reinterpret_cast<const float4 *>(c.pcaT32);
        const float4 *ATlo = reinterpret_cast<const float4 *>(c.pcaT32lo);
        const float sh = c.ff_sqrt_t1[0], sl = c.ff_sqrt_t1[1];
        for (int blk = grp; 8 * blk < nd; blk += G) {
            float w[8], wl[8];
#pragma unroll
            for (int r = 0; r < 8; ++r) w[r] = wl[r] = 0.0f;
            const size_t first = static_cast<size_t>(n_pad / 4) + 2 * blk;  // row k = 2 (index 1)
            const float4 *a = AT + first, *al = ATlo + first;
            for (int k = 2; k <= nd; ++k, a += n_pad / 4, al += n_pad / 4) {
                const float z = row[k];
                const float4 a0 = __ldg(a), a1 = __ldg(a + 1);
                const float4 l0 = __ldg(al), l1 = __ldg(al + 1);
                w[0] = fmaf(a0.x, z, w[0]);
                w[1] = fmaf(a0.y, z, w[1]);
                w[2] = fmaf(a0.z, z, w[2]);
                w[3] = fmaf(a0.w, z, w[3]);
                w[4] = fmaf(a1.x, z, w[4]);
                w[5] = fmaf(a1.y, z, w[5]);
                w[6] = fmaf(a1.z, z, w[6]);
                w[7] = fmaf(a1.w, z, w[7]);
                wl[0] = fmaf(l0.x, z, wl[0]);
                wl[1] = fmaf(l0.y, z, wl[1]);
                wl[2] = fmaf(l0.z, z, wl[2]);
                wl[3] = fmaf(l0.w, z, wl[3]);
                wl[4] = fmaf(l1.x, z, wl[4]);
                wl[5] = fmaf(l1.y, z, wl[5]);
                wl[6] = fmaf(l1.z, z, wl[6]);
                wl[7] = fmaf(l1.w, z, wl[7]);
            }
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                const int i = 8 * blk + r + 1;
                // (w + wl) (sh + sl), the small products first
                if (i <= nd) out[i] = fmaf(w[r], sh, fmaf(wl[r], sh, w[r] * sl));
            }
        }
    }
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
    const BridgeTables t(c);
    const int32_t *level_start = c.level_start;
    const int n_levels = c.n_levels;
    // nodes b and b + stride of one level (both independent): float takes
    // their exponentials in packed form
    // the float path's constants in registers once per phase (read from the
    // contract inside the loop, the stores to the row would make the
    // compiler load them again at every node)
    const PathConst kc = sizeof(T) == 4 ? PathConst(c) : PathConst();
    auto two_nodes = [&](int b, bool second, int stride) {
        int4 s0, s1;
        if constexpr (sizeof(T) == 4) {
            // the steps carry float(date) in their last field
            const float w0 = bridge_node<float, false>(t, row, b, s0);
            if (second) {
                const float w1 = bridge_node<float, false>(t, row, b + stride, s1);
                acc.template add2<TYPE>(s0.x, s1.x, w0, w1, kc, __int_as_float(s0.w), __int_as_float(s1.w));
            } else {
                acc.template add<TYPE>(s0.x, w0, kc);
            }
        } else {
            double omega, sigma, dt;
            market_of(c, omega, sigma, dt);
            const T W0 = bridge_node<T>(t, row, b, s0);
            acc.template add<TYPE>(s0.x, W0, omega, sigma, static_cast<T>(__int_as_float(s0.w)) * dt);
            if (second) {
                const T W1 = bridge_node<T>(t, row, b + stride, s1);
                acc.template add<TYPE>(s1.x, W1, omega, sigma, static_cast<T>(__int_as_float(s1.w)) * dt);
            }
        }
    };
    // With G threads per point and the subtree table: the top levels (up to
    // the one that leaves G intervals) level by level with a barrier after
    // each, then each thread its own interval's subtree, level by level and
    // without barriers (a subtree reads only its own nodes and its ends).
    const int top = (G > 1 && c.sub_start) ? min(n_levels, __ffs(G)) : n_levels;
    for (int lvl = 0; lvl < top; ++lvl) {
        const int b_end = __ldg(level_start + lvl + 1);
        for (int b = __ldg(level_start + lvl) + grp; b < b_end; b += 2 * G) two_nodes(b, b + G < b_end, G);
        if (G > 1) __syncthreads();
    }
    if (top < n_levels) {
        const int32_t *ss = c.sub_start + grp;
        for (int lvl = top; lvl < n_levels; ++lvl, ss += G + 1) {
            const int b_end = __ldg(ss + 1);
            for (int b = __ldg(ss); b < b_end; b += 2) two_nodes(b, b + 1 < b_end, 1);
        }
    }
}

// Bridge with a compile-time schedule (n = N dates after t_1) and W~ in
// registers: the breadth-first order, the endpoints and the weights are
// constants, so each node is one shared-memory load of z and four flops.
// Used by the float path when one thread owns one point (P = 256).
struct BridgeSchedule {
    static constexpr int kMax = 128;
    int m[kMax], l[kMax], r[kMax];
    double wr[kMax], c[kMax];  // W_m = W_l + wr (W_r - W_l) + c sqrt(dt) z
    int count;
};

__host__ __device__ constexpr double cx_sqrt(double v) {  // Newton's method, for compile-time constants only
    if (v <= 0.0) return 0.0;
    double x = v > 1.0 ? v : 1.0;
    for (int i = 0; i < 64; ++i) x = 0.5 * (x + v / x);
    return x;
}

__host__ __device__ constexpr BridgeSchedule make_schedule(int n) {
    BridgeSchedule s{};
    int ql[2 * BridgeSchedule::kMax + 2] = {}, qr[2 * BridgeSchedule::kMax + 2] = {};
    int head = 0, tail = 0, k = 0;
    s.m[k] = n; s.l[k] = 0; s.r[k] = 0; s.wr[k] = 0.0; s.c[k] = cx_sqrt(static_cast<double>(n)); ++k;
    ql[tail] = 0; qr[tail] = n; ++tail;
    while (head < tail) {
        const int a = ql[head], b = qr[head];
        ++head;
        if (b - a < 2) continue;
        const int mm = (a + b) / 2;
        s.m[k] = mm; s.l[k] = a; s.r[k] = b;
        s.wr[k] = static_cast<double>(mm - a) / (b - a);
        s.c[k] = cx_sqrt(static_cast<double>(mm - a) * (b - mm) / (b - a));
        ++k;
        ql[tail] = a; qr[tail] = mm; ++tail;
        ql[tail] = mm; qr[tail] = b; ++tail;
    }
    s.count = k;
    return s;
}

template <int N, int TYPE>
__device__ __forceinline__ void bridge_registers(const ContractDev &c, const float *row, PathAcc<float> &acc) {
    constexpr BridgeSchedule S = make_schedule(N);
    static_assert(S.count == N, "bridge schedule size");
    const PathConst k(c);
    float W[N + 1];  // the path of unit spacing
    W[0] = 0.0f;
    auto node = [&](int b) {
        const float z = row[b + 1];  // z of dimension b (stored by dimension)
        const float Wl = W[S.l[b]], Wr = W[S.r[b]];
        const float Wm = fmaf(static_cast<float>(S.c[b]), z, fmaf(static_cast<float>(S.wr[b]), Wr - Wl, Wl));
        W[S.m[b]] = Wm;
        return Wm;
    };
    // nodes in schedule order, their exponentials two at a time
#pragma unroll
    for (int b = 0; b + 1 < N; b += 2) {
        const float W0 = node(b), W1 = node(b + 1);
        acc.template add2<TYPE>(S.m[b], S.m[b + 1], W0, W1, k);
    }
    if constexpr (N % 2 == 1) {
        const float W0 = node(N - 1);
        acc.template add<TYPE>(S.m[N - 1], W0, k);
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
    const int n = c.n;
    if constexpr (sizeof(T) == 8) {
        double omega, sigma, dt;
        market_of(c, omega, sigma, dt);
        double s_i = static_cast<double>(1 + grp) * dt;
        const double ds = static_cast<double>(c.groups) * dt;
        for (int i = 1 + grp; i <= n; i += c.groups, s_i += ds) {
            T Wi = T(0);
            const double *Ai = c.pca64 + static_cast<size_t>(i - 1) * n;
            for (int k = 0; k < n; ++k) Wi += __ldg(Ai + k) * row[k + 1];
            Wi *= c.sqrt_t1;
            acc.template add<TYPE>(i, Wi, omega, sigma, s_i);
        }
    } else {
        const PathConst kc(c);
        const int n_pad = (n + 15) & ~15;
        for (int i = 1 + grp; i <= n; i += c.groups) {
            float w = 0.0f;  // unit spacing
            for (int k = 0; k < n; ++k) w = fmaf(__ldg(c.pcaT32 + static_cast<size_t>(k) * n_pad + (i - 1)), row[k + 1], w);
            acc.template add<TYPE>(i, w, kc);
        }
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
    const PathConst kc(c);
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
        for (int r = 0; r < 16; r += 2) {  // dates i, i + 1 (unit-spacing path): exponentials in packed form
            const int i = rb * 16 + r + 1;
            if (i + 1 <= n) {
#pragma unroll
                for (int j = 0; j < PB; ++j) acc[j].template add2<TYPE>(i, i + 1, w[j][r], w[j][r + 1], kc);
            } else if (i <= n) {
#pragma unroll
                for (int j = 0; j < PB; ++j) acc[j].template add<TYPE>(i, w[j][r], kc);
            }
        }
    }
}

// Standard construction: W~(s_i) = sqrt(dt) (z_1 + ... + z_i).  The G
// threads of a point split its dates into G contiguous blocks: each sums its
// block's z, the sums of the earlier blocks (through shared memory, added in
// block order) give its starting value, and it walks its block again adding
// every date to its accumulator.

__shared__ double forward_block_sums[kThreads];  // one per thread, shared by the product types' instances

template <typename T, int TYPE>
__device__ void forward_phase(const ContractDev &c, const T *zw, int stride, PathAcc<T> &acc) {
    T *block_sum = reinterpret_cast<T *>(forward_block_sums);
    const int P = 1 << c.tile_log2;
    const int pt = threadIdx.x & (P - 1);
    const int g = threadIdx.x >> c.tile_log2;
    const int n = c.n;
    const int per = (n + c.groups - 1) / c.groups;
    const int i0 = 1 + g * per, i1 = min(n, (g + 1) * per);  // this thread's dates (may be none)
    const T *row = zw + pt * stride;                          // row[i] = z of dimension i - 1
    T w = T(0);
    if (c.groups > 1) {
        for (int i = i0; i <= i1; ++i) w += row[i];
        block_sum[threadIdx.x] = w;
        __syncthreads();
        w = T(0);
        for (int h = 0; h < g; ++h) w += block_sum[h * P + pt];
    }
    if constexpr (sizeof(T) == 8) {
        double omega, sigma, dt;
        market_of(c, omega, sigma, dt);
        for (int i = i0; i <= i1; ++i) {
            w += row[i];
            acc.template add<TYPE>(i, w * c.sqrt_t1, omega, sigma, small_int_to<T>(i) * dt);
        }
    } else {
        const PathConst kc(c);
        int i = i0;
        for (; i + 1 <= i1; i += 2) {  // two dates at a time (unit spacing): exponentials in packed form
            const float w0 = w + row[i];
            w = w0 + row[i + 1];
            acc.template add2<TYPE>(i, i + 1, w0, w, kc);
        }
        if (i <= i1) {
            w += row[i];
            acc.template add<TYPE>(i, w, kc);
        }
    }
}

// Phase 2 for one product type: returns, for threads t < P, the merged
// accumulator of point t in `acc` (other threads' acc is unspecified).
template <typename T, int CONS, int TYPE>
__device__ void path_phase(const ContractDev &c, T *zw, int stride, PathAcc<T> &acc) {
    const int P = 1 << c.tile_log2;
    if constexpr (CONS == QMCCPW_BB) {
        acc.init(TYPE, threadIdx.x < P);
        if constexpr (sizeof(T) == 4) {
            if (c.z_by_dim) {  // set exactly when the register bridge applies
                const float *row = zw + threadIdx.x * stride;
                if (c.n == 63) bridge_registers<63, TYPE>(c, row, acc);
                else bridge_registers<15, TYPE>(c, row, acc);
                return;
            }
        }
        bridge_phase<T, TYPE>(c, zw, stride, acc);
        if (c.groups == 1) return;
        __syncthreads();
        stage_partial(zw, P, threadIdx.x >> c.tile_log2, threadIdx.x & (P - 1), acc);
        __syncthreads();
        if (threadIdx.x < P) merge_partials(zw, P, c.groups, threadIdx.x, TYPE, acc);
        return;
    } else if constexpr (CONS == QMCCPW_STD) {
        acc.init(TYPE, threadIdx.x < P);
        forward_phase<T, TYPE>(c, zw, stride, acc);
        if (c.groups == 1) return;
        __syncthreads();
        stage_partial(zw, P, threadIdx.x >> c.tile_log2, threadIdx.x & (P - 1), acc);
        __syncthreads();
        if (threadIdx.x < P) merge_partials(zw, P, c.groups, threadIdx.x, TYPE, acc);
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
                for (int j = 0; j < 4; ++j) stage_partial(zw, P, slot, pts[j], a4[j]);
            } else if (P == 64) {
                PathAcc<float> a2[2];
                int pts[2];
                pca_gemm_phase<2, TYPE>(c, zw, stride, a2, slot, slots, pts);
                __syncthreads();
#pragma unroll
                for (int j = 0; j < 2; ++j) stage_partial(zw, P, slot, pts[j], a2[j]);
            } else {
                PathAcc<float> a1[1];
                int pts[1];
                pca_gemm_phase<1, TYPE>(c, zw, stride, a1, slot, slots, pts);
                __syncthreads();
                stage_partial(zw, P, slot, pts[0], a1[0]);
            }
            __syncthreads();
            if (threadIdx.x < P) merge_partials(zw, P, slots, threadIdx.x, TYPE, acc);
            return;
        }
    }
    acc.init(TYPE, threadIdx.x < P);
    pca_rows_phase<T, TYPE>(c, zw, stride, acc);
    if (c.groups == 1) return;
    __syncthreads();
    stage_partial(zw, P, threadIdx.x >> c.tile_log2, threadIdx.x & (P - 1), acc);
    __syncthreads();
    if (threadIdx.x < P) merge_partials(zw, P, c.groups, threadIdx.x, TYPE, acc);
    }
}

// the first Sobol' point of the current tile, per dimension (phase 1)
constexpr int kTileStartDims = 1024;
__shared__ uint32_t tile_start[kTileStartDims];

// One tile of a work item: tile `tile` (points tile*P .. tile*P+P-1 of the
// contract, the last tile ragged) of replicate `rep` (index into the plan's
// randomisation tables), its four tile sums added to the item's
// accumulator item_acc (shared memory: tile_acc).
// Point t of the contract is Sobol' point point_k0 + c.k_first + t
// (point_k0: diagnostics; k_first: the contract's first point); point_out,
// when set, receives every point's values (diagnostics).  `smem` is the CTA's dynamic shared memory
// (fused_smem_bytes); every thread of the CTA calls this.
template <typename T, int CONS>
__device__ __forceinline__ void run_item(const ContractDev &c, const uint32_t *__restrict__ sobol_table,
                                         const uint32_t *__restrict__ sobol_shift, int jstride, uint32_t rep,
                                         uint64_t tile, uint64_t point_k0, double *point_out, double *item_acc,
                                         unsigned char *smem) {
    const int P = 1 << c.tile_log2;
    const int n = c.n;
    const int stride = c.row_stride;
    T *zw = reinterpret_cast<T *>(smem);
    point_k0 += c.k_first;

    // ---- phase 1: Sobol' + inverse normal -> zw[point][slot]
    if (n > 0) {
        const uint32_t *tab = sobol_table + static_cast<size_t>(rep) * 32u * jstride;
        const uint32_t *shf = sobol_shift + static_cast<size_t>(rep) * jstride;
        const int chunk = 1 << c.chunk_log2;
        const int nchunks = P >> c.chunk_log2;
        // the tile's first point, one walk per dimension, when the tile starts
        // on a multiple of P (every run then starts from it by the bits of
        // its own offset); otherwise each run walks from its own index
        const uint64_t k_tile = point_k0 + tile * static_cast<uint64_t>(P);
        const bool from_tile = nchunks > 1 && (k_tile & static_cast<uint64_t>(P - 1)) == 0 && n <= kTileStartDims;
        if (from_tile) {
            for (int j = threadIdx.x; j < n; j += kThreads)
                tile_start[j] = sobol_first(tab, jstride, j, __ldg(shf + j), static_cast<uint32_t>(k_tile));
            __syncthreads();
        }
        // n >= 32: a warp takes whole chunks, its lanes consecutive dimensions
        // (stores to one row: no bank conflicts); smaller n: (chunk, dim) items
        const bool by_warp = n >= 32;
        const int step = by_warp ? kThreads / 32 : kThreads;
        const int first = by_warp ? (threadIdx.x >> 5) : threadIdx.x;
        const int work = by_warp ? nchunks * ((n + 31) >> 5) : nchunks * n;
        for (int it = first; it < work; it += step) {
            int j, ch;
            int slot;
            if (by_warp) {
                const int per = (n + 31) >> 5;            // 32-wide dimension blocks per chunk
                ch = it / per;
                const int idx = (it - ch * per) * 32 + (threadIdx.x & 31);
                if (idx >= n) continue;
                if (c.slot_dim) {
                    // the shared-memory bridge: lanes take 32 consecutive slots of the
                    // row (distinct banks), each the dimension whose node sits there
                    slot = idx + 1;
                    j = __ldg(c.slot_dim + slot);
                } else {
                    j = idx;
                    slot = c.z_by_dim ? j + 1 + c.slot_shift : __ldg(&c.steps[j + c.slot_shift].m);
                }
            } else {
                j = it % n;
                ch = it / n;
                slot = c.z_by_dim ? j + 1 + c.slot_shift : __ldg(&c.steps[j + c.slot_shift].m);
            }
            T *dst = zw + static_cast<size_t>(ch * chunk) * stride + slot;
            // points at or past N (ragged last tile) are never generated: their
            // index could pass 2^32; they are zero-filled and left out of the sums
            const uint64_t first_local = tile * P + static_cast<uint64_t>(ch) * chunk;
            const int len = first_local >= c.N ? 0 : static_cast<int>(min(static_cast<uint64_t>(chunk), c.N - first_local));
            if (len > 0) {
                const uint32_t k0 = static_cast<uint32_t>(point_k0 + first_local);
                const uint32_t off = static_cast<uint32_t>(ch * chunk);
                const uint32_t y0 = from_tile ? sobol_from_gray(tab, jstride, j, tile_start[j], off ^ (off >> 1))
                                              : sobol_first(tab, jstride, j, __ldg(shf + j), k0);
                if constexpr (sizeof(T) == 4) {
                    sobol_point_deferred(
                        tab, jstride, j, y0, k0, len, c.chunk_log2,
                        [&](int s, uint32_t y) { dst[s * stride] = Arith<float>::inv_normal(y); },
                        [&](int s, float2 z) {
                            dst[s * stride] = z.x;
                            dst[(s + 1) * stride] = z.y;
                        });
                } else {
                    sobol_points(tab, jstride, j, y0, k0, len, c.chunk_log2,
                                 [&](int s, uint32_t y) { dst[s * stride] = Arith<T>::inv_normal(y); });
                }
            }
            for (int s = len; s < chunk; ++s) dst[s * stride] = T(0);
        }
    }
    for (int pt = threadIdx.x; pt < P; pt += kThreads) zw[pt * stride] = T(0);
    if (c.slot_shift) {  // the leading coordinate is integrated out: its slot holds 0
        const int lead_slot = c.z_by_dim ? 1 : __ldg(&c.steps[0].m);
        for (int pt = threadIdx.x; pt < P; pt += kThreads) zw[pt * stride + lead_slot] = T(0);
    }
    __syncthreads();

    using V = typename std::conditional<sizeof(T) == 8, double, ff>::type;
    const int pt = threadIdx.x;
    const uint64_t local_point = tile * P + pt;
    V v[4];
    for (int g = 0; g < 4; ++g) v[g] = V{};
    if constexpr (CONS == QMCCPW_BB_LEAD || CONS == QMCCPW_PCA_LEAD) {
        // ---- phase 2: the rest of the whole path R_1..R_d (leading Gaussian 0)
        T *rbuf = zw;
        if constexpr (CONS == QMCCPW_BB_LEAD) {
            bridge_store<T>(c, zw, stride);
        } else {
            rbuf = zw + static_cast<size_t>(P) * stride;
            lead_pca_store<T>(c, zw, rbuf, stride);
        }
        __syncthreads();
        // ---- phase 3: the switch point and the values of the point, tile sum
        if (pt < P && local_point < c.N) {
            lead_values<T>(c, rbuf + pt * stride, v);
            if (point_out) {
                for (int g = 0; g < 4; ++g) {
                    if constexpr (sizeof(T) == 8) point_out[local_point * 4 + g] = v[g];
                    else point_out[local_point * 4 + g] = ff_to_double(v[g]);
                }
            }
        }
    } else {
        // ---- phase 2: path construction and running sums, merged per point
        PathAcc<T> acc;
        switch (c.type) {
            case QMCCPW_ARITH_ASIAN_CALL: path_phase<T, CONS, QMCCPW_ARITH_ASIAN_CALL>(c, zw, stride, acc); break;
            case QMCCPW_BINARY_ASIAN: path_phase<T, CONS, QMCCPW_BINARY_ASIAN>(c, zw, stride, acc); break;
            case QMCCPW_LOOKBACK_FIXED_CALL: path_phase<T, CONS, QMCCPW_LOOKBACK_FIXED_CALL>(c, zw, stride, acc); break;
            default: path_phase<T, CONS, QMCCPW_GEOMETRIC_ASIAN_CALL>(c, zw, stride, acc); break;
        }
        // ---- phase 3: conditional values of the point, tile sum
        if (pt < P && local_point < c.N) {
            T xhat, dhat;
            finish_functional(c, acc, xhat, dhat);
            if constexpr (sizeof(T) == 8) values_fp64(c, xhat, dhat, v);
            else values_mixed(c, xhat, dhat, v);
            if (point_out) {
                double *o = point_out + local_point * 4;
                for (int g = 0; g < 4; ++g) {
                    if constexpr (sizeof(T) == 8) o[g] = v[g];
                    else o[g] = ff_to_double(v[g]);
                }
            }
        }
    }
    tile_acc(item_acc, v, smem);
}

// ---------------------------------------------------------------------------
// per-replicate compensated reduction
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

// Replicate estimate from its `tiles` item slots (4 doubles each, in item
// order): thread t of a 256-thread block sums slots t, t + 256, ... with
// compensated arithmetic, then a fixed tree merges the 256 partial sums;
// thread g < 4 returns Greek g divided by N (other threads: 0).
// `part` is 256 x 4 shared Neumaier pairs.  Every thread of the block calls it.
__device__ __forceinline__ double reduce_replicate(const double *__restrict__ first, uint64_t tiles, uint64_t N,
                                                   Neumaier (*part)[4]) {
    Neumaier acc[4] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
    for (uint64_t t = threadIdx.x; t < tiles; t += 256)
        for (int g = 0; g < 4; ++g) acc[g].add(__ldcg(first + t * 4 + g));  // L2: written by other CTAs
    for (int g = 0; g < 4; ++g) part[threadIdx.x][g] = acc[g];
    __syncthreads();
    for (int half = 128; half > 0; half >>= 1) {
        if (threadIdx.x < half)
            for (int g = 0; g < 4; ++g) part[threadIdx.x][g].add(part[threadIdx.x + half][g]);
        __syncthreads();
    }
    const double v = threadIdx.x < 4 ? part[0][threadIdx.x].value() / static_cast<double>(N) : 0.0;
    __syncthreads();  // part is free again on return
    return v;
}

// Mean over the R replicate estimates of Greek g (rows of 4 doubles from
// `rows`) and the standard error of that mean, sd / sqrt(R) with the (R - 1)
// sample variance (Sec. 5); both sums compensated, in replicate order.
__device__ void replicate_stats(const double *__restrict__ rows, int R, int g, double &mean, double &se) {
    Neumaier s = {0, 0};
    for (int r = 0; r < R; ++r) s.add(rows[r * 4 + g]);
    mean = s.value() / R;
    Neumaier dev = {0, 0};
    for (int r = 0; r < R; ++r) {
        const double e = rows[r * 4 + g] - mean;
        dev.add(e * e);
    }
    se = sqrt(dev.value() / (static_cast<double>(R) * (R - 1)));
}

}  // namespace
}  // namespace qmccpw
