// PCA construction on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// W~ = A z with A A^T = Sigma (eq. WboldTilde); for equal spacing
// A = sqrt(dt) * Ahat where Ahat (the factor for dt = 1) depends on n only.
// One CTA (256 threads; 512 in the streamed variant) per tile of 128 points
// (a work item is a run of consecutive tiles of one replicate):
//   1. Sobol' + inverse normal as in the CUDA-core kernel; z is split into
//      hi + lo parts (bf16 or tf32) written straight into the operand layout
//      (K-major, 128-byte swizzle, so a warp's stores hit distinct banks).
//   2. One thread issues the split product with FP32 accumulation in tensor
//      memory, M = 128 points, N = dates, K = dimensions: D1 = Z_hi Ahat_hi^T
//      and D2 = the small products (tf32: Z_lo Ahat_hi^T + Z_hi Ahat_lo^T;
//      bf16, Ahat in three parts: Z_lo Ahat_hi^T + Z_hi Ahat_mid^T +
//      Z_lo Ahat_mid^T + Z_hi Ahat_lo^T).
//   3. The epilogue reads D1 + D2 with tcgen05.ld (warp w owns TMEM lanes
//      32(w%4)..+31, warpgroup w/4 one half of the columns), scales by
//      sqrt(dt) and forms the path sums; then the conditional step and the
//      tile sum exactly as in the CUDA-core kernel.
// Exact leading product: the tensor core's FP32 accumulation does not round
// to nearest, and a bias of ~1 ulp of |D| per instruction shifts every path
// the same way (averaging over points does not remove it).  So the hi parts
// lie on fixed grids (z: 2^-5 for bf16, 2^-8 for tf32, with |z| < 6.4 from
// u >= 2^-33; Ahat: 2^-e with e the largest that keeps max|Ahat| 2^e within
// the 8 or 11 significant bits), every product and partial sum of D1 is then
// a multiple of one quantum and far below 2^24 quanta, and D1 is exact.  The
// small terms go to their own accumulator D2, where the same ulp errors are
// 2^-9 (tf32) to 2^-4 (bf16) of |W~| smaller.
// Fixed matrix, random points: rounding z costs every point an independent,
// zero-mean error that the average over points removes, but rounding Ahat
// is one fixed perturbation of the factor, hence of the covariance of every
// simulated path, and no number of points removes it.  A bf16 hi + lo pair
// leaves Ahat off by up to 2^-15 (~2e-6 relative bias of the estimates at
// d = 16..64, about ten standard errors on the d = 64 benchmark); so bf16
// carries Ahat in three parts (hi on its grid, mid and lo each the bf16 of
// what remains, ~2^-23), while tf32 keeps two (off by <= 2^-20, at the
// float floor).  z keeps two parts in both: its rounding is new for every
// point, and so is the product z_lo x Ahat_lo that tf32 leaves out (at most
// 2^-18, zero-mean).
// Two variants, each for bf16 and tf32: d <= 65 (N = K = 64; Ahat resident,
// staged by one bulk TMA copy per contract) and d <= 257 (N = K = 256; Ahat
// streamed from L2 in K-chunks, see pca_tcs_kernel).
// Every wait on an mbarrier is bounded: on expiry the kernel records an
// error code, releases its tensor memory and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "qmccpw_internal.h"
#include "qmccpw_device.cuh"
#include "tc_ptx.cuh"

namespace qmccpw {
namespace {

constexpr int kM = 128;        // points per tile (UMMA M)
constexpr int kNpad = 64;      // dates and dimensions, padded (UMMA N and K)
// ---- operand element addressing ----------------------------------------------
// Element (row, k) of Z (kM rows), K-major with the 128-byte swizzle: K
// columns of 128 bytes each hold kM rows of 128 bytes; the 16-byte unit u of
// row r sits at u ^ (r % 8).  With lanes over k a warp's stores cover whole
// 128-byte rows, so they fall in distinct banks.
template <int ESIZE>
__device__ __forceinline__ uint32_t z_offset(int row, int k) {
    const uint32_t kb = static_cast<uint32_t>(k) * ESIZE;
    return (kb >> 7) * (kM * 128u) + static_cast<uint32_t>(row) * 128u +
           ((((kb >> 4) & 7u) ^ (static_cast<uint32_t>(row) & 7u)) << 4) + (kb & 15u);
}
// Start of the K slice [kb, kb + 32 bytes) of Z for one instruction.
__device__ __forceinline__ uint32_t z_slice(uint32_t base, uint32_t kb) { return base + (kb >> 7) * (kM * 128u) + (kb & 127u); }

// hi + lo split of z for two adjacent dimensions (k even, k + 1) of one
// point: hi on the fixed grid (2^-5 bf16, 2^-8 tf32; rounding by the
// add-and-subtract of 1.5 2^23, exact for |z| 2^8 < 2^22), so it is exact in
// the operand type.  Stored as one 32-bit word per part for bf16 (hi is
// exact, so its bf16 is the top half of its bits, gathered by one byte
// permutation; lo is rounded to nearest even by the packed conversion), one
// 64-bit word per part for tf32.  hs = z kScale rounded to an integer;
// lo = z - hs / kScale is exact, so one FMA forms it.  `off` is element k's
// offset (4- or 8-byte aligned: the swizzle permutes whole 16-byte units).
template <int KIND>
__device__ __forceinline__ void split_store_pair(unsigned char *hi_base, unsigned char *lo_base, uint32_t off,
                                                 float2 z) {
    constexpr float kScale = KIND == 0 ? 32.0f : 256.0f;
    const float2 hs = add2(fma2(z, f2(kScale), f2(12582912.0f)), f2(-12582912.0f));
    const float2 h = mul2(hs, f2(1.0f / kScale));
    const float2 l = fma2(hs, f2(-1.0f / kScale), z);
    if constexpr (KIND == 0) {
        const __nv_bfloat162 lw = __floats2bfloat162_rn(l.x, l.y);  // .x (element k) in the low half
        *reinterpret_cast<uint32_t *>(hi_base + off) = __byte_perm(__float_as_uint(h.x), __float_as_uint(h.y), 0x7632);
        *reinterpret_cast<__nv_bfloat162 *>(lo_base + off) = lw;
    } else {
        const uint2 hb = make_uint2(__float_as_uint(h.x), __float_as_uint(h.y));
        const uint2 lb = make_uint2((__float_as_uint(l.x) + 0x1000u) & 0xFFFFE000u,
                                    (__float_as_uint(l.y) + 0x1000u) & 0xFFFFE000u);
        *reinterpret_cast<uint2 *>(hi_base + off) = hb;
        *reinterpret_cast<uint2 *>(lo_base + off) = lb;
    }
}

// Path sums of this thread's point over its warpgroup's share of the dates
// (NWG warpgroups, each NPAD / NWG consecutive columns): W~ = sqrt(dt)
// (D1 + D2), D2 at column offset NPAD.
// `half` is the warpgroup's share, `quarter` the warp's position in its
// warpgroup (TMEM lanes 32 quarter .. 32 quarter + 31).
template <int TYPE, int NPAD, int NWG>
__device__ void epilogue_sums(const ContractDev &c, uint32_t tmem, PathAcc<float> &acc, int half, int quarter) {
    static_assert((NPAD / NWG) % 16 == 0, "whole 16-column loads per warpgroup");
    const uint32_t lane_base = static_cast<uint32_t>(32 * quarter) << 16;
    const PathConst k(c);
    acc.init(TYPE, half == 0);
    const int last = min(c.n, (half + 1) * (NPAD / NWG));  // dates beyond n are padding
#pragma unroll 1
    for (int col = half * (NPAD / NWG); col < last; col += 16) {
        float d1[16], d2[16];
        tmem_ld16x2(tmem + lane_base + static_cast<uint32_t>(col), tmem + lane_base + static_cast<uint32_t>(col + NPAD),
                    d1, d2);
#pragma unroll
        for (int i = 0; i < 16; i += 2) {  // dates two at a time, in packed form (unit-spacing path D1 + D2)
            const int date = col + i + 1;
            const float2 w = add2(make_float2(d1[i], d1[i + 1]), make_float2(d2[i], d2[i + 1]));
            if (date + 1 <= c.n)
                acc.template add2<TYPE>(date, date + 1, w.x, w.y, k);
            else if (date <= c.n)
                acc.template add<TYPE>(date, w.x, k);
        }
    }
}

template <int NPAD, int NWG>
__device__ __forceinline__ void epilogue_dispatch(const ContractDev &c, uint32_t tmem, PathAcc<float> &acc,
                                                  int half, int quarter) {
    switch (c.type) {
        case QMCCPW_ARITH_ASIAN_CALL:
            epilogue_sums<QMCCPW_ARITH_ASIAN_CALL, NPAD, NWG>(c, tmem, acc, half, quarter);
            break;
        case QMCCPW_BINARY_ASIAN: epilogue_sums<QMCCPW_BINARY_ASIAN, NPAD, NWG>(c, tmem, acc, half, quarter); break;
        case QMCCPW_LOOKBACK_FIXED_CALL:
            epilogue_sums<QMCCPW_LOOKBACK_FIXED_CALL, NPAD, NWG>(c, tmem, acc, half, quarter);
            break;
        default: epilogue_sums<QMCCPW_GEOMETRIC_ASIAN_CALL, NPAD, NWG>(c, tmem, acc, half, quarter); break;
    }
}

// Merge the NWG warpgroups' partial sums of each point (in date order), the
// conditional step and the tile sum, added to the work item's total in
// item_acc (shared by both variants).
template <int NWG>
__device__ __forceinline__ void finish_tile(const LaunchParams &p, const ContractDev &c, double *item_acc,
                                           uint64_t tile, PathAcc<float> &acc, unsigned char *scratch) {
    const int warp = threadIdx.x >> 5;
    const int point = 32 * (warp & 3) + (threadIdx.x & 31);
    if (warp < 4 * NWG) stage_partial(scratch, kM, warp >> 2, point, acc, kM * NWG);  // not the product warp
    __syncthreads();
    ff v[4] = {{0.0f, 0.0f}, {0.0f, 0.0f}, {0.0f, 0.0f}, {0.0f, 0.0f}};
    const uint64_t local_point = tile * kM + point;
    if (warp < 4) {
        merge_partials(scratch, kM, NWG, point, c.type, acc, kM * NWG);
        if (local_point < c.N) {
            float xhat, dhat;
            finish_functional(c, acc, xhat, dhat);
            values_mixed(c, xhat, dhat, v);
            if (p.point_out) {
                double *o = p.point_out + local_point * 4;
                for (int g = 0; g < 4; ++g) o[g] = ff_to_double(v[g]);
            }
        }
    }
    tile_acc(item_acc, v, scratch);
}

// Two Gray-code chains (dimensions ja and jb) over the same run of points.
// A full aligned run of 4..64 points is unrolled with both dimensions'
// direction integers in registers and the inverse normal's tail test taken
// out of the unrolled body: emitz(s, z) receives the central values of point
// s and a bit per point records a tail draw; after the run each recorded
// point (rare) is rebuilt from the run's first point by the bits of its Gray
// index and its exact values emitted again.  Other runs go point by point,
// emit(s, y_ja(k0+s), y_jb(k0+s)).
template <int LG, typename EmitZ>
__device__ __forceinline__ void chain_pair_run_deferred(const uint32_t *__restrict__ tab, int jstride, int ja,
                                                        int jb, uint32_t ya, uint32_t yb, EmitZ &&emitz) {
    uint32_t va[LG], vb[LG];
#pragma unroll
    for (int b = 0; b < LG; ++b) {
        va[b] = __ldg(tab + b * jstride + ja);
        vb[b] = __ldg(tab + b * jstride + jb);
    }
    const uint32_t ya0 = ya, yb0 = yb;
    uint64_t redo = 0;
#pragma unroll
    for (int s = 0; s < (1 << LG); ++s) {
        if (s > 0) {
            ya ^= va[ctz_const(s)];
            yb ^= vb[ctz_const(s)];
        }
        float2 z;
        if (Arith<float>::inv_normal2_central(ya, yb, z)) redo |= 1ull << s;
        emitz(s, z);
    }
    while (redo) {
        const int s = __ffsll(static_cast<long long>(redo)) - 1;
        redo &= redo - 1ull;
        const uint32_t g = static_cast<uint32_t>(s) ^ (static_cast<uint32_t>(s) >> 1);
        uint32_t a = ya0, b2 = yb0;
#pragma unroll
        for (int b = 0; b < LG; ++b)
            if ((g >> b) & 1u) {
                a ^= va[b];
                b2 ^= vb[b];
            }
        emitz(s, Arith<float>::inv_normal2(a, b2));
    }
}

template <typename Emit, typename EmitZ>
__device__ __forceinline__ void sobol_chain_deferred(const uint32_t *__restrict__ tab, int jstride, int ja, int jb,
                                                     uint32_t ya, uint32_t yb, uint32_t k0, int len, int chunk_log2,
                                                     Emit &&emit, EmitZ &&emitz) {
    if (len == (1 << chunk_log2) && (k0 & (static_cast<uint32_t>(len) - 1u)) == 0u) {
        switch (chunk_log2) {
            case 2: chain_pair_run_deferred<2>(tab, jstride, ja, jb, ya, yb, emitz); return;
            case 3: chain_pair_run_deferred<3>(tab, jstride, ja, jb, ya, yb, emitz); return;
            case 4: chain_pair_run_deferred<4>(tab, jstride, ja, jb, ya, yb, emitz); return;
            case 5: chain_pair_run_deferred<5>(tab, jstride, ja, jb, ya, yb, emitz); return;
            case 6: chain_pair_run_deferred<6>(tab, jstride, ja, jb, ya, yb, emitz); return;
            default: break;
        }
    }
    for (int s = 0; s < len; ++s) {
        if (s > 0) {
            const int b = __ffs(k0 + s) - 1;
            ya ^= __ldg(tab + b * jstride + ja);
            yb ^= __ldg(tab + b * jstride + jb);
        }
        emit(s, ya, yb);
    }
}

// Phase 1 of both variants: Sobol' + inverse normal of the tile's points for
// dimensions j0 <= j < j1, split and stored into Z at column col0 + j - j0.
// A lane takes two adjacent dimensions (j even relative to j0) over a chunk
// of consecutive points, the two Gray-code chains side by side, so each step
// evaluates the inverse normal of two draws at once and stores both
// dimensions' parts in one word; a warp covers 64 dimensions of a row
// (128-byte swizzled rows: conflict-free).  Points past N are 0.  Columns of Z
// at or beyond n meet only zero Ahat columns: an odd last dimension is
// paired with a copy of itself in the next (padding) column.  `warp` counts
// the NW warps that share the work.
// The first Sobol' point of the current tile, per dimension (the streamed
// variant): with it every run starts from the tile's point by the bits of its
// own offset (sobol_from_gray) instead of a walk over the bits of its index.
// The resident variant (at most 64 dimensions) measured 0.7% slower with it
// (one more barrier per tile), so its runs walk from their own index.
constexpr int kTcTileDims = 256;
__shared__ uint32_t tc_tile_start[kTcTileDims];

// Fill tc_tile_start for dimensions 0..n-1 (every thread of the CTA; the
// caller synchronises); false when the tile does not start on a multiple of
// kM, whose runs then walk from their own index.
__device__ __forceinline__ bool tile_start_dims(const LaunchParams &p, const ContractDev &c, uint32_t rep,
                                                uint64_t tile) {
    const uint64_t k_tile = p.point_k0 + c.k_first + tile * static_cast<uint64_t>(kM);
    if ((k_tile & static_cast<uint64_t>(kM - 1)) != 0 || c.n > kTcTileDims || (kM >> c.chunk_log2) < 2) return false;
    const uint32_t *tab = p.sobol_table + static_cast<size_t>(rep) * 32u * p.jstride;
    const uint32_t *shf = p.sobol_shift + static_cast<size_t>(rep) * p.jstride;
    for (int j = static_cast<int>(threadIdx.x); j < c.n; j += static_cast<int>(blockDim.x))
        tc_tile_start[j] = sobol_first(tab, p.jstride, j, __ldg(shf + j), static_cast<uint32_t>(k_tile));
    return true;
}

template <int KIND, int NW>
__device__ __forceinline__ void sobol_to_z(const LaunchParams &p, const ContractDev &c, uint32_t rep, uint64_t tile,
                                           unsigned char *z_hi, unsigned char *z_lo, int j0, int j1, int col0,
                                           bool from_tile, int warp) {
    constexpr int ES = KIND == 0 ? 2 : 4;
    const uint32_t *tab = p.sobol_table + static_cast<size_t>(rep) * 32u * p.jstride;
    const uint32_t *shf = p.sobol_shift + static_cast<size_t>(rep) * p.jstride;
    const int chunk = 1 << c.chunk_log2;
    const int nchunks = kM >> c.chunk_log2;
    const int per = (j1 - j0 + 63) >> 6;
    const int work = nchunks * per;
    for (int it = warp; it < work; it += NW) {
        const int ch = it / per;
        const int rel = (it - ch * per) * 64 + 2 * (threadIdx.x & 31);
        const int ja = j0 + rel;
        if (ja >= j1) continue;
        const int col = col0 + rel;
        const int jb = ja + 1 < j1 ? ja + 1 : ja;  // odd last dimension: its own copy (in bounds of the tables)
        const uint64_t first_local = tile * kM + static_cast<uint64_t>(ch) * chunk;
        const int len = first_local >= c.N ? 0 : static_cast<int>(min(static_cast<uint64_t>(chunk), c.N - first_local));
        const int row0 = ch * chunk;
        if (len > 0) {
            const uint32_t k0 = static_cast<uint32_t>(p.point_k0 + c.k_first + first_local);
            uint32_t ya, yb;
            if (from_tile) {
                const uint32_t off = static_cast<uint32_t>(row0);
                sobol_from_gray_pair(tab, p.jstride, ja, jb, tc_tile_start[ja], tc_tile_start[jb], off ^ (off >> 1),
                                     ya, yb);
            } else {
                sobol_first_pair(tab, p.jstride, ja, jb, __ldg(shf + ja), __ldg(shf + jb), k0, ya, yb);
            }
            auto emit = [&](int s, uint32_t a, uint32_t b) {
                split_store_pair<KIND>(z_hi, z_lo, z_offset<ES>(row0 + s, col), Arith<float>::inv_normal2(a, b));
            };
            auto emitz = [&](int s, float2 z) { split_store_pair<KIND>(z_hi, z_lo, z_offset<ES>(row0 + s, col), z); };
            sobol_chain_deferred(tab, p.jstride, ja, jb, ya, yb, k0, len, c.chunk_log2, emit, emitz);
        }
        for (int s = len; s < chunk; ++s)
            split_store_pair<KIND>(z_hi, z_lo, z_offset<ES>(row0 + s, col), make_float2(0.0f, 0.0f));
    }
}

struct TcShared {
    uint64_t bar_b, bar_mma;
    uint32_t tmem_addr;
    int32_t loaded_n;
    int32_t abort;
};

// dynamic shared memory rounded up to the 1024-byte alignment of swizzled operands
__device__ __forceinline__ unsigned char *aligned_smem(unsigned char *raw) {
    const uint32_t a = smem_u32(raw);
    return raw + (((a + 1023u) & ~1023u) - a);
}

template <int KIND>
__global__ void __launch_bounds__(kThreads, KIND == 0 ? 3 : 2) pca_tc_kernel(const __grid_constant__ LaunchParams p) {
    constexpr int ES = KIND == 0 ? 2 : 4;                  // element bytes
    constexpr uint32_t kOpBytesZ = kM * kNpad * ES;        // one split part of Z
    constexpr uint32_t kOpBytesB = kNpad * kNpad * ES;     // one split part of Ahat
    constexpr int kPartsB = KIND == 0 ? 3 : 2;             // Ahat parts: bf16 hi/mid/lo, tf32 hi/lo
    constexpr uint32_t kIdesc = instr_desc(KIND == 0 ? 1u : 2u, kNpad);
    constexpr uint32_t kLbo = 128, kSbo = (kNpad / (16 / ES)) * 128;
    constexpr uint32_t kCols = 2 * kNpad;                  // D1 and D2

    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *z_hi = aligned_smem(smem_raw);
    unsigned char *z_lo = z_hi + kOpBytesZ;
    unsigned char *b_hi = z_lo + kOpBytesZ;                // the other parts follow (one bulk copy)
    unsigned char *scratch = b_hi + kPartsB * kOpBytesB;   // partial sums, tile values
    __shared__ TcShared sh;

    const int warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        mbar_init(&sh.bar_b, 1);
        mbar_init(&sh.bar_mma, 1);
        sh.loaded_n = -1;
        sh.abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tmem_alloc(&sh.tmem_addr, kCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sh.tmem_addr;
    // padding columns (k >= n) of Z are never written by the Sobol' phase
    for (uint32_t i = threadIdx.x; i < 2 * kOpBytesZ / 4; i += kThreads) reinterpret_cast<uint32_t *>(z_hi)[i] = 0u;

    uint32_t b_phase = 0, mma_phase = 0;
    __shared__ WorkItem work;
    __shared__ double item_acc[8];
    item_acc_clear(item_acc);
    while (true) {
      next_work(p, work);
      if (work.item >= p.item_end) break;
      // the item stays in shared memory (`work`); tiles per replicate fit 32 bits
      for (uint32_t tile = static_cast<uint32_t>(work.tile); tile < work.tile_end; ++tile) {
        const ContractDev &c = p.contracts[work.ci];
        const uint32_t rep = work.rep;
        const int n = c.n;

        // ---- Ahat (hi, lo) for this n: one bulk copy when n changes (only
        // at an item's first tile, after the barrier that ends next_work)
        if (sh.loaded_n != n) {
            if (threadIdx.x == 0) {
                mbar_expect_tx(&sh.bar_b, kPartsB * kOpBytesB);
                bulk_copy_g2s(b_hi, c.tc_operand, kPartsB * kOpBytesB, &sh.bar_b);
            }
            if (!mbar_wait(&sh.bar_b, b_phase & 1u)) atomicExch(&sh.abort, 1);  // 1: the copy may still land
            ++b_phase;
            __syncthreads();
            if (threadIdx.x == 0) sh.loaded_n = n;
        }
        if (sh.abort) break;

        // ---- phase 1: Sobol' + inverse normal -> split operand
        sobol_to_z<KIND, kThreads / 32>(p, c, rep, tile, z_hi, z_lo, 0, n, 0, false, warp);
        fence_proxy_async();  // generic-proxy stores -> visible to the tensor core
        tc_fence_before();
        __syncthreads();
        tc_fence_after();

        // ---- phase 2: the split product into tensor memory
        if (threadIdx.x == 0) {
            const uint32_t bh = smem_u32(b_hi), b2 = bh + kOpBytesB, b3 = b2 + kOpBytesB;
#pragma unroll
            for (int ks = 0; ks < kNpad / (32 / ES); ++ks) {  // K per instruction: 16 bf16 or 8 tf32 = 32 bytes
                const uint32_t kb = static_cast<uint32_t>(ks) * 32u;     // Z: byte offset along K
                const uint32_t koff = static_cast<uint32_t>(ks) * 256u;  // Ahat: two core matrices along K
                const uint64_t zh = smem_desc_sw128(z_slice(smem_u32(z_hi), kb));
                const uint64_t zl = smem_desc_sw128(z_slice(smem_u32(z_lo), kb));
                const uint32_t acc = ks > 0 ? 1u : 0u;
                mma<KIND>(tmem, zh, smem_desc(bh + koff, kLbo, kSbo), kIdesc, acc);
                mma<KIND>(tmem + kNpad, zl, smem_desc(bh + koff, kLbo, kSbo), kIdesc, acc);
                mma<KIND>(tmem + kNpad, zh, smem_desc(b2 + koff, kLbo, kSbo), kIdesc, 1u);
                if constexpr (KIND == 0) {  // bf16: Ahat mid is b2, lo is b3
                    mma<KIND>(tmem + kNpad, zl, smem_desc(b2 + koff, kLbo, kSbo), kIdesc, 1u);
                    mma<KIND>(tmem + kNpad, zh, smem_desc(b3 + koff, kLbo, kSbo), kIdesc, 1u);
                }
            }
            mma_commit(&sh.bar_mma);
        }
        if (!mbar_wait(&sh.bar_mma, mma_phase & 1u)) atomicExch(&sh.abort, 2);  // 2: products may still run
        __syncthreads();
        if (sh.abort) break;  // an unfinished accumulator is never read or summed
        ++mma_phase;
        tc_fence_after();

        // ---- phase 3: path sums from D, merged across the two warpgroups
        PathAcc<float> acc;
        epilogue_dispatch<kNpad, 2>(c, tmem, acc, warp >> 2, warp & 3);
        tc_fence_before();
        finish_tile<2>(p, c, item_acc, tile, acc, scratch);
      }
      if (sh.abort) break;  // read after a barrier: the same in every thread
      item_flush<ff>(p.tile_sums + work.item * 4, item_acc);
    }

    // release tensor memory (also after an abort: first, with the same bounded
    // wait, let the copy or the products the expired wait left in flight land)
    tc_fence_before();
    __syncthreads();
    if (sh.abort && threadIdx.x == 0) {
        if (sh.abort == 1) mbar_wait(&sh.bar_b, (b_phase - 1u) & 1u);
        else mbar_wait(&sh.bar_mma, mma_phase & 1u);
        if (p.error_flag) atomicExch(p.error_flag, QMCCPW_ERR_TIMEOUT);
    }
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, kCols);
    }
}

// d up to 257 (N = K = 256), Ahat streamed.  Ahat (384 KB bf16 in three
// parts, 512 KB tf32 in two) does not fit beside Z, so it comes from L2 in
// K-chunks of 16 dimensions (all parts of a chunk in one bulk TMA copy, 24 or
// 32 KB) through a ring of chunk buffers (three for bf16, two for tf32; six
// for bf16, with Z in two slots, measured 2.5% slower).
// Z is produced in blocks of 64 dimensions (one 128-byte swizzle column of
// bf16, two of tf32) and the products of a block run while the next block is
// produced: 16 producer warps write Z and arrive on the block's "full"
// barrier; a 17th warp, the product warp, waits for each block, issues its
// products chunk by chunk as the Ahat chunks land, refills each chunk buffer
// once the products that read it are done (tcgen05.commit to the buffer's
// barrier), and commits the block's Z slot free.  Z hi/lo holds all 256
// columns for bf16 (128 KB, four block slots); for tf32 the same 128 KB holds
// 128 columns (two block slots), a slot reused once its block's products are
// done.  Measured at d = 256 (N = 2^20, R = 16): bf16 25.1 -> 23.8 ms, tf32
// 27.5 -> 23.6 ms per launch; the products read about 90 bytes of shared
// memory per clock while they run, so the producers' stores compete with
// them and the overlap gains less than the product phase's share.
// A buffer's next chunk wraps to the first chunks of the next tile, which
// are fetched while the epilogue of this one runs.  D1 and D2 take all 512
// TMEM columns: one CTA per SM.  Without any overlap (the product phase
// after the whole Sobol' phase) the product phase was 44% of the kernel.
constexpr int kNbig = 256;
// Four warpgroups share each point's dates in the epilogue: 16 warps.  15 of
// them produce Z; the 16th is the product warp during production and joins
// the epilogue (512 threads, up to 128 registers).  A 17th warp for the
// products instead (544 threads: five warps on one SM sub-partition cap the
// registers at 96) measured 1-6% slower.
constexpr int kThreadsS = 512;
constexpr int kProducerWarpsS = 15;
constexpr int kEpilogueWarpsS = 16;

template <int KIND> struct Streamed {
    static constexpr int ES = KIND == 0 ? 2 : 4;
    static constexpr int Kc = 16;                          // K per chunk
    static constexpr int Kz = KIND == 0 ? 256 : 128;       // Z columns resident at a time
    static constexpr int Bd = 64;                          // dimensions per produced block
    static constexpr int Slots = Kz / Bd;                  // block slots of Z
    static constexpr int Nb = KIND == 0 ? 3 : 2;           // Ahat chunk buffers
    static constexpr int Parts = KIND == 0 ? 3 : 2;        // Ahat parts
    static constexpr uint32_t ZPart = kM * Kz * ES;        // one split part of Z
    static constexpr uint32_t ChunkPart = kNbig * Kc * ES; // one part of one chunk (8 or 16 KB)
    static constexpr uint32_t ChunkBytes = Parts * ChunkPart;  // 24 KB bf16, 32 KB tf32
};

struct TcSharedS {
    uint64_t bar_b[3], bar_f[3];       // Ahat chunk buffer landed / free again
    uint64_t bar_full[4], bar_free[4]; // Z block slot written by the producers / read by the products
    uint64_t bar_mma;                  // every product of the tile done
    uint32_t tmem_addr;
    int32_t abort;
};

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

template <int KIND>
__global__ void __launch_bounds__(kThreadsS, 1) pca_tcs_kernel(const __grid_constant__ LaunchParams p) {
    using S = Streamed<KIND>;
    constexpr uint32_t kIdesc = instr_desc(KIND == 0 ? 1u : 2u, kNbig);
    constexpr uint32_t kLbo = 128;
    constexpr uint32_t kSboB = (S::Kc * S::ES / 16) * 128;  // 8-row groups of a chunk
    constexpr uint32_t kCols = 2 * kNbig;
    constexpr int kSteps = S::Kc * S::ES / 32;             // instructions (32 bytes of K) per chunk
    constexpr int kChunksPerBlock = S::Bd / S::Kc;

    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *z_hi = aligned_smem(smem_raw);
    unsigned char *z_lo = z_hi + S::ZPart;
    unsigned char *bbuf = z_lo + S::ZPart;                 // S::Nb chunk buffers
    unsigned char *scratch = bbuf + S::Nb * S::ChunkBytes;
    __shared__ TcSharedS sh;
    __shared__ WorkItem work;

    const int warp = threadIdx.x >> 5;
    const bool producer = warp < kProducerWarpsS;
    const bool issuer = warp == kProducerWarpsS && (threadIdx.x & 31) == 0;
    if (threadIdx.x == 0) {
        for (int i = 0; i < S::Nb; ++i) {
            mbar_init(&sh.bar_b[i], 1);
            mbar_init(&sh.bar_f[i], 1);
        }
        for (int i = 0; i < S::Slots; ++i) {
            mbar_init(&sh.bar_full[i], 32 * kProducerWarpsS);
            mbar_init(&sh.bar_free[i], 1);
        }
        mbar_init(&sh.bar_mma, 1);
        sh.abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tmem_alloc(&sh.tmem_addr, kCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sh.tmem_addr;
    for (uint32_t i = threadIdx.x; i < 2 * S::ZPart / 4; i += kThreadsS) reinterpret_cast<uint32_t *>(z_hi)[i] = 0u;

    // the product thread's state: barrier phases, the running chunk index q
    // (chunk q sits in buffer q % Nb), the operand whose next Nb chunks are in
    // flight or resident
    uint32_t b_ph[3] = {0, 0, 0}, f_ph[3] = {0, 0, 0}, full_ph[4] = {0, 0, 0, 0};
    uint64_t q = 0;
    const void *loaded = nullptr;
    bool ok = true;  // the product thread: no wait has expired
    // the producers' uses of each Z slot (parity of its "free" barrier)
    uint32_t slot_uses[4] = {0, 0, 0, 0};
    uint32_t mma_ph = 0;
    auto fetch = [&](const void *op, int chunk, int buf) {
        mbar_expect_tx(&sh.bar_b[buf], S::ChunkBytes);
        bulk_copy_g2s(bbuf + buf * S::ChunkBytes, static_cast<const unsigned char *>(op) + chunk * S::ChunkBytes,
                      S::ChunkBytes, &sh.bar_b[buf]);
    };
    auto wait_b = [&](int buf) {
        ok = ok && mbar_wait(&sh.bar_b[buf], b_ph[buf] & 1u);
        ++b_ph[buf];
    };
    auto wait_f = [&](int buf) {
        ok = ok && mbar_wait(&sh.bar_f[buf], f_ph[buf] & 1u);
        ++f_ph[buf];
    };

    __shared__ double item_acc[8];
    item_acc_clear(item_acc);
    while (true) {
      // the stop decision travels with the item: thread 0 reads the abort
      // flag here and ends the loop for all (an expired wait stops it)
      next_work(p, work, threadIdx.x == 0 && sh.abort);
      if (work.item >= p.item_end) break;
      // the item stays in shared memory (`work`); tiles per replicate fit 32 bits
      for (uint32_t tile = static_cast<uint32_t>(work.tile); tile < work.tile_end; ++tile) {
        const ContractDev &c = p.contracts[work.ci];
        const uint32_t rep = work.rep;
        const int nch = (c.n + S::Kc - 1) / S::Kc;        // chunks holding dimensions below n (>= 5)
        const int nblk = (c.n + S::Bd - 1) / S::Bd;
        const bool from_tile = tile_start_dims(p, c, rep, tile);
        __syncthreads();

        if (producer) {
            // ---- Sobol' + inverse normal -> Z, one 64-dimension block at a time
            for (int b = 0; b < nblk; ++b) {
                const int slot = b % S::Slots;
                // the slot's block of this tile before: its products must be done
                if (b >= S::Slots && !sh.abort &&
                    !mbar_wait(&sh.bar_free[slot], (slot_uses[slot] - 1u) & 1u))
                    atomicExch(&sh.abort, 2);
                ++slot_uses[slot];
                const int j0 = b * S::Bd, j1 = min(c.n, j0 + S::Bd);
                sobol_to_z<KIND, kProducerWarpsS>(p, c, rep, tile, z_hi, z_lo, j0, j1, j0 % S::Kz, from_tile, warp);
                fence_proxy_async();  // generic-proxy stores -> visible to the tensor core
                mbar_arrive(&sh.bar_full[slot]);
            }
        } else if (warp == kProducerWarpsS) {
          if (issuer) {
            // ---- the products of each block as it fills
            if (ok && loaded != c.tc_operand) {
                // first tile, or a contract with another d: let the prefetch of
                // the previous operand land, then fetch this one's first chunks
                if (loaded != nullptr)
                    for (int i = 0; i < S::Nb; ++i) wait_b(static_cast<int>((q + i) % S::Nb));
                if (ok) {
                    for (int i = 0; i < S::Nb; ++i) fetch(c.tc_operand, i, static_cast<int>((q + i) % S::Nb));
                    loaded = c.tc_operand;
                }
            }
            int cc = 0;
            for (int b = 0; b < nblk && ok; ++b) {
                const int slot = b % S::Slots;
                ok = mbar_wait(&sh.bar_full[slot], full_ph[slot] & 1u);
                ++full_ph[slot];
                if (!ok) break;
                tc_fence_after();
                const int c_end = min(nch, (b + 1) * kChunksPerBlock);
                for (; cc < c_end && ok; ++cc, ++q) {
                    const int buf = static_cast<int>(q % S::Nb);
                    wait_b(buf);
                    if (!ok) break;
                    const uint32_t bh = smem_u32(bbuf + buf * S::ChunkBytes), b2 = bh + S::ChunkPart,
                                   b3 = b2 + S::ChunkPart;
#pragma unroll
                    for (int ks = 0; ks < kSteps; ++ks) {
                        const uint32_t kb = static_cast<uint32_t>(((cc * S::Kc) % S::Kz) * S::ES + ks * 32);  // Z byte offset
                        const uint32_t koff = static_cast<uint32_t>(ks) * 256u;  // chunk: two core matrices
                        const uint64_t zh = smem_desc_sw128(z_slice(smem_u32(z_hi), kb));
                        const uint64_t zl = smem_desc_sw128(z_slice(smem_u32(z_lo), kb));
                        const uint32_t acc = (cc | ks) ? 1u : 0u;
                        mma<KIND>(tmem, zh, smem_desc(bh + koff, kLbo, kSboB), kIdesc, acc);
                        mma<KIND>(tmem + kNbig, zl, smem_desc(bh + koff, kLbo, kSboB), kIdesc, acc);
                        mma<KIND>(tmem + kNbig, zh, smem_desc(b2 + koff, kLbo, kSboB), kIdesc, 1u);
                        if constexpr (KIND == 0) {  // bf16: Ahat mid is b2, lo is b3
                            mma<KIND>(tmem + kNbig, zl, smem_desc(b2 + koff, kLbo, kSboB), kIdesc, 1u);
                            mma<KIND>(tmem + kNbig, zh, smem_desc(b3 + koff, kLbo, kSboB), kIdesc, 1u);
                        }
                    }
                    mma_commit(&sh.bar_f[buf]);
                    if (cc >= 1) {
                        // chunk cc-1's products are done with their buffer: refill it with
                        // chunk cc-1+Nb (past the last: the first chunks of the next tile)
                        const int pb = static_cast<int>((q - 1) % S::Nb);
                        wait_f(pb);
                        const int next = cc - 1 + S::Nb;
                        if (ok) fetch(c.tc_operand, next < nch ? next : next - nch, pb);
                    }
                }
                mma_commit(&sh.bar_free[slot]);  // the slot is free once this block's products are done
            }
            if (ok) {  // the last chunk's buffer: then chunk Nb-1 of the next tile
                const int pb = static_cast<int>((q - 1) % S::Nb);
                wait_f(pb);
                if (ok) fetch(c.tc_operand, S::Nb - 1, pb);
            }
            mma_commit(&sh.bar_mma);  // arrives when every product issued above is done
            if (!ok) atomicExch(&sh.abort, 1);
          }
          __syncwarp();  // the rest of the product warp waits here, not in a poll beside the issuing lane
        }
        if (!mbar_wait(&sh.bar_mma, mma_ph & 1u)) atomicExch(&sh.abort, 2);  // 2: products may still run
        ++mma_ph;
        __syncthreads();
        if (sh.abort) break;  // an unfinished accumulator is never read or summed
        tc_fence_after();

        // ---- path sums from D1 + D2 (the first 16 warps), then values and the tile sum
        PathAcc<float> acc;
        if (warp < kEpilogueWarpsS) epilogue_dispatch<kNbig, kEpilogueWarpsS / 4>(c, tmem, acc, warp >> 2, warp & 3);
        tc_fence_before();
        finish_tile<kEpilogueWarpsS / 4>(p, c, item_acc, tile, acc, scratch);
      }
      if (sh.abort) break;  // read after a barrier: the same in every thread
      item_flush<ff>(p.tile_sums + work.item * 4, item_acc);
    }

    // the prefetched chunks, and products an expired wait left running, must
    // land before the CTA exits (bounded waits again)
    if (threadIdx.x == 0 && sh.abort == 2) mbar_wait(&sh.bar_mma, (mma_ph - 1u) & 1u);
    if (issuer && ok && loaded != nullptr) {
        for (int i = 0; i < S::Nb; ++i) wait_b(static_cast<int>((q + i) % S::Nb));
        if (!ok) atomicExch(&sh.abort, 1);
    }
    tc_fence_before();
    __syncthreads();
    if (sh.abort && threadIdx.x == 0 && p.error_flag) atomicExch(p.error_flag, QMCCPW_ERR_TIMEOUT);
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, kCols);
    }
}

// Failure-path check of the bounded wait: an mbarrier that nothing arrives at
// (count 1, no arrive, no copy), waited on with the kernels' own poll loop and
// a short limit; the wait must give up and the kernel exit normally.
__global__ void bounded_wait_probe_kernel(uint64_t limit_ns, int *status) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const bool done = mbar_wait(&bar, 0u, limit_ns);
    __syncthreads();
    if (threadIdx.x == 0) *status = done ? QMCCPW_OK : QMCCPW_ERR_TIMEOUT;
}

}  // namespace

int launch_bounded_wait_probe(uint64_t limit_ns, int *status, void *stream) {
    bounded_wait_probe_kernel<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(limit_ns, status);
    return static_cast<int>(cudaGetLastError());
}

size_t pca_tc_smem_bytes(int kind) {
    // staging of the warpgroups' partial sums (4 arrays of kM x 4 entries at most) and the
    // float-float tile sum (8 x kThreads floats)
    const size_t scratch = std::max<size_t>(16 * kM * 4, 8 * kThreads * sizeof(float));
    if (kind == 2)
        return 1024 + 2 * static_cast<size_t>(Streamed<0>::ZPart) + Streamed<0>::Nb * Streamed<0>::ChunkBytes + scratch;
    if (kind == 3)
        return 1024 + 2 * static_cast<size_t>(Streamed<1>::ZPart) + Streamed<1>::Nb * Streamed<1>::ChunkBytes + scratch;
    const size_t es = kind == 0 ? 2 : 4, parts = kind == 0 ? 3 : 2;
    return 1024 + 2 * kM * kNpad * es + parts * kNpad * kNpad * es + scratch;
}

int pca_tc_max_n(int kind) { return kind >= 2 ? kNbig : kNpad; }

int pca_tc_prepare(int kind, size_t smem_bytes) {
    const int b = static_cast<int>(smem_bytes);
    const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
    cudaError_t e = kind == 0   ? cudaFuncSetAttribute(pca_tc_kernel<0>, a, b)
                    : kind == 1 ? cudaFuncSetAttribute(pca_tc_kernel<1>, a, b)
                    : kind == 2 ? cudaFuncSetAttribute(pca_tcs_kernel<0>, a, b)
                                : cudaFuncSetAttribute(pca_tcs_kernel<1>, a, b);
    return static_cast<int>(e);
}

// Resident CTAs per SM from the kernel's resources: shared memory (dynamic,
// static and the per-block reservation), registers (allocated per warp in
// units of 256), threads and tensor-memory columns (D1 + D2 of every
// resident CTA within the SM's 512).  The runtime's occupancy query gave one
// CTA per SM for these kernels (a 152-CTA grid on 152 SMs) where the
// profiler's launch statistics show room for three, so the count is formed
// here; a grid larger than fits would only queue, the work list is dynamic.
int pca_tc_occupancy(int kind, size_t smem_bytes, int *blocks) {
    cudaFuncAttributes fa{};
    cudaError_t e = kind == 0   ? cudaFuncGetAttributes(&fa, pca_tc_kernel<0>)
                    : kind == 1 ? cudaFuncGetAttributes(&fa, pca_tc_kernel<1>)
                    : kind == 2 ? cudaFuncGetAttributes(&fa, pca_tcs_kernel<0>)
                                : cudaFuncGetAttributes(&fa, pca_tcs_kernel<1>);
    if (e != cudaSuccess) return static_cast<int>(e);
    int dev = 0, smem_sm = 0, reserved = 0, regs_sm = 0, threads_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return static_cast<int>(e);
    if ((e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&threads_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev)) != cudaSuccess)
        return static_cast<int>(e);
    const size_t per_block = smem_bytes + fa.sharedSizeBytes + static_cast<size_t>(reserved);
    const int by_smem = static_cast<int>(static_cast<size_t>(smem_sm) / per_block);
    const int threads = kind >= 2 ? kThreadsS : kThreads;
    const int regs_warp = ((fa.numRegs * 32 + 255) / 256) * 256;
    const int by_regs = regs_warp > 0 ? (regs_sm / regs_warp) / (threads / 32) : 0;
    const int by_threads = threads_sm / threads;
    const int by_tmem = 512 / (kind >= 2 ? 2 * kNbig : 2 * kNpad);
    *blocks = std::max(0, std::min(std::min(by_smem, by_regs), std::min(by_threads, by_tmem)));
    return 0;
}

int launch_pca_tc(const LaunchParams &p, int kind, size_t smem_bytes, int grid, void *stream) {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (kind == 0) pca_tc_kernel<0><<<grid, kThreads, smem_bytes, s>>>(p);
    else if (kind == 1) pca_tc_kernel<1><<<grid, kThreads, smem_bytes, s>>>(p);
    else if (kind == 2) pca_tcs_kernel<0><<<grid, kThreadsS, smem_bytes, s>>>(p);
    else pca_tcs_kernel<1><<<grid, kThreadsS, smem_bytes, s>>>(p);
    return static_cast<int>(cudaGetLastError());
}

// Host: Ahat = A / sqrt(dt) (the factor for unit spacing) split into parts
// of the operand type: hi = Ahat rounded to the grid 2^-e, e the largest
// with max|Ahat| 2^e <= 2^8 - 1/2 (bf16) or 2^11 - 1/2 (tf32), so hi is exact
// in the operand type and hi x z_hi products accumulate exactly; tf32: lo =
// the rest, rounded; bf16: mid = the rest rounded to bf16, lo = what mid
// leaves, rounded.  Layout K-major without swizzle in 8 x 16-byte core
// matrices: kinds 0 and 1 one 64 x 64 block per part, parts in order; kinds
// 2 and 3 K-chunks of 16 dimensions, each chunk all parts (256 x 16 each) in
// order, so one bulk copy brings a whole chunk.
void pca_tc_operand(int kind, int n, const std::vector<double> &A_unit, std::vector<unsigned char> &out) {
    const bool tf32 = kind == 1 || kind == 3;
    const int es = tf32 ? 4 : 2;
    const int parts = tf32 ? 2 : 3;
    const int T = 16 / es;
    const int npad = pca_tc_max_n(kind);
    const int kc = Streamed<0>::Kc;
    const size_t part_bytes = kind >= 2 ? static_cast<size_t>(npad) * kc * es : static_cast<size_t>(npad) * npad * es;
    out.assign(static_cast<size_t>(parts) * npad * npad * es, 0);
    double amax = 0.0;
    for (double a : A_unit) amax = std::max(amax, std::fabs(a));
    const double lim = tf32 ? 2047.5 : 255.5;
    const int e = amax > 0.0 ? static_cast<int>(std::floor(std::log2(lim / amax))) : 0;
    const double scale = std::ldexp(1.0, e);
    auto offset = [&](int row, int k, int part) -> size_t {
        if (kind >= 2) {
            const int c = k / kc, kk = k % kc;
            return (static_cast<size_t>(c) * parts + part) * part_bytes +
                   static_cast<size_t>(((row >> 3) * (kc / T) + kk / T) * 128 + (row & 7) * 16 + (kk % T) * es);
        }
        return part * part_bytes +
               static_cast<size_t>(((row >> 3) * (npad / T) + k / T) * 128 + (row & 7) * 16 + (k % T) * es);
    };
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < n; ++k) {
            const double a = A_unit[static_cast<size_t>(i) * n + k];
            const double h = std::nearbyint(a * scale) / scale;  // exact in 8 (11) significant bits
            if (!tf32) {
                const __nv_bfloat16 hb = __float2bfloat16_rn(static_cast<float>(h));
                const __nv_bfloat16 mb = __float2bfloat16_rn(static_cast<float>(a - h));
                const __nv_bfloat16 lb =
                    __float2bfloat16_rn(static_cast<float>(a - h - static_cast<double>(__bfloat162float(mb))));
                std::memcpy(&out[offset(i, k, 0)], &hb, 2);
                std::memcpy(&out[offset(i, k, 1)], &mb, 2);
                std::memcpy(&out[offset(i, k, 2)], &lb, 2);
            } else {
                const float hf = static_cast<float>(h);
                const float l = static_cast<float>(a - h);
                uint32_t hb, lb;
                std::memcpy(&hb, &hf, 4);
                std::memcpy(&lb, &l, 4);
                lb = (lb + 0x1000u) & 0xFFFFE000u;
                std::memcpy(&out[offset(i, k, 0)], &hb, 4);
                std::memcpy(&out[offset(i, k, 1)], &lb, 4);
            }
        }
}

}  // namespace qmccpw
