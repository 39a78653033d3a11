// PCA construction on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// W~ = A z with A A^T = Sigma (eq. WboldTilde); for equal spacing
// A = sqrt(dt) * Ahat where Ahat (the factor for dt = 1) depends on n only.
// One CTA (256 threads) per work item of 128 points:
//   1. Sobol' + inverse normal as in the CUDA-core kernel, but z is split
//      into hi + lo parts (bf16 or tf32) written straight into the K-major
//      canonical operand layout (8-row x 16-byte core matrices).
//   2. One thread issues D = Z_hi Ahat_hi^T + Z_lo Ahat_hi^T + Z_hi Ahat_lo^T
//      (the 3-term split product, FP32 accumulation in tensor memory),
//      M = 128 points, N = 64 dates, K = 64 dimensions; Ahat hi/lo stays
//      resident in shared memory (staged by a bulk TMA copy).
//   3. The epilogue reads D with tcgen05.ld (warp w owns TMEM lanes
//      32(w%4)..+31, warpgroup w/4 one half of the columns), scales by
//      sqrt(dt) and forms the path sums; then the conditional step and the
//      tile sum exactly as in the CUDA-core kernel.
// Every wait on an mbarrier is bounded: on expiry the kernel records an
// error code, releases its tensor memory and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <vector>

#include "qmccpw_internal.h"
#include "qmccpw_device.cuh"

namespace qmccpw {
namespace {

constexpr int kM = 128;        // points per tile (UMMA M)
constexpr int kNpad = 64;      // dates and dimensions, padded (UMMA N and K)
constexpr uint64_t kWaitLimitNs = 2000000000ull;  // give up on an mbarrier after 2 s

// ---- PTX wrappers ---------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// Poll the barrier for the given phase parity; false if kWaitLimitNs passed.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
    const uint32_t addr = smem_u32(bar);
    const uint64_t start = global_ns();
    while (true) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(addr), "r"(parity)
            : "memory");
        if (done) return true;
        if (global_ns() - start > kWaitLimitNs) return false;
    }
}

__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t *dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst_smem)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// Shared-memory matrix descriptor, K-major, no swizzle: core matrices of
// 8 rows x 16 bytes; LBO = distance of K-adjacent core matrices, SBO = of
// row-adjacent (8-row) groups; bits 46-48 = 0b001.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= static_cast<uint64_t>((addr & 0x3FFFFu) >> 4);
    d |= static_cast<uint64_t>((lbo & 0x3FFFFu) >> 4) << 16;
    d |= static_cast<uint64_t>((sbo & 0x3FFFFu) >> 4) << 32;
    d |= static_cast<uint64_t>(1) << 46;
    return d;  // base offset 0, relative LBO mode, no swizzle
}

// Instruction descriptor: FP32 accumulate, A and B of format `fmt`
// (kind::f16: 1 = bf16; kind::tf32: 2 = tf32), both K-major, M = 128, N = 64.
__host__ __device__ constexpr uint32_t instr_desc(uint32_t fmt, int n = kNpad) {
    return (1u << 4) | (fmt << 7) | (fmt << 10) | (static_cast<uint32_t>(n >> 3) << 17) |
           (static_cast<uint32_t>(kM >> 4) << 24);
}

template <int KIND>
__device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t accum) {
    if constexpr (KIND == 0) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
            : "memory");
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
            : "memory");
    }
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// ---- operand element addressing ----------------------------------------------
// Element (row, k) of a K-major operand with kNpad columns of ESIZE bytes:
// core matrix (row/8, k/T) of 128 bytes, T = 16/ESIZE elements per row.
template <int ESIZE, int NPAD = kNpad>
__device__ __forceinline__ uint32_t operand_offset(int row, int k) {
    constexpr int T = 16 / ESIZE;
    return static_cast<uint32_t>(((row >> 3) * (NPAD / T) + k / T) * 128 + (row & 7) * 16 + (k % T) * ESIZE);
}

// hi + lo split of a float for the 3-term product
template <int KIND>
__device__ __forceinline__ void split_store(unsigned char *hi_base, unsigned char *lo_base, uint32_t off, float z) {
    if constexpr (KIND == 0) {
        const __nv_bfloat16 h = __float2bfloat16_rn(z);
        const __nv_bfloat16 l = __float2bfloat16_rn(z - __bfloat162float(h));
        *reinterpret_cast<__nv_bfloat16 *>(hi_base + off) = h;
        *reinterpret_cast<__nv_bfloat16 *>(lo_base + off) = l;
    } else {
        // tf32 keeps 10 explicit mantissa bits: round to nearest at bit 13
        const uint32_t b = __float_as_uint(z);
        const uint32_t hb = (b + 0x1000u) & 0xFFFFE000u;
        const float h = __uint_as_float(hb);
        const float l = z - h;
        const uint32_t lb = (__float_as_uint(l) + 0x1000u) & 0xFFFFE000u;
        *reinterpret_cast<uint32_t *>(hi_base + off) = hb;
        *reinterpret_cast<uint32_t *>(lo_base + off) = lb;
    }
}

template <int KIND, int TYPE, int NPAD = kNpad>
__device__ void epilogue_sums(const ContractDev &c, uint32_t tmem, PathAcc<float> &acc, int point) {
    const int warp = threadIdx.x >> 5;
    const int half = warp >> 2;                 // warpgroup: which half of the dates
    const uint32_t lane_base = static_cast<uint32_t>(32 * (warp & 3)) << 16;
    const float sdt_hi = c.ff_sqrt_t1[0], sdt_lo = c.ff_sqrt_t1[1];
    const float omega = static_cast<float>(c.omega), sigma = static_cast<float>(c.sigma), dt = static_cast<float>(c.dt);
    acc.init(TYPE, half == 0);
#pragma unroll
    for (int blk = 0; blk < NPAD / 32; ++blk) {
        const int col = half * (NPAD / 2) + blk * 16;
        float d[16];
        tmem_ld16(tmem + lane_base + static_cast<uint32_t>(col), d);
        const float s0 = static_cast<float>(col + 1) * dt;
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const int date = col + i + 1;  // W~ at s_date
            if (date <= c.n)
                acc.template add<TYPE>(date, fmaf(d[i], sdt_hi, d[i] * sdt_lo), omega, sigma, fmaf(static_cast<float>(i), dt, s0));
        }
    }
    (void)point;
}

struct TcShared {
    uint64_t bar_b, bar_mma;
    uint32_t tmem_addr;
    int32_t loaded_n;
    int32_t abort;
};

template <int KIND>
__global__ void __launch_bounds__(kThreads, 2) pca_tc_kernel(const __grid_constant__ LaunchParams p) {
    constexpr int ES = KIND == 0 ? 2 : 4;                  // element bytes
    constexpr uint32_t kOpBytesZ = kM * kNpad * ES;        // one split part of Z
    constexpr uint32_t kOpBytesB = kNpad * kNpad * ES;     // one split part of Ahat
    constexpr uint32_t kIdesc = instr_desc(KIND == 0 ? 1u : 2u);
    constexpr uint32_t kLbo = 128, kSbo = (kNpad / (16 / ES)) * 128;

    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char *z_hi = smem;
    unsigned char *z_lo = z_hi + kOpBytesZ;
    unsigned char *b_hi = z_lo + kOpBytesZ;                // b_lo follows b_hi (one bulk copy)
    unsigned char *b_lo = b_hi + kOpBytesB;
    unsigned char *scratch = b_lo + kOpBytesB;             // partial sums, tile values
    __shared__ TcShared sh;

    const int warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        mbar_init(&sh.bar_b, 1);
        mbar_init(&sh.bar_mma, 1);
        sh.loaded_n = -1;
        sh.abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tmem_alloc(&sh.tmem_addr, kNpad);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sh.tmem_addr;
    // padding columns (k >= n) of Z are never written by the Sobol' phase
    for (uint32_t i = threadIdx.x; i < 2 * kOpBytesZ / 4; i += kThreads) reinterpret_cast<uint32_t *>(z_hi)[i] = 0u;

    uint32_t b_phase = 0, mma_phase = 0;
    __shared__ uint64_t next_item;
    while (true) {
        // dynamic schedule: CTAs take the next item as they finish one (the
        // result of an item never depends on which CTA ran it)
        if (threadIdx.x == 0) next_item = p.item_begin + atomicAdd(p.work_counter, 1ull);
        __syncthreads();
        const uint64_t item = next_item;
        if (item >= p.item_end) break;
        const int ci = find_contract(p.item_base, p.count, item);
        const ContractDev &c = p.contracts[ci];
        const int n = c.n;
        const uint64_t local = item - c.item_base;
        const uint32_t rep = static_cast<uint32_t>(local / static_cast<uint64_t>(c.tiles)) + p.rep_offset;
        const uint64_t tile = local % static_cast<uint64_t>(c.tiles);

        // ---- Ahat (hi, lo) for this n: one bulk copy when n changes
        __syncthreads();
        if (sh.loaded_n != n) {
            if (threadIdx.x == 0) {
                mbar_expect_tx(&sh.bar_b, 2 * kOpBytesB);
                bulk_copy_g2s(b_hi, c.tc_operand, 2 * kOpBytesB, &sh.bar_b);
            }
            if (!mbar_wait(&sh.bar_b, b_phase & 1u)) atomicExch(&sh.abort, 1);
            ++b_phase;
            __syncthreads();
            if (threadIdx.x == 0) sh.loaded_n = n;
        }
        if (sh.abort) break;

        // ---- phase 1: Sobol' + inverse normal -> split operand
        const uint32_t *tab = p.sobol_table + static_cast<size_t>(rep) * 32u * p.jstride;
        const uint32_t *shf = p.sobol_shift + static_cast<size_t>(rep) * p.jstride;
        const int chunk = 1 << c.chunk_log2;
        const int nchunks = kM >> c.chunk_log2;
        const bool by_warp = n >= 32;
        const int step = by_warp ? kThreads / 32 : kThreads;
        const int first = by_warp ? (threadIdx.x >> 5) : static_cast<int>(threadIdx.x);
        const int work = by_warp ? nchunks * ((n + 31) >> 5) : nchunks * n;
        for (int it = first; it < work; it += step) {
            int j, ch;
            if (by_warp) {
                const int per = (n + 31) >> 5;
                ch = it / per;
                j = (it - ch * per) * 32 + (threadIdx.x & 31);
                if (j >= n) continue;
            } else {
                j = it % n;
                ch = it / n;
            }
            const uint64_t first_local = tile * kM + static_cast<uint64_t>(ch) * chunk;
            const int len = first_local >= c.N ? 0 : static_cast<int>(min(static_cast<uint64_t>(chunk), c.N - first_local));
            const int row0 = ch * chunk;
            if (len > 0) {
                const uint32_t k0 = static_cast<uint32_t>(p.point_k0 + first_local);
                uint32_t y = sobol_first(tab, p.jstride, j, __ldg(shf + j), k0);
                split_store<KIND>(z_hi, z_lo, operand_offset<ES>(row0, j), Arith<float>::inv_normal(y));
                for (int s = 1; s < len; ++s) {
                    y ^= __ldg(tab + (__ffs(k0 + s) - 1) * p.jstride + j);
                    split_store<KIND>(z_hi, z_lo, operand_offset<ES>(row0 + s, j), Arith<float>::inv_normal(y));
                }
            }
            for (int s = len; s < chunk; ++s) split_store<KIND>(z_hi, z_lo, operand_offset<ES>(row0 + s, j), 0.0f);
        }
        fence_proxy_async();  // generic-proxy stores -> visible to the tensor core
        tc_fence_before();
        __syncthreads();
        tc_fence_after();

        // ---- phase 2: the split product into tensor memory
        if (threadIdx.x == 0) {
            const uint32_t za[2] = {smem_u32(z_hi), smem_u32(z_lo)};
            const uint32_t ba[2] = {smem_u32(b_hi), smem_u32(b_lo)};
            const int pa[3] = {0, 1, 0}, pb[3] = {0, 0, 1};  // (hi,hi), (lo,hi), (hi,lo)
            uint32_t accum = 0;
#pragma unroll
            for (int t = 0; t < 3; ++t)
#pragma unroll
                for (int ks = 0; ks < kNpad / (32 / ES); ++ks) {  // K per instruction: 16 bf16 or 8 tf32 = 32 bytes
                    const uint32_t koff = static_cast<uint32_t>(ks) * 256u;
                    mma<KIND>(tmem, smem_desc(za[pa[t]] + koff, kLbo, kSbo), smem_desc(ba[pb[t]] + koff, kLbo, kSbo),
                              kIdesc, accum);
                    accum = 1;
                }
            mma_commit(&sh.bar_mma);
        }
        if (!mbar_wait(&sh.bar_mma, mma_phase & 1u)) atomicExch(&sh.abort, 1);
        ++mma_phase;
        tc_fence_after();

        // ---- phase 3: path sums from D, merged across the two warpgroups
        PathAcc<float> acc;
        const int point = 32 * (warp & 3) + (threadIdx.x & 31);
        switch (c.type) {
            case QMCCPW_ARITH_ASIAN_CALL: epilogue_sums<KIND, QMCCPW_ARITH_ASIAN_CALL>(c, tmem, acc, point); break;
            case QMCCPW_BINARY_ASIAN: epilogue_sums<KIND, QMCCPW_BINARY_ASIAN>(c, tmem, acc, point); break;
            case QMCCPW_LOOKBACK_FIXED_CALL: epilogue_sums<KIND, QMCCPW_LOOKBACK_FIXED_CALL>(c, tmem, acc, point); break;
            default: epilogue_sums<KIND, QMCCPW_GEOMETRIC_ASIAN_CALL>(c, tmem, acc, point); break;
        }
        tc_fence_before();
        stage_partial<float>(scratch, kM, warp >> 2, point, acc);
        __syncthreads();
        ff v[4] = {{0.0f, 0.0f}, {0.0f, 0.0f}, {0.0f, 0.0f}, {0.0f, 0.0f}};
        const uint64_t local_point = tile * kM + point;
        if (warp < 4) {
            merge_partials<float>(scratch, kM, 2, point, c.type, acc);
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
        tile_sum(p, item, v, scratch);
    }

    // release tensor memory (also after an abort)
    tc_fence_before();
    __syncthreads();
    if (sh.abort && threadIdx.x == 0 && p.error_flag) atomicExch(p.error_flag, QMCCPW_ERR_TIMEOUT);
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, kNpad);
    }
}

}  // namespace

size_t pca_tc_smem_bytes(int kind) {
    const size_t es = kind == 0 ? 2 : 4;
    const size_t ops = 2 * kM * kNpad * es + 2 * kNpad * kNpad * es;
    const size_t scratch = 4 * kThreads * sizeof(double) > 4 * kThreads * 12 ? 4 * kThreads * sizeof(double)
                                                                            : 4 * kThreads * 12;
    return ops + scratch;
}

int pca_tc_npad() { return kNpad; }

int pca_tc_prepare(int kind, size_t smem_bytes) {
    cudaError_t e = kind == 0 ? cudaFuncSetAttribute(pca_tc_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                     static_cast<int>(smem_bytes))
                              : cudaFuncSetAttribute(pca_tc_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                     static_cast<int>(smem_bytes));
    return static_cast<int>(e);
}

int pca_tc_occupancy(int kind, size_t smem_bytes, int *blocks) {
    cudaError_t e = kind == 0
                        ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, pca_tc_kernel<0>, kThreads, smem_bytes)
                        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, pca_tc_kernel<1>, kThreads, smem_bytes);
    return static_cast<int>(e);
}

int launch_pca_tc(const LaunchParams &p, int kind, size_t smem_bytes, int grid, void *stream) {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (kind == 0) pca_tc_kernel<0><<<grid, kThreads, smem_bytes, s>>>(p);
    else pca_tc_kernel<1><<<grid, kThreads, smem_bytes, s>>>(p);
    return static_cast<int>(cudaGetLastError());
}

// Host: Ahat = A / sqrt(dt) (the factor for unit spacing), split into hi + lo
// of the operand type and laid out K-major in 8 x 16-byte core matrices.
void pca_tc_operand(int kind, int n, const std::vector<double> &A_unit, std::vector<unsigned char> &out) {
    const int es = kind == 0 ? 2 : 4;
    const int T = 16 / es;
    const size_t part = static_cast<size_t>(kNpad) * kNpad * es;
    out.assign(2 * part, 0);
    auto offset = [&](int row, int k) {
        return static_cast<size_t>(((row >> 3) * (kNpad / T) + k / T) * 128 + (row & 7) * 16 + (k % T) * es);
    };
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < n; ++k) {
            const double a = A_unit[static_cast<size_t>(i) * n + k];
            const size_t off = offset(i, k);
            if (kind == 0) {
                const __nv_bfloat16 h = __float2bfloat16_rn(static_cast<float>(a));
                const __nv_bfloat16 l = __float2bfloat16_rn(static_cast<float>(a - static_cast<double>(__bfloat162float(h))));
                std::memcpy(&out[off], &h, 2);
                std::memcpy(&out[part + off], &l, 2);
            } else {
                const float af = static_cast<float>(a);
                uint32_t b;
                std::memcpy(&b, &af, 4);
                const uint32_t hb = (b + 0x1000u) & 0xFFFFE000u;
                float h;
                std::memcpy(&h, &hb, 4);
                const float l = static_cast<float>(a - static_cast<double>(h));
                uint32_t lb;
                std::memcpy(&lb, &l, 4);
                lb = (lb + 0x1000u) & 0xFFFFE000u;
                std::memcpy(&out[off], &hb, 4);
                std::memcpy(&out[part + off], &lb, 4);
            }
        }
}

}  // namespace qmccpw
