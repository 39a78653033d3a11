// The fused QMC-CPW kernel for sm_103a (one launch per batch segment) and
// the reduction, statistics and set-up kernels.
//
// A launch covers the work items (contract, replicate, run of tiles) of one
// construction; each CTA takes items from an atomic counter in order, runs
// each tile of an item through the three phases of run_item (fused_body.cuh)
// and writes the item's compensated tile total to its slot.  A second kernel
// sums each replicate's item slots with compensated (Neumaier) arithmetic in
// a fixed order; a third forms mean and standard error over replicates.
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "fused_body.cuh"
#include "qmccpw_internal.h"

namespace qmccpw {

namespace {

// CONS is the construction of every contract this launch covers (the host
// launches one grid per construction over that construction's items).
// Register budget: the float PCA product's register block needs up to 128
// registers and the double forms more than 80 (two CTAs per SM); the other
// float forms fit three CTAs per SM.
template <typename T, int CONS>
__global__ void __launch_bounds__(kThreads, (sizeof(T) == 4 && CONS != QMCCPW_PCA) ? 3 : 2)
    fused_kernel(const __grid_constant__ LaunchParams p) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ WorkItem work;
    __shared__ double item_acc[8];
    item_acc_clear(item_acc);
    while (true) {
        next_work(p, work);
        if (work.item >= p.item_end) break;
        // the item stays in shared memory (`work`); tiles per replicate fit 32 bits
        for (uint32_t tile = static_cast<uint32_t>(work.tile); tile < work.tile_end; ++tile)
            run_item<T, CONS>(p.contracts[work.ci], p.sobol_table, p.sobol_shift, p.jstride, work.rep, tile,
                              p.point_k0, p.point_out, item_acc, smem);
        item_flush<PointValue<T>>(p.tile_sums + work.item * 4, item_acc);
    }
}

// ---------------------------------------------------------------------------
// per-replicate compensated reduction of the item slots, then statistics
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) reduce_kernel(const ContractDev *__restrict__ contracts,
                                                     const uint64_t *__restrict__ rep_owner,
                                                     const double *__restrict__ tile_sums,
                                                     double *__restrict__ per_rep) {
    __shared__ Neumaier part[256][4];
    const uint64_t slot = blockIdx.x;  // global replicate slot
    const ContractDev &c = contracts[rep_owner[slot]];
    const uint64_t r = slot - c.rep_base;
    const uint64_t first = c.item_base + r * static_cast<uint64_t>(c.items);
    const double v = reduce_replicate(tile_sums + first * 4, static_cast<uint64_t>(c.items), c.N, part);
    if (threadIdx.x < 4) per_rep[slot * 4 + threadIdx.x] = v;
}

__global__ void stats_kernel(const ContractDev *__restrict__ contracts, int count,
                             const double *__restrict__ per_rep, double *__restrict__ stats) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= count * 4) return;
    const int ci = t >> 2, g = t & 3;
    const ContractDev &c = contracts[ci];
    replicate_stats(per_rep + c.rep_base * 4, c.R, g, stats[ci * 8 + g], stats[ci * 8 + 4 + g]);
}

// The same statistics for replicate estimates assembled elsewhere (contract
// i's R[i] rows start at row first_row[i] of per_rep).
__global__ void gathered_stats_kernel(const double *__restrict__ per_rep, const int64_t *__restrict__ first_row,
                                      const int32_t *__restrict__ R, int count, double *__restrict__ stats) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= count * 4) return;
    const int ci = t >> 2, g = t & 3;
    replicate_stats(per_rep + first_row[ci] * 4, R[ci], g, stats[ci * 8 + g], stats[ci * 8 + 4 + g]);
}

// Copy replicate slot s of a batch (4 doubles) to row dst_row[s] of dst.
__global__ void scatter_replicates_kernel(const double *__restrict__ per_rep, const int64_t *__restrict__ dst_row,
                                          uint64_t slots, double *__restrict__ dst) {
    const uint64_t t = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x;
    if (t >= slots * 4) return;
    dst[dst_row[t >> 2] * 4 + (t & 3)] = per_rep[t];
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

size_t fused_smem_bytes(int precision, int construction, int n, int tile_log2) {
    const size_t elem = (precision == QMCCPW_FP64) ? 8 : 4;
    const size_t zw = static_cast<size_t>(1u << tile_log2) * tile_row_elems(construction, n) * elem;
    // staging of partial accumulators: up to 4 * kThreads (slot, point) entries of kStageBytes
    // (double: x, dsum, m; float: x, yw, yn, m), >= 4 * kThreads doubles for the tile sum
    const size_t red = 4 * kThreads * static_cast<size_t>(kStageBytes);
    return ((zw > red ? zw : red) + 15) & ~size_t(15);
}

// Raise each kernel's dynamic shared-memory limit to what the per-block
// opt-in maximum leaves beside that kernel's static shared memory.
template <typename T>
static cudaError_t set_limit(void (*kernel)(LaunchParams), int optin) {
    cudaFuncAttributes fa{};
    cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                optin - static_cast<int>(fa.sharedSizeBytes));
}

template <typename T>
static cudaError_t set_limit_all(int optin) {
    cudaError_t e = set_limit<T>(fused_kernel<T, QMCCPW_BB>, optin);
    if (e == cudaSuccess) e = set_limit<T>(fused_kernel<T, QMCCPW_PCA>, optin);
    if (e == cudaSuccess) e = set_limit<T>(fused_kernel<T, QMCCPW_STD>, optin);
    if (e == cudaSuccess) e = set_limit<T>(fused_kernel<T, QMCCPW_BB_LEAD>, optin);
    if (e == cudaSuccess) e = set_limit<T>(fused_kernel<T, QMCCPW_PCA_LEAD>, optin);
    return e;
}

template <typename T>
static auto fused_for(int construction) -> void (*)(LaunchParams) {
    switch (construction) {
        case QMCCPW_BB: return fused_kernel<T, QMCCPW_BB>;
        case QMCCPW_STD: return fused_kernel<T, QMCCPW_STD>;
        case QMCCPW_BB_LEAD: return fused_kernel<T, QMCCPW_BB_LEAD>;
        case QMCCPW_PCA_LEAD: return fused_kernel<T, QMCCPW_PCA_LEAD>;
        default: return fused_kernel<T, QMCCPW_PCA>;
    }
}

int fused_set_smem_limit(int precision, size_t optin_bytes) {
    const int b = static_cast<int>(optin_bytes);
    return static_cast<int>(precision == QMCCPW_FP64 ? set_limit_all<double>(b) : set_limit_all<float>(b));
}

int fused_occupancy(int precision, int construction, size_t smem_bytes, int *blocks_per_sm) {
    const void *f = precision == QMCCPW_FP64 ? reinterpret_cast<const void *>(fused_for<double>(construction))
                                             : reinterpret_cast<const void *>(fused_for<float>(construction));
    return static_cast<int>(cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, f, kThreads, smem_bytes));
}

int launch_fused(const LaunchParams &p, int precision, int construction, size_t smem_bytes, int grid, void *stream) {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (precision == QMCCPW_FP64) fused_for<double>(construction)<<<grid, kThreads, smem_bytes, s>>>(p);
    else fused_for<float>(construction)<<<grid, kThreads, smem_bytes, s>>>(p);
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

int launch_gathered_stats(const double *per_rep, const int64_t *first_row, const int32_t *R, int count,
                          double *stats, void *stream) {
    gathered_stats_kernel<<<(count * 4 + 127) / 128, 128, 0, static_cast<cudaStream_t>(stream)>>>(
        per_rep, first_row, R, count, stats);
    return static_cast<int>(cudaGetLastError());
}

int launch_scatter_replicates(const double *per_rep, const int64_t *dst_row, uint64_t slots, double *dst,
                              void *stream) {
    scatter_replicates_kernel<<<static_cast<unsigned>((slots * 4 + 255) / 256), 256, 0,
                                static_cast<cudaStream_t>(stream)>>>(per_rep, dst_row, slots, dst);
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
