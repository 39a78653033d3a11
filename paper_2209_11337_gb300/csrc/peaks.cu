// Pipe micro-benchmarks: the issue rates that bound the fused kernels, timed
// with CUDA events on this GPU (the roofline denominators of the float and
// double paths and of the tensor-core product).  Each kernel runs long
// chains of independent operations of one kind, enough of them per warp and
// enough warps per SM that the pipe, not latency, sets the rate; the result
// is folded into a value that is stored only under a condition that never
// holds, so the compiler keeps every operation.
//   FP32 FFMA and packed FFMA2 (2 and 4 flops per instruction), FP64 DFMA,
//   the SFU approximations ex2 / lg2 / rcp, and tcgen05.mma kind::f16 (bf16)
//   and kind::tf32 with M = 128, N = 256, FP32 accumulation in tensor memory.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "qmccpw_internal.h"
#include "tc_ptx.cuh"

namespace qmccpw {
namespace {

constexpr int kChains = 8;      // independent chains per thread
constexpr int kUnroll = 16;     // chain steps per loop iteration

__global__ void __launch_bounds__(256) ffma_kernel(float b, float c, int iters, float *sink) {
    float x[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = 1.0f + 1e-3f * static_cast<float>(threadIdx.x + i);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int i = 0; i < kChains; ++i) x[i] = fmaf(x[i], b, c);
    }
    float s = 0.0f;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += x[i];
    if (s == 1234.5f) sink[threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) ffma2_kernel(float b, float c, int iters, float *sink) {
    float2 x[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = make_float2(1.0f + 1e-3f * static_cast<float>(threadIdx.x + i), 1.5f);
    const float2 b2 = make_float2(b, b), c2 = make_float2(c, c);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int i = 0; i < kChains; ++i) x[i] = __ffma2_rn(x[i], b2, c2);
    }
    float s = 0.0f;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += x[i].x + x[i].y;
    if (s == 1234.5f) sink[threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) dfma_kernel(double b, double c, int iters, float *sink) {
    double x[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = 1.0 + 1e-3 * static_cast<double>(threadIdx.x + i);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int i = 0; i < kChains; ++i) x[i] = fma(x[i], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += x[i];
    if (s == 1234.5) sink[threadIdx.x] = static_cast<float>(s);
}

// SFU chains: x <- 2^-x (fixed point ~0.64), x <- log2(x) + 2 (fixed point 4),
// x <- 1/x + 1/2 (fixed point ~1.28); the adds run on the FMA pipe, at
// several times the SFU rate.
template <int OP>
__device__ __forceinline__ float sfu_step(float x) {
    float y;
    if constexpr (OP == 0) {
        asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(-x));
    } else if constexpr (OP == 1) {
        asm volatile("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
        y += 2.0f;
    } else {
        asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
        y += 0.5f;
    }
    return y;
}

template <int OP>
__global__ void __launch_bounds__(256) sfu_kernel(int iters, float *sink) {
    float x[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = 1.5f + 1e-3f * static_cast<float>(threadIdx.x + i);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int i = 0; i < kChains; ++i) x[i] = sfu_step<OP>(x[i]);
    }
    float s = 0.0f;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += x[i];
    if (s == 1234.5f) sink[threadIdx.x] = s;
}

// tcgen05: one thread per CTA issues `iters` products D += A B^T (M = 128,
// N = 256, K = 16 bf16 or 8 tf32: 32 bytes of K), A and B K-major without
// swizzle in shared memory (contents irrelevant to the rate: zeros), D in
// 256 tensor-memory columns (two CTAs per SM fill the 512).  The wait for
// the last product is bounded; on expiry the kernel records an error.
constexpr int kTcM = 128, kTcN = 256;

template <int KIND>
__global__ void __launch_bounds__(128) tc_kernel(int iters, int *error_flag) {
    __shared__ __align__(1024) unsigned char a[kTcM * 32];
    __shared__ __align__(1024) unsigned char b[kTcN * 32];
    __shared__ uint64_t bar;
    __shared__ uint32_t tmem_addr;
    for (int i = threadIdx.x; i < kTcM * 8; i += blockDim.x) reinterpret_cast<uint32_t *>(a)[i] = 0u;
    for (int i = threadIdx.x; i < kTcN * 8; i += blockDim.x) reinterpret_cast<uint32_t *>(b)[i] = 0u;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (threadIdx.x < 32) tmem_alloc(&tmem_addr, kTcN);
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_addr;
    if (threadIdx.x == 0) {
        // 8-row groups 256 bytes apart (two core matrices along K), K-adjacent core matrices 128 bytes apart
        const uint64_t ad = smem_desc(smem_u32(a), 128, 256), bd = smem_desc(smem_u32(b), 128, 256);
        constexpr uint32_t idesc = instr_desc(KIND == 0 ? 1u : 2u, kTcN, kTcM);
        for (int i = 0; i < iters; ++i) mma<KIND>(tmem, ad, bd, idesc, i > 0 ? 1u : 0u);
        mma_commit(&bar);
        if (!mbar_wait(&bar, 0u) && error_flag) atomicExch(error_flag, QMCCPW_ERR_TIMEOUT);
    }
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x < 32) {
        tc_fence_after();
        tmem_dealloc(tmem, kTcN);
    }
}

struct Timer {
    cudaEvent_t a = nullptr, b = nullptr;
    Timer() {
        cudaEventCreate(&a);
        cudaEventCreate(&b);
    }
    ~Timer() {
        cudaEventDestroy(a);
        cudaEventDestroy(b);
    }
};

// best of `reps` timed launches (after one warm-up), in seconds
template <typename Launch>
cudaError_t best_time(Launch &&launch, int reps, double *sec) {
    Timer t;
    launch();
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return e;
    double best = 1e30;
    for (int r = 0; r < reps; ++r) {
        cudaEventRecord(t.a);
        launch();
        cudaEventRecord(t.b);
        if ((e = cudaEventSynchronize(t.b)) != cudaSuccess) return e;
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, t.a, t.b);
        best = std::min(best, static_cast<double>(ms) * 1e-3);
    }
    *sec = best;
    return cudaGetLastError();
}

}  // namespace

int measure_pipe_peaks(int device, qmccpw_pipe_peaks *out) {
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return static_cast<int>(e);
    int sms = 0;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device)) != cudaSuccess)
        return static_cast<int>(e);
    float *sink = nullptr;
    int *flag = nullptr;
    if ((e = cudaMalloc(&sink, 1024 * sizeof(float))) != cudaSuccess) return static_cast<int>(e);
    if ((e = cudaMalloc(&flag, sizeof(int))) != cudaSuccess) {
        cudaFree(sink);
        return static_cast<int>(e);
    }
    cudaMemset(flag, 0, sizeof(int));
    const int grid = sms * 8, threads = 256, reps = 5;
    const double thr = static_cast<double>(grid) * threads;
    const double per_iter = static_cast<double>(kChains) * kUnroll;  // operations per thread per iteration
    double s = 0.0;
    const int it32 = 4096, it64 = 128, itsfu = 1024;
    do {
        if ((e = best_time([&] { ffma_kernel<<<grid, threads>>>(0.999f, 1e-3f, it32, sink); }, reps, &s))) break;
        out->fp32_fma_tflops = 2.0 * per_iter * it32 * thr / s * 1e-12;
        if ((e = best_time([&] { ffma2_kernel<<<grid, threads>>>(0.999f, 1e-3f, it32 / 2, sink); }, reps, &s))) break;
        out->fp32_fma2_tflops = 4.0 * per_iter * (it32 / 2) * thr / s * 1e-12;
        if ((e = best_time([&] { dfma_kernel<<<grid, threads>>>(0.999, 1e-3, it64, sink); }, reps, &s))) break;
        out->fp64_fma_tflops = 2.0 * per_iter * it64 * thr / s * 1e-12;
        if ((e = best_time([&] { sfu_kernel<0><<<grid, threads>>>(itsfu, sink); }, reps, &s))) break;
        out->sfu_ex2_gops = per_iter * itsfu * thr / s * 1e-9;
        if ((e = best_time([&] { sfu_kernel<1><<<grid, threads>>>(itsfu, sink); }, reps, &s))) break;
        out->sfu_lg2_gops = per_iter * itsfu * thr / s * 1e-9;
        if ((e = best_time([&] { sfu_kernel<2><<<grid, threads>>>(itsfu, sink); }, reps, &s))) break;
        out->sfu_rcp_gops = per_iter * itsfu * thr / s * 1e-9;
        // 100 KB of (unused) dynamic shared memory keeps two CTAs per SM, the
        // two that fill its 512 tensor-memory columns
        const int tc_grid = 2 * sms, tc_iters = 4096, tc_smem = 100 * 1024;
        if ((e = cudaFuncSetAttribute(tc_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, tc_smem)) ||
            (e = cudaFuncSetAttribute(tc_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, tc_smem)))
            break;
        const double mma_flops = 2.0 * kTcM * kTcN * 16;  // one kind::f16 product (K = 16)
        if ((e = best_time([&] { tc_kernel<0><<<tc_grid, 128, tc_smem>>>(tc_iters, flag); }, reps, &s))) break;
        out->tc_bf16_tflops = mma_flops * tc_iters * tc_grid / s * 1e-12;
        if ((e = best_time([&] { tc_kernel<1><<<tc_grid, 128, tc_smem>>>(tc_iters, flag); }, reps, &s))) break;
        out->tc_tf32_tflops = 0.5 * mma_flops * tc_iters * tc_grid / s * 1e-12;  // K = 8
    } while (false);
    int status = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&status, flag, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(sink);
    cudaFree(flag);
    if (e != cudaSuccess) return static_cast<int>(e);
    return status ? -status : 0;
}

}  // namespace qmccpw
