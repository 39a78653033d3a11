// The FP64 serving kernel (serve_impl.cuh).
#include "serve_impl.cuh"

namespace qmccpw {

int serve_f64_prepare(size_t optin_bytes) { return serve_prepare_kernel(serve_kernel<double, true>, optin_bytes); }

int serve_f64_occupancy(size_t smem_bytes, int *blocks_per_sm) {
    return static_cast<int>(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        blocks_per_sm, reinterpret_cast<const void *>(serve_kernel<double, true>), kThreads, smem_bytes));
}

int serve_f64_launch(const ServeParams &p, size_t smem_bytes, int grid, void *stream) {
    return serve_launch_kernel(serve_kernel<double, true>, p, smem_bytes, grid, stream);
}

}  // namespace qmccpw
