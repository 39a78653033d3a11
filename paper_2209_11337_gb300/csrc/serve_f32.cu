// The MIXED-precision serving kernels (serve_impl.cuh): with the PCA
// product (two CTAs per SM) and without it (three).
#include "serve_impl.cuh"

namespace qmccpw {

int serve_f32_prepare(bool with_pca, size_t optin_bytes) {
    return with_pca ? serve_prepare_kernel(serve_kernel<float, true>, optin_bytes)
                    : serve_prepare_kernel(serve_kernel<float, false>, optin_bytes);
}

int serve_f32_occupancy(bool with_pca, size_t smem_bytes, int *blocks_per_sm) {
    const void *f = with_pca ? reinterpret_cast<const void *>(serve_kernel<float, true>)
                             : reinterpret_cast<const void *>(serve_kernel<float, false>);
    return static_cast<int>(cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, f, kThreads, smem_bytes));
}

int serve_f32_launch(const ServeParams &p, bool with_pca, size_t smem_bytes, int grid, void *stream) {
    return with_pca ? serve_launch_kernel(serve_kernel<float, true>, p, smem_bytes, grid, stream)
                    : serve_launch_kernel(serve_kernel<float, false>, p, smem_bytes, grid, stream);
}

}  // namespace qmccpw
