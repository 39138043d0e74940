// grad_wide.cu -- instantiations of the wide-lattice adjoint (L = 48, 64, 128; FP32, FP64).
#include "ffbs_launch.cuh"
#include "grad_wide.cuh"

namespace hqmc {


template <typename T, int L>
static cudaError_t gw_occ(int *blocks) {
    auto k = grad_wide_kernel<T, L>;
    cudaError_t e = raise_smem_limit(k, WideGeo<T, L>::BYTES);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k, WideGeo<T, L>::NT, WideGeo<T, L>::BYTES);
}

cudaError_t grad_wide_occupancy(int L, bool fp64, int *blocks) {
    switch (L) {
#define HQMC_CASE(n) \
    case n: return fp64 ? gw_occ<double, n>(blocks) : gw_occ<float, n>(blocks);
        HQMC_WIDE_SIZES(HQMC_CASE)
#undef HQMC_CASE
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_grad_wide(int L, bool fp64, const DevState &st, const GradLaunch &gk, int grid, cudaStream_t s) {
    switch (L) {
#define HQMC_CASE(n)                                                                                    \
    case n:                                                                                             \
        if (fp64)                                                                                       \
            grad_wide_kernel<double, n><<<grid, WideGeo<double, n>::NT, WideGeo<double, n>::BYTES, s>>>(st, gk); \
        else                                                                                            \
            grad_wide_kernel<float, n><<<grid, WideGeo<float, n>::NT, WideGeo<float, n>::BYTES, s>>>(st, gk);    \
        return cudaGetLastError();
        HQMC_WIDE_SIZES(HQMC_CASE)
#undef HQMC_CASE
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace hqmc
