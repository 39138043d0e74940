// grad_launch.cuh -- per-precision launch helpers of the adjoint kernel (included once by
// grad_f32.cu and once by grad_f64.cu so the two precisions compile in parallel).
#pragma once

#include "ffbs_launch.cuh"
#include "grad.cuh"

namespace hqmc {

constexpr int kGradWarps = 4;

template <typename T, int L>
static cudaError_t grad_go(const DevState &st, const GradLaunch &gk, int grid, cudaStream_t s) {
    grad_kernel<T, L><<<grid, kGradWarps * 32, grad_smem_bytes_t<T, L>(kGradWarps), s>>>(st, gk);
    return cudaGetLastError();
}

template <typename T, int L>
static cudaError_t grad_occ(int *blocks) {
    const size_t sm = grad_smem_bytes_t<T, L>(kGradWarps);
    auto k = grad_kernel<T, L>;
    cudaError_t e = raise_smem_limit(k, sm);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k, kGradWarps * 32, sm);
}

template <typename T>
static cudaError_t grad_dispatch(int L, const DevState &st, const GradLaunch &gk, int grid, cudaStream_t s) {
    switch (L) {
#define HQMC_CASE(n) \
    case n: return grad_go<T, n>(st, gk, grid, s);
        HQMC_FFBS_SIZES(HQMC_CASE)
#undef HQMC_CASE
        default: return cudaErrorInvalidValue;
    }
}

template <typename T>
static cudaError_t grad_occ_dispatch(int L, int *blocks) {
    switch (L) {
#define HQMC_CASE(n) \
    case n: return grad_occ<T, n>(blocks);
        HQMC_FFBS_SIZES(HQMC_CASE)
#undef HQMC_CASE
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace hqmc
