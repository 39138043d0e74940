// ffbs_launch.cuh -- per-precision launch helpers of the FFBS kernel (included by
// ffbs_f32.cu, ffbs_f64.cu and their Gaussian-field twins ffbs_f32g.cu, ffbs_f64g.cu, so
// the four compile in parallel).
#pragma once

#include "ffbs.cuh"

namespace hqmc {

#define HQMC_FFBS_SIZES(X) X(2) X(3) X(4) X(6) X(8) X(12) X(16) X(24) X(32)

// launch only: the shared-memory attribute is set beforehand by ffbs_occ (never
// during stream capture)
template <typename T, int L, bool G>
static cudaError_t ffbs_go(const DevState &st, const FfbsLaunch &fl, int grid, int wpc, cudaStream_t s) {
    const size_t sm = ffbs_smem_bytes_t<T, L>(wpc);
    if (fl.stencil) {
        if (fl.general) ffbs_kernel<T, L, true, true, G><<<grid, wpc * 32, sm, s>>>(st, fl);
        else ffbs_kernel<T, L, false, true, G><<<grid, wpc * 32, sm, s>>>(st, fl);
    } else {
        if (fl.general) ffbs_kernel<T, L, true, false, G><<<grid, wpc * 32, sm, s>>>(st, fl);
        else ffbs_kernel<T, L, false, false, G><<<grid, wpc * 32, sm, s>>>(st, fl);
    }
    return cudaGetLastError();
}

// Raises a kernel's dynamic shared-memory limit to at least `bytes`, never lowers it: the
// limit belongs to the whole process, and another context (or the no-allocation entry
// point) may launch the same kernel with a wider CTA.
template <typename K>
static cudaError_t raise_smem_limit(K kernel, size_t bytes) {
    cudaFuncAttributes fa{};
    cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
    if (e != cudaSuccess) return e;
    if (size_t(fa.maxDynamicSharedSizeBytes) >= bytes) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes));
}

// raises the kernel's dynamic shared-memory limit as needed and reports resident CTAs per SM
template <typename T, int L, bool G>
static cudaError_t ffbs_occ(int wpc, int *blocks) {
    const size_t sm = ffbs_smem_bytes_t<T, L>(wpc);
    cudaError_t e = cudaSuccess;
    for (auto kx : {ffbs_kernel<T, L, true, false, G>, ffbs_kernel<T, L, true, true, G>, ffbs_kernel<T, L, false, true, G>}) {
        e = raise_smem_limit(kx, sm);
        if (e != cudaSuccess) return e;
    }
    auto k = ffbs_kernel<T, L, false, false, G>;
    e = raise_smem_limit(k, sm);
    if (e != cudaSuccess) return e;
    // both instantiations are held to the same launch bounds; the closed-loop one sizes the grid
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k, wpc * 32, sm);
}

template <typename T, bool G>
static cudaError_t ffbs_dispatch(int L, const DevState &st, const FfbsLaunch &fl, int grid, int wpc,
                                 cudaStream_t s) {
    switch (L) {
#define HQMC_CASE(n) \
    case n: return ffbs_go<T, n, G>(st, fl, grid, wpc, s);
        HQMC_FFBS_SIZES(HQMC_CASE)
#undef HQMC_CASE
        default: return cudaErrorInvalidValue;
    }
}

template <typename T, bool G>
static cudaError_t ffbs_occ_dispatch(int L, int wpc, int *blocks) {
    switch (L) {
#define HQMC_CASE(n) \
    case n: return ffbs_occ<T, n, G>(wpc, blocks);
        HQMC_FFBS_SIZES(HQMC_CASE)
#undef HQMC_CASE
        default: return cudaErrorInvalidValue;
    }
}

template <typename T>
static size_t ffbs_smem_dispatch(int L, int wpc) {
    switch (L) {
#define HQMC_CASE(n) \
    case n: return ffbs_smem_bytes_t<T, n>(wpc);
        HQMC_FFBS_SIZES(HQMC_CASE)
#undef HQMC_CASE
        default: return 0;
    }
}

}  // namespace hqmc
