// ffbs_wide.cu -- instantiations of the wide-lattice FFBS kernel (L = 48, 64, 128; FP32
// and FP64) and its host-side geometry.
#include "ffbs_launch.cuh"
#include "ffbs_wide.cuh"

namespace hqmc {

#define HQMC_WIDE_SIZES(X) X(48) X(64) X(128)

bool ffbs_wide_supported(int L) {
    switch (L) {
#define HQMC_CASE(n) \
    case n: return true;
        HQMC_WIDE_SIZES(HQMC_CASE)
#undef HQMC_CASE
        default: return false;
    }
}

// worldlines held by one CTA (the work unit is this many worldlines of one spin)
int ffbs_wide_wpc(int L) {
    switch (L) {
#define HQMC_CASE(n) \
    case n: return WideGeo<float, n>::WPC;
        HQMC_WIDE_SIZES(HQMC_CASE)
#undef HQMC_CASE
        default: return 0;
    }
}

template <typename T, int L>
static cudaError_t wide_occ(int *blocks) {
    if constexpr (sizeof(T) == 4) {
        cudaError_t e = raise_smem_limit(ffbs_wide_kernel<T, L, true>, WideGeo<T, L>::BYTES);
        if (e != cudaSuccess) return e;
    }
    auto k = ffbs_wide_kernel<T, L, false>;
    cudaError_t e = raise_smem_limit(k, WideGeo<T, L>::BYTES);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k, WideGeo<T, L>::NT, WideGeo<T, L>::BYTES);
}

cudaError_t ffbs_wide_occupancy(int L, bool fp64, int *blocks) {
    switch (L) {
#define HQMC_CASE(n) \
    case n: return fp64 ? wide_occ<double, n>(blocks) : wide_occ<float, n>(blocks);
        HQMC_WIDE_SIZES(HQMC_CASE)
#undef HQMC_CASE
        default: return cudaErrorInvalidValue;
    }
}

// launch only: the shared-memory limit is raised beforehand (never during stream capture)
cudaError_t launch_ffbs_wide(int L, bool fp64, const DevState &st, const FfbsLaunch &fl, int grid, cudaStream_t s) {
    switch (L) {
#define HQMC_CASE(n)                                                                                        \
    case n:                                                                                                 \
        if (fp64)                                                                                           \
            ffbs_wide_kernel<double, n, false><<<grid, WideGeo<double, n>::NT, WideGeo<double, n>::BYTES, s>>>(st, fl); \
        else if (fl.ckpt_K > 0)                                                                            \
            ffbs_wide_kernel<float, n, true><<<grid, WideGeo<float, n>::NT, WideGeo<float, n>::BYTES, s>>>(st, fl);     \
        else                                                                                                \
            ffbs_wide_kernel<float, n, false><<<grid, WideGeo<float, n>::NT, WideGeo<float, n>::BYTES, s>>>(st, fl);    \
        return cudaGetLastError();
        HQMC_WIDE_SIZES(HQMC_CASE)
#undef HQMC_CASE
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace hqmc
