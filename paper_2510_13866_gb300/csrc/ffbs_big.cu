// ffbs_big.cu -- instantiations of the wide-lattice FFBS kernel (FP32, L = 48, 64, 128).
#include "ffbs_big.cuh"

namespace hqmc {

#define HQMC_BIG_SIZES(X) X(48) X(64) X(128)

bool ffbs_big_supported(int L) {
    switch (L) {
#define HQMC_CASE(n) \
    case n: return true;
        HQMC_BIG_SIZES(HQMC_CASE)
#undef HQMC_CASE
        default: return false;
    }
}

size_t ffbs_big_smem(int L) {
    switch (L) {
#define HQMC_CASE(n) \
    case n: return BigGeo<n>::BYTES;
        HQMC_BIG_SIZES(HQMC_CASE)
#undef HQMC_CASE
        default: return 0;
    }
}

int ffbs_big_threads(int L) {
    switch (L) {
#define HQMC_CASE(n) \
    case n: return BigGeo<n>::NT;
        HQMC_BIG_SIZES(HQMC_CASE)
#undef HQMC_CASE
        default: return 0;
    }
}

template <int L>
static cudaError_t big_occ(int *blocks) {
    auto k = ffbs_big_kernel<L>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(BigGeo<L>::BYTES));
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k, BigGeo<L>::NT, BigGeo<L>::BYTES);
}

cudaError_t ffbs_big_occupancy(int L, int *blocks) {
    switch (L) {
#define HQMC_CASE(n) \
    case n: return big_occ<n>(blocks);
        HQMC_BIG_SIZES(HQMC_CASE)
#undef HQMC_CASE
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_ffbs_big(int L, const DevState &st, const FfbsLaunch &fl, int grid, cudaStream_t s) {
    switch (L) {
#define HQMC_CASE(n)                                                                  \
    case n:                                                                           \
        ffbs_big_kernel<n><<<grid, BigGeo<n>::NT, BigGeo<n>::BYTES, s>>>(st, fl);     \
        return cudaGetLastError();
        HQMC_BIG_SIZES(HQMC_CASE)
#undef HQMC_CASE
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace hqmc
