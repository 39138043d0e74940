// ffbs_wide.cu -- instantiations of the wide-lattice FFBS kernel (L = 48, 64, 128; FP32
// and FP64) for Hirsch-field classes, and the host-side geometry.
#include "ffbs_launch.cuh"
#include "ffbs_wide.cuh"

namespace hqmc {

cudaError_t ffbs_wide_occupancy_g(int L, bool fp64, int *blocks);
cudaError_t launch_ffbs_wide_g(int L, bool fp64, const DevState &st, const FfbsLaunch &fl, int grid, cudaStream_t s);

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

// both Gaussian flags get their limits; the grid follows the smaller residency
cudaError_t ffbs_wide_occupancy(int L, bool fp64, int *blocks) {
    cudaError_t e = wide_occ_dispatch<false>(L, fp64, blocks);
    if (e != cudaSuccess) return e;
    int bg = 0;
    e = ffbs_wide_occupancy_g(L, fp64, &bg);
    if (e == cudaSuccess && bg > 0 && bg < *blocks) *blocks = bg;
    return e;
}

cudaError_t launch_ffbs_wide(int L, bool fp64, const DevState &st, const FfbsLaunch &fl, int grid, cudaStream_t s) {
    return fl.gauss ? launch_ffbs_wide_g(L, fp64, st, fl, grid, s) : wide_launch_dispatch<false>(L, fp64, st, fl, grid, s);
}

}  // namespace hqmc
