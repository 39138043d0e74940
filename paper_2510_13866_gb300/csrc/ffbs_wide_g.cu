// ffbs_wide_g.cu -- instantiations of the wide-lattice FFBS kernel for classes with
// Gaussian-field (U < 0) chains.
#include "ffbs_launch.cuh"
#include "ffbs_wide.cuh"

namespace hqmc {

cudaError_t ffbs_wide_occupancy_g(int L, bool fp64, int *blocks) { return wide_occ_dispatch<true>(L, fp64, blocks); }

cudaError_t launch_ffbs_wide_g(int L, bool fp64, const DevState &st, const FfbsLaunch &fl, int grid, cudaStream_t s) {
    return wide_launch_dispatch<true>(L, fp64, st, fl, grid, s);
}

}  // namespace hqmc
