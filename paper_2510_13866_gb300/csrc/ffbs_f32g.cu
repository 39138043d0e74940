// ffbs_f32g.cu -- FP32 instantiations of the FFBS kernel for classes with Gaussian-field
// (U < 0) chains.
#include "ffbs_launch.cuh"

namespace hqmc {
cudaError_t launch_ffbs_f32g(int L, const DevState &st, const FfbsLaunch &fl, int grid, int wpc, cudaStream_t s) {
    return ffbs_dispatch<float, true>(L, st, fl, grid, wpc, s);
}
cudaError_t ffbs_occupancy_f32g(int L, int wpc, int *blocks) { return ffbs_occ_dispatch<float, true>(L, wpc, blocks); }
}  // namespace hqmc
