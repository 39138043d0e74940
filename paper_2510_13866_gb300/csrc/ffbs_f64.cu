// ffbs_f64.cu -- FP64 instantiations of the FFBS kernel (the plain comparison form;
// Hirsch-field classes).
#include "ffbs_launch.cuh"

namespace hqmc {
cudaError_t launch_ffbs_f64(int L, const DevState &st, const FfbsLaunch &fl, int grid, int wpc, cudaStream_t s) {
    return ffbs_dispatch<double, false>(L, st, fl, grid, wpc, s);
}
cudaError_t ffbs_occupancy_f64(int L, int wpc, int *blocks) { return ffbs_occ_dispatch<double, false>(L, wpc, blocks); }
size_t ffbs_smem_f64(int L, int wpc) { return ffbs_smem_dispatch<double>(L, wpc); }
}  // namespace hqmc
