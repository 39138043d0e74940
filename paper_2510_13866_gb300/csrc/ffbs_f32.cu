// ffbs_f32.cu -- FP32 instantiations of the FFBS kernel (Hirsch-field classes).
#include "ffbs_launch.cuh"

namespace hqmc {
cudaError_t launch_ffbs_f32(int L, const DevState &st, const FfbsLaunch &fl, int grid, int wpc, cudaStream_t s) {
    return ffbs_dispatch<float, false>(L, st, fl, grid, wpc, s);
}
cudaError_t ffbs_occupancy_f32(int L, int wpc, int *blocks) { return ffbs_occ_dispatch<float, false>(L, wpc, blocks); }
size_t ffbs_smem_f32(int L, int wpc) { return ffbs_smem_dispatch<float>(L, wpc); }
}  // namespace hqmc
