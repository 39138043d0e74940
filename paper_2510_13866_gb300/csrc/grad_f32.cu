// grad_f32.cu -- FP32 instantiations of the adjoint kernel.
#include "grad_launch.cuh"

namespace hqmc {
cudaError_t launch_grad_f32(int L, const DevState &st, const GradLaunch &gk, int grid, cudaStream_t s) {
    return grad_dispatch<float>(L, st, gk, grid, s);
}
cudaError_t grad_occupancy_f32(int L, int *blocks) { return grad_occ_dispatch<float>(L, blocks); }
}  // namespace hqmc
