// grad_f64.cu -- FP64 instantiations of the adjoint kernel.
#include "grad_launch.cuh"

namespace hqmc {
cudaError_t launch_grad_f64(int L, const DevState &st, const GradLaunch &gk, int grid, cudaStream_t s) {
    return grad_dispatch<double>(L, st, gk, grid, s);
}
cudaError_t grad_occupancy_f64(int L, int *blocks) { return grad_occ_dispatch<double>(L, blocks); }
}  // namespace hqmc
