// rd_k_brusselator.cu -- instantiations of the fused step kernel for one model
// family (kept in its own translation unit so the families compile in
// parallel).
#include "rd_step_kernel.cuh"

namespace rdk {

cudaError_t launch_brusselator(int storage, int tsteps, const LaunchArgs& a, int grid,
                        size_t smem, cudaStream_t st, int* occ) {
    return launch_model<MBrusselator>(storage, tsteps, a, grid, smem, st, occ);
}

size_t smem_brusselator(int storage, int tsteps, int ty, int vw) {
    return smem_for<MBrusselator>(storage, tsteps, ty, vw);
}

}  // namespace rdk
