// rd_k_air.cu -- instantiations of the fused step kernel for one model
// family (kept in its own translation unit so the families compile in
// parallel).
#include "rd_step_kernel.cuh"

namespace rdk {

cudaError_t launch_air(int storage, int tsteps, const LaunchArgs& a, int grid,
                        size_t smem, cudaStream_t st, int* occ) {
    return launch_model<MAir>(storage, tsteps, a, grid, smem, st, occ);
}

size_t smem_air(int storage, int tsteps, int ty, int vw) {
    return smem_for<MAir>(storage, tsteps, ty, vw);
}

}  // namespace rdk
