// rd_k_diffusion.cu -- instantiations of the fused step kernel for one model
// family (kept in its own translation unit so the families compile in
// parallel).
#include "rd_step_kernel.cuh"

namespace rdk {

cudaError_t launch_diffusion(int storage, int tsteps, const LaunchArgs& a, int grid,
                        size_t smem, cudaStream_t st, int* occ) {
    return launch_model<MDiffusion>(storage, tsteps, a, grid, smem, st, occ);
}

size_t smem_diffusion(int storage, int tsteps, int ty, int vw) {
    return smem_for<MDiffusion>(storage, tsteps, ty, vw);
}

}  // namespace rdk
