// rd_k_ch_front.cu -- instantiations of the fused step kernel for one model
// family (kept in its own translation unit so the families compile in
// parallel).
#include "rd_step_kernel.cuh"

namespace rdk {

cudaError_t launch_ch_front(int storage, int tsteps, const LaunchArgs& a, int grid,
                        size_t smem, cudaStream_t st, int* occ) {
    return launch_model<MChFront>(storage, tsteps, a, grid, smem, st, occ);
}

size_t smem_ch_front(int storage, int tsteps, int ty, int vw) {
    return smem_for<MChFront>(storage, tsteps, ty, vw);
}

}  // namespace rdk
