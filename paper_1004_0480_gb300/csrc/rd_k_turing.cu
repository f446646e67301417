// rd_k_turing.cu -- instantiations of the fused step kernels for the Turing
// model of Table 1 (its own translation unit, so the families compile in
// parallel).
#include "rd_model_turing.h"
#include "rd_step_kernel.cuh"

namespace rdk {

cudaError_t launch_turing(int storage, int tsteps, const LaunchArgs& a, int grid, size_t smem,
                          cudaStream_t st, int* occ) {
    return launch_model<MTuring>(storage, tsteps, a, grid, smem, st, occ);
}

size_t smem_turing(int storage, int tsteps, int ty, int vw) {
    return smem_for<MTuring>(storage, tsteps, ty, vw);
}

}  // namespace rdk
