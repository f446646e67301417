// rd_k_ch_table1.cu -- instantiations of the fused step kernels for the
// phase separation behind a front of Table 1, row 3 (its own translation
// unit, so the families compile in parallel).
#include "rd_step_kernel.cuh"

namespace rdk {

cudaError_t launch_ch_table1(int storage, int tsteps, const LaunchArgs& a, int grid,
                             size_t smem, cudaStream_t st, int* occ) {
    return launch_model<MChTable1>(storage, tsteps, a, grid, smem, st, occ);
}

size_t smem_ch_table1(int storage, int tsteps, int ty, int vw) {
    return smem_for<MChTable1>(storage, tsteps, ty, vw);
}

}  // namespace rdk
