// rd_k19_brusselator.cu -- instantiations of the 19-point step kernel for one model
// family (its own translation unit, so the families compile in parallel).
#include "rd_step19_kernel.cuh"

namespace rdk {

cudaError_t launch19_brusselator(int storage, const LaunchArgs& a, int grid, size_t smem,
                        cudaStream_t st, int* occ) {
    return launch19_model<MBrusselator>(storage, a, grid, smem, st, occ);
}

}  // namespace rdk
