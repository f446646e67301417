// rd_k19_turing.cu -- instantiations of the 19-point step kernel for the
// Turing model of Table 1.
#include "rd_model_turing.h"
#include "rd_step19_kernel.cuh"

namespace rdk {

cudaError_t launch19_turing(int storage, const LaunchArgs& a, int grid, size_t smem,
                            cudaStream_t st, int* occ) {
    return launch19_model<MTuring>(storage, a, grid, smem, st, occ);
}

}  // namespace rdk
