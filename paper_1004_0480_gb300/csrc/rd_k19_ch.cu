// rd_k19_ch.cu -- instantiations of the two-launch 19-point step for the
// models with a Cahn-Hilliard species (the front model and the phase
// separation of Table 1, row 3), in their own translation unit so the
// families compile in parallel.
#include "rd_step19_kernel.cuh"

namespace rdk {

cudaError_t launch19_ch_front(int storage, int pass, const LaunchArgs& a, int grid, size_t smem,
                              cudaStream_t st, int* occ) {
    return launch19_ch_model<MChFront>(storage, pass, a, grid, smem, st, occ);
}

cudaError_t launch19_ch_table1(int storage, int pass, const LaunchArgs& a, int grid, size_t smem,
                               cudaStream_t st, int* occ) {
    return launch19_ch_model<MChTable1>(storage, pass, a, grid, smem, st, occ);
}

}  // namespace rdk
