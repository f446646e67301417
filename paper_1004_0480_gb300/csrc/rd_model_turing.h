// rd_model_turing.h -- the activator-inhibitor Turing system of the paper's
// Table 1 (row 2) as a model of the step kernels, and its launchers.
//   dc1/dt = D1 Lap c1 + c1 - c1^3 - c2
//   dc2/dt = D2 Lap c2 + gamma (c1 - alpha c2 - beta)
#pragma once

#include "rd_internal.h"

namespace rdk {

#ifdef __CUDACC__
// p[0] = alpha, p[1] = beta, p[2] = gamma.  ``react`` returns dt * R_s(c).
struct MTuring {
    static constexpr int S = 2;
    static constexpr bool CH = false;
    __device__ __forceinline__ static void react(const InstDesc& d, const float* c, float* inc) {
        const float c1 = c[0], c2 = c[1];
        const float cube = __fmul_rn(__fmul_rn(c1, c1), c1);
        const float f = __fsub_rn(__fsub_rn(c1, cube), c2);
        const float g = __fmul_rn(d.p[2], __fsub_rn(__fmaf_rn(-d.p[0], c2, c1), d.p[1]));
        inc[0] = __fmul_rn(d.dt, f);
        inc[1] = __fmul_rn(d.dt, g);
    }
};
#endif

// 7-point kernels (any steps per launch) and their shared memory; the
// 19-point kernel (one step per launch).  Same contracts as the other models.
cudaError_t launch_turing(int storage, int tsteps, const LaunchArgs& a, int grid, size_t smem,
                          cudaStream_t st, int* occ);
size_t smem_turing(int storage, int tsteps, int ty, int vw);
cudaError_t launch19_turing(int storage, const LaunchArgs& a, int grid, size_t smem,
                            cudaStream_t st, int* occ);

}  // namespace rdk
