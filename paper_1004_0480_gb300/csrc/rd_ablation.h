// rd_ablation.h -- the paper's Shared and Moving Tiles kernel designs
// (Section 4.1, Tables 4-5) for the 19-point step, as ablation baselines.
#pragma once

#include "rd_internal.h"

namespace rdk {

// One 19-point step of a single instance (a.use_one) with the kernel
// ``kernel`` (RD_KERNEL_SHARED or RD_KERNEL_TILES); the grid follows from
// the grid size.  FP32 state, no held layer, point source or wind.
cudaError_t launch_ablation(int kernel, int model, const LaunchArgs& a, cudaStream_t st);

}  // namespace rdk
