// rd_step19.h -- host-side declarations of the 19-point step kernels (the
// isotropic Laplacian of eqs. (3)-(4)), one step per launch, for the models
// without Cahn-Hilliard.
#pragma once

#include <stddef.h>

#include "rd_internal.h"

namespace rdk {

// Shared-memory ring of the 19-point kernel: planes q-1 .. q+4 rotate
// through 6 slots; a slot holds, per species, (ty + 2) rows of kTileQ + 2
// four-cell vectors and a four-cell guard at both ends.  96 halo fetch
// descriptors follow the ring.
constexpr int kRing19 = 6;
__host__ __device__ inline int plane_elems19(int ty) {
    return (ty + 2) * (kTileQ + 2) * 4 + 2 * 4;
}
__host__ __device__ inline size_t smem19_bytes(int nspecies, int ebytes, int ty) {
    return (size_t)kRing19 * nspecies * plane_elems19(ty) * ebytes + 96 * 16;
}
// The same with ``mu_plane``: one more float plane per slot (the second
// launch of a Cahn-Hilliard step, which reads mu beside the state).
__host__ __device__ inline size_t smem19_pass_bytes(int nfields, int ebytes, bool mu_plane,
                                                    int ty) {
    return smem19_bytes(nfields, ebytes, ty) +
           (mu_plane ? (size_t)kRing19 * plane_elems19(ty) * 4 : 0);
}
inline int threads19(int ty) { return kTileQ * ty + 32; }

// Single-instance launchers (one translation unit per model).  With
// occ != nullptr they only report the CTAs per SM.
cudaError_t launch19_diffusion(int storage, const LaunchArgs& a, int grid, size_t smem,
                               cudaStream_t st, int* occ);
cudaError_t launch19_brusselator(int storage, const LaunchArgs& a, int grid, size_t smem,
                                 cudaStream_t st, int* occ);
cudaError_t launch19_air(int storage, const LaunchArgs& a, int grid, size_t smem,
                         cudaStream_t st, int* occ);
// The two launches of a 19-point Cahn-Hilliard step (pass 1: mu, pass 2: the
// update); ``smem`` is the larger of the two passes' needs (smem19_ch_bytes).
cudaError_t launch19_ch_front(int storage, int pass, const LaunchArgs& a, int grid, size_t smem,
                              cudaStream_t st, int* occ);
cudaError_t launch19_ch_table1(int storage, int pass, const LaunchArgs& a, int grid, size_t smem,
                               cudaStream_t st, int* occ);
inline size_t smem19_ch_bytes(int ebytes, int ty) {
    return smem19_pass_bytes(3, ebytes, true, ty);
}

}  // namespace rdk
