// rd_resident.h -- the resident step kernel: many steps of one instance in a
// single cooperative launch, for grids whose state stays in L2.
#pragma once

#include "rd_internal.h"

namespace rdk {

// Grid barrier of a resident launch, in the context's scratch.  ``count``
// counts CTA arrivals over the launch (barrier k is passed once it reaches
// k * grid) and ``err`` is raised by a CTA whose wait ran out; the host
// zeroes both before every launch.  ``failed`` is sticky: set with ``err``,
// read and cleared by the host when it synchronises.
struct ResidentBar {
    unsigned count;
    unsigned err;
    unsigned failed;
    unsigned pad;
};

// How a resident launch covers the grid: tiles of ty x tz full x rows
// (y by z), each advanced up to K steps per round in shared memory from a
// halo of K rows and planes; one grid barrier per round.
struct ResidentPlan {
    int K;              // steps per round, 1..kResidentMaxK
    int ty, tz;         // tile rows (y) and planes (z)
    int nty, ntz;       // tiles along y and z
    int rw;             // shared-memory row stride in elements
    int grid;           // CTAs (all resident at once)
    int threads;        // per CTA
    int smem;           // dynamic shared memory per CTA (bytes)
    int tma;            // 1: tiles arrive as tensor-memory boxes
};

constexpr int kResidentMaxK = 4;
// Steps of one launch; the host splits longer runs (keeps the barrier count
// far from wrapping and each launch short).
constexpr int kResidentMaxSteps = 1 << 16;

// Plan for a problem (FP32 or BF16 state, a 7-point model without
// Cahn-Hilliard; ``plain`` as LaunchArgs::plain, which picks the kernel
// variant whose occupancy counts).  ``tma_ok``: y and z are not periodic
// (a box cannot wrap), so tiles may arrive as tensor-memory boxes when
// rows are at most 256 elements.  K, ty, tz > 0 fix those choices
// (clamped to the grid); 0 leaves them to a cost model.
// cudaErrorInvalidValue when no candidate fits shared memory (very wide
// rows, or a forced tile too large).
cudaError_t plan_resident(int model, int storage, bool plain, bool tma_ok, int nx, int ny,
                          int nz, int K, int ty, int tz, ResidentPlan* out);

// Advance a single instance (a.use_one) by ``nsteps`` >= 1 steps reading
// level a.one.par ^ a.parity.  Each round of the plan's K steps is one
// transition between the two levels: the result is in the other level when
// ceil(nsteps / K) is odd.  7-point stencil, a model without
// Cahn-Hilliard, no 3-D wind; FP32 or BF16 state.  The launch is cooperative
// (every CTA resident).  ``phantom`` > 0 makes every barrier wait for that
// many CTAs that do not exist, so the first one runs out (the test of the
// timeout); 0 otherwise.
cudaError_t launch_resident(int model, int storage, const LaunchArgs& a, const ResidentPlan& p,
                            int nsteps, ResidentBar* bar, unsigned phantom, cudaStream_t st);

}  // namespace rdk
