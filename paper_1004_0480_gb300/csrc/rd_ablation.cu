// rd_ablation.cu -- the paper's two kernel designs for the 19-point step
// (Section 4.1, Tables 4-5), restated for this GPU as ablation baselines
// beside the z-marching kernels.  FP32 state, one step per launch, problems
// without held layers, point source or wind (the paper's kernels handle its
// boundary layers in separate launches; here every load maps its
// coordinates through the face rules instead, which composes them at edges
// exactly as the 19-point march does).
//
// Shared method (Table 4, Figure 3): a 3-D block of BW x BH x BD threads,
// one cell each, over an x-y tile that overlaps its neighbours by one cell
// on every side; the threads on the tile's rim only load.  The block walks
// up z holding BD planes in shared memory: it updates the BD - 2 inner
// planes, keeps the top two as the next bottom two and loads BD - 2 new
// ones.  Every load is a plain coalesced global load (a warp is one
// 32-cell row).
//
// Moving Tiles (Table 5, Figure 4): a block of BW x BH x BD threads over a
// y-z tile (overlapping by one row and plane), walking along x in windows
// of BW cells: shared memory holds, per row, the cell left of the current
// window, the window and the next window (2 BW + 1 cells); each step
// updates the window, slides the next window into its place and loads the
// one after.  The paper's BW = 16 matched the half-warp coalescing rules of
// its first-generation GPUs; here BW = 32, one warp per row.
#include "rd_ablation.h"
#include "rd_model_turing.h"
#include "rd_step_kernel.cuh"

namespace rdk {
namespace {

constexpr int kShW = 32, kShH = 8, kShD = 4;   // Shared: 30 x 6 x 2 updates per iteration
constexpr int kMtW = 32, kMtH = 8, kMtD = 4;   // Moving Tiles: 32 x 6 x 2 per window

// Coordinate i mapped into [0, n) by an axis's rule: wrapped when periodic,
// else clamped (zero flux: a ghost one cell out is the face cell).  Only
// ghosts at distance one feed an update; other out-of-range cells are
// loaded by rim threads that do not compute, and only need to be in range.
__device__ __forceinline__ int face_rule(int i, int n, bool periodic) {
    if (periodic) return wrapi(i, n);
    return i < 0 ? 0 : (i >= n ? n - 1 : i);
}

// One cell of eq. (5) with the 19-point Laplacian of eqs. (3)-(4):
// c + dt R(c) + k6 (2 x faces + edges - 24 c), k6 = D dt / (6 h^2);
// ``at(s, dx, dy, dz)`` returns the neighbour value of species s.
template <class M, class F>
__device__ __forceinline__ void update19(const InstDesc& sd, const float (&k6)[M::S], F at,
                                         float (&out)[M::S]) {
    constexpr int S = M::S;
    float cv[S], inc[S];
#pragma unroll
    for (int s = 0; s < S; ++s) cv[s] = at(s, 0, 0, 0);
    M::react(sd, cv, inc);
#pragma unroll
    for (int s = 0; s < S; ++s) {
        const float face = (at(s, -1, 0, 0) + at(s, 1, 0, 0)) + (at(s, 0, -1, 0) + at(s, 0, 1, 0)) +
                           (at(s, 0, 0, -1) + at(s, 0, 0, 1));
        const float exy = (at(s, -1, -1, 0) + at(s, 1, -1, 0)) + (at(s, -1, 1, 0) + at(s, 1, 1, 0));
        const float exz = (at(s, -1, 0, -1) + at(s, 1, 0, -1)) + (at(s, -1, 0, 1) + at(s, 1, 0, 1));
        const float eyz = (at(s, 0, -1, -1) + at(s, 0, 1, -1)) + (at(s, 0, -1, 1) + at(s, 0, 1, 1));
        const float lap6 = fmaf(-24.0f, cv[s], fmaf(2.0f, face, (exy + exz) + eyz));
        out[s] = cv[s] + fmaf(k6[s], lap6, inc[s]);
    }
}

template <class M>
__global__ void __launch_bounds__(kShW * kShH * kShD)
rd_shared19_kernel(const __grid_constant__ LaunchArgs a) {
    constexpr int S = M::S;
    __shared__ float cs[S][kShD][kShH][kShW];
    const InstDesc& sd = a.one;
    const int tx = threadIdx.x, ty = threadIdx.y, tz = threadIdx.z;
    const int nx = sd.nx, ny = sd.ny, nz = sd.nz;
    const int x = blockIdx.x * (kShW - 2) + tx - 1;   // the cell this thread loads
    const int y = blockIdx.y * (kShH - 2) + ty - 1;
    const long long row = (long long)face_rule(y, ny, sd.per_y) * sd.pitch + face_rule(x, nx, sd.per_x);
    const int lin = sd.par ^ a.parity;
    const float* const gin = reinterpret_cast<const float*>(sd.base[lin][0]);
    float* const gout = reinterpret_cast<float*>(sd.base[lin ^ 1][0]);
    const long long fstride = S > 1 ? reinterpret_cast<const float*>(sd.base[lin][1]) - gin : 0;
    const long long plane = sd.plane;
    // rim threads load only; x, y >= 0 for all others
    const bool computes = tx > 0 && tx < kShW - 1 && ty > 0 && ty < kShH - 1 && x < nx && y < ny;
    float k6[S];
#pragma unroll
    for (int s = 0; s < S; ++s) k6[s] = __fdiv_rn(sd.kx[s], 6.0f);
    auto load = [&](int z) {
        const long long off = (long long)face_rule(z, nz, sd.per_z) * plane + row;
#pragma unroll
        for (int s = 0; s < S; ++s) cs[s][tz][ty][tx] = gin[s * fstride + off];
    };
    int zb = -1;                       // the plane held by tz = 0
    load(zb + tz);
    for (;;) {
        __syncthreads();
        const int z = zb + tz;         // tz = 1 .. kShD-2 update planes zb+1 .. zb+kShD-2
        if (computes && tz > 0 && tz < kShD - 1 && z < nz) {
            float o[S];
            update19<M>(sd, k6,
                        [&](int s, int dx, int dy, int dz) {
                            return cs[s][tz + dz][ty + dy][tx + dx];
                        },
                        o);
#pragma unroll
            for (int s = 0; s < S; ++s) gout[s * fstride + z * plane + (long long)y * sd.pitch + x] = o[s];
        }
        if (zb + kShD - 1 >= nz) break;   // planes up to nz - 1 are done
        __syncthreads();
        if (tz >= kShD - 2) {
#pragma unroll
            for (int s = 0; s < S; ++s) cs[s][tz - (kShD - 2)][ty][tx] = cs[s][tz][ty][tx];
        }
        __syncthreads();
        zb += kShD - 2;
        if (tz >= 2) load(zb + tz);
    }
}

template <class M>
__global__ void __launch_bounds__(kMtW * kMtH * kMtD)
rd_tiles19_kernel(const __grid_constant__ LaunchArgs a) {
    constexpr int S = M::S;
    constexpr int W2 = 2 * kMtW + 1;
    __shared__ float cs[S][kMtD][kMtH][W2];
    const InstDesc& sd = a.one;
    const int tx = threadIdx.x, ty = threadIdx.y, tz = threadIdx.z;
    const int nx = sd.nx, ny = sd.ny, nz = sd.nz;
    const int y = blockIdx.x * (kMtH - 2) + ty - 1;   // the row this thread loads
    const int z = blockIdx.y * (kMtD - 2) + tz - 1;
    const int lin = sd.par ^ a.parity;
    const float* const gin = reinterpret_cast<const float*>(sd.base[lin][0]);
    float* const gout = reinterpret_cast<float*>(sd.base[lin ^ 1][0]);
    const long long fstride = S > 1 ? reinterpret_cast<const float*>(sd.base[lin][1]) - gin : 0;
    const long long rowbase = (long long)face_rule(z, nz, sd.per_z) * sd.plane +
                              (long long)face_rule(y, ny, sd.per_y) * sd.pitch;
    const bool computes = ty > 0 && ty < kMtH - 1 && tz > 0 && tz < kMtD - 1 && y < ny && z < nz;
    const bool px = sd.per_x;
    float k6[S];
#pragma unroll
    for (int s = 0; s < S; ++s) k6[s] = __fdiv_rn(sd.kx[s], 6.0f);
    auto ld = [&](int s, int x) { return gin[s * fstride + rowbase + face_rule(x, nx, px)]; };
    // element 0: the cell left of the window; 1..kMtW: the window; then the next window
#pragma unroll
    for (int s = 0; s < S; ++s) {
        cs[s][tz][ty][tx + 1] = ld(s, tx);
        cs[s][tz][ty][kMtW + tx + 1] = ld(s, kMtW + tx);
        if (tx == 0) cs[s][tz][ty][0] = ld(s, -1);
    }
    const int nwin = (nx + kMtW - 1) / kMtW;
    for (int k = 0; k < nwin; ++k) {
        __syncthreads();
        const int x = k * kMtW + tx;
        if (computes && x < nx) {
            float o[S];
            update19<M>(sd, k6,
                        [&](int s, int dx, int dy, int dz) {
                            return cs[s][tz + dz][ty + dy][tx + 1 + dx];
                        },
                        o);
#pragma unroll
            for (int s = 0; s < S; ++s)
                gout[s * fstride + (long long)z * sd.plane + (long long)y * sd.pitch + x] = o[s];
        }
        if (k + 1 == nwin) break;
        __syncthreads();
#pragma unroll
        for (int s = 0; s < S; ++s) {
            if (tx == kMtW - 1) cs[s][tz][ty][0] = cs[s][tz][ty][kMtW];
            cs[s][tz][ty][tx + 1] = cs[s][tz][ty][kMtW + tx + 1];
        }
        __syncthreads();
#pragma unroll
        for (int s = 0; s < S; ++s) cs[s][tz][ty][kMtW + tx + 1] = ld(s, (k + 2) * kMtW + tx);
    }
}

template <class M>
cudaError_t launch_ablation_model(int kernel, const LaunchArgs& a, cudaStream_t st) {
    const InstDesc& d = a.one;
    if (kernel == RD_KERNEL_SHARED) {
        const dim3 block(kShW, kShH, kShD);
        const dim3 grid((d.nx + kShW - 3) / (kShW - 2), (d.ny + kShH - 3) / (kShH - 2));
        rd_shared19_kernel<M><<<grid, block, 0, st>>>(a);
        return cudaGetLastError();
    }
    if (kernel == RD_KERNEL_TILES) {
        const dim3 block(kMtW, kMtH, kMtD);
        const dim3 grid((d.ny + kMtH - 3) / (kMtH - 2), (d.nz + kMtD - 3) / (kMtD - 2));
        rd_tiles19_kernel<M><<<grid, block, 0, st>>>(a);
        return cudaGetLastError();
    }
    return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_ablation(int kernel, int model, const LaunchArgs& a, cudaStream_t st) {
    if (!a.use_one) return cudaErrorInvalidValue;
    switch (model) {
    case RD_MODEL_DIFFUSION: return launch_ablation_model<MDiffusion>(kernel, a, st);
    case RD_MODEL_BRUSSELATOR: return launch_ablation_model<MBrusselator>(kernel, a, st);
    case RD_MODEL_AIR: return launch_ablation_model<MAir>(kernel, a, st);
    case RD_MODEL_TURING: return launch_ablation_model<MTuring>(kernel, a, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace rdk
