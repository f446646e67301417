// rd_ablation.cu -- the paper's two kernel designs for the 19-point step
// (Section 4.1, Tables 4-5), restated for this GPU as ablation baselines
// beside the z-marching kernels.  FP32 state, one step per launch, problems
// without held layers, point source or wind (the paper's kernels handle its
// boundary layers in separate launches; here every load maps its
// coordinates through the face rules instead, which composes them at edges
// exactly as the 19-point march does).
//
// Shared method (Section 4.1, Figure 3): a 3-D block of BW x BH x BD
// threads, one cell each, over an x-y tile that overlaps its neighbours by
// one cell on every side; the threads on the tile's rim only load.  The
// block walks up z keeping a window of planes in shared memory, so each
// plane is read from global memory once per tile.  Here the window is a
// ring of BD + 2 plane slots indexed by the plane number: every thread
// layer updates one plane per iteration (BD planes), then loads one new
// plane into the slot of a plane no longer needed.  Every load is a plain
// coalesced global load (a warp is one 32-cell row).
//
// Moving Tiles (Section 4.1, Figure 4): a block of BW x BH x BD threads
// over a y-z tile (overlapping by one row and plane) that walks along x in
// windows of BW cells.  Here each row keeps a ring of three windows
// indexed by the window number (the one before, the current one, the next
// one): the current window is updated with its x neighbours taken across
// the slot boundaries, then the window after the next one is loaded into
// the slot of the window before.  The paper's 16-cell window matched the
// half-warp coalescing rules of its first-generation GPUs; here BW = 32,
// one warp per row.
#include "rd_ablation.h"
#include "rd_model_turing.h"
#include "rd_step_kernel.cuh"

namespace rdk {
namespace {

constexpr int kShW = 32, kShH = 8, kShD = 4;   // Shared: 30 x 6 x 4 updates per iteration
constexpr int kShR = kShD + 2;                  // plane slots in the ring
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
    __shared__ float cs[S][kShR][kShH][kShW];
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
    // the rim loads only; x, y >= 0 elsewhere
    const bool inner = tx > 0 && tx < kShW - 1 && ty > 0 && ty < kShH - 1 && x < nx && y < ny;
    float k6[S];
#pragma unroll
    for (int s = 0; s < S; ++s) k6[s] = __fdiv_rn(sd.kx[s], 6.0f);
    // plane z lives in slot (z + 1) mod kShR (z >= -1)
    auto slot = [](int z) { return (z + 1) % kShR; };
    auto load = [&](int z) {
        const long long off = (long long)face_rule(z, nz, sd.per_z) * plane + row;
        const int sl = slot(z);
#pragma unroll
        for (int s = 0; s < S; ++s) cs[s][sl][ty][tx] = gin[s * fstride + off];
    };
    // planes -1 .. kShD fill the ring
    for (int z = tz - 1; z <= kShD; z += kShD) load(z);
    for (int zb = 0; zb < nz; zb += kShD) {
        __syncthreads();
        const int z = zb + tz;                 // the plane this layer updates
        if (inner && z < nz) {
            const int sm = slot(z - 1), s0 = slot(z), sp = slot(z + 1);
            float o[S];
            update19<M>(sd, k6,
                        [&](int s, int dx, int dy, int dz) {
                            const int sl = dz < 0 ? sm : (dz > 0 ? sp : s0);
                            return cs[s][sl][ty + dy][tx + dx];
                        },
                        o);
#pragma unroll
            for (int s = 0; s < S; ++s)
                gout[s * fstride + z * plane + (long long)y * sd.pitch + x] = o[s];
        }
        __syncthreads();
        // planes zb + kShD + 1 .. zb + 2 kShD replace zb - 1 .. zb + kShD - 2
        if (zb + kShD < nz) load(zb + kShD + 1 + tz);
    }
}

template <class M>
__global__ void __launch_bounds__(kMtW * kMtH * kMtD)
rd_tiles19_kernel(const __grid_constant__ LaunchArgs a) {
    constexpr int S = M::S;
    __shared__ float cs[S][kMtD][kMtH][3][kMtW];
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
    const bool inner = ty > 0 && ty < kMtH - 1 && tz > 0 && tz < kMtD - 1 && y < ny && z < nz;
    const bool px = sd.per_x;
    float k6[S];
#pragma unroll
    for (int s = 0; s < S; ++s) k6[s] = __fdiv_rn(sd.kx[s], 6.0f);
    // window w (cells w kMtW .. w kMtW + kMtW - 1) lives in slot (w + 1) mod 3
    auto load = [&](int w) {
        const int sl = (w + 1) % 3;
        const int xx = face_rule(w * kMtW + tx, nx, px);
#pragma unroll
        for (int s = 0; s < S; ++s) cs[s][tz][ty][sl][tx] = gin[s * fstride + rowbase + xx];
    };
    load(-1);
    load(0);
    load(1);
    const int nwin = (nx + kMtW - 1) / kMtW;
    for (int w = 0; w < nwin; ++w) {
        __syncthreads();
        const int x = w * kMtW + tx;
        if (inner && x < nx) {
            const int sm = w % 3, s0 = (w + 1) % 3, sp = (w + 2) % 3;
            float o[S];
            update19<M>(sd, k6,
                        [&](int s, int dx, int dy, int dz) {
                            // x neighbours across the window boundaries
                            const int xi = tx + dx;
                            const int sl = xi < 0 ? sm : (xi >= kMtW ? sp : s0);
                            const int xe = xi < 0 ? xi + kMtW : (xi >= kMtW ? xi - kMtW : xi);
                            return cs[s][tz + dz][ty + dy][sl][xe];
                        },
                        o);
#pragma unroll
            for (int s = 0; s < S; ++s)
                gout[s * fstride + (long long)z * sd.plane + (long long)y * sd.pitch + x] = o[s];
        }
        __syncthreads();
        if (w + 1 < nwin) load(w + 2);      // into the slot of window w - 1
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
