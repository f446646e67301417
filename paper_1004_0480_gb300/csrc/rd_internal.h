// rd_internal.h -- device-side descriptors shared by the step kernels and
// the host runtime of the GB300 reaction-diffusion library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "rd.h"

namespace rdk {

constexpr int kMaxThreads = 512;     // upper bound of step-kernel CTA size
constexpr int kTileQ = 16;           // tile width in 4-cell vectors (64 cells)
constexpr int kMaxS = RD_MAX_SPECIES;

// One instance (context) as the step kernels see it.  Written by the host,
// read by every CTA that works on the instance.
struct InstDesc {
    char* base[2][kMaxS];      // field of species s at time level l
    int nx, ny, nz;
    int pitch;                 // elements per row (multiple of 16 bytes)
    long long plane;           // elements per plane (pitch * ny)
    int par;                   // level read when the launch parity is 0
    int per_x, per_y, per_z;   // periodic axes
    unsigned held_mask[kMaxS]; // bit f: face f of species s is a held layer
    float held_val[kMaxS][6];
    float kx[kMaxS], ky[kMaxS], kz[kMaxS];   // D[s][axis] * dt / h^2
    float dt;
    float p[8];                // model constants, see the model structs
    const float* courant;      // u_x(z) * dt / h per plane, or nullptr
    // 3-D wind (Table 1, row 4): Courant number along y, and along z
    // wz_amp * sin(n * wz_omega) at step n, computed in double precision;
    // stepn[l] is the step index of the state held in time level l (the
    // launch reading level l writes stepn[l ^ 1] = stepn[l] + 1); nullptr
    // without a 3-D wind.  The x Courant number is the courant table.
    long long* stepn;
    double wz_amp, wz_omega;
    float cy;
    float* mu;                 // 19-point Cahn-Hilliard models: the chemical
                               // potential of species 2 (float, the state's
                               // pitch and plane size), written by the first
                               // of the two launches of a step; else nullptr
    int src_x, src_y, src_z, src_s;          // src_s < 0: no source
    float src_amt;             // emission per step: rate * dt
    int ntx, nty, nzc, zchunk; // work items: ntx * nty * nzc
    int wrap_elems;            // periodic x with nx % 4 != 0: some halo
                               // vectors straddle the wrap point
    long long item_begin;      // first global item index of this instance
    long long launch_cap;      // batches: launches of the current step call
                               // that step this instance (it is left alone
                               // from then on); -1: every launch
    const char* mem_lo[2];     // the instance's state and scratch allocations,
    const char* mem_hi[2];     // [lo, hi): the debug build's global bounds
};

struct LaunchArgs {
    const InstDesc* desc;      // device array of ninst descriptors (batches)
    int ninst;
    int parity;                // launch parity (0/1): level read = par ^ parity
    long long nitems;          // total work items over all instances
    int ty;                    // tile height in rows (width is kTileQ vectors)
    int use_one;               // 1: a single instance, described by ``one``
    int regcap;                // one-step kernel: 1 = at most 64 registers
    int plain;                 // every instance has no held layer, source or
                               // wind, and isotropic diffusivities
    int wind3;                 // some instance has the 3-D wind (kernels take
                               // the variant with upwind along y and z)
    int vw;                    // cells per thread of the one-step 7-point
                               // kernel: 4 (16 threads per tile row) or 8
    unsigned long long* work;  // batches that pull items: work[0] the
                               // work-item counter (zero between launches),
                               // work[1] the launches completed in the
                               // current step call; nullptr: a CTA takes
                               // every gridDim-th item
    InstDesc one;              // the instance of a single-instance launch
};

// Per-model launchers (one translation unit each).  With occ != nullptr
// they only report the CTAs per SM for that shared-memory size.
cudaError_t launch_diffusion(int storage, int tsteps, const LaunchArgs& a, int grid,
                             size_t smem, cudaStream_t st, int* occ);
cudaError_t launch_brusselator(int storage, int tsteps, const LaunchArgs& a, int grid,
                               size_t smem, cudaStream_t st, int* occ);
cudaError_t launch_ch_front(int storage, int tsteps, const LaunchArgs& a, int grid,
                            size_t smem, cudaStream_t st, int* occ);
cudaError_t launch_air(int storage, int tsteps, const LaunchArgs& a, int grid,
                       size_t smem, cudaStream_t st, int* occ);
cudaError_t launch_ch_table1(int storage, int tsteps, const LaunchArgs& a, int grid,
                             size_t smem, cudaStream_t st, int* occ);
// Dynamic shared memory (bytes) and CTA size of one step kernel variant.
size_t smem_diffusion(int storage, int tsteps, int ty, int vw);
size_t smem_brusselator(int storage, int tsteps, int ty, int vw);
size_t smem_ch_front(int storage, int tsteps, int ty, int vw);
size_t smem_air(int storage, int tsteps, int ty, int vw);
size_t smem_ch_table1(int storage, int tsteps, int ty, int vw);
int step_threads(int model, int tsteps, int ty);

// Auxiliary kernels (rd_aux.cu).
cudaError_t launch_pack(const float* dense, char* field, int storage, int nx, int ny,
                        int nz, int pitch, unsigned held_mask, const float* held_val,
                        cudaStream_t st);
cudaError_t launch_unpack(const char* field, float* dense, int storage, int nx, int ny,
                          int nz, int pitch, cudaStream_t st);
// Deterministic two-pass FP64 reduction: out[0]=sum, out[1]=sum of squares,
// out[2]=non-finite count.  partials holds reduce_blocks() * 3 doubles.
int reduce_blocks();
cudaError_t launch_reduce(const char* field, int storage, int nx, int ny, int nz,
                          int pitch, double* partials, double* out, cudaStream_t st);

// The debug build's error word (rd_debug.cu): read it, and reset it with
// ``clear``; always 0 in the normal build.
cudaError_t debug_word(unsigned long long* out, bool clear);

}  // namespace rdk
