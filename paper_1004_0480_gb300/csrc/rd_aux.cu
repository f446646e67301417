// rd_aux.cu -- field packing and FP64 reductions (sm_103a).
#include <cuda_bf16.h>
#include <math.h>

#include "rd_internal.h"

namespace rdk {

namespace {

constexpr int kReduceBlocks = 608;    // fixed: 4 per SM of a 152-SM part
constexpr int kReduceThreads = 256;

template <class ST> __device__ __forceinline__ float to_f(ST v);
template <> __device__ __forceinline__ float to_f<float>(float v) { return v; }
template <> __device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 v) {
    return __bfloat162float(v);
}
template <class ST> __device__ __forceinline__ ST from_f(float v);
template <> __device__ __forceinline__ float from_f<float>(float v) { return v; }
template <> __device__ __forceinline__ __nv_bfloat16 from_f<__nv_bfloat16>(float v) {
    return __float2bfloat16_rn(v);
}

struct Held {
    float v[6];
};

// dense (z, y, x) float32 -> pitched field; held layers take their value
template <class ST>
__global__ void pack_kernel(const float* __restrict__ dense, ST* __restrict__ field, int nx,
                            int ny, int nz, int pitch, unsigned held, Held hv) {
    const long long n = (long long)nx * ny * nz;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % nx);
        const long long zy = i / nx;
        const int y = (int)(zy % ny);
        const int z = (int)(zy / ny);
        float v = dense[i];
        if (held) {
            if ((held & 1u) && x == 0) v = hv.v[0];
            else if ((held & 2u) && x == nx - 1) v = hv.v[1];
            else if ((held & 4u) && y == 0) v = hv.v[2];
            else if ((held & 8u) && y == ny - 1) v = hv.v[3];
            else if ((held & 16u) && z == 0) v = hv.v[4];
            else if ((held & 32u) && z == nz - 1) v = hv.v[5];
        }
        field[((long long)z * ny + y) * pitch + x] = from_f<ST>(v);
    }
}

template <class ST>
__global__ void unpack_kernel(const ST* __restrict__ field, float* __restrict__ dense, int nx,
                              int ny, int nz, int pitch) {
    const long long n = (long long)nx * ny * nz;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % nx);
        const long long zy = i / nx;
        dense[i] = to_f<ST>(field[zy * pitch + x]);
    }
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// pass 1: block b accumulates rows b, b+G, ... in FP64
template <class ST>
__global__ void __launch_bounds__(kReduceThreads)
reduce_pass1(const ST* __restrict__ field, int nx, int nrows, int pitch,
             double* __restrict__ partials) {
    double s = 0.0, q = 0.0, bad = 0.0;
    for (int row = blockIdx.x; row < nrows; row += gridDim.x) {
        const ST* r = field + (long long)row * pitch;
        for (int x = threadIdx.x; x < nx; x += blockDim.x) {
            const float f = to_f<ST>(r[x]);
            if (isfinite(f)) {
                const double d = (double)f;
                s += d;
                q = fma(d, d, q);
            } else {
                bad += 1.0;
            }
        }
    }
    __shared__ double sh[3][kReduceThreads / 32];
    s = warp_sum(s);
    q = warp_sum(q);
    bad = warp_sum(bad);
    const int w = threadIdx.x / 32, lane = threadIdx.x % 32;
    if (lane == 0) { sh[0][w] = s; sh[1][w] = q; sh[2][w] = bad; }
    __syncthreads();
    if (threadIdx.x < 3) {
        double t = 0.0;
        for (int i = 0; i < kReduceThreads / 32; ++i) t += sh[threadIdx.x][i];
        partials[blockIdx.x * 3 + threadIdx.x] = t;
    }
}

// pass 2: one block folds the partials in a fixed order
__global__ void __launch_bounds__(kReduceThreads)
reduce_pass2(const double* __restrict__ partials, int nblocks, double* __restrict__ out) {
    double acc[3] = {0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
        for (int k = 0; k < 3; ++k) acc[k] += partials[b * 3 + k];
    __shared__ double sh[3][kReduceThreads / 32];
    const int w = threadIdx.x / 32, lane = threadIdx.x % 32;
    for (int k = 0; k < 3; ++k) {
        const double v = warp_sum(acc[k]);
        if (lane == 0) sh[k][w] = v;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double t = 0.0;
        for (int i = 0; i < kReduceThreads / 32; ++i) t += sh[threadIdx.x][i];
        out[threadIdx.x] = t;
    }
}

int grid_for(long long n) {
    long long g = (n + 255) / 256;
    if (g > 4096) g = 4096;
    if (g < 1) g = 1;
    return (int)g;
}

}  // namespace

cudaError_t launch_pack(const float* dense, char* field, int storage, int nx, int ny, int nz,
                        int pitch, unsigned held_mask, const float* held_val,
                        cudaStream_t st) {
    Held hv;
    for (int i = 0; i < 6; ++i) hv.v[i] = held_val ? held_val[i] : 0.0f;
    const int g = grid_for((long long)nx * ny * nz);
    if (storage == RD_STORE_F32)
        pack_kernel<float><<<g, 256, 0, st>>>(dense, reinterpret_cast<float*>(field), nx, ny,
                                              nz, pitch, held_mask, hv);
    else
        pack_kernel<__nv_bfloat16><<<g, 256, 0, st>>>(
            dense, reinterpret_cast<__nv_bfloat16*>(field), nx, ny, nz, pitch, held_mask, hv);
    return cudaGetLastError();
}

cudaError_t launch_unpack(const char* field, float* dense, int storage, int nx, int ny, int nz,
                          int pitch, cudaStream_t st) {
    const int g = grid_for((long long)nx * ny * nz);
    if (storage == RD_STORE_F32)
        unpack_kernel<float><<<g, 256, 0, st>>>(reinterpret_cast<const float*>(field), dense,
                                                nx, ny, nz, pitch);
    else
        unpack_kernel<__nv_bfloat16><<<g, 256, 0, st>>>(
            reinterpret_cast<const __nv_bfloat16*>(field), dense, nx, ny, nz, pitch);
    return cudaGetLastError();
}

int reduce_blocks() { return kReduceBlocks; }

cudaError_t launch_reduce(const char* field, int storage, int nx, int ny, int nz, int pitch,
                          double* partials, double* out, cudaStream_t st) {
    const int nrows = ny * nz;
    if (storage == RD_STORE_F32)
        reduce_pass1<float><<<kReduceBlocks, kReduceThreads, 0, st>>>(
            reinterpret_cast<const float*>(field), nx, nrows, pitch, partials);
    else
        reduce_pass1<__nv_bfloat16><<<kReduceBlocks, kReduceThreads, 0, st>>>(
            reinterpret_cast<const __nv_bfloat16*>(field), nx, nrows, pitch, partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    reduce_pass2<<<1, kReduceThreads, 0, st>>>(partials, kReduceBlocks, out);
    return cudaGetLastError();
}

}  // namespace rdk
