// rd_noalloc.cu -- FP64 moments of a field without any device allocation.
//
// Some callers cannot allocate device memory at the moment they need a
// conservation check: a thread that is capturing a CUDA graph (cudaMalloc
// and cudaFree are not allowed inside a stream capture), a serving loop
// that runs under a fixed memory budget planned at start-up, or a health
// monitor that must not call cudaMalloc/cudaFree because those calls can
// synchronise the device and stall the other streams.  rd_moments_noalloc
// serves them: it computes the same sums as rd_mass, with the same two-pass
// FP64 reduction, but keeps its per-block partial sums in a file-scope
// device array instead of a context's scratch buffer.
//
// The array is a fixed 608 x 3 doubles (14,592 bytes) that every GPU which
// loads this library holds until the process exits.  Its device address is
// looked up once per device, on the first call made with that device
// current, and kept until the process exits: a device reset (or a release
// and re-creation of the primary context) reloads the module and leaves the
// kept address stale, so the entry point must not be used on that device
// again afterwards.  All calls on a device share the array, and each call overwrites
// all of it before reading it, so nothing has to be cleared between calls;
// but two calls whose kernels overlap on the GPU (different streams, no
// ordering between them) race on the array and may return wrong sums.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <climits>
#include <mutex>

#include "rd.h"

namespace {

constexpr int kBlocks = 608;       // partial sums: one triple per block
constexpr int kThreads = 256;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_partials[kBlocks * 3];

std::mutex g_mu;
double* g_dev_ptr[kMaxDevices] = {};

template <class ST> __device__ __forceinline__ float as_float(ST v);
template <> __device__ __forceinline__ float as_float<float>(float v) { return v; }
template <> __device__ __forceinline__ float as_float<__nv_bfloat16>(__nv_bfloat16 v) {
    return __bfloat162float(v);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// pass 1: block b sums rows b, b + kBlocks, ... (x strided over threads)
template <class ST>
__global__ void __launch_bounds__(kThreads)
moments_pass1(const ST* __restrict__ field, int nx, int nrows, long long pitch,
              double* __restrict__ partials) {
    double s = 0.0, q = 0.0, bad = 0.0;
    for (int row = blockIdx.x; row < nrows; row += gridDim.x) {
        const ST* r = field + (long long)row * pitch;
        for (int x = threadIdx.x; x < nx; x += blockDim.x) {
            const float f = as_float<ST>(r[x]);
            if (isfinite(f)) {
                const double d = (double)f;
                s += d;
                q = fma(d, d, q);
            } else {
                bad += 1.0;
            }
        }
    }
    __shared__ double sh[3][kThreads / 32];
    s = warp_sum(s);
    q = warp_sum(q);
    bad = warp_sum(bad);
    const int w = threadIdx.x / 32, lane = threadIdx.x % 32;
    if (lane == 0) { sh[0][w] = s; sh[1][w] = q; sh[2][w] = bad; }
    __syncthreads();
    if (threadIdx.x < 3) {
        double t = 0.0;
        for (int i = 0; i < kThreads / 32; ++i) t += sh[threadIdx.x][i];
        partials[blockIdx.x * 3 + threadIdx.x] = t;
    }
}

// pass 2: one block folds the partials in a fixed order into out[0..2]
__global__ void __launch_bounds__(kThreads)
moments_pass2(const double* __restrict__ partials, double* __restrict__ out) {
    double acc[3] = {0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < kBlocks; b += blockDim.x)
        for (int k = 0; k < 3; ++k) acc[k] += partials[b * 3 + k];
    __shared__ double sh[3][kThreads / 32];
    const int w = threadIdx.x / 32, lane = threadIdx.x % 32;
    for (int k = 0; k < 3; ++k) {
        const double v = warp_sum(acc[k]);
        if (lane == 0) sh[k][w] = v;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double t = 0.0;
        for (int i = 0; i < kThreads / 32; ++i) t += sh[threadIdx.x][i];
        out[threadIdx.x] = t;
    }
}

// Device address of g_partials on the current device (looked up once).
rd_status scratch_address(double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return RD_ECUDA;
    if (dev < 0 || dev >= kMaxDevices) return RD_EUNSUPPORTED;   // device index too large
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_dev_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_partials);
        if (e != cudaSuccess) return RD_ECUDA;
        g_dev_ptr[dev] = static_cast<double*>(p);
    }
    *out = g_dev_ptr[dev];
    return RD_OK;
}

}  // namespace

extern "C" {

rd_status rd_moments_noalloc(const void* field, int32_t storage, int32_t nx, int32_t ny,
                             int32_t nz, int64_t pitch, double* out, void* stream) {
    if (!field || !out) return RD_EINVAL;
    if (storage != RD_STORE_F32 && storage != RD_STORE_BF16) return RD_EINVAL;
    if (nx < 1 || ny < 1 || nz < 1) return RD_EINVAL;          // empty grid
    if (pitch < nx) return RD_EINVAL;                          // rows overlap
    // beyond the supported maximum: pitch and ny * nz each at most 2^31 - 1
    if (pitch > INT_MAX || (long long)ny * nz > INT_MAX) return RD_EINVAL;
    double* partials = nullptr;
    rd_status st = scratch_address(&partials);
    if (st != RD_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int nrows = ny * nz;
    if (storage == RD_STORE_F32)
        moments_pass1<float><<<kBlocks, kThreads, 0, s>>>(static_cast<const float*>(field), nx,
                                                          nrows, pitch, partials);
    else
        moments_pass1<__nv_bfloat16><<<kBlocks, kThreads, 0, s>>>(
            static_cast<const __nv_bfloat16*>(field), nx, nrows, pitch, partials);
    if (cudaGetLastError() != cudaSuccess) return RD_ECUDA;
    moments_pass2<<<1, kThreads, 0, s>>>(partials, out);
    if (cudaGetLastError() != cudaSuccess) return RD_ECUDA;
    return RD_OK;
}

}  // extern "C"
