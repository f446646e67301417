// rd_debug.cu -- the error word of the bounds-checked debug build and its
// C ABI (rd_debug_bounds).  In the normal build the entry point exists and
// answers RD_EUNSUPPORTED.
#include <cuda_runtime.h>

#include "rd.h"
#include "rd_debug.cuh"

namespace rdk {

#ifdef RD_DEBUG_BOUNDS
__device__ unsigned long long rd_dbg_word = 0;

namespace {
// Records one violation without touching memory: any shared address is out
// of range for a launch with no dynamic shared memory.
__global__ void dbg_selftest_kernel() {
    __shared__ int probe;
    if (threadIdx.x == 0) dbg_shared_ok(&probe, 4, kSiteSelfTest);
}
}  // namespace

// Read (and with ``clear`` reset) the error word.
cudaError_t debug_word(unsigned long long* out, bool clear) {
    cudaError_t e = cudaMemcpyFromSymbol(out, rd_dbg_word, sizeof(*out));
    if (e != cudaSuccess || !clear) return e;
    const unsigned long long zero = 0;
    return cudaMemcpyToSymbol(rd_dbg_word, &zero, sizeof(zero));
}
#else
cudaError_t debug_word(unsigned long long* out, bool) {
    *out = 0;
    return cudaSuccess;
}
#endif

}  // namespace rdk

extern "C" rd_status rd_debug_bounds(uint64_t* word, int32_t op) {
#ifdef RD_DEBUG_BOUNDS
    if (!word || op < 0 || op > 2) return RD_EINVAL;
    if (op == 2) {
        rdk::dbg_selftest_kernel<<<1, 32>>>();
        if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess)
            return RD_ECUDA;
    }
    unsigned long long w = 0;
    if (rdk::debug_word(&w, op >= 1) != cudaSuccess) return RD_ECUDA;
    *word = w;
    return RD_OK;
#else
    (void)word;
    (void)op;
    return RD_EUNSUPPORTED;
#endif
}
