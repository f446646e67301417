// rd_debug.cuh -- bounds checks of the bounds-checked debug build.
//
// Compiled with RD_DEBUG_BOUNDS (a separate library variant, built with
// relocatable device code so every kernel shares one error word), the step
// kernels check every shared-memory access made through the load, store and
// copy helpers against the launch's dynamic shared memory, and every global
// access against the instance's two allocations (state, scratch).  An
// access out of range is not made (a load yields 0) and the first one is
// recorded in the device word rd_dbg_word:
//   bit 63 set, bits 40..55 the site code below, bits 0..39 the byte offset
//   of the access from the start of the window it missed (two's complement).
// Nothing traps; rd_sync reads the word and reports RD_EBOUNDS.  Without
// RD_DEBUG_BOUNDS every check compiles to nothing.
#pragma once

#include "rd_internal.h"

namespace rdk {

// where a violation was met
enum DbgSite : int {
    kSiteSharedLoad = 1,     // a load from shared memory (helpers)
    kSiteSharedStore = 2,    // a store to shared memory (helpers)
    kSiteCopyDst = 3,        // the shared destination of an asynchronous copy
    kSiteCopySrc = 4,        // the global source of a copy
    kSiteStateStore = 5,     // a store of new state
    kSiteTable = 6,          // the Courant table or the step counter
    kSiteMu = 7,             // the mu field (19-point Cahn-Hilliard)
    kSiteHaloDesc = 8,       // the halo fetch descriptors
    kSiteStateLoad = 9,      // a direct load of state (resident kernel)
    kSiteSelfTest = 0xFFFF   // rd_debug_bounds' self-test
};

#ifdef RD_DEBUG_BOUNDS
extern __device__ unsigned long long rd_dbg_word;

__device__ __forceinline__ void dbg_record(int site, long long offset) {
    const unsigned long long code = (1ull << 63) | ((unsigned long long)(site & 0xFFFF) << 40) |
                                    ((unsigned long long)offset & ((1ull << 40) - 1));
    atomicCAS(&rd_dbg_word, 0ull, code);
}

// Is [p, p + bytes) inside the launch's dynamic shared memory?
__device__ __forceinline__ bool dbg_shared_ok(const void* p, int bytes, int site) {
    extern __shared__ __align__(16) unsigned char rd_dbg_dyn[];
    unsigned dyn;
    asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn));
    const char* c = static_cast<const char*>(p);
    const char* lo = reinterpret_cast<const char*>(rd_dbg_dyn);
    if (c >= lo && c + bytes <= lo + dyn) return true;
    dbg_record(site, c - lo);
    return false;
}

// Is [p, p + bytes) inside the instance's state or scratch allocation?
__device__ __forceinline__ bool dbg_global_ok(const InstDesc& sd, const void* p, int bytes,
                                              int site) {
    const char* c = static_cast<const char*>(p);
#pragma unroll
    for (int r = 0; r < 2; ++r)
        if (c >= sd.mem_lo[r] && c + bytes <= sd.mem_hi[r]) return true;
    dbg_record(site, c - sd.mem_lo[0]);
    return false;
}

// Shared-memory check of a pointer that may point to either space (the
// helpers serve both): global pointers are checked where the instance is
// known.
__device__ __forceinline__ bool dbg_any_ok(const void* p, int bytes, int site) {
    return !__isShared(p) || dbg_shared_ok(p, bytes, site);
}
#define RD_DBG_SHARED(p, n, site) dbg_shared_ok((p), (n), (site))
#define RD_DBG_ANY(p, n, site) dbg_any_ok((p), (n), (site))
#define RD_DBG_GLOBAL(sd, p, n, site) dbg_global_ok((sd), (p), (n), (site))
#else
#define RD_DBG_SHARED(p, n, site) true
#define RD_DBG_ANY(p, n, site) true
#define RD_DBG_GLOBAL(sd, p, n, site) true
#endif

}  // namespace rdk
