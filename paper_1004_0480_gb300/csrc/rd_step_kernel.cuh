// rd_step_kernel.cuh -- the fused forward-Euler step kernels (sm_103a).
//
// Three kernels share the per-cell update functions below, so every launch
// shape gives the same bits: rd_step_kernel (T steps per launch, described
// here), rd_step1_kernel (one step per launch, models without
// Cahn-Hilliard) and rd_stepch_kernel (one step per launch, the front
// model); the last two are described where they are defined.
//
// rd_step_kernel: one launch advances T steps of eq. (5) for every species
// of every work item.  A work item is an x-y tile of 64 x TY cells and a chunk of z planes
// of one instance.  The CTA marches up the chunk, as the paper's Shared
// method does (Section 4.1, Table 4), restated for this hardware:
//
//  * thread layout: one thread per 4-cell vector position of the tile
//    widened by a halo (one vector each side in x, L rows each side in y),
//    i.e. (16 + 2) x (TY + 2L) threads.  As in the paper's overlapped
//    blocks, halo threads load (and at inner levels compute) but never
//    store.  A thread keeps its position for the whole march, so all index
//    and boundary arithmetic is done once per work item.
//  * level 0: planes of the current state arrive in a shared-memory ring by
//    per-thread cp.async copies, several planes ahead.
//  * level l = 1..L: as soon as level l-1 has planes q-1, q, q+1, plane q of
//    level l is computed from them; every level keeps a few planes in shared
//    memory.  Level L goes to global memory.  All levels advance once per
//    plane, with a single barrier per plane.
//  * Without Cahn-Hilliard L = T and level l is the state after l steps.
//    With it L = 2T: odd levels hold mu = f'(c) - kappa Lap c, even levels
//    the state -- the paper's "Laplacian, boundary rule, Laplacian"
//    biharmonic (Section 4.1), fused into the march.
//
// Boundary rules, applied at every level:
//   periodic axis  halo cells are real cells at wrapped coordinates;
//   zero flux      a neighbour outside the domain is the cell itself (the
//                  ghost equals the face cell), so outside cells are never
//                  read or loaded;
//   held layer     (Dirichlet) the cell's new value is its bc value.
// Every value at every level comes from the same per-cell update with
// explicitly rounded operations, and inner levels are rounded to the storage
// type, so a T-step launch reproduces T one-step launches bit for bit.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

#include "rd_debug.cuh"
#include "rd_internal.h"

namespace rdk {

constexpr int kVEC = 4;               // cells per thread position (x)
constexpr int kNQ = kTileQ + 2;       // vector positions per row incl. halo
constexpr int kRW = kNQ * kVEC;       // elements per shared-memory row

// ---------------------------------------------------------------- storage
template <class ST> struct Store;

// Loads and stores of 4-cell vectors and single cells in either space, and
// asynchronous global-to-shared copies.  In the bounds-checked debug build
// (rd_debug.cuh) each checks its shared-memory side and skips an access out
// of range (a load then yields 0); global sides are checked by the callers,
// which know the instance.
template <> struct Store<float> {
    __device__ __forceinline__ static void load(const float* p, float (&v)[4]) {
        if (!RD_DBG_ANY(p, 16, kSiteSharedLoad)) { v[0] = v[1] = v[2] = v[3] = 0.0f; return; }
        const float4 t = *reinterpret_cast<const float4*>(p);
        v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
    }
    __device__ __forceinline__ static void store(float* p, const float (&v)[4]) {
        if (!RD_DBG_ANY(p, 16, kSiteSharedStore)) return;
        *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
    }
    __device__ __forceinline__ static float get(const float* p) {
        if (!RD_DBG_ANY(p, 4, kSiteSharedLoad)) return 0.0f;
        return *p;
    }
    __device__ __forceinline__ static float round(float x) { return x; }
    __device__ __forceinline__ static void cp_async(float* smem, const float* g) {
        if (!RD_DBG_SHARED(smem, 16, kSiteCopyDst)) return;
        const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(g) : "memory");
    }
    // copy only where ``pred`` holds (no branch)
    __device__ __forceinline__ static void cp_async_if(float* smem, const float* g, int pred) {
        if (pred && !RD_DBG_SHARED(smem, 16, kSiteCopyDst)) return;
        const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
        asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %2, 0;\n"
                     " @p cp.async.cg.shared.global [%0], [%1], 16;\n}\n" ::"r"(s), "l"(g),
                     "r"(pred)
                     : "memory");
    }
    // one element (4 bytes), asynchronously
    __device__ __forceinline__ static void cp_async_elem(float* smem, const float* g) {
        if (!RD_DBG_SHARED(smem, 4, kSiteCopyDst)) return;
        const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(g) : "memory");
    }
};

template <> struct Store<__nv_bfloat16> {
    __device__ __forceinline__ static void load(const __nv_bfloat16* p, float (&v)[4]) {
        if (!RD_DBG_ANY(p, 8, kSiteSharedLoad)) { v[0] = v[1] = v[2] = v[3] = 0.0f; return; }
        const uint2 t = *reinterpret_cast<const uint2*>(p);
        v[0] = __uint_as_float(t.x << 16);
        v[1] = __uint_as_float(t.x & 0xffff0000u);
        v[2] = __uint_as_float(t.y << 16);
        v[3] = __uint_as_float(t.y & 0xffff0000u);
    }
    __device__ __forceinline__ static void store(__nv_bfloat16* p, const float (&v)[4]) {
        if (!RD_DBG_ANY(p, 8, kSiteSharedStore)) return;
        __nv_bfloat162 a = __floats2bfloat162_rn(v[0], v[1]);
        __nv_bfloat162 b = __floats2bfloat162_rn(v[2], v[3]);
        *reinterpret_cast<uint2*>(p) =
            make_uint2(*reinterpret_cast<unsigned*>(&a), *reinterpret_cast<unsigned*>(&b));
    }
    __device__ __forceinline__ static float get(const __nv_bfloat16* p) {
        if (!RD_DBG_ANY(p, 2, kSiteSharedLoad)) return 0.0f;
        return __bfloat162float(*p);
    }
    __device__ __forceinline__ static float round(float x) {
        return __bfloat162float(__float2bfloat16_rn(x));
    }
    __device__ __forceinline__ static void cp_async(__nv_bfloat16* smem, const __nv_bfloat16* g) {
        if (!RD_DBG_SHARED(smem, 8, kSiteCopyDst)) return;
        const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(g) : "memory");
    }
    // 2-byte elements have no asynchronous copy: element copies are plain
    __device__ __forceinline__ static void cp_async_elem(__nv_bfloat16* smem,
                                                         const __nv_bfloat16* g) {
        if (!RD_DBG_SHARED(smem, 2, kSiteCopyDst)) return;
        *smem = *g;
    }
    __device__ __forceinline__ static void cp_async_if(__nv_bfloat16* smem,
                                                       const __nv_bfloat16* g, int pred) {
        if (pred && !RD_DBG_SHARED(smem, 8, kSiteCopyDst)) return;
        const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
        asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %2, 0;\n"
                     " @p cp.async.ca.shared.global [%0], [%1], 8;\n}\n" ::"r"(s), "l"(g),
                     "r"(pred)
                     : "memory");
    }
};

__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N> __device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

__device__ __forceinline__ int wrapi(int i, int n) {
    int r = i % n;
    return r < 0 ? r + n : r;
}

// Entry z of the Courant table ``tab`` (0 without a table).
__device__ __forceinline__ float courant_at(const InstDesc& sd, const float* tab, int z) {
    if (!tab || !RD_DBG_GLOBAL(sd, tab + z, 4, kSiteTable)) return 0.0f;
    return tab[z];
}

// ----------------------------------------------------------------- models
// Per-cell pieces of eq. (1).  ``react`` returns dt * R_s(c) per species.
struct MDiffusion {
    static constexpr int S = 1;
    static constexpr bool CH = false;
    __device__ __forceinline__ static void react(const InstDesc&, const float*, float* inc) {
        inc[0] = 0.0f;
    }
};

// Brusselator: R_u = a - (b+1) u + u^2 v, R_v = b u - u^2 v.
// p[0] = a, p[1] = b + 1, p[2] = b.
struct MBrusselator {
    static constexpr int S = 2;
    static constexpr bool CH = false;
    __device__ __forceinline__ static void react(const InstDesc& d, const float* c, float* inc) {
        const float u = c[0], v = c[1];
        const float uuv = __fmul_rn(__fmul_rn(u, u), v);
        const float f = __fadd_rn(__fmaf_rn(-d.p[1], u, d.p[0]), uuv);
        const float g = __fsub_rn(__fmul_rn(d.p[2], u), uuv);
        inc[0] = __fmul_rn(d.dt, f);
        inc[1] = __fmul_rn(d.dt, g);
    }
};

// Photochemistry NO, NO2, O3: NO2 -> NO + O3 (j), NO + O3 -> NO2 (k).
// p[0] = j, p[1] = k.
struct MAir {
    static constexpr int S = 3;
    static constexpr bool CH = false;
    __device__ __forceinline__ static void react(const InstDesc& d, const float* c, float* inc) {
        const float ph = __fmul_rn(d.p[0], c[1]);
        const float ti = __fmul_rn(__fmul_rn(d.p[1], c[0]), c[2]);
        const float net = __fmul_rn(d.dt, __fsub_rn(ph, ti));
        inc[0] = net;
        inc[1] = -net;
        inc[2] = net;
    }
};

// Models with a Cahn-Hilliard species (species 2, c) share one shape: the
// chemical potential mu = g(c) - p[2] Lap_h c, where Lap_h c = (sum of the
// 6 neighbours - 6 c) is the Laplacian times h^2, and the update
// c += p[1] Lap_h mu + dt R_c, with no Fickian term for c (the biharmonic
// as "Laplacian, boundary rule, Laplacian", Section 4.1).

// mu from g(c) and the 6 neighbours of c
__device__ __forceinline__ float ch_mu(float g, float pk, float c, float xm, float xp, float ym,
                                       float yp, float zm, float zp) {
    const float s6 = __fadd_rn(__fadd_rn(__fadd_rn(xm, xp), __fadd_rn(ym, yp)), __fadd_rn(zm, zp));
    const float lap = __fmaf_rn(-6.0f, c, s6);
    return __fmaf_rn(-pk, lap, g);
}

// Front a + b -> c with Cahn-Hilliard c.
// p[0] = dt k, p[1] = dt M / h^2, p[2] = kappa / h^2.
struct MChFront {
    static constexpr int S = 3;
    static constexpr bool CH = true;
    __device__ __forceinline__ static void react(const InstDesc& d, const float* c, float* inc) {
        const float q = __fmul_rn(__fmul_rn(d.p[0], c[0]), c[1]);
        inc[0] = -q;
        inc[1] = -q;
        inc[2] = q;
    }
    // g(c) = f'(c) = 2c(c-1)(2c-1), the derivative of the double well
    __device__ __forceinline__ static float g(const InstDesc&, float c) {
        const float c2 = __fadd_rn(c, c);
        return __fmul_rn(__fmul_rn(c2, __fsub_rn(c, 1.0f)), __fsub_rn(c2, 1.0f));
    }
    // mu = f'(c) - (kappa/h^2) (sum of 6 neighbours - 6 c)
    __device__ __forceinline__ static float mu(const InstDesc& d, float c, float xm, float xp,
                                               float ym, float yp, float zm, float zp) {
        return ch_mu(g(d, c), d.p[2], c, xm, xp, ym, yp, zm, zp);
    }
};

// The phase separation behind a front of Table 1 (row 3): c1 + c2 -> c3 at
// k1 c1 c2, the sink k2 c1 c3 taken from c1 and c3, and
// dc3/dt += -lambda Lap(eps c3 - gamma c3^3 + sigma Lap c3).
// p[0] = dt k1, p[1] = -dt lambda / h^2, p[2] = -sigma / h^2, p[3] = dt k2,
// p[4] = eps, p[5] = gamma.
struct MChTable1 {
    static constexpr int S = 3;
    static constexpr bool CH = true;
    __device__ __forceinline__ static void react(const InstDesc& d, const float* c, float* inc) {
        const float q1 = __fmul_rn(__fmul_rn(d.p[0], c[0]), c[1]);
        const float q2 = __fmul_rn(__fmul_rn(d.p[3], c[0]), c[2]);
        inc[0] = -__fadd_rn(q1, q2);
        inc[1] = -q1;
        inc[2] = __fsub_rn(q1, q2);
    }
    // g(c) = eps c - gamma c^3
    __device__ __forceinline__ static float g(const InstDesc& d, float c) {
        return __fmul_rn(c, __fmaf_rn(-d.p[5], __fmul_rn(c, c), d.p[4]));
    }
    __device__ __forceinline__ static float mu(const InstDesc& d, float c, float xm, float xp,
                                               float ym, float yp, float zm, float zp) {
        return ch_mu(g(d, c), d.p[2], c, xm, xp, ym, yp, zm, zp);
    }
};

// One cell of eq. (5) for a species with Fickian transport:
// c + inc + sum_a k_a (c[-1] + c[+1] - 2c), k_a = D_a dt / h^2.
__device__ __forceinline__ float euler_cell(float c, float xm, float xp, float ym, float yp,
                                            float zm, float zp, float kx, float ky, float kz,
                                            float inc) {
    const float c2 = __fadd_rn(c, c);
    const float lx = __fsub_rn(__fadd_rn(xm, xp), c2);
    const float ly = __fsub_rn(__fadd_rn(ym, yp), c2);
    const float lz = __fsub_rn(__fadd_rn(zm, zp), c2);
    inc = __fmaf_rn(kz, lz, inc);
    inc = __fmaf_rn(ky, ly, inc);
    inc = __fmaf_rn(kx, lx, inc);
    return __fadd_rn(c, inc);
}

// Same for equal diffusivities on the three axes (k = D dt / h^2):
// c + inc + k (sum of the 6 neighbours - 6 c).
__device__ __forceinline__ float euler_cell_iso(float c, float xm, float xp, float ym, float yp,
                                                float zm, float zp, float k, float inc) {
    const float s6 = __fadd_rn(__fadd_rn(__fadd_rn(xm, xp), __fadd_rn(ym, yp)), __fadd_rn(zm, zp));
    const float lap = __fmaf_rn(-6.0f, c, s6);
    return __fadd_rn(c, __fmaf_rn(k, lap, inc));
}

// ------------------------------------------------------- shared-memory map
// Every level keeps its planes in shared memory; slots are the low bits of
// the plane index.  Level 0 is a ring of 8 planes per species, P of them in
// flight ahead of the plane being consumed; an inner level has 4 plane
// buffers (a mu level holds one field).  The z neighbours a thread needs
// are its own position in planes q-1 and q+1, which it wrote (or copied)
// itself; only the x/y neighbours in plane q come from other threads, and
// that plane was completed before the last barrier.  Hence one barrier per
// plane suffices when
//   level 0:  P <= 8 - 3 (read up to two planes after arrival; the
//             Cahn-Hilliard state level reads it three planes after: P <= 4)
//   inner:    4 buffers (read up to three planes after it is written).
// Each plane is rows(ty) rows of kRW elements plus a kVEC guard at both ends.
template <class M, class ST, int T> struct Layout {
    static constexpr int S = M::S;
    static constexpr bool CH = M::CH;
    static constexpr int L = CH ? 2 * T : T;
    static constexpr int RING0 = 8;
    static constexpr int P = CH ? 4 : 5;     // level-0 planes in flight
    static constexpr int NBUF = 4;           // planes of an inner level
    __host__ __device__ static constexpr bool is_mu(int l) { return CH && (l & 1); }
    __host__ __device__ static int rows(int ty) { return ty + 2 * L; }
    __host__ __device__ static int plane_elems(int ty) { return rows(ty) * kRW + 2 * kVEC; }
    __host__ __device__ static size_t level_bytes(int l, int ty) {
        const size_t pe = plane_elems(ty);
        if (l == 0) return (size_t)RING0 * S * pe * sizeof(ST);
        if (is_mu(l)) return (size_t)NBUF * pe * sizeof(float);
        return (size_t)NBUF * S * pe * sizeof(ST);
    }
    __host__ __device__ static size_t level_offset(int l, int ty) {
        size_t o = 0;
        for (int i = 0; i < l; ++i) o += level_bytes(i, ty);
        return o;
    }
    __host__ __device__ static size_t total(int ty) { return level_offset(L, ty); }
    __host__ __device__ static int threads(int ty) { return kNQ * rows(ty); }
};

// Per-thread geometry of a work item (fixed for the whole march).
struct Pos {
    int own;          // shared-memory element offset of the thread's vector
    int offm, offp;   // vector above / below (own vector at a zero-flux y face)
    int offl;         // element left of the vector (own element 0 at x = 0)
    int xs, y;        // global x of element 0 and global y (unwrapped)
    int xhi;          // element holding x = nx-1 at a zero-flux face, else -1
};

// 7-point neighbourhood of the thread's vector in one level: centre and the
// z neighbours from planes Pc / Pm / Pp at the thread's own position, x and
// y neighbours from plane Pc.
template <class E>
__device__ __forceinline__ void gather7(const E* Pc, const E* Pm, const E* Pp, const Pos& ps,
                                        float (&c)[kVEC], float (&xm)[kVEC], float (&xp)[kVEC],
                                        float (&ym)[kVEC], float (&yp)[kVEC],
                                        float (&zm)[kVEC], float (&zp)[kVEC]) {
    Store<E>::load(Pc + ps.own, c);
    Store<E>::load(Pm + ps.own, zm);
    Store<E>::load(Pp + ps.own, zp);
    Store<E>::load(Pc + ps.offm, ym);
    Store<E>::load(Pc + ps.offp, yp);
    const float left = Store<E>::get(Pc + ps.offl);
    const float right = Store<E>::get(Pc + ps.own + kVEC);
#pragma unroll
    for (int e = 0; e < kVEC; ++e) {
        xm[e] = e ? c[e - 1] : left;
        xp[e] = (e < kVEC - 1) ? c[e + 1] : right;
    }
    if (ps.xhi >= 0) {
#pragma unroll
        for (int e = 0; e < kVEC; ++e)
            if (e == ps.xhi) xp[e] = c[e];
    }
}

// The instance a work item belongs to: the launch's own descriptor (kernel
// parameter space, read as constants) for single-instance launches, else a
// shared-memory copy of the batch entry.
template <bool ONE>
__device__ __forceinline__ const InstDesc& desc_of(const LaunchArgs& a, const InstDesc& copy) {
    if constexpr (ONE) return a.one;
    else return copy;
}

// Fetch the descriptor of the instance owning ``item`` into ``copy`` (batch
// launches); one barrier-separated pass per change of instance.
__device__ __forceinline__ void load_desc(const LaunchArgs& a, long long item, InstDesc& copy,
                                          int& s_inst, int& cur_inst) {
    const int tid = threadIdx.x;
    for (int i = tid; i < a.ninst; i += blockDim.x) {
        const long long b0 = a.desc[i].item_begin;
        const long long b1 = (i + 1 < a.ninst) ? a.desc[i + 1].item_begin : a.nitems;
        if (item >= b0 && item < b1) s_inst = i;
    }
    __syncthreads();
    if (s_inst != cur_inst) {
        cur_inst = s_inst;
        const int* src = reinterpret_cast<const int*>(a.desc + cur_inst);
        int* dst = reinterpret_cast<int*>(&copy);
        for (int i = tid; i < (int)(sizeof(InstDesc) / sizeof(int)); i += blockDim.x) dst[i] = src[i];
    }
    __syncthreads();
}

// Work items of a CTA.  A single instance's items cost the same, so a CTA
// takes every gridDim-th one; a batch's may differ (partial tiles, short
// last z-chunks, unequal instances), so when the host passes the batch's
// counter (a.work) its CTAs pull the next item as they finish one.  Each CTA's last pull fails (its
// ticket is at least nitems); the CTA holding the launch's last ticket,
// nitems + gridDim - 1, pulls after every other CTA has finished its
// items, so it also counts the launch as completed (work[1]) and zeroes
// the item counter for the next launch.  Called by every thread of the CTA
// together; the item loops end with a block barrier, so s_item is free to
// overwrite.
__device__ __forceinline__ long long pull_item(const LaunchArgs& a, long long& s_item) {
    if (threadIdx.x == 0) {
        const unsigned long long t = atomicAdd(a.work, 1ull);
        if (t == (unsigned long long)a.nitems + gridDim.x - 1) {
            atomicAdd(a.work + 1, 1ull);
            atomicExch(a.work, 0ull);
        }
        s_item = (long long)t;
    }
    __syncthreads();
    return s_item;
}
// A batch member whose launches for the current step call are used up
// (rd_batch_step_each) is left alone: its items are skipped, its fields
// keep the level its last step wrote.  The same for every thread.
template <bool ONE>
__device__ __forceinline__ bool member_done(const LaunchArgs& a, const InstDesc& sd) {
    if (ONE || !a.work || sd.launch_cap < 0) return false;
    return (long long)a.work[1] >= sd.launch_cap;
}
template <bool ONE>
__device__ __forceinline__ long long first_item(const LaunchArgs& a, long long& s_item) {
    if (ONE || !a.work) return blockIdx.x;
    return pull_item(a, s_item);
}
template <bool ONE>
__device__ __forceinline__ long long next_item(const LaunchArgs& a, long long item,
                                               long long& s_item) {
    if (ONE || !a.work) return item + gridDim.x;
    return pull_item(a, s_item);
}

// Held (Dirichlet) layers: the first face in -x,+x,-y,+y,-z,+z wins.
__device__ __forceinline__ void held_layers(const InstDesc& sd, int s, int xs, int y, int q,
                                            float (&o)[kVEC]) {
    const unsigned hm = sd.held_mask[s];
    if (!hm) return;
#pragma unroll
    for (int e = 0; e < kVEC; ++e) {
        const int x = xs + e;
        float hv = o[e];
        if ((hm & 32u) && q == sd.nz - 1) hv = sd.held_val[s][5];
        if ((hm & 16u) && q == 0) hv = sd.held_val[s][4];
        if ((hm & 8u) && y == sd.ny - 1) hv = sd.held_val[s][3];
        if ((hm & 4u) && y == 0) hv = sd.held_val[s][2];
        if ((hm & 2u) && x == sd.nx - 1) hv = sd.held_val[s][1];
        if ((hm & 1u) && x == 0) hv = sd.held_val[s][0];
        o[e] = hv;
    }
}

// Faces of the grid that a thread's 4 cells (x = xs..xs+3, row y, plane
// q) lie on, as bits in the order of held_mask: -x, +x, -y, +y, -z, +z.
__device__ __forceinline__ unsigned xy_faces(int xs, int y, int nx, int ny) {
    return (xs <= 0 && xs + kVEC > 0 ? 1u : 0u) | (xs <= nx - 1 && xs + kVEC > nx - 1 ? 2u : 0u) |
           (y == 0 ? 4u : 0u) | (y == ny - 1 ? 8u : 0u);
}
__device__ __forceinline__ unsigned z_faces(int q, int nz) {
    return (q == 0 ? 16u : 0u) | (q == nz - 1 ? 32u : 0u);
}

// held_layers for a thread whose face bits are known: the same result, the
// per-cell tests run only where a held face is touched
__device__ __forceinline__ void held_layers_at(const InstDesc& sd, int s, unsigned faces, int xs,
                                               int y, int q, float (&o)[kVEC]) {
    if (sd.held_mask[s] & faces) held_layers(sd, s, xs, y, q, o);
}

// First-order upwind along one axis with Courant number cu = u dt / h:
// in -= cu (c - c[-1]) for cu > 0, cu (c[+1] - c) for cu < 0 (Section 4.1).
__device__ __forceinline__ void upwind_axis(float cu, const float (&c)[kVEC],
                                            const float (&cm)[kVEC], const float (&cp)[kVEC],
                                            float (&in)[kVEC]) {
    if (cu > 0.0f) {
#pragma unroll
        for (int e = 0; e < kVEC; ++e) in[e] = __fmaf_rn(-cu, __fsub_rn(c[e], cm[e]), in[e]);
    } else if (cu < 0.0f) {
#pragma unroll
        for (int e = 0; e < kVEC; ++e) in[e] = __fmaf_rn(-cu, __fsub_rn(cp[e], c[e]), in[e]);
    }
}

// Courant numbers along y and z of the 3-D wind for the launch reading time
// level ``lin`` (zero without it): u_z = wz_amp sin(n wz_omega) at the step
// index n of that level, evaluated in double precision.  The CTA taking an
// instance's first work item also records n + 1 as the step index of the
// level it writes (read by the next launch, never by this one).
__device__ __forceinline__ void wind3d(const InstDesc& sd, int lin, long long local, float& cy,
                                       float& cz) {
    cy = 0.0f;
    cz = 0.0f;
    if (!sd.stepn) return;
    if (!RD_DBG_GLOBAL(sd, sd.stepn, 16, kSiteTable)) return;
    const long long n = sd.stepn[lin];
    cy = sd.cy;
    cz = (float)(sd.wz_amp * sin((double)n * sd.wz_omega));
    if (local == 0 && threadIdx.x == 0) sd.stepn[lin ^ 1] = n + 1;
}

// New value of one species on the thread's 4 cells (eq. (5)): reaction
// increment ``inc`` (dt R), point source, upwind advection, Fickian
// transport; held layers are applied by the caller.  Shared by every
// kernel so that all launch shapes give identical bits.
__device__ __forceinline__ void species_core(const InstDesc& sd, int s, const float (&c)[kVEC],
                                             const float (&xm)[kVEC], const float (&xp)[kVEC],
                                             const float (&ym)[kVEC], const float (&yp)[kVEC],
                                             const float (&zm)[kVEC], const float (&zp)[kVEC],
                                             const float (&inc)[kVEC], float cx, bool src_here,
                                             bool px, int xs, float (&o)[kVEC], float cy = 0.0f,
                                             float cz = 0.0f) {
    const float kx = sd.kx[s], ky = sd.ky[s], kz = sd.kz[s];
    const bool src_s = src_here && s == sd.src_s;
    const bool iso = kx == ky && kx == kz;
    // every test below is uniform over the 4 cells: taken once, not per cell
    float in[kVEC];
#pragma unroll
    for (int e = 0; e < kVEC; ++e) in[e] = inc[e];
    if (src_s) {
#pragma unroll
        for (int e = 0; e < kVEC; ++e)
            if ((px ? wrapi(xs + e, sd.nx) : xs + e) == sd.src_x) in[e] = __fadd_rn(in[e], sd.src_amt);
    }
    // first-order upwind advection, Courant number cx = u dt / h
    if (cx > 0.0f) {
#pragma unroll
        for (int e = 0; e < kVEC; ++e) in[e] = __fmaf_rn(-cx, __fsub_rn(c[e], xm[e]), in[e]);
    } else if (cx < 0.0f) {
#pragma unroll
        for (int e = 0; e < kVEC; ++e) in[e] = __fmaf_rn(-cx, __fsub_rn(xp[e], c[e]), in[e]);
    }
    // the same along y and z (the 3-D wind of Table 1, row 4)
    upwind_axis(cy, c, ym, yp, in);
    upwind_axis(cz, c, zm, zp, in);
    if (iso) {
#pragma unroll
        for (int e = 0; e < kVEC; ++e)
            o[e] = euler_cell_iso(c[e], xm[e], xp[e], ym[e], yp[e], zm[e], zp[e], kx, in[e]);
    } else {
#pragma unroll
        for (int e = 0; e < kVEC; ++e)
            o[e] = euler_cell(c[e], xm[e], xp[e], ym[e], yp[e], zm[e], zp[e], kx, ky, kz, in[e]);
    }
}

// species_core followed by the held layers
__device__ __forceinline__ void species_update(const InstDesc& sd, int s, const float (&c)[kVEC],
                                               const float (&xm)[kVEC], const float (&xp)[kVEC],
                                               const float (&ym)[kVEC], const float (&yp)[kVEC],
                                               const float (&zm)[kVEC], const float (&zp)[kVEC],
                                               const float (&inc)[kVEC], float cx, bool src_here,
                                               bool px, int xs, int y, int q, float (&o)[kVEC]) {
    species_core(sd, s, c, xm, xp, ym, yp, zm, zp, inc, cx, src_here, px, xs, o);
    held_layers(sd, s, xs, y, q, o);
}

// ------------------------------------------------------------------ kernel
template <class M, class ST, int T, bool ONE>
__global__ void __launch_bounds__(kMaxThreads, 2) rd_step_kernel(const __grid_constant__ LaunchArgs a) {
    using LY = Layout<M, ST, T>;
    constexpr int S = M::S;
    constexpr bool CH = M::CH;
    constexpr int L = LY::L;
    constexpr int P = LY::P;

    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ InstDesc sdm;
    __shared__ int s_inst;
    __shared__ long long s_item;

    const int tid = threadIdx.x;
    const int TY = a.ty;
    const int NR = LY::rows(TY);
    const int PE = LY::plane_elems(TY);
    const int r = tid / kNQ;             // row of the thread's position
    const int v = tid - r * kNQ;         // vector of the thread's position

    // plane X of state level m, species s; plane X of mu level m
    auto state_plane = [&](int m, int s, int X) -> ST* {
        const int slot = (m == 0) ? (X & (LY::RING0 - 1)) : (X & (LY::NBUF - 1));
        return reinterpret_cast<ST*>(smem + LY::level_offset(m, TY)) + (size_t)(slot * S + s) * PE +
               kVEC;
    };
    auto mu_plane = [&](int m, int X) -> float* {
        return reinterpret_cast<float*>(smem + LY::level_offset(m, TY)) +
               (size_t)(X & (LY::NBUF - 1)) * PE + kVEC;
    };

    int cur_inst = -1;
    if (tid == 0) s_inst = 0;
    for (long long item = first_item<ONE>(a, s_item); item < a.nitems;
         item = next_item<ONE>(a, item, s_item)) {
        if constexpr (!ONE) load_desc(a, item, sdm, s_inst, cur_inst);
        const InstDesc& sd = desc_of<ONE>(a, sdm);
        if (member_done<ONE>(a, sd)) continue;   // block-uniform

        const int nx = sd.nx, ny = sd.ny, nz = sd.nz;
        const bool px = sd.per_x, py = sd.per_y, pz = sd.per_z;
        const long long local = item - sd.item_begin;
        const int txi = (int)(local % sd.ntx);
        const int tyi = (int)((local / sd.ntx) % sd.nty);
        const int zc = (int)(local / ((long long)sd.ntx * sd.nty));
        const int x0 = txi * kTileQ * kVEC, y0 = tyi * TY;
        const int z0 = zc * sd.zchunk;
        const int z1 = min(z0 + sd.zchunk, nz);
        const int lin = sd.par ^ a.parity;

        // ---- per-thread geometry
        Pos ps;
        ps.y = y0 - L + r;
        ps.xs = x0 - kVEC + v * kVEC;
        const bool yin = py || (ps.y >= 0 && ps.y < ny);
        const bool xin = px || (ps.xs + kVEC > 0 && ps.xs < nx);
        const bool in_dom = r < NR && yin && xin;
        ps.own = r * kRW + v * kVEC;
        ps.offm = (!py && ps.y == 0) ? ps.own : ps.own - kRW;
        ps.offp = (!py && ps.y == ny - 1) ? ps.own : ps.own + kRW;
        ps.offl = (!px && ps.xs == 0) ? ps.own : ps.own - 1;
        ps.xhi = (!px && ps.xs <= nx - 1 && nx - 1 < ps.xs + kVEC) ? nx - 1 - ps.xs : -1;
        const int yw = py ? wrapi(ps.y, ny) : ps.y;
        // global load of the thread's vector: 1 = one copy, 2 = wrapped
        // element by element, 0 = none
        int ld_mode = 0;
        long long ld_off = 0;
        if (in_dom) {
            const long long row = (long long)yw * sd.pitch;
            if (ps.xs >= 0 && ps.xs < nx && (!px || ps.xs + kVEC <= nx)) {
                ld_mode = 1;
                ld_off = row + ps.xs;
            } else if (px) {
                const int xw = wrapi(ps.xs, nx);
                if (xw % kVEC == 0 && xw + kVEC <= nx) { ld_mode = 1; ld_off = row + xw; }
                else { ld_mode = 2; ld_off = row; }
            }
        }
        // levels this position computes: bit l (l = L: the stored tile)
        unsigned lbits = 0;
        if (in_dom) {
#pragma unroll
            for (int l = 1; l < L; ++l)
                if (r >= l && r < NR - l) lbits |= 1u << l;
            if (r >= L && r < L + TY && v >= 1 && v <= kTileQ && ps.y >= 0 && ps.y < ny &&
                ps.xs < nx)
                lbits |= 1u << L;
        }
        const long long st_off = (long long)ps.y * sd.pitch + ps.xs;
        const bool src_col = sd.src_s >= 0 && yw == sd.src_y;

        // ---- loads: plane ``nld`` (wrapped index zld) into the level-0 ring
        const int pbeg = z0 - L, pend = z1 + L;
        int nld = pbeg;
        int zld = pz ? wrapi(nld, nz) : nld;
        auto issue = [&]() {
            if (nld < pend && ld_mode != 0 && (pz || (nld >= 0 && nld < nz))) {
                const long long zoff = (long long)zld * sd.plane + ld_off;
#pragma unroll
                for (int s = 0; s < S; ++s) {
                    const ST* g = reinterpret_cast<const ST*>(sd.base[lin][s]) + zoff;
                    ST* dst = state_plane(0, s, nld) + ps.own;
                    if (ld_mode == 1) {
                        if (RD_DBG_GLOBAL(sd, g, 4 * (int)sizeof(ST), kSiteCopySrc))
                            Store<ST>::cp_async(dst, g);
                    } else {
#pragma unroll
                        for (int e = 0; e < kVEC; ++e) {
                            const ST* ge = g + wrapi(ps.xs + e, nx);
                            if (RD_DBG_GLOBAL(sd, ge, (int)sizeof(ST), kSiteCopySrc) &&
                                RD_DBG_SHARED(dst + e, (int)sizeof(ST), kSiteCopyDst))
                                dst[e] = *ge;
                        }
                    }
                }
            }
            ++nld;
            if (!pz) zld = nld;
            else if (++zld == nz) zld = 0;
            cp_async_commit();
        };

#pragma unroll 1
        for (int j = 0; j < P; ++j) issue();
        int zcur = pz ? wrapi(pbeg, nz) : pbeg;   // wrapped index of plane p
#pragma unroll 1
        for (int p = pbeg; p < pend; ++p) {
            issue();
            cp_async_wait<P>();
            __syncthreads();
#pragma unroll
            for (int l = 1; l <= L; ++l) {
                const int q = p - l;
                const bool valid = q >= z0 - L + l && q < z1 + L - l && (pz || (q >= 0 && q < nz));
                if (!valid || !(lbits & (1u << l))) continue;
                const bool fin = (l == L);
                int zw = q;
                if (pz) { zw = zcur - l; while (zw < 0) zw += nz; }
                // z neighbours: the face plane itself at a zero-flux z face
                const int qm = (!pz && q == 0) ? q : q - 1;
                const int qp = (!pz && q == nz - 1) ? q : q + 1;
                if constexpr (CH) {
                    if (LY::is_mu(l)) {
                        // mu of the Cahn-Hilliard species from state level l-1
                        float c[kVEC], xm[kVEC], xp[kVEC], ym[kVEC], yp[kVEC], zm[kVEC], zp[kVEC];
                        gather7<ST>(state_plane(l - 1, 2, q), state_plane(l - 1, 2, qm),
                                    state_plane(l - 1, 2, qp), ps, c, xm, xp, ym, yp, zm, zp);
                        float mo[kVEC];
#pragma unroll
                        for (int e = 0; e < kVEC; ++e)
                            mo[e] = M::mu(sd, c[e], xm[e], xp[e], ym[e], yp[e], zm[e], zp[e]);
                        Store<float>::store(mu_plane(l, q) + ps.own, mo);
                        continue;
                    }
                }
                // state update from level ls (and, for Cahn-Hilliard, mu at l-1)
                const int ls = CH ? l - 2 : l - 1;
                float inc[S][kVEC];
                {
                    float cen[S][kVEC];
#pragma unroll
                    for (int s = 0; s < S; ++s) Store<ST>::load(state_plane(ls, s, q) + ps.own, cen[s]);
#pragma unroll
                    for (int e = 0; e < kVEC; ++e) {
                        float cv[S], iv[S];
#pragma unroll
                        for (int s = 0; s < S; ++s) cv[s] = cen[s][e];
                        M::react(sd, cv, iv);
#pragma unroll
                        for (int s = 0; s < S; ++s) inc[s][e] = iv[s];
                    }
                }
                const float cx = courant_at(sd, sd.courant, zw);
                const bool src_here = src_col && zw == sd.src_z;
#pragma unroll
                for (int s = 0; s < S; ++s) {
                    float o[kVEC];
                    if (CH && s == 2) {
                        // c += dt M / h^2 * (7-point Laplacian of mu)
                        float m0[kVEC], mxm[kVEC], mxp[kVEC], mym[kVEC], myp[kVEC], mzm[kVEC],
                            mzp[kVEC], c[kVEC];
                        gather7<float>(mu_plane(l - 1, q), mu_plane(l - 1, qm), mu_plane(l - 1, qp),
                                       ps, m0, mxm, mxp, mym, myp, mzm, mzp);
                        Store<ST>::load(state_plane(ls, 2, q) + ps.own, c);
#pragma unroll
                        for (int e = 0; e < kVEC; ++e) {
                            const float s6 = __fadd_rn(
                                __fadd_rn(__fadd_rn(mxm[e], mxp[e]), __fadd_rn(mym[e], myp[e])),
                                __fadd_rn(mzm[e], mzp[e]));
                            const float lap = __fmaf_rn(-6.0f, m0[e], s6);
                            o[e] = __fadd_rn(c[e], __fmaf_rn(sd.p[1], lap, inc[s][e]));
                        }
                    } else {
                        float c[kVEC], xm[kVEC], xp[kVEC], ym[kVEC], yp[kVEC], zm[kVEC], zp[kVEC];
                        gather7<ST>(state_plane(ls, s, q), state_plane(ls, s, qm),
                                    state_plane(ls, s, qp), ps, c, xm, xp, ym, yp, zm, zp);
                        species_update(sd, s, c, xm, xp, ym, yp, zm, zp, inc[s], cx, src_here, px,
                                       ps.xs, ps.y, q, o);
                    }
                    if (CH && s == 2) held_layers(sd, s, ps.xs, ps.y, q, o);
                    if (fin) {
                        ST* g = reinterpret_cast<ST*>(sd.base[lin ^ 1][s]) +
                                (long long)q * sd.plane + st_off;
                        if (RD_DBG_GLOBAL(sd, g, 4 * (int)sizeof(ST), kSiteStateStore))
                            Store<ST>::store(g, o);
                    } else {
                        // inner level, rounded exactly as a stored state
                        Store<ST>::store(state_plane(l, s, q) + ps.own, o);
                    }
                }
            }
            if (pz && ++zcur == nz) zcur = 0;
        }
        cp_async_wait<0>();
        __syncthreads();
    }
}

// ------------------------------------------------------ one-step kernel
// The T = 1 path of the models without Cahn-Hilliard.  16 x TY compute
// threads, one per 4-cell vector of a 64 x TY tile, plus one halo warp that
// fetches the tile's halo (one row above and below, one vector left and
// right; the 7-point stencil needs no corners).  Planes arrive in a 6-slot
// shared-memory ring: while plane q is computed, planes q-1..q+1 are
// resident and q+2..q+4 in flight (P = 5 copy groups ahead of q-1).  A
// compute thread reads its own vector in planes q-1, q, q+1 and its four
// neighbours in plane q.  The slot refilled at step q held plane q-2: its
// neighbour reads ended two barriers earlier and its own-vector reads
// precede the refill in the owner's program order, so one barrier per plane
// suffices.  The halo warp runs its own copy loop with the same barriers.
template <class M, class ST> struct Layout1 {
    static constexpr int S = M::S;
    static constexpr int RING = 6;
    static constexpr int P = 5;
    __host__ __device__ static int plane_elems(int ty) { return (ty + 2) * kRW + 2 * kVEC; }
    __host__ __device__ static size_t total(int ty) {
        return (size_t)RING * S * plane_elems(ty) * sizeof(ST) + 96 * sizeof(int4);
    }
    __host__ __device__ static int threads(int ty) { return kTileQ * ty + 32; }
};

// How one vector is fetched: 1 = one async copy, 2 = element by element
// (wrapped x, or clamped x for a vector straddling a zero-flux face), 0 =
// nothing (a vector wholly outside a zero-flux x face, or a row outside a
// face that is never read: the kernels take the face cell from the
// thread's own vector instead, see xface_offsets).
struct Fetch {
    int mode;
    int goff;    // element offset of row + x within a plane
    int soff;    // byte offset of the position within a plane buffer
    int xs;      // global x of the vector's first element (unwrapped)
};

template <class ST>
__device__ __forceinline__ Fetch make_fetch(int yrow, int xs, int nx, int ny, int pitch, bool px,
                                            bool py, int soff_elems, bool clamp) {
    Fetch f{0, 0, soff_elems * (int)sizeof(ST), xs};
    int yw = yrow;
    if (py) {
        yw = wrapi(yrow, ny);
    } else if (yrow < 0 || yrow >= ny) {
        if (!clamp) return f;                     // never read
        yw = yrow < 0 ? 0 : ny - 1;               // ghost row = face row
    }
    const int row = yw * pitch;
    if (xs >= 0 && xs + kVEC <= nx) {
        f.mode = 1;
        f.goff = row + xs;
    } else if (px) {
        const int xw = wrapi(xs, nx);
        if (xw % kVEC == 0 && xw + kVEC <= nx) { f.mode = 1; f.goff = row + xw; }
        else { f.mode = 2; f.goff = row; }
    } else if (clamp) {
        if (xs < nx && xs + kVEC > 0) {           // straddles the face: ghost
            f.mode = 2;                           // cells = face cell
            f.goff = row;
        }
    } else if (xs >= 0 && xs < nx) {
        f.mode = 1;                               // last vector: tail in the row padding
        f.goff = row + xs;
    }
    return f;
}

// one fetch of every species of a plane; ``elems`` is true where mode 2 can
// occur (zero-flux x faces, periodic x with nx not a multiple of 4); its
// element copies are 4-byte async copies for FP32, plain loads for BF16
template <class ST, int S>
__device__ __forceinline__ void fetch_all(const Fetch& f, unsigned char* plane_buf, int pe_bytes,
                                          const ST* gplane, long long fstride, int nx,
                                          bool elems, bool px, const InstDesc& sd) {
#pragma unroll
    for (int s = 0; s < S; ++s) {
        const ST* src = gplane + s * fstride + f.goff;
        const int ok =
            f.mode == 1 && RD_DBG_GLOBAL(sd, src, 4 * (int)sizeof(ST), kSiteCopySrc);
        Store<ST>::cp_async_if(reinterpret_cast<ST*>(plane_buf + s * pe_bytes + f.soff), src, ok);
    }
    if (elems && f.mode == 2) {
#pragma unroll
        for (int s = 0; s < S; ++s) {
            ST* d = reinterpret_cast<ST*>(plane_buf + s * pe_bytes + f.soff);
#pragma unroll
            for (int e = 0; e < kVEC; ++e) {
                const int x = f.xs + e;
                const int xi = px ? wrapi(x, nx) : (x < 0 ? 0 : (x >= nx ? nx - 1 : x));
                const ST* src = gplane + s * fstride + f.goff + xi;
                if (RD_DBG_GLOBAL(sd, src, (int)sizeof(ST), kSiteCopySrc))
                    Store<ST>::cp_async_elem(d + e, src);
            }
        }
    }
}

// Byte offsets, from a thread's own vector in a plane buffer, of the x
// neighbours beside it: the element left of element 0 and right of element
// 3.  At a zero-flux x face the ghost there equals the face cell, which is
// the thread's own element 0 (left face) or 3 (a vector ending at the right
// face), so those offsets point into the own vector and the vectors outside
// the face are never copied (element-by-element copies of them had cost a
// quarter of the step).  A vector straddling the right face (nx not a
// multiple of 4) holds its clamped ghosts itself.
template <class ST>
__device__ __forceinline__ void xface_offsets(int xs, int nx, bool px, int& loff, int& roff) {
    constexpr int EB = (int)sizeof(ST);
    loff = (!px && xs == 0) ? 0 : -EB;
    roff = (!px && xs + kVEC == nx) ? (kVEC - 1) * EB : kVEC * EB;
}

template <class ST>
__device__ __forceinline__ void lds_vec(const unsigned char* p, float (&v)[kVEC]) {
    Store<ST>::load(reinterpret_cast<const ST*>(p), v);
}
template <class ST>
__device__ __forceinline__ float lds_one(const unsigned char* p) {
    return Store<ST>::get(reinterpret_cast<const ST*>(p));
}

// Zero-flux ghost cells are copied in as face values at distance one (rows,
// planes, and vectors straddling the face), as the paper sets its boundary
// layer before each step; a thread at an x face reads its x neighbour
// beyond the face from its own vector (xface_offsets).  Every other
// neighbour sits at a fixed offset from the thread's own vector.  An upwind
// inflow face sees a zero gradient, and a held layer's ghost only feeds the
// held cell's own update, which is replaced by its bc value, so this is
// exact for every one-step problem.
// PLAIN: no held layer, point source or wind, and every species isotropic;
// the update then needs no per-plane or per-species branches.  W3: the
// 3-D wind (upwind along y and z too; never with PLAIN).
template <class M, class ST, bool ONE, int MINB, bool PLAIN, bool W3>
__global__ void __launch_bounds__(kMaxThreads, MINB)
rd_step1_kernel(const __grid_constant__ LaunchArgs a) {
    using LY = Layout1<M, ST>;
    constexpr int S = M::S;
    constexpr int P = LY::P;
    constexpr int RING = LY::RING;
    constexpr int EB = (int)sizeof(ST);
    constexpr int RWB = kRW * EB;                            // bytes per shared row

    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ InstDesc sdm;
    __shared__ int s_inst;
    __shared__ long long s_item;

    const int tid = threadIdx.x;
    const int TY = a.ty;
    const int PEB = LY::plane_elems(TY) * EB;                // bytes per species plane
    const int SLOTB = S * PEB;                               // bytes per ring slot
    unsigned char* const ring = smem + kVEC * EB;            // slot 0, species 0
    int4* const hfetch = reinterpret_cast<int4*>(smem + RING * SLOTB);
    const int ncomp = kTileQ * TY;
    const bool halo_warp = tid >= ncomp;
    const int r = tid / kTileQ;
    const int v = tid - r * kTileQ;
    const int own_b = ((r + 1) * kRW + (v + 1) * kVEC) * EB;

    int cur_inst = -1;
    if (tid == 0) s_inst = 0;
    for (long long item = first_item<ONE>(a, s_item); item < a.nitems;
         item = next_item<ONE>(a, item, s_item)) {
        if constexpr (!ONE) load_desc(a, item, sdm, s_inst, cur_inst);
        const InstDesc& sd = desc_of<ONE>(a, sdm);
        if (member_done<ONE>(a, sd)) continue;   // block-uniform

        const int nx = sd.nx, ny = sd.ny, nz = sd.nz, pitch = sd.pitch;
        const bool px = sd.per_x, py = sd.per_y, pz = sd.per_z;
        // element-wise copies: periodic x with nx % 4 != 0, and zero-flux x faces
        const bool elems = sd.wrap_elems || !sd.per_x;
        const long long local = item - sd.item_begin;
        const int txi = (int)(local % sd.ntx);
        const int tyi = (int)((local / sd.ntx) % sd.nty);
        const int zc = (int)(local / ((long long)sd.ntx * sd.nty));
        const int x0 = txi * kTileQ * kVEC, y0 = tyi * TY;
        const int z0 = zc * sd.zchunk;
        const int z1 = min(z0 + sd.zchunk, nz);
        const int lin = sd.par ^ a.parity;
        const ST* const gin = reinterpret_cast<const ST*>(sd.base[lin][0]);
        ST* const gout = reinterpret_cast<ST*>(sd.base[lin ^ 1][0]);
        // the fields of one instance and time level are evenly spaced
        const long long fstride = S > 1 ? reinterpret_cast<const ST*>(sd.base[lin][1]) - gin : 0;
        const long long plane = sd.plane;

        // ---- halo lanes: up to three halo vectors each, described in shared
        // memory (2 TY side vectors, then 2 x 16 row vectors)
        if (halo_warp) {
            const int hl = tid - ncomp;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const int j = hl + 32 * k;
                Fetch f{0, 0, 0, 0};
                if (j < 2 * TY) {
                    const int hr = j >> 1;
                    const bool right = j & 1;
                    const int xh = right ? x0 + kTileQ * kVEC : x0 - kVEC;
                    f = make_fetch<ST>(y0 + hr, xh, nx, ny, pitch, px, py,
                                       (hr + 1) * kRW + (right ? kNQ - 1 : 0) * kVEC, true);
                } else if (j < 2 * TY + 2 * kTileQ) {
                    const int jj = j - 2 * TY;
                    const bool bottom = jj >= kTileQ;
                    const int hv = jj - (bottom ? kTileQ : 0);
                    f = make_fetch<ST>(bottom ? y0 + TY : y0 - 1, x0 + hv * kVEC, nx, ny, pitch, px,
                                       py, (bottom ? TY + 1 : 0) * kRW + (hv + 1) * kVEC, true);
                }
                if (RD_DBG_SHARED(hfetch + j, 16, kSiteHaloDesc))
                    hfetch[j] = make_int4(f.mode, f.goff, f.soff, f.xs);
            }
        }
        // ---- compute threads: own vector and its neighbours
        const int y = y0 + r;
        const int xs = x0 + v * kVEC;
        const bool computes = !halo_warp && y < ny && xs < nx;
        const bool src_col = sd.src_s >= 0 && (py ? wrapi(y, ny) : y) == sd.src_y;
        const unsigned xyf = xy_faces(xs, y, nx, ny);
        const Fetch fo = halo_warp ? Fetch{0, 0, 0, 0}
                                   : make_fetch<ST>(y, xs, nx, ny, pitch, px, py, own_b / EB, true);
        int loff, roff;                           // x neighbours beside the own vector
        xface_offsets<ST>(xs, nx, px, loff, roff);
        float cy = 0.0f, cz = 0.0f;               // 3-D wind
        if constexpr (W3) wind3d(sd, lin, local, cy, cz);
        __syncthreads();   // halo descriptors written

        // ---- the march: plane nld is fetched P planes ahead into slot sl;
        // plane z0 - 1 goes to slot 0, plane q to slot (q - z0 + 1) mod RING
        int nld = z0 - 1;
        int zld = pz ? wrapi(nld, nz) : nld;      // plane index the copy reads
        auto issue = [&](int sl) {
            // zero-flux z: the face plane is copied in as the ghost plane
            const bool in_z = pz || (nld >= 0 && nld < nz);
            if (nld <= z1) {
                const int zs = in_z ? zld : (nld < 0 ? 0 : nz - 1);
                const ST* gld = gin + (long long)zs * plane;
                unsigned char* buf = ring + sl * SLOTB;
                if (halo_warp) {
                    const int hl = tid - ncomp;
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        int4 h = make_int4(0, 0, 0, 0);
                        if (RD_DBG_SHARED(hfetch + hl + 32 * k, 16, kSiteHaloDesc))
                            h = hfetch[hl + 32 * k];
                        fetch_all<ST, S>(Fetch{h.x, h.y, h.z, h.w}, buf, PEB, gld, fstride, nx,
                                         elems, px, sd);
                    }
                } else {
                    fetch_all<ST, S>(fo, buf, PEB, gld, fstride, nx, elems, px, sd);
                }
            }
            ++nld;
            if (!pz) zld = nld;
            else if (++zld == nz) zld = 0;
            cp_async_commit();
        };
#pragma unroll 1
        for (int j = 0; j < P; ++j) issue(j);
        int zq = pz ? wrapi(z0, nz) : z0;       // wrapped index of plane q
        ST* gst = gout + (long long)z0 * plane + (long long)y * pitch + xs;
        const float* courant = sd.courant;
        int sc = 1;                               // ring slot of plane q
        // own vectors of planes q-1 and q, carried down the march
        float own_m[S][kVEC], own_0[S][kVEC];
#pragma unroll 1
        for (int q = z0; q < z1; ++q) {
            const int sm = sc == 0 ? RING - 1 : sc - 1;
            const int sp = sc == RING - 1 ? 0 : sc + 1;
            // planes up to q + 1 must have landed: of the P + (q - z0 + 1)
            // groups issued so far, all but the newest P - 2
            issue(sc >= RING - P + 1 ? sc + P - 1 - RING : sc + P - 1);
            cp_async_wait<P - 2>();
            __syncthreads();
            if (!halo_warp) {
                // every neighbour at a fixed offset; ghosts were copied in
                const unsigned char* Pc = ring + sc * SLOTB + own_b;
                const unsigned char* Pp = ring + sp * SLOTB + own_b;
                if (q == z0) {
                    const unsigned char* Pm = ring + sm * SLOTB + own_b;
#pragma unroll
                    for (int s = 0; s < S; ++s) {
                        lds_vec<ST>(Pm + s * PEB, own_m[s]);
                        lds_vec<ST>(Pc + s * PEB, own_0[s]);
                    }
                }
                float own_p[S][kVEC], inc[S][kVEC];
#pragma unroll
                for (int s = 0; s < S; ++s) lds_vec<ST>(Pp + s * PEB, own_p[s]);
                auto& cen = own_0;
#pragma unroll
                for (int e = 0; e < kVEC; ++e) {
                    float cv[S], iv[S];
#pragma unroll
                    for (int s = 0; s < S; ++s) cv[s] = cen[s][e];
                    M::react(sd, cv, iv);
#pragma unroll
                    for (int s = 0; s < S; ++s) inc[s][e] = iv[s];
                }
                const float cx = courant_at(sd, courant, zq);
                const bool src_here = src_col && zq == sd.src_z;
                const unsigned faces = xyf | z_faces(q, nz);
#pragma unroll
                for (int s = 0; s < S; ++s) {
                    const unsigned char* Ps = Pc + s * PEB;
                    float xm[kVEC], xp[kVEC], ym[kVEC], yp[kVEC], o[kVEC];
                    const float (&zm)[kVEC] = own_m[s];
                    const float (&zp)[kVEC] = own_p[s];
                    lds_vec<ST>(Ps - RWB, ym);
                    lds_vec<ST>(Ps + RWB, yp);
                    const float left = lds_one<ST>(Ps + loff);
                    const float right = lds_one<ST>(Ps + roff);
#pragma unroll
                    for (int e = 0; e < kVEC; ++e) {
                        xm[e] = e ? cen[s][e - 1] : left;
                        xp[e] = (e < kVEC - 1) ? cen[s][e + 1] : right;
                    }
                    if constexpr (PLAIN) {
                        // the same arithmetic species_update takes for this case
                        const float k = sd.kx[s];
#pragma unroll
                        for (int e = 0; e < kVEC; ++e)
                            o[e] = euler_cell_iso(cen[s][e], xm[e], xp[e], ym[e], yp[e], zm[e],
                                                  zp[e], k, inc[s][e]);
                    } else {
                        species_core(sd, s, cen[s], xm, xp, ym, yp, zm, zp, inc[s], cx, src_here,
                                     px, xs, o, cy, cz);
                        held_layers_at(sd, s, faces, xs, y, q, o);
                    }
                    if (computes &&
                        RD_DBG_GLOBAL(sd, gst + s * fstride, 4 * (int)sizeof(ST), kSiteStateStore))
                        Store<ST>::store(gst + s * fstride, o);
                }
#pragma unroll
                for (int s = 0; s < S; ++s)
#pragma unroll
                    for (int e = 0; e < kVEC; ++e) {
                        own_m[s][e] = own_0[s][e];
                        own_0[s][e] = own_p[s][e];
                    }
            }
            gst += plane;
            sc = sc == RING - 1 ? 0 : sc + 1;
            if (!pz) zq = q + 1;
            else if (++zq == nz) zq = 0;
        }
        cp_async_wait<0>();
        __syncthreads();
    }
}
}  // namespace rdk

#include "rd_step1w_kernel.cuh"
#include "rd_stepch_kernel.cuh"

namespace rdk {

// Launch helper used by the per-model translation units.
template <class M, class ST, int T, bool ONE>
cudaError_t launch_one(const LaunchArgs& a, int grid, size_t smem, cudaStream_t st, int* occ) {
    // the one-step kernel needs an even tile height (16 ty compute threads,
    // then a whole halo warp); an odd one -- the last launch of a call whose
    // tuning steps 2 or 3 per launch -- runs the multi-level kernel at T = 1
    const bool lean = (T == 1 && !M::CH) && !(a.ty & 1);
    constexpr bool lean_ch = (T == 1 && M::CH);
    void (*k)(const LaunchArgs);
    // 8 cells per thread: the one-step kernel of rd_step1w_kernel.cuh
    const bool wide = lean && a.vw == 8;
    if constexpr (lean_ch) {
        k = a.plain ? rd_stepch_kernel<M, ST, ONE, true> : rd_stepch_kernel<M, ST, ONE, false>;
    } else if (wide) {
        k = a.plain  ? rd_step1w_kernel<M, ST, ONE, true, false>
            : a.wind3 ? rd_step1w_kernel<M, ST, ONE, false, true>
                      : rd_step1w_kernel<M, ST, ONE, false, false>;
    } else if (lean) {
        // register budget of the one-step kernel: 128 (regcap 0) or 64 (regcap 1)
        if (a.plain)
            k = a.regcap ? rd_step1_kernel<M, ST, ONE, 2, true, false>
                         : rd_step1_kernel<M, ST, ONE, 1, true, false>;
        else if (a.wind3)
            k = a.regcap ? rd_step1_kernel<M, ST, ONE, 2, false, true>
                         : rd_step1_kernel<M, ST, ONE, 1, false, true>;
        else
            k = a.regcap ? rd_step1_kernel<M, ST, ONE, 2, false, false>
                         : rd_step1_kernel<M, ST, ONE, 1, false, false>;
    } else {
        k = rd_step_kernel<M, ST, T, ONE>;
    }
    // dynamic shared memory granted so far, per kernel variant (4: the
    // multi-level kernel at T = 1; 5, 6: the one-step kernel with 3-D wind;
    // 7, 8, 9: the 8-cell kernel, plain, 3-D wind, general)
    static size_t configured[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    const int variant = wide ? (a.plain ? 7 : a.wind3 ? 8 : 9)
                        : (T == 1 && !M::CH && !lean) ? 4
                        : (lean && !a.plain && a.wind3) ? 5 + (a.regcap ? 1 : 0)
                        : (lean && a.regcap ? 1 : 0) + ((lean || lean_ch) && a.plain ? 2 : 0);
    size_t& conf = configured[variant];
    if (smem > conf) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        conf = smem;
    }
    const int threads = wide      ? Layout1w<M, ST>::threads(a.ty)
                        : lean    ? Layout1<M, ST>::threads(a.ty)
                        : lean_ch ? LayoutCH<ST>::threads(a.ty)
                                  : Layout<M, ST, T>::threads(a.ty);
    if (threads > kMaxThreads) return cudaErrorInvalidConfiguration;
    if (occ) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k, threads, smem);
    k<<<grid, threads, smem, st>>>(a);
    return cudaGetLastError();
}

template <class M, bool ONE>
cudaError_t launch_var(int storage, int tsteps, const LaunchArgs& a, int grid, size_t smem,
                       cudaStream_t st, int* occ) {
    if (storage == RD_STORE_F32) {
        switch (tsteps) {
        case 1: return launch_one<M, float, 1, ONE>(a, grid, smem, st, occ);
        case 2: return launch_one<M, float, 2, ONE>(a, grid, smem, st, occ);
        case 3: if constexpr (!M::CH) return launch_one<M, float, 3, ONE>(a, grid, smem, st, occ);
                break;
        default: break;
        }
    } else {
        switch (tsteps) {
        case 1: return launch_one<M, __nv_bfloat16, 1, ONE>(a, grid, smem, st, occ);
        case 2: return launch_one<M, __nv_bfloat16, 2, ONE>(a, grid, smem, st, occ);
        case 3:
            if constexpr (!M::CH) return launch_one<M, __nv_bfloat16, 3, ONE>(a, grid, smem, st, occ);
            break;
        default: break;
        }
    }
    return cudaErrorInvalidValue;
}

template <class M>
cudaError_t launch_model(int storage, int tsteps, const LaunchArgs& a, int grid, size_t smem,
                         cudaStream_t st, int* occ) {
    return a.use_one ? launch_var<M, true>(storage, tsteps, a, grid, smem, st, occ)
                     : launch_var<M, false>(storage, tsteps, a, grid, smem, st, occ);
}

template <class M>
size_t smem_for(int storage, int tsteps, int ty, int vw = 4) {
    if (tsteps == 1 && !M::CH && vw == 8)
        return storage == RD_STORE_F32 ? Layout1w<M, float>::total(ty)
                                       : Layout1w<M, __nv_bfloat16>::total(ty);
    if (storage == RD_STORE_F32) {
        switch (tsteps) {
        case 1: return M::CH ? LayoutCH<float>::total(ty)
                             : (ty & 1) ? Layout<M, float, 1>::total(ty) : Layout1<M, float>::total(ty);
        case 2: return Layout<M, float, 2>::total(ty);
        case 3: return Layout<M, float, 3>::total(ty);
        }
    } else {
        switch (tsteps) {
        case 1: return M::CH ? LayoutCH<__nv_bfloat16>::total(ty)
                             : (ty & 1) ? Layout<M, __nv_bfloat16, 1>::total(ty)
                                        : Layout1<M, __nv_bfloat16>::total(ty);
        case 2: return Layout<M, __nv_bfloat16, 2>::total(ty);
        case 3: return Layout<M, __nv_bfloat16, 3>::total(ty);
        }
    }
    return 0;
}

}  // namespace rdk
