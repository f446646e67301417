// rd_resident.cu -- the resident step kernel (RD_KERNEL_RESIDENT): one
// cooperative launch advances many steps of a problem whose state stays in
// L2, a few steps per grid barrier.
//
// The one-step march kernels pay, per step, a launch and the fill of a
// plane pipeline for every work item; on a grid of a megabyte or so (the
// 64^3 inert-diffusion problem) that latency, not memory, sets the rate.
// Here every CTA of a cooperative launch (all CTAs resident at once) owns
// tiles of ty x tz full x rows.  A round of K steps copies a tile's rows
// with a halo of K rows and planes into shared memory (16-byte asynchronous
// copies that bypass L1, since other SMs wrote the level), computes levels
// 1..K on regions shrinking by one row and plane per side per level, and
// writes level K of the tile's own rows; then the grid meets at a barrier
// and the two time levels swap roles.  A halo row beyond a zero-flux face
// is never loaded: its neighbour reads resolve to the face row, as the
// march kernels' ghost copies do; periodic rows wrap.  Each level is
// rounded to the state's type, and every cell is updated by the march
// kernels' per-cell code (euler_cell_iso, species_core, held_layers_at) on
// the same neighbour values, so results equal the march kernel's bit for
// bit.  K levels need a halo of K: (ty+2K)(tz+2K) rows are loaded for ty*tz
// rows kept, and levels below K are computed on the overlaps as well; the
// plan (plan_resident) trades that against one barrier per round.
//
// The barrier counts CTA arrivals over the whole launch: barrier k is
// passed once the count reaches k times the grid, so nothing is reset
// between rounds.  Thread 0 of a CTA arrives with a release add after the
// CTA's barrier and waits with acquire loads; the CTA's next copies follow
// another CTA barrier.  Every wait is bounded: after 0.2 s (the GPU's
// global timer) the waiting CTA raises the barrier's error word and leaves;
// every other CTA sees the word while it waits and leaves too, and rd_sync
// reports RD_ETIMEOUT.  The host zeroes the count and the word before every
// launch.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <vector>

#include "rd_model_turing.h"
#include "rd_resident.h"
#include "rd_step_kernel.cuh"

namespace rdk {
namespace {

constexpr unsigned long long kWaitNs = 200000000ull;   // 0.2 s per barrier wait
constexpr unsigned kPollLimit = 1u << 24;               // backstop on the polls
constexpr int kResSmemMax = 200 * 1024;                 // shared memory a plan may take
constexpr int kResThreads = 512;                        // threads per CTA

// Tensor maps of the state's two time levels, each a 4-D tensor (row
// elements of the pitch, rows, planes, species) whose box is one tile with
// its K-halo for every species.
struct ResidentMaps {
    CUtensorMap map[2];
};

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void red_release_add(unsigned* p, unsigned v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned ld_relaxed(const unsigned* p) {
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid-wide barrier ``k`` (1, 2, ...) of the launch, waits bounded; false
// when the launch must stop.  ``phantom`` CTAs never arrive (0 except in
// the test of the timeout).
__device__ bool grid_barrier(ResidentBar* bar, unsigned k, unsigned phantom) {
    __shared__ int go;
    __syncthreads();
    if (threadIdx.x == 0) {
        go = 1;
        red_release_add(&bar->count, 1u);
        const unsigned target = k * (gridDim.x + phantom);
        const unsigned long long t0 = global_ns();
        unsigned polls = 0;
        while (ld_acquire(&bar->count) < target) {
            if ((++polls & 15) == 0) {
                if (ld_relaxed(&bar->err)) { go = 0; break; }
                if (polls > kPollLimit || global_ns() - t0 > kWaitNs) {
                    atomicExch(&bar->err, 1u);
                    atomicExch(&bar->failed, 1u);
                    go = 0;
                    break;
                }
            }
        }
    }
    __syncthreads();
    return go != 0;
}

// 16-byte copy global -> shared that bypasses L1 (the debug build checks
// both sides and skips a copy out of range).
__device__ __forceinline__ void copy16(const InstDesc& sd, void* smem, const void* g) {
    if (!RD_DBG_SHARED(smem, 16, kSiteCopyDst) || !RD_DBG_GLOBAL(sd, g, 16, kSiteStateLoad))
        return;
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(g) : "memory");
}

// Tensor-memory copies (TMA) of a tile: one 4-D box (row elements x rows x
// planes x species) per tile and round, issued by one thread and counted
// on a shared-memory mbarrier.
__device__ __forceinline__ unsigned smem_addr(const void* p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(unsigned long long* b) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(b)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* b, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(b)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* b, unsigned parity) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_addr(b)), "r"(parity)
        : "memory");
    return done != 0;
}
// Wait for phase ``parity`` of the mbarrier, bounded by kWaitNs.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* b, unsigned parity) {
    const unsigned long long t0 = global_ns();
    for (unsigned polls = 0;; ++polls) {
        if (mbar_try_wait(b, parity)) return true;
        if (polls > kPollLimit || global_ns() - t0 > kWaitNs) return false;
    }
}
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int x, int y, int z,
                                            int w, unsigned long long* b) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_addr(dst)),
        "l"(map), "r"(x), "r"(y), "r"(z), "r"(w), "r"(smem_addr(b))
        : "memory");
}

// Global index of the unwrapped row (or plane) ``v`` on an axis of n:
// wrapped on a periodic axis (v lies within a few periods of the axis, so
// conditional steps replace a division); false beyond a zero-flux face.
__device__ __forceinline__ bool map_row(int v, int n, bool per, int& out) {
    if (per) {
        while (v < 0) v += n;
        while (v >= n) v -= n;
        out = v;
        return true;
    }
    out = v;
    return v >= 0 && v < n;
}

// q = a / b, r = a % b for 0 <= a < 2^20, 0 < b < 2^20, through the
// correctly rounded float reciprocal ``rb`` of b: (a + 0.5) / b lies at
// least 0.5 / b from an integer, and the float product errs by under
// 3 * 2^-24 relative, which stays below that margin while a < 2^20.
__device__ __forceinline__ void divmod_small(int a, int b, float rb, int& q, int& r) {
    q = __float2int_rz(__fmul_rn(__int2float_rn(a) + 0.5f, rb));
    r = a - q * b;
}

// A thread's place in the CTA's walks over regions of ``cols`` columns
// (items row-major, the CTA's threads taking consecutive items): its first
// item's column and row, and one stride of blockDim.x items, split once.
struct Lane {
    int col, row, dcol, drow;
    __device__ __forceinline__ explicit Lane(int cols) {
        const int t = threadIdx.x, T = blockDim.x;
        col = t % cols;
        row = t / cols;
        dcol = T % cols;
        drow = T / cols;
    }
};

// A thread's walk over the items of a region whose rows are numbered
// lz * iy + ly; each step is adds and compares.
struct Walk {
    int col, ly, lz;          // the current item
    int dcol, dly, dlz;       // one stride of blockDim.x items
    __device__ __forceinline__ Walk(const Lane& l, int iy) {
        const float rb = __frcp_rn(__int2float_rn(iy));
        col = l.col;
        dcol = l.dcol;
        divmod_small(l.row, iy, rb, lz, ly);
        divmod_small(l.drow, iy, rb, dlz, dly);
    }
    __device__ __forceinline__ void next(int cols, int iy) {
        col += dcol;
        ly += dly;
        lz += dlz;
        if (col >= cols) { col -= cols; ++ly; }
        if (ly >= iy) { ly -= iy; ++lz; }
    }
};

// 512 threads per CTA (1024, which the plain update would fit in 64
// registers, measured no faster: the rounds are not bound by per-thread
// latency).
// TMA: the tile and its K-halo arrive as one tensor-memory box per round
// (``tm`` holds the tensor maps of the two time levels); else per-thread
// 16-byte copies.  Rows of a zero-flux halo that lie beyond the face are
// filled with zeros by the box and never read.
template <class M, class ST, bool PLAIN, bool TMA>
__global__ void __launch_bounds__(kResThreads, 1)
rd_resident_kernel(const __grid_constant__ LaunchArgs a, const ResidentPlan p, int nsteps,
                   ResidentBar* bar, unsigned phantom, const __grid_constant__ ResidentMaps tm) {
    constexpr int S = M::S;
    constexpr int ES = (int)sizeof(ST);
    constexpr int CE = 16 / ES;                        // elements per 16-byte copy
    extern __shared__ __align__(16) unsigned char res_smem[];
    __shared__ unsigned long long mbar;
    __shared__ int tma_ok;
    const InstDesc& sd = a.one;
    const int nx = sd.nx, ny = sd.ny, nz = sd.nz, pitch = sd.pitch;
    const bool px = sd.per_x, py = sd.per_y, pz = sd.per_z;
    const int nvx = (nx + kVEC - 1) / kVEC;
    const long long plane = sd.plane;
    const int K = p.K, ty = p.ty, tz = p.tz, rw = p.rw;
    const int RY = ty + 2 * K;                         // local rows per plane (layout)
    const int PW = RY * rw;                            // elements per local plane
    const int fsm = PW * (tz + 2 * K);                 // elements per species
    // buffers start on a 128-byte boundary (the box destination)
    ST* const sbase = reinterpret_cast<ST*>(
        res_smem + ((128u - (smem_addr(res_smem) & 127u)) & 127u));
    const int cpr = rw / CE;                           // copies per row
    const int ntiles = p.nty * p.ntz;
    const int rounds = (nsteps + K - 1) / K;
    // x neighbours beyond the row ends
    const int xl0 = px ? nx - 1 : 0;                   // left of cell 0
    const int xr0 = px ? 0 : nx - 1;                   // right of cell nx - 1
    const Lane lcopy(cpr), lcell(nvx);
    unsigned tma_phase = 0;
    if constexpr (TMA) {
        if (threadIdx.x == 0) mbar_init(&mbar);
        __syncthreads();
    }
    int lin = sd.par ^ a.parity;
    for (int r = 0; r < rounds; ++r) {
        const int H = min(K, nsteps - r * K);          // steps and halo of this round
        const ST* const gin = reinterpret_cast<const ST*>(sd.base[lin][0]);
        ST* const gout = reinterpret_cast<ST*>(sd.base[lin ^ 1][0]);
        const long long fstride =
            S > 1 ? reinterpret_cast<const ST*>(sd.base[lin][1]) - gin : 0;
        for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
            const int oy = (tile % p.nty) * ty, oz = (tile / p.nty) * tz;   // owned origin
            // local row 0 is unwrapped row oy - K (plane oz - K); a round of
            // H < K steps uses the rows from o = K - H on
            const int y0 = oy - K, z0 = oz - K, o = K - H;
            const int ry = ty + 2 * H, rz = tz + 2 * H;
            // level 0: the rows of the tile and its halo
            if constexpr (TMA) {
                if (threadIdx.x == 0) {
                    // order the CTA's generic accesses (last tile's reads of
                    // the buffers, the grid barrier's acquire) before the
                    // asynchronous copy
                    asm volatile("fence.proxy.async;" ::: "memory");
                    const unsigned bytes = (unsigned)(S * fsm * ES);
                    bool ok = RD_DBG_SHARED(sbase, (int)bytes, kSiteCopyDst);
                    if (ok) {
                        mbar_expect_tx(&mbar, bytes);
                        tma_load_4d(sbase, &tm.map[lin], 0, y0, z0, 0, &mbar);
                        ok = mbar_wait_bounded(&mbar, tma_phase);
                        if (!ok) mbar_wait_bounded(&mbar, tma_phase);   // copies in flight
                    }
                    tma_phase ^= 1u;
                    tma_ok = ok;
                    if (!ok) {
                        atomicExch(&bar->err, 1u);
                        atomicExch(&bar->failed, 1u);
                    }
                }
                __syncthreads();
                if (!tma_ok) return;
            } else {
#pragma unroll
                for (int s = 0; s < S; ++s)
                    for (Walk w(lcopy, ry); w.lz < rz; w.next(cpr, ry)) {
                        int y, z;
                        const int ly = o + w.ly, lz = o + w.lz;
                        if (!map_row(y0 + ly, ny, py, y) || !map_row(z0 + lz, nz, pz, z))
                            continue;
                        copy16(sd, sbase + s * fsm + lz * PW + ly * rw + w.col * CE,
                               gin + s * fstride + (long long)z * plane + (long long)y * pitch +
                                   w.col * CE);
                    }
                asm volatile("cp.async.wait_all;\n" ::: "memory");
                __syncthreads();
            }
            for (int j = 1; j <= H; ++j) {
                const ST* const src = sbase + ((j - 1) & 1) * S * fsm;
                ST* const dst = sbase + (j & 1) * S * fsm;
                const int iy = ty + 2 * (H - j), iz = tz + 2 * (H - j);
                const bool last = j == H;
                for (Walk w(lcell, iy); w.lz < iz; w.next(nvx, iy)) {
                    const int ly = o + j + w.ly, lz = o + j + w.lz;
                    int y, z;
                    if (!map_row(y0 + ly, ny, py, y) || !map_row(z0 + lz, nz, pz, z)) continue;
                    // the last level keeps the tile's own rows (a last tile may
                    // reach past the grid's end)
                    if (last && (y0 + ly >= ny || z0 + lz >= nz)) continue;
                    const int xs = w.col * kVEC;
                    // neighbour rows and planes: beyond a zero-flux face, the face
                    const int own = lz * PW + ly * rw;
                    const int rym = own - ((!py && y == 0) ? 0 : rw);
                    const int ryq = own + ((!py && y == ny - 1) ? 0 : rw);
                    const int rzm = own - ((!pz && z == 0) ? 0 : PW);
                    const int rzq = own + ((!pz && z == nz - 1) ? 0 : PW);
                    const bool tail = xs + kVEC >= nx;  // holds cell nx - 1
                    const int elast = nx - 1 - xs;
                    const int xl = xs > 0 ? xs - 1 : xl0;
                    const int xr = tail ? xr0 : xs + kVEC;
                    float cen[S][kVEC], inc[S][kVEC];
#pragma unroll
                    for (int s = 0; s < S; ++s) Store<ST>::load(src + s * fsm + own + xs, cen[s]);
#pragma unroll
                    for (int e = 0; e < kVEC; ++e) {
                        float cv[S], iv[S];
#pragma unroll
                        for (int s = 0; s < S; ++s) cv[s] = cen[s][e];
                        M::react(sd, cv, iv);
#pragma unroll
                        for (int s = 0; s < S; ++s) inc[s][e] = iv[s];
                    }
                    const float cx = PLAIN ? 0.0f : courant_at(sd, sd.courant, z);
                    const bool src_here = sd.src_s >= 0 && y == sd.src_y && z == sd.src_z;
                    const unsigned faces = xy_faces(xs, y, nx, ny) | z_faces(z, nz);
#pragma unroll
                    for (int s = 0; s < S; ++s) {
                        const ST* f = src + s * fsm;
                        float yv[kVEC], yw[kVEC], zv[kVEC], zw[kVEC], xm[kVEC], xp[kVEC], o[kVEC];
                        Store<ST>::load(f + rym + xs, yv);
                        Store<ST>::load(f + ryq + xs, yw);
                        Store<ST>::load(f + rzm + xs, zv);
                        Store<ST>::load(f + rzq + xs, zw);
                        const float left = Store<ST>::get(f + own + xl);
                        const float right = Store<ST>::get(f + own + xr);
#pragma unroll
                        for (int e = 0; e < kVEC; ++e) {
                            xm[e] = e ? cen[s][e - 1] : left;
                            xp[e] = (e < kVEC - 1 && !(tail && e == elast)) ? cen[s][e + 1]
                                                                             : right;
                        }
                        if constexpr (PLAIN) {
                            const float k = sd.kx[s];
#pragma unroll
                            for (int e = 0; e < kVEC; ++e)
                                o[e] = euler_cell_iso(cen[s][e], xm[e], xp[e], yv[e], yw[e],
                                                      zv[e], zw[e], k, inc[s][e]);
                        } else {
                            species_core(sd, s, cen[s], xm, xp, yv, yw, zv, zw, inc[s], cx,
                                         src_here, px, xs, o);
                            held_layers_at(sd, s, faces, xs, y, z, o);
                        }
                        if (last) {
                            ST* g = gout + s * fstride + (long long)z * plane +
                                    (long long)y * pitch + xs;
                            if (RD_DBG_GLOBAL(sd, g, kVEC * ES, kSiteStateStore))
                                Store<ST>::store(g, o);
                        } else {
                            // the level rounded to the state's type, as a march
                            // kernel stores it
                            Store<ST>::store(dst + s * fsm + own + xs, o);
                        }
                    }
                }
                __syncthreads();
            }
        }
        if (r + 1 < rounds && !grid_barrier(bar, (unsigned)(r + 1), phantom)) return;
        lin ^= 1;
    }
}

using KernelFn = void (*)(const LaunchArgs, const ResidentPlan, int, ResidentBar*, unsigned,
                          const ResidentMaps);

template <class M, class ST>
KernelFn kernel_for(bool plain, bool tma) {
    if (tma) return plain ? rd_resident_kernel<M, ST, true, true> : rd_resident_kernel<M, ST, false, true>;
    return plain ? rd_resident_kernel<M, ST, true, false> : rd_resident_kernel<M, ST, false, false>;
}

// cuTensorMapEncodeTiled from the driver, found once through the runtime
// (no link against the driver library); null when unavailable.
using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                              const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                              const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                              CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeFn encoder() {
    static const EncodeFn fn = []() -> EncodeFn {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000,
                                             cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return nullptr;
        return reinterpret_cast<EncodeFn>(f);
    }();
    return fn;
}

// The two levels' tensor maps for plan ``p``; false if they cannot be made
// (the launch then copies per thread).  Every stride is a multiple of 16
// bytes (rows are padded to 128 bytes, fields to 256) and the box's inner
// extent, rw elements, is too.
template <class ST>
bool encode_maps(const InstDesc& d, int S, const ResidentPlan& p, ResidentMaps* out) {
    constexpr int ES = (int)sizeof(ST);
    const EncodeFn enc = encoder();
    if (!enc) return false;
    for (int l = 0; l < 2; ++l) {
        const long long level = (long long)d.plane * d.nz * ES;
        const long long fbytes =
            S > 1 ? (long long)(d.base[l][1] - d.base[l][0]) : (level + 15) / 16 * 16;
        const cuuint64_t dims[4] = {(cuuint64_t)d.pitch, (cuuint64_t)d.ny, (cuuint64_t)d.nz,
                                    (cuuint64_t)S};
        const cuuint64_t strides[3] = {(cuuint64_t)d.pitch * ES, (cuuint64_t)d.plane * ES,
                                       (cuuint64_t)fbytes};
        const cuuint32_t box[4] = {(cuuint32_t)p.rw, (cuuint32_t)(p.ty + 2 * p.K),
                                   (cuuint32_t)(p.tz + 2 * p.K), (cuuint32_t)S};
        const cuuint32_t estr[4] = {1, 1, 1, 1};
        const CUtensorMapDataType dt =
            ES == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
        if (enc(&out->map[l], dt, 4, d.base[l][0], dims, strides, box, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) !=
            CUDA_SUCCESS)
            return false;
    }
    return true;
}

// Cost model of a plan, in microseconds per step: a round costs a barrier,
// then per tile a CTA handles, a copy round trip, the copies and the cell
// updates its threads make (levels 1..K over the shrinking regions), with
// the SM's CTAs sharing its issue slots.  The constants are measured
// orders of magnitude on this GPU; only the ranking of plans matters.
// With tensor-memory copies the per-thread copies vanish and the box's
// round trip remains.
constexpr double kBarrierUs = 1.4, kCopyTripUs = 0.66, kCopyUs = 0.24, kUpdateUs = 0.37;

double plan_cost(int S, int nvx, int rw, int ES, int K, int ty, int tz, long long tiles,
                 long long grid, int sms, int nt, bool tma) {
    const double threads = nt;
    const long long waves = (tiles + grid - 1) / grid;
    const long long per_sm = (grid + sms - 1) / sms;
    const double copies =
        tma ? 0.0
            : std::ceil((double)S * (ty + 2 * K) * (tz + 2 * K) * (rw * ES / 16) / threads);
    double updates = 0.0;
    for (int j = 1; j <= K; ++j)
        updates += std::ceil((double)(ty + 2 * (K - j)) * (tz + 2 * (K - j)) * nvx / threads);
    const double tile_us = kCopyTripUs + (copies * kCopyUs + updates * S * kUpdateUs) * per_sm;
    return (kBarrierUs + waves * tile_us) / K;
}

// Candidate tile extents along an axis of n rows: powers of two below n,
// and n; or the forced extent.
std::vector<int> extents(int n, int forced) {
    std::vector<int> v;
    if (forced > 0) {
        v.push_back(std::min(forced, n));
        return v;
    }
    for (int t = 1; t < n; t *= 2) v.push_back(t);
    v.push_back(n);
    return v;
}

template <class M, class ST>
cudaError_t plan_st(bool plain, bool tma_ok, int nx, int ny, int nz, int Kf, int tyf, int tzf,
                    ResidentPlan* out) {
    constexpr int S = M::S;
    constexpr int ES = (int)sizeof(ST);
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int nvx = (nx + kVEC - 1) / kVEC;
    const int rw = (nvx * kVEC + 16 / ES - 1) / (16 / ES) * (16 / ES);
    // tensor-memory copies: a box extent is at most 256 elements, and the
    // driver must offer the encoder
    const bool tma = tma_ok && rw <= 256 && S <= 256 && encoder() != nullptr;
    const KernelFn kfn = kernel_for<M, ST>(plain, tma);
    const int nt = kResThreads;
    e = cudaFuncSetAttribute(reinterpret_cast<const void*>(kfn),
                             cudaFuncAttributeMaxDynamicSharedMemorySize, kResSmemMax + 128);
    if (e != cudaSuccess) return e;
    const std::vector<int> tys = extents(ny, tyf), tzs = extents(nz, tzf);
    double best = 1e300;
    bool found = false;
    for (int K = 1; K <= kResidentMaxK; ++K) {
        if (Kf > 0 && K != std::min(Kf, kResidentMaxK)) continue;
        for (int ty : tys)
            for (int tz : tzs) {
                const long long bufs = K == 1 ? 1 : 2;
                const long long buf_bytes =
                    bufs * S * (ty + 2 * K) * (tz + 2 * K) * (long long)rw * ES;
                if (buf_bytes > kResSmemMax) continue;
                if (tma && (ty + 2 * K > 256 || tz + 2 * K > 256)) continue;
                const long long smem = buf_bytes + 128;   // 128-byte alignment of the buffers
                int occ = 0;
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kfn, nt, (size_t)smem);
                if (e != cudaSuccess) return e;
                if (occ < 1) continue;
                const long long nty = (ny + ty - 1) / ty, ntz = (nz + tz - 1) / tz;
                const long long tiles = nty * ntz;
                if (tiles > INT_MAX) continue;    // the kernel counts tiles in int
                const long long grid = std::min<long long>(tiles, (long long)occ * sms);
                const double cost =
                    plan_cost(S, nvx, rw, ES, K, ty, tz, tiles, grid, sms, nt, tma);
                if (cost < best) {
                    best = cost;
                    found = true;
                    *out = ResidentPlan{K,  ty,         tz, (int)nty,   (int)ntz,
                                        rw, (int)grid, nt, (int)smem, tma ? 1 : 0};
                }
            }
    }
    return found ? cudaSuccess : cudaErrorInvalidValue;
}

template <class M>
cudaError_t plan_model(int storage, bool plain, bool tma_ok, int nx, int ny, int nz, int K,
                       int ty, int tz, ResidentPlan* out) {
    if (storage == RD_STORE_F32)
        return plan_st<M, float>(plain, tma_ok, nx, ny, nz, K, ty, tz, out);
    if (storage == RD_STORE_BF16)
        return plan_st<M, __nv_bfloat16>(plain, tma_ok, nx, ny, nz, K, ty, tz, out);
    return cudaErrorInvalidValue;
}

template <class M, class ST>
cudaError_t launch_st(const LaunchArgs& a, const ResidentPlan& p, int nsteps, ResidentBar* bar,
                      unsigned phantom, cudaStream_t st) {
    ResidentMaps maps{};
    // the maps name this launch's addresses; without them, per-thread copies
    const bool tma = p.tma && encode_maps<ST>(a.one, M::S, p, &maps);
    const KernelFn k = kernel_for<M, ST>(a.plain != 0, tma);
    if (!tma && p.tma) {
        const cudaError_t e = cudaFuncSetAttribute(reinterpret_cast<const void*>(k),
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   kResSmemMax + 128);
        if (e != cudaSuccess) return e;
    }
    LaunchArgs args = a;
    ResidentPlan plan = p;
    void* params[] = {&args, &plan, &nsteps, &bar, &phantom, &maps};
    return cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(k), dim3(p.grid),
                                       dim3(p.threads), params, (size_t)p.smem, st);
}

template <class M>
cudaError_t launch_model(int storage, const LaunchArgs& a, const ResidentPlan& p, int nsteps,
                         ResidentBar* bar, unsigned phantom, cudaStream_t st) {
    if (storage == RD_STORE_F32) return launch_st<M, float>(a, p, nsteps, bar, phantom, st);
    if (storage == RD_STORE_BF16)
        return launch_st<M, __nv_bfloat16>(a, p, nsteps, bar, phantom, st);
    return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t plan_resident(int model, int storage, bool plain, bool tma_ok, int nx, int ny,
                          int nz, int K, int ty, int tz, ResidentPlan* out) {
    switch (model) {
    case RD_MODEL_DIFFUSION:
        return plan_model<MDiffusion>(storage, plain, tma_ok, nx, ny, nz, K, ty, tz, out);
    case RD_MODEL_BRUSSELATOR:
        return plan_model<MBrusselator>(storage, plain, tma_ok, nx, ny, nz, K, ty, tz, out);
    case RD_MODEL_AIR:
        return plan_model<MAir>(storage, plain, tma_ok, nx, ny, nz, K, ty, tz, out);
    case RD_MODEL_TURING:
        return plan_model<MTuring>(storage, plain, tma_ok, nx, ny, nz, K, ty, tz, out);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_resident(int model, int storage, const LaunchArgs& a, const ResidentPlan& p,
                            int nsteps, ResidentBar* bar, unsigned phantom, cudaStream_t st) {
    if (!a.use_one || nsteps < 1 || p.K < 1 || p.grid < 1) return cudaErrorInvalidValue;
    switch (model) {
    case RD_MODEL_DIFFUSION:
        return launch_model<MDiffusion>(storage, a, p, nsteps, bar, phantom, st);
    case RD_MODEL_BRUSSELATOR:
        return launch_model<MBrusselator>(storage, a, p, nsteps, bar, phantom, st);
    case RD_MODEL_AIR: return launch_model<MAir>(storage, a, p, nsteps, bar, phantom, st);
    case RD_MODEL_TURING:
        return launch_model<MTuring>(storage, a, p, nsteps, bar, phantom, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace rdk
