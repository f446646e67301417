// rd_step_kernel.cuh -- the fused forward-Euler step kernel (sm_103a).
//
// One kernel advances T steps of eq. (5) for every species of a work item.
// A work item is an x-y tile of TX x TY cells and a chunk of z planes of one
// instance.  The CTA marches up the chunk (the z-march of the paper's
// Shared method, Section 4.1 / Table 4, restated for this hardware):
//
//   level 0   planes of the current state arrive in a shared-memory ring by
//             16-byte cp.async copies, kPrefetch planes ahead, with the tile
//             widened by a halo of L cells in y and one 16-byte vector in x;
//   level l   1 <= l <= L: each new plane of level l is computed from three
//             planes (q-1, q, q+1) of level l-1 as soon as they exist;
//             level L is written to global memory with 16-byte stores.
//
// Without Cahn-Hilliard, L = T and level l is the state after l steps.
// With it, L = 2T: odd levels hold mu = f'(c) - kappa Lap c, even levels the
// state, so the biharmonic term is the paper's "Laplacian, boundary rule,
// Laplacian" (Section 4.1) fused into one pass.
//
// Boundary rules are applied where neighbours are read, at every level:
//   periodic axis  halo cells are real cells at wrapped coordinates, loaded
//                  and updated like any other cell;
//   zero-flux axis a neighbour outside the domain is replaced by the cell
//                  itself (ghost = face cell), so out-of-domain halo cells
//                  are never read and never loaded;
//   held layer     (Dirichlet) the cell's new value is its bc value.
// Every cell value, at every level, comes from the same per-cell update with
// explicitly rounded operations, so a T-step launch gives bit-for-bit the
// same state as T one-step launches.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

#include "rd_internal.h"

namespace rdk {

// ---------------------------------------------------------------- storage
template <class ST> struct Store;

template <> struct Store<float> {
    static constexpr int VEC = 4;
    __device__ __forceinline__ static void load(const float* p, float (&v)[4]) {
        float4 t = *reinterpret_cast<const float4*>(p);
        v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
    }
    __device__ __forceinline__ static void store(float* p, const float (&v)[4]) {
        *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
    }
    __device__ __forceinline__ static float get(const float* p) { return *p; }
};

template <> struct Store<__nv_bfloat16> {
    static constexpr int VEC = 8;
    __device__ __forceinline__ static void load(const __nv_bfloat16* p, float (&v)[8]) {
        uint4 t = *reinterpret_cast<const uint4*>(p);
        const unsigned w[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            v[2 * i] = __uint_as_float(w[i] << 16);
            v[2 * i + 1] = __uint_as_float(w[i] & 0xffff0000u);
        }
    }
    __device__ __forceinline__ static void store(__nv_bfloat16* p, const float (&v)[8]) {
        unsigned w[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
            w[i] = *reinterpret_cast<unsigned*>(&h);
        }
        *reinterpret_cast<uint4*>(p) = make_uint4(w[0], w[1], w[2], w[3]);
    }
    __device__ __forceinline__ static float get(const __nv_bfloat16* p) {
        return __bfloat162float(*p);
    }
};

// N consecutive elements of type E (float or bfloat16) as floats, moved with
// 16-byte shared-memory accesses.
template <class E, int N> struct Vec;
template <int N> struct Vec<float, N> {
    __device__ __forceinline__ static void load(const float* p, float (&v)[N]) {
#pragma unroll
        for (int i = 0; i < N / 4; ++i) {
            float4 t = reinterpret_cast<const float4*>(p)[i];
            v[4 * i] = t.x; v[4 * i + 1] = t.y; v[4 * i + 2] = t.z; v[4 * i + 3] = t.w;
        }
    }
    __device__ __forceinline__ static void store(float* p, const float (&v)[N]) {
#pragma unroll
        for (int i = 0; i < N / 4; ++i)
            reinterpret_cast<float4*>(p)[i] =
                make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
    }
    __device__ __forceinline__ static float get(const float* p) { return *p; }
};
template <int N> struct Vec<__nv_bfloat16, N> {
    static_assert(N % 8 == 0, "bf16 vectors are 8 wide");
    __device__ __forceinline__ static void load(const __nv_bfloat16* p, float (&v)[N]) {
#pragma unroll
        for (int i = 0; i < N / 8; ++i) {
            float t[8];
            Store<__nv_bfloat16>::load(p + 8 * i, t);
#pragma unroll
            for (int e = 0; e < 8; ++e) v[8 * i + e] = t[e];
        }
    }
    __device__ __forceinline__ static void store(__nv_bfloat16* p, const float (&v)[N]) {
#pragma unroll
        for (int i = 0; i < N / 8; ++i) {
            float t[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) t[e] = v[8 * i + e];
            Store<__nv_bfloat16>::store(p + 8 * i, t);
        }
    }
    __device__ __forceinline__ static float get(const __nv_bfloat16* p) {
        return __bfloat162float(*p);
    }
};

// 7-point neighbourhood of N cells of one row: centre plus the two
// neighbours along each axis.  Planes P0 (this z), Pm (z-1), Pp (z+1) are
// already chosen by the z rule; rows off/offm/offp by the y rule; the x rule
// for zero-flux faces replaces an outside neighbour by the cell itself.
template <class E, int N>
__device__ __forceinline__ void gather7(const E* P0, const E* Pm, const E* Pp, int off,
                                        int offm, int offp, bool xb, int xs, int nx,
                                        float (&c)[N], float (&xm)[N], float (&xp)[N],
                                        float (&ym)[N], float (&yp)[N], float (&zm)[N],
                                        float (&zp)[N]) {
    Vec<E, N>::load(P0 + off, c);
    Vec<E, N>::load(P0 + offm, ym);
    Vec<E, N>::load(P0 + offp, yp);
    Vec<E, N>::load(Pm + off, zm);
    Vec<E, N>::load(Pp + off, zp);
    const float left = Vec<E, N>::get(P0 + off - 1);
    const float right = Vec<E, N>::get(P0 + off + N);
#pragma unroll
    for (int e = 0; e < N; ++e) {
        xm[e] = e ? c[e - 1] : left;
        xp[e] = (e < N - 1) ? c[e + 1] : right;
    }
    if (xb) {
#pragma unroll
        for (int e = 0; e < N; ++e) {
            if (xs + e == 0) xm[e] = c[e];
            if (xs + e == nx - 1) xp[e] = c[e];
        }
    }
}

// ------------------------------------------------------------ async copies
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem)
                 : "memory");
}
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

// ----------------------------------------------------------------- models
// Per-cell pieces of eq. (1).  ``react`` returns dt * R_s(c) for every
// species (the increment before transport terms).
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
    // mu = f'(c) - (kappa/h^2) (sum of 6 neighbours - 6 c), f'(c) = 2c(c-1)(2c-1)
    __device__ __forceinline__ static float mu(const InstDesc& d, float c, float xm, float xp,
                                               float ym, float yp, float zm, float zp) {
        const float c2 = __fadd_rn(c, c);
        const float fp = __fmul_rn(__fmul_rn(c2, __fsub_rn(c, 1.0f)), __fsub_rn(c2, 1.0f));
        const float s6 = __fadd_rn(__fadd_rn(__fadd_rn(xm, xp), __fadd_rn(ym, yp)),
                                   __fadd_rn(zm, zp));
        const float lap = __fmaf_rn(-6.0f, c, s6);
        return __fmaf_rn(-d.p[2], lap, fp);
    }
};

// One cell of eq. (5) for a species with Fickian transport: c + inc +
// sum_a k_a (c[-1] + c[+1] - 2c) with k_a = D_a dt / h^2.
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

// First-order upwind advection increment for Courant number cx = u dt / h.
__device__ __forceinline__ float upwind(float inc, float cx, float c, float xm, float xp) {
    return cx >= 0.0f ? __fmaf_rn(-cx, __fsub_rn(c, xm), inc)
                      : __fmaf_rn(-cx, __fsub_rn(xp, c), inc);
}

// Held (Dirichlet) layer test, faces in order -x,+x,-y,+y,-z,+z.
__device__ __forceinline__ bool held_value(const InstDesc& d, int s, int x, int y, int z,
                                           float& v) {
    const unsigned m = d.held_mask[s];
    if (!m) return false;
    if ((m & 1u) && x == 0) { v = d.held_val[s][0]; return true; }
    if ((m & 2u) && x == d.nx - 1) { v = d.held_val[s][1]; return true; }
    if ((m & 4u) && y == 0) { v = d.held_val[s][2]; return true; }
    if ((m & 8u) && y == d.ny - 1) { v = d.held_val[s][3]; return true; }
    if ((m & 16u) && z == 0) { v = d.held_val[s][4]; return true; }
    if ((m & 32u) && z == d.nz - 1) { v = d.held_val[s][5]; return true; }
    return false;
}

// ------------------------------------------------------- shared-memory map
// Plane buffers: NR rows of RS elements plus a VEC-element guard at each
// end; ring slots per level as described above.
template <class M, class ST, int T> struct Layout {
    static constexpr int VEC = Store<ST>::VEC;
    static constexpr int S = M::S;
    static constexpr bool CH = M::CH;
    static constexpr int L = CH ? 2 * T : T;
    static constexpr int RING_STATE = CH ? 4 : 3;
    static constexpr int RING0 = RING_STATE + kPrefetch;
    static constexpr int RING_MU = 3;

    __host__ __device__ static bool is_mu(int l) { return CH && (l & 1); }
    __host__ __device__ static int plane_elems(int tq, int ty) {
        return (ty + 2 * L) * (tq + 2) * VEC + 2 * VEC;
    }
    // bytes of level l's ring (l = 0 .. L-1)
    __host__ __device__ static size_t level_bytes(int l, int tq, int ty) {
        const size_t pe = plane_elems(tq, ty);
        if (l == 0) return RING0 * S * pe * sizeof(ST);
        if (is_mu(l)) return RING_MU * pe * sizeof(float);
        return RING_STATE * S * pe * sizeof(ST);
    }
    __host__ __device__ static size_t level_offset(int l, int tq, int ty) {
        size_t o = 0;
        for (int i = 0; i < l; ++i) o += level_bytes(i, tq, ty);
        return o;
    }
    __host__ __device__ static size_t total(int tq, int ty) { return level_offset(L, tq, ty); }
};

// ------------------------------------------------------------------ kernel
template <class M, class ST, int T>
__global__ void __launch_bounds__(kThreads) rd_step_kernel(const LaunchArgs a) {
    using SX = Store<ST>;
    using LY = Layout<M, ST, T>;
    constexpr int VEC = SX::VEC;
    constexpr int S = M::S;
    constexpr bool CH = M::CH;
    constexpr int L = LY::L;

    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ InstDesc sd;
    __shared__ int s_inst;

    const int tid = threadIdx.x;
    const int tq = a.tq, TY = a.ty;
    const int nq = tq + 2;
    const int RS = nq * VEC;
    const int NR = TY + 2 * L;
    const int PE = LY::plane_elems(tq, TY);

    int cur_inst = -1;
    if (tid == 0) s_inst = 0;
    for (long long item = blockIdx.x; item < a.nitems; item += gridDim.x) {
        // ---- which instance owns this item
        if (a.ninst == 1) {
            if (tid == 0) s_inst = 0;
        } else {
            for (int i = tid; i < a.ninst; i += kThreads) {
                const long long b0 = a.desc[i].item_begin;
                const long long b1 = (i + 1 < a.ninst) ? a.desc[i + 1].item_begin : a.nitems;
                if (item >= b0 && item < b1) s_inst = i;
            }
        }
        __syncthreads();
        if (s_inst != cur_inst) {
            cur_inst = s_inst;
            const int* src = reinterpret_cast<const int*>(a.desc + cur_inst);
            int* dst = reinterpret_cast<int*>(&sd);
            for (int i = tid; i < (int)(sizeof(InstDesc) / sizeof(int)); i += kThreads)
                dst[i] = src[i];
        }
        __syncthreads();

        const int nx = sd.nx, ny = sd.ny, nz = sd.nz, pitch = sd.pitch;
        const long long plane = sd.plane;
        const bool px = sd.per_x, py = sd.per_y, pz = sd.per_z;
        const long long local = item - sd.item_begin;
        const int tx = (int)(local % sd.ntx);
        const int tyi = (int)((local / sd.ntx) % sd.nty);
        const int zc = (int)(local / ((long long)sd.ntx * sd.nty));
        const int x0 = tx * tq * VEC, y0 = tyi * TY;
        const int z0 = zc * sd.zchunk;
        const int z1 = min(z0 + sd.zchunk, nz);
        const int lin = sd.par ^ a.parity;

        // -------------------------------------------------------- loader
        auto ring0 = [&](int s, int slot) -> ST* {
            return reinterpret_cast<ST*>(smem) + (size_t)(slot * S + s) * PE + VEC;
        };
        auto load_plane = [&](int q) {
            if (!pz && (q < 0 || q >= nz)) return;
            const int zw = pz ? wrapi(q, nz) : q;
            const int slot = wrapi(q, LY::RING0);
            const int per_s = NR * nq;
            for (int u = tid; u < S * per_s; u += kThreads) {
                const int s = u / per_s;
                const int rem = u - s * per_s;
                const int r = rem / nq;
                const int v = rem - r * nq;
                const int y = y0 - L + r;
                int yw = y;
                if (py) yw = wrapi(y, ny);
                else if (y < 0 || y >= ny) continue;
                const int xs = x0 - VEC + v * VEC;
                ST* dst = ring0(s, slot) + r * RS + v * VEC;
                const ST* row = reinterpret_cast<const ST*>(sd.base[lin][s]) +
                                (size_t)zw * plane + (size_t)yw * pitch;
                if (xs >= 0 && xs < nx) {
                    if (!px || xs + VEC <= nx) { cp_async16(dst, row + xs); continue; }
                } else if (!px) {
                    continue;                         // zero-flux halo: never read
                } else {
                    // a wrapped vector is copied whole only from a 16-byte
                    // aligned start that does not cross the wrap point
                    const int xw = wrapi(xs, nx);
                    if (xw % VEC == 0 && xw + VEC <= nx) { cp_async16(dst, row + xw); continue; }
                }
                // periodic vector straddling the wrap point: element-wise
#pragma unroll
                for (int e = 0; e < VEC; ++e) dst[e] = row[wrapi(xs + e, nx)];
            }
        };

        // ---------------------------------------------- per-level compute
        // level l: q = plane, reads level l-1 (and l-2 for the CH state)
        auto level_ptr = [&](int l, int s, int q) -> void* {
            if (l == 0) return ring0(s, wrapi(q, LY::RING0));
            unsigned char* b = smem + LY::level_offset(l, tq, TY);
            if (LY::is_mu(l)) return reinterpret_cast<float*>(b) + (size_t)wrapi(q, LY::RING_MU) * PE + VEC;
            return reinterpret_cast<ST*>(b) +
                   (size_t)(wrapi(q, LY::RING_STATE) * S + s) * PE + VEC;
        };

        const int pbeg = z0 - L, pend = z1 + L;
#pragma unroll 1
        for (int j = 0; j < kPrefetch; ++j) {
            if (pbeg + j < pend) load_plane(pbeg + j);
            cp_async_commit();
        }
#pragma unroll 1
        for (int p = pbeg; p < pend; ++p) {
            if (p + kPrefetch < pend) load_plane(p + kPrefetch);
            cp_async_commit();
            cp_async_wait<kPrefetch>();
            __syncthreads();
#pragma unroll
            for (int l = 1; l <= L; ++l) {
                const int q = p - l;
                const bool valid = q >= z0 - L + l && q < z1 + L - l && (pz || (q >= 0 && q < nz));
                if (valid) {
                    const bool fin = (l == L);
                    const bool mu_lvl = LY::is_mu(l);
                    // state source level for Fickian terms and centres
                    const int ls = (CH && !mu_lvl) ? l - 2 : l - 1;
                    int qm = q - 1, qp = q + 1;
                    if (!pz) { if (q == 0) qm = q; if (q == nz - 1) qp = q; }
                    const int zw = pz ? wrapi(q, nz) : q;
                    const float cx = sd.courant ? sd.courant[zw] : 0.0f;
                    const int r_lo = l, r_hi = NR - l;
                    const int v_lo = fin ? 1 : 0, v_hi = fin ? nq - 1 : nq;
                    const int nv = v_hi - v_lo;
                    const int nunits = (r_hi - r_lo) * nv;
                    for (int u = tid; u < nunits; u += kThreads) {
                        const int rr = u / nv;
                        const int r = r_lo + rr;
                        const int v = v_lo + (u - rr * nv);
                        const int y = y0 - L + r;
                        if (!py && (y < 0 || y >= ny)) continue;
                        const int xs = x0 - VEC + v * VEC;
                        if (!px && (xs + VEC <= 0 || xs >= nx)) continue;
                        if (fin && (y >= ny || xs >= nx)) continue;
                        const int yw = py ? wrapi(y, ny) : y;
                        int rm = r - 1, rp = r + 1;
                        if (!py) { if (y == 0) rm = r; if (y == ny - 1) rp = r; }
                        const bool xb = !px && (xs <= 0 || xs + VEC >= nx);
                        const int off = r * RS + v * VEC;
                        const int offm = rm * RS + v * VEC;
                        const int offp = rp * RS + v * VEC;

                        if (mu_lvl) {
                            // mu of the Cahn-Hilliard species from level l-1
                            const ST* P0 = (const ST*)level_ptr(l - 1, 2, q);
                            const ST* Pm = (const ST*)level_ptr(l - 1, 2, qm);
                            const ST* Pp = (const ST*)level_ptr(l - 1, 2, qp);
                            float c[VEC], xm[VEC], xp[VEC], ym[VEC], yp[VEC], zm[VEC], zp[VEC];
                            gather7<ST, VEC>(P0, Pm, Pp, off, offm, offp, xb, xs, nx, c, xm, xp, ym, yp, zm, zp);
                            float mo[VEC];
#pragma unroll
                            for (int e = 0; e < VEC; ++e)
                                mo[e] = MChFront::mu(sd, c[e], xm[e], xp[e], ym[e], yp[e], zm[e], zp[e]);
                            Vec<float, VEC>::store((float*)level_ptr(l, 0, q) + off, mo);
                            continue;
                        }

                        // centres of all species, then the reaction increments
                        float cen[S][VEC], inc[S][VEC];
#pragma unroll
                        for (int s = 0; s < S; ++s)
                            SX::load((const ST*)level_ptr(ls, s, q) + off, cen[s]);
#pragma unroll
                        for (int e = 0; e < VEC; ++e) {
                            float cv[S], iv[S];
#pragma unroll
                            for (int s = 0; s < S; ++s) cv[s] = cen[s][e];
                            M::react(sd, cv, iv);
#pragma unroll
                            for (int s = 0; s < S; ++s) inc[s][e] = iv[s];
                        }
                        const bool src_here = sd.src_s >= 0 && zw == sd.src_z && yw == sd.src_y;
#pragma unroll
                        for (int s = 0; s < S; ++s) {
                            float o[VEC];
                            if (CH && s == 2) {
                                const float* U0 = (const float*)level_ptr(l - 1, 0, q);
                                const float* Um = (const float*)level_ptr(l - 1, 0, qm);
                                const float* Up = (const float*)level_ptr(l - 1, 0, qp);
                                float m0[VEC], mxm[VEC], mxp[VEC], mym[VEC], myp[VEC], mzm[VEC], mzp[VEC];
                                gather7<float, VEC>(U0, Um, Up, off, offm, offp, xb, xs, nx, m0, mxm, mxp, mym, myp, mzm, mzp);
#pragma unroll
                                for (int e = 0; e < VEC; ++e) {
                                    const float s6 = __fadd_rn(__fadd_rn(__fadd_rn(mxm[e], mxp[e]),
                                                                         __fadd_rn(mym[e], myp[e])),
                                                               __fadd_rn(mzm[e], mzp[e]));
                                    const float lap = __fmaf_rn(-6.0f, m0[e], s6);
                                    const float in = __fmaf_rn(sd.p[1], lap, inc[s][e]);
                                    o[e] = __fadd_rn(cen[s][e], in);
                                }
                            } else {
                                const ST* P0 = (const ST*)level_ptr(ls, s, q);
                                const ST* Pm = (const ST*)level_ptr(ls, s, qm);
                                const ST* Pp = (const ST*)level_ptr(ls, s, qp);
                                float c[VEC], xm[VEC], xp[VEC], ym[VEC], yp[VEC], zm[VEC], zp[VEC];
                                gather7<ST, VEC>(P0, Pm, Pp, off, offm, offp, xb, xs, nx, c, xm, xp, ym, yp, zm, zp);
                                const float kx = sd.kx[s], ky = sd.ky[s], kz = sd.kz[s];
#pragma unroll
                                for (int e = 0; e < VEC; ++e) {
                                    float in = inc[s][e];
                                    if (src_here && s == sd.src_s) {
                                        const int xw = px ? wrapi(xs + e, nx) : xs + e;
                                        if (xw == sd.src_x) in = __fadd_rn(in, sd.src_amt);
                                    }
                                    if (cx != 0.0f) in = upwind(in, cx, c[e], xm[e], xp[e]);
                                    o[e] = euler_cell(c[e], xm[e], xp[e], ym[e], yp[e], zm[e], zp[e],
                                                      kx, ky, kz, in);
                                }
                            }
                            if (sd.held_mask[s]) {
#pragma unroll
                                for (int e = 0; e < VEC; ++e) {
                                    float hv;
                                    if (held_value(sd, s, xs + e, y, q, hv)) o[e] = hv;
                                }
                            }
                            if (fin) {
                                ST* g = reinterpret_cast<ST*>(sd.base[lin ^ 1][s]) +
                                        (size_t)q * plane + (size_t)y * pitch + xs;
                                SX::store(g, o);
                            } else {
                                SX::store((ST*)level_ptr(l, s, q) + off, o);
                            }
                        }
                    }
                }
                __syncthreads();
            }
        }
        cp_async_wait<0>();
        __syncthreads();
    }
}

// Launch helper used by the per-model translation units.
template <class M, class ST, int T>
cudaError_t launch_one(const LaunchArgs& a, int grid, size_t smem, cudaStream_t st, int* occ) {
    auto k = rd_step_kernel<M, ST, T>;
    static size_t configured = 0;
    if (smem > configured) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        configured = smem;
    }
    if (occ) {
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k, kThreads, smem);
    }
    k<<<grid, kThreads, smem, st>>>(a);
    return cudaGetLastError();
}

template <class M>
cudaError_t launch_model(int storage, int tsteps, const LaunchArgs& a, int grid, size_t smem,
                         cudaStream_t st, int* occ) {
    if (storage == RD_STORE_F32) {
        switch (tsteps) {
        case 1: return launch_one<M, float, 1>(a, grid, smem, st, occ);
        case 2: return launch_one<M, float, 2>(a, grid, smem, st, occ);
        case 3: if constexpr (!M::CH) return launch_one<M, float, 3>(a, grid, smem, st, occ);
                break;
        default: break;
        }
    } else {
        switch (tsteps) {
        case 1: return launch_one<M, __nv_bfloat16, 1>(a, grid, smem, st, occ);
        case 2: return launch_one<M, __nv_bfloat16, 2>(a, grid, smem, st, occ);
        case 3: if constexpr (!M::CH) return launch_one<M, __nv_bfloat16, 3>(a, grid, smem, st, occ);
                break;
        default: break;
        }
    }
    return cudaErrorInvalidValue;
}

template <class M>
size_t smem_for(int storage, int tsteps, int tq, int ty) {
    if (storage == RD_STORE_F32) {
        switch (tsteps) {
        case 1: return Layout<M, float, 1>::total(tq, ty);
        case 2: return Layout<M, float, 2>::total(tq, ty);
        case 3: return Layout<M, float, 3>::total(tq, ty);
        }
    } else {
        switch (tsteps) {
        case 1: return Layout<M, __nv_bfloat16, 1>::total(tq, ty);
        case 2: return Layout<M, __nv_bfloat16, 2>::total(tq, ty);
        case 3: return Layout<M, __nv_bfloat16, 3>::total(tq, ty);
        }
    }
    return 0;
}

}  // namespace rdk
