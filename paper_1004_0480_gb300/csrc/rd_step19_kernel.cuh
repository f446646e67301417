// rd_step19_kernel.cuh -- one forward-Euler step of eq. (5) with the
// 19-point Laplacian of eqs. (3)-(4), for the models without Cahn-Hilliard
// (sm_103a).
//
// Work items, thread layout and copies follow the one-step 7-point kernel
// (rd_step1_kernel): one thread per 4-cell vector of a 64 x TY tile plus one
// halo warp, planes of the current state copied into a shared-memory ring
// by per-thread cp.async several planes ahead, one barrier per plane.  What
// differs:
//
//  * Neighbourhood.  A cell reads the 3x3 block of its own plane (weights
//    -24 centre, 2 faces, 1 diagonals) and the 5-point cross of the planes
//    below and above (2 centre, 1 faces); corners weigh 0.  The diagonals
//    need the tile's four corner vectors, which the halo warp also copies.
//  * Per-plane sums carried down the march.  When plane k arrives, a
//    thread forms at each of its 4 cells, with X = xm + xp + ym + yp,
//        Z_k = 2 c + X                 (plane k as a z-neighbour)
//        W_k = 2 X + the 4 diagonals   (plane k as the centre plane)
//    so that 6 h^2 Lap c on plane q = W_q - 24 c_q + Z_{q-1} + Z_{q+1}.
//    Z_{q-1}, Z_q, W_q and c_q stay in registers; each plane is read from
//    shared memory once, on arrival (plane q+1 at step q).
//  * Ring reuse.  A plane's last reads are its arrival and, with wind, the
//    two elements beside a thread's own row at its own step, so the copy
//    issued at step q may overwrite plane q-2, whose reads all ended before
//    the barrier of step q-1: the 7-point kernel's ring of 6 slots with
//    P = 5 copy groups ahead of q-1.  The first step of a work item also
//    reads the neighbours of plane z0-1, whose slot the copy of step z0+1
//    refills; one more barrier after those reads keeps the rule.
//
// Boundary rules are those of the 7-point kernels: ghost rows, planes and
// vectors are copied in under each axis's rule (zero flux: the face value;
// periodic: wrapped), and a thread at a zero-flux x face reads the cells
// beyond it from its own column (xface_offsets), so an edge ghost composes
// the rules of the two axes it crosses, as the paper fills its edges after
// its faces (Section 4.1); a held layer's cell takes its bc value.
#pragma once

#include "rd_step19.h"
#include "rd_step_kernel.cuh"

namespace rdk {

// PASS 0: one step of a model without Cahn-Hilliard.  For the models with a
// Cahn-Hilliard species (species 2, c) a step is two launches, the paper's
// "Laplacian, boundary rule, Laplacian" (Section 4.1): PASS 1 writes the
// chemical potential mu = g(c) - p[2] h^2 Lap c of every cell to the
// instance's mu field, PASS 2 then updates a, b and c, reading mu as one more
// field of the ring (its ghost cells copied in under the same rules, which
// is the paper's "boundary rule" applied to mu) and adding p[1] h^2 Lap mu
// to c.  The ring of PASS 1 holds species 2 only.
template <class M, class ST, int PASS> struct Layout19 {
    static constexpr int S = M::S;
    static constexpr int NS = PASS == 1 ? 1 : S;    // state fields per slot
    static constexpr bool MUF = PASS == 2;          // plus one float mu plane
    static constexpr int RING = kRing19;
    static constexpr int P = 5;
    static_assert(RING == P + 1, "the copy of step q refills the slot of plane q - 2");
    static_assert(PASS == 0 || M::CH, "passes 1 and 2 are for Cahn-Hilliard models");
    __host__ __device__ static int plane_elems(int ty) { return plane_elems19(ty); }
    __host__ __device__ static size_t total(int ty) {
        return smem19_pass_bytes(NS, (int)sizeof(ST), MUF, ty);
    }
    __host__ __device__ static int threads(int ty) { return kTileQ * ty + 32; }
};

// Own vector c and the sums Z, W of one species plane at the thread's 4
// cells; ``p`` points at the own vector in the ring, ``loff`` / ``roff``
// are the byte offsets of the x neighbours beside it (xface_offsets: at a
// zero-flux x face, the thread's own face cell, also in the rows above and
// below, where the edge ghost composes both faces' rules).
template <class ST>
__device__ __forceinline__ void plane_sums19(const unsigned char* p, int loff, int roff,
                                             float (&c)[kVEC], float (&zs)[kVEC],
                                             float (&ws)[kVEC]) {
    constexpr int RWB = kRW * (int)sizeof(ST);
    float ym[kVEC], yp[kVEC];
    lds_vec<ST>(p, c);
    lds_vec<ST>(p - RWB, ym);
    lds_vec<ST>(p + RWB, yp);
    const unsigned char* pl = p + loff;
    const unsigned char* pr = p + roff;
    const float l = lds_one<ST>(pl), r = lds_one<ST>(pr);
    const float ul = lds_one<ST>(pl - RWB), ur = lds_one<ST>(pr - RWB);
    const float dl = lds_one<ST>(pl + RWB), dr = lds_one<ST>(pr + RWB);
#pragma unroll
    for (int e = 0; e < kVEC; ++e) {
        const float xm = e ? c[e - 1] : l;
        const float xp = e < kVEC - 1 ? c[e + 1] : r;
        const float yml = e ? ym[e - 1] : ul;
        const float ymr = e < kVEC - 1 ? ym[e + 1] : ur;
        const float ypl = e ? yp[e - 1] : dl;
        const float ypr = e < kVEC - 1 ? yp[e + 1] : dr;
        const float cross = __fadd_rn(__fadd_rn(xm, xp), __fadd_rn(ym[e], yp[e]));
        const float diag = __fadd_rn(__fadd_rn(yml, ymr), __fadd_rn(ypl, ypr));
        zs[e] = __fmaf_rn(2.0f, c[e], cross);
        ws[e] = __fmaf_rn(2.0f, cross, diag);
    }
}

// New value of one species on the thread's 4 cells: c + inc + k6 * lap6,
// k6 = D dt / (6 h^2), lap6 = 6 h^2 Lap c, plus the point source and
// first-order upwind advection (Courant number cx, x neighbours from the
// own vector and the elements ``left`` / ``right`` beside it).
template <bool PLAIN>
__device__ __forceinline__ void species19(const InstDesc& sd, int s, float k6,
                                          const float (&c)[kVEC], const float (&lap6)[kVEC],
                                          const float (&inc)[kVEC], float cx, float left,
                                          float right, bool src_here, bool px, int xs,
                                          float (&o)[kVEC]) {
    float in[kVEC];
#pragma unroll
    for (int e = 0; e < kVEC; ++e) in[e] = inc[e];
    if constexpr (!PLAIN) {
        if (src_here && s == sd.src_s) {
#pragma unroll
            for (int e = 0; e < kVEC; ++e)
                if ((px ? wrapi(xs + e, sd.nx) : xs + e) == sd.src_x)
                    in[e] = __fadd_rn(in[e], sd.src_amt);
        }
        if (cx > 0.0f) {
#pragma unroll
            for (int e = 0; e < kVEC; ++e) {
                const float xm = e ? c[e - 1] : left;
                in[e] = __fmaf_rn(-cx, __fsub_rn(c[e], xm), in[e]);
            }
        } else if (cx < 0.0f) {
#pragma unroll
            for (int e = 0; e < kVEC; ++e) {
                const float xp = e < kVEC - 1 ? c[e + 1] : right;
                in[e] = __fmaf_rn(-cx, __fsub_rn(xp, c[e]), in[e]);
            }
        }
    }
#pragma unroll
    for (int e = 0; e < kVEC; ++e) o[e] = __fadd_rn(c[e], __fmaf_rn(k6, lap6[e], in[e]));
}

// One float field of a plane (the mu plane of PASS 2), fetched with the
// state's descriptor: the same rows, pitch and ghost rules.  ``mu0`` is the
// address of the mu plane's element 0.
template <class ST>
__device__ __forceinline__ void fetch_mu(const Fetch& f, unsigned char* mu0,
                                         const float* gplane, int nx, bool elems, bool px,
                                         const InstDesc& sd) {
    float* d = reinterpret_cast<float*>(mu0 + f.soff / (int)sizeof(ST) * 4);
    const int ok = f.mode == 1 && RD_DBG_GLOBAL(sd, gplane + f.goff, 16, kSiteMu);
    Store<float>::cp_async_if(d, gplane + f.goff, ok);
    if (elems && f.mode == 2) {
#pragma unroll
        for (int e = 0; e < kVEC; ++e) {
            const int x = f.xs + e;
            const int xi = px ? wrapi(x, nx) : (x < 0 ? 0 : (x >= nx ? nx - 1 : x));
            if (RD_DBG_GLOBAL(sd, gplane + f.goff + xi, 4, kSiteMu))
                Store<float>::cp_async_elem(d + e, gplane + f.goff + xi);
        }
    }
}

// PLAIN: no held layer, point source or wind.  PASS: see Layout19.  W3:
// the 3-D wind (upwind along y and z too; never with PLAIN, PASS 0 only).
template <class M, class ST, bool ONE, bool PLAIN, int PASS, bool W3 = false>
__global__ void __launch_bounds__(kMaxThreads, 1)
rd_step19_kernel(const __grid_constant__ LaunchArgs a) {
    using LY = Layout19<M, ST, PASS>;
    constexpr int S = M::S;
    constexpr int NS = LY::NS;
    constexpr bool MUF = LY::MUF;
    // fields whose plane sums are formed: every state field (PASS 0), c
    // (PASS 1), a, b and mu (PASS 2; c needs only its own cells there)
    constexpr int NSUM = PASS == 2 ? 3 : NS;
    constexpr int P = LY::P;
    constexpr int RING = LY::RING;
    constexpr int EB = (int)sizeof(ST);

    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ InstDesc sdm;
    __shared__ int s_inst;
    __shared__ long long s_item;

    const int tid = threadIdx.x;
    const int TY = a.ty;
    const int PE = LY::plane_elems(TY);
    const int PEB = PE * EB;                                 // bytes per state plane
    const int SLOTB = NS * PEB + (MUF ? PE * 4 : 0);         // bytes per ring slot
    unsigned char* const ring = smem + kVEC * EB;            // slot 0, field 0
    int4* const hfetch = reinterpret_cast<int4*>(smem + RING * SLOTB);
    const int ncomp = kTileQ * TY;
    const bool halo_warp = tid >= ncomp;
    const int r = tid / kTileQ;
    const int v = tid - r * kTileQ;
    const int own_e = (r + 1) * kRW + (v + 1) * kVEC;        // element offset in a plane
    const int own_b = own_e * EB;
    // the mu plane of a slot (PASS 2) starts at NS * PEB; its guard is
    // kVEC floats, the state planes' kVEC elements of ST
    const int mu0_b = NS * PEB + kVEC * (4 - EB);            // element 0, from a slot
    const int mu_own_b = mu0_b + own_e * 4;

    int cur_inst = -1;
    if (tid == 0) s_inst = 0;
    for (long long item = first_item<ONE>(a, s_item); item < a.nitems;
         item = next_item<ONE>(a, item, s_item)) {
        if constexpr (!ONE) load_desc(a, item, sdm, s_inst, cur_inst);
        const InstDesc& sd = desc_of<ONE>(a, sdm);
        if (member_done<ONE>(a, sd)) continue;   // block-uniform

        const int nx = sd.nx, ny = sd.ny, nz = sd.nz, pitch = sd.pitch;
        const bool px = sd.per_x, py = sd.per_y, pz = sd.per_z;
        const bool elems = sd.wrap_elems || !sd.per_x;
        const long long local = item - sd.item_begin;
        const int txi = (int)(local % sd.ntx);
        const int tyi = (int)((local / sd.ntx) % sd.nty);
        const int zc = (int)(local / ((long long)sd.ntx * sd.nty));
        const int x0 = txi * kTileQ * kVEC, y0 = tyi * TY;
        const int z0 = zc * sd.zchunk;
        const int z1 = min(z0 + sd.zchunk, nz);
        const int lin = sd.par ^ a.parity;
        const ST* const gin = reinterpret_cast<const ST*>(sd.base[lin][PASS == 1 ? 2 : 0]);
        ST* const gout = reinterpret_cast<ST*>(sd.base[lin ^ 1][0]);
        const long long fstride =
            NS > 1 ? reinterpret_cast<const ST*>(sd.base[lin][1]) - gin : 0;
        const long long plane = sd.plane;

        // ---- halo lanes: 2 TY side vectors, 2 x 16 row vectors, then the 4
        // corner vectors (rows -1 and TY, vector columns -1 and 16)
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
                } else if (j < 2 * TY + 2 * kTileQ + 4) {
                    const int jj = j - 2 * TY - 2 * kTileQ;
                    const bool bottom = jj >= 2;
                    const bool right = jj & 1;
                    f = make_fetch<ST>(bottom ? y0 + TY : y0 - 1,
                                       right ? x0 + kTileQ * kVEC : x0 - kVEC, nx, ny, pitch, px,
                                       py,
                                       (bottom ? TY + 1 : 0) * kRW + (right ? kNQ - 1 : 0) * kVEC,
                                       true);
                }
                if (RD_DBG_SHARED(hfetch + j, 16, kSiteHaloDesc))
                    hfetch[j] = make_int4(f.mode, f.goff, f.soff, f.xs);
            }
        }
        // ---- compute threads: own vector
        const int y = y0 + r;
        const int xs = x0 + v * kVEC;
        const bool computes = !halo_warp && y < ny && xs < nx;
        const bool src_col = sd.src_s >= 0 && (py ? wrapi(y, ny) : y) == sd.src_y;
        const unsigned xyf = xy_faces(xs, y, nx, ny);
        const Fetch fo = halo_warp ? Fetch{0, 0, 0, 0}
                                   : make_fetch<ST>(y, xs, nx, ny, pitch, px, py, own_e, true);
        int loff, roff;                           // x neighbours beside the own vector
        xface_offsets<ST>(xs, nx, px, loff, roff);
        int loff_f = 0, roff_f = 0;               // the same in the float mu plane
        if constexpr (MUF) xface_offsets<float>(xs, nx, px, loff_f, roff_f);
        // k6: D dt / (6 h^2) per species; PASS 1: p[2] / 6 (mu); PASS 2:
        // k6[2] = p[1] / 6 (the mobility term of c)
        float k6[S];
#pragma unroll
        for (int s = 0; s < S; ++s) k6[s] = __fdiv_rn(sd.kx[s], 6.0f);
        if constexpr (PASS == 1) k6[0] = __fdiv_rn(sd.p[2], 6.0f);
        if constexpr (PASS == 2) k6[2] = __fdiv_rn(sd.p[1], 6.0f);
        float cy = 0.0f, cz = 0.0f;               // 3-D wind
        if constexpr (W3 && PASS == 0) wind3d(sd, lin, local, cy, cz);
        __syncthreads();   // halo descriptors written

        // ---- the march: plane nld is fetched P planes ahead into slot sl;
        // plane z0 - 1 goes to slot 0, plane q to slot (q - z0 + 1) mod RING
        int nld = z0 - 1;
        int zld = pz ? wrapi(nld, nz) : nld;
        auto issue = [&](int sl) {
            const bool in_z = pz || (nld >= 0 && nld < nz);
            if (nld <= z1) {
                const int zs = in_z ? zld : (nld < 0 ? 0 : nz - 1);
                const ST* gld = gin + (long long)zs * plane;
                const float* gmu = nullptr;
                if constexpr (MUF) gmu = sd.mu + (long long)zs * plane;
                unsigned char* buf = ring + sl * SLOTB;
                if (halo_warp) {
                    const int hl = tid - ncomp;
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        int4 h = make_int4(0, 0, 0, 0);
                        if (RD_DBG_SHARED(hfetch + hl + 32 * k, 16, kSiteHaloDesc))
                            h = hfetch[hl + 32 * k];
                        const Fetch f{h.x, h.y, h.z, h.w};
                        fetch_all<ST, NS>(f, buf, PEB, gld, fstride, nx, elems, px, sd);
                        if constexpr (MUF) fetch_mu<ST>(f, buf + mu0_b, gmu, nx, elems, px, sd);
                    }
                } else {
                    fetch_all<ST, NS>(fo, buf, PEB, gld, fstride, nx, elems, px, sd);
                    if constexpr (MUF) fetch_mu<ST>(fo, buf + mu0_b, gmu, nx, elems, px, sd);
                }
            }
            ++nld;
            if (!pz) zld = nld;
            else if (++zld == nz) zld = 0;
            cp_async_commit();
        };
        // plane sums of field f of the slot at ``base`` (own vector address)
        auto sums = [&](const unsigned char* base, int f, float (&c)[kVEC], float (&zs)[kVEC],
                        float (&ws)[kVEC]) {
            if (MUF && f == NSUM - 1)
                plane_sums19<float>(base - own_b + mu_own_b, loff_f, roff_f, c, zs, ws);
            else
                plane_sums19<ST>(base + f * PEB, loff, roff, c, zs, ws);
        };
#pragma unroll 1
        for (int j = 0; j < P; ++j) issue(j);
        int zq = pz ? wrapi(z0, nz) : z0;
        ST* gst = gout + (long long)z0 * plane + (long long)y * pitch + xs;
        float* gmu_st = nullptr;
        if constexpr (PASS == 1) gmu_st = sd.mu + (long long)z0 * plane + (long long)y * pitch + xs;
        const float* courant = sd.courant;
        int sc = 1;                               // ring slot of plane q
        // sums of planes q-1 and q, and the own vector of plane q
        float zsum_m[NSUM][kVEC], zsum_0[NSUM][kVEC], wsum_0[NSUM][kVEC], c_0[NSUM][kVEC];
        float cc_0[kVEC];                         // PASS 2: own c of plane q
#pragma unroll 1
        for (int q = z0; q < z1; ++q) {
            const int sm = sc == 0 ? RING - 1 : sc - 1;
            const int sp = sc == RING - 1 ? 0 : sc + 1;
            // overwrite plane q - 2; planes up to q + 1 must have landed
            issue(sc + P - 1 >= RING ? sc + P - 1 - RING : sc + P - 1);
            cp_async_wait<P - 2>();
            __syncthreads();
            const unsigned char* Pc = ring + sc * SLOTB + own_b;
            if (q == z0) {   // block-uniform
                if (!halo_warp) {
                    const unsigned char* Pm = ring + sm * SLOTB + own_b;
#pragma unroll
                    for (int f = 0; f < NSUM; ++f) {
                        float cm[kVEC], wm[kVEC];
                        sums(Pm, f, cm, zsum_m[f], wm);
                        sums(Pc, f, c_0[f], zsum_0[f], wsum_0[f]);
                    }
                    if constexpr (PASS == 2) lds_vec<ST>(Pc + 2 * PEB, cc_0);
                }
                __syncthreads();   // plane z0 - 1 is refilled at the next step
            }
            if (!halo_warp) {
                const unsigned char* Pp = ring + sp * SLOTB + own_b;
                float c_p[NSUM][kVEC], zsum_p[NSUM][kVEC], wsum_p[NSUM][kVEC];
                float cc_p[kVEC];
#pragma unroll
                for (int f = 0; f < NSUM; ++f) sums(Pp, f, c_p[f], zsum_p[f], wsum_p[f]);
                if constexpr (PASS == 2) lds_vec<ST>(Pp + 2 * PEB, cc_p);
                // 6 h^2 Lap of each summed field on plane q
                float lap6[NSUM][kVEC];
#pragma unroll
                for (int f = 0; f < NSUM; ++f)
#pragma unroll
                    for (int e = 0; e < kVEC; ++e)
                        lap6[f][e] = __fmaf_rn(-24.0f, c_0[f][e],
                                               __fadd_rn(__fadd_rn(zsum_m[f][e], zsum_p[f][e]),
                                                         wsum_0[f][e]));
                if constexpr (PASS == 1) {
                    // mu = g(c) - (p[2] / 6) 6 h^2 Lap c
                    float mu[kVEC];
#pragma unroll
                    for (int e = 0; e < kVEC; ++e)
                        mu[e] = __fmaf_rn(-k6[0], lap6[0][e], M::g(sd, c_0[0][e]));
                    if (computes && RD_DBG_GLOBAL(sd, gmu_st, 16, kSiteMu))
                        Store<float>::store(gmu_st, mu);
                } else {
                    // state of plane q: a, b (and every PASS 0 species) from
                    // the summed fields, c of PASS 2 from its own vector
                    float cen[S][kVEC], inc[S][kVEC];
#pragma unroll
                    for (int s = 0; s < S; ++s)
#pragma unroll
                        for (int e = 0; e < kVEC; ++e)
                            cen[s][e] = (PASS == 2 && s == 2) ? cc_0[e] : c_0[s][e];
#pragma unroll
                    for (int e = 0; e < kVEC; ++e) {
                        float cv[S], iv[S];
#pragma unroll
                        for (int s = 0; s < S; ++s) cv[s] = cen[s][e];
                        M::react(sd, cv, iv);
#pragma unroll
                        for (int s = 0; s < S; ++s) inc[s][e] = iv[s];
                    }
                    if (W3 && (cy != 0.0f || cz != 0.0f)) {
                        // upwind along y and z (3-D wind): y neighbours from
                        // plane q, z neighbours from the thread's own column
                        // in planes q - 1 (still in the ring) and q + 1
                        const unsigned char* Pm = ring + sm * SLOTB + own_b;
#pragma unroll
                        for (int s = 0; s < S; ++s) {
                            float ym[kVEC], yp[kVEC], zm[kVEC];
                            lds_vec<ST>(Pc + s * PEB - kRW * EB, ym);
                            lds_vec<ST>(Pc + s * PEB + kRW * EB, yp);
                            lds_vec<ST>(Pm + s * PEB, zm);
                            upwind_axis(cy, cen[s], ym, yp, inc[s]);
                            upwind_axis(cz, cen[s], zm, c_p[s < NSUM ? s : 0], inc[s]);
                        }
                    }
                    const float cx = PLAIN ? 0.0f : courant_at(sd, courant, zq);
                    const bool src_here = src_col && zq == sd.src_z;
                    const unsigned faces = xyf | z_faces(q, nz);
#pragma unroll
                    for (int s = 0; s < S; ++s) {
                        float o[kVEC];
                        // PASS 2, c: the Laplacian is that of mu (summed field 2)
                        const float(&ls)[kVEC] = lap6[(PASS == 2 && s == 2) ? 2 : (s < NSUM ? s : 0)];
                        float left = 0.0f, right = 0.0f;
                        if (!PLAIN && cx != 0.0f) {
                            left = lds_one<ST>(Pc + s * PEB + loff);
                            right = lds_one<ST>(Pc + s * PEB + roff);
                        }
                        species19<PLAIN>(sd, s, k6[s], cen[s], ls, inc[s], cx, left, right,
                                         src_here, px, xs, o);
                        if constexpr (!PLAIN) held_layers_at(sd, s, faces, xs, y, q, o);
                        if (computes && RD_DBG_GLOBAL(sd, gst + s * fstride, 4 * (int)sizeof(ST),
                                                      kSiteStateStore))
                            Store<ST>::store(gst + s * fstride, o);
                    }
                }
#pragma unroll
                for (int f = 0; f < NSUM; ++f)
#pragma unroll
                    for (int e = 0; e < kVEC; ++e) {
                        zsum_m[f][e] = zsum_0[f][e];
                        zsum_0[f][e] = zsum_p[f][e];
                        wsum_0[f][e] = wsum_p[f][e];
                        c_0[f][e] = c_p[f][e];
                    }
                if constexpr (PASS == 2)
#pragma unroll
                    for (int e = 0; e < kVEC; ++e) cc_0[e] = cc_p[e];
            }
            gst += plane;
            if constexpr (PASS == 1) gmu_st += plane;
            sc = sc == RING - 1 ? 0 : sc + 1;
            if (!pz) zq = q + 1;
            else if (++zq == nz) zq = 0;
        }
        cp_async_wait<0>();
        __syncthreads();
    }
}

// Launch helper used by the per-model translation units: even tile heights
// (16 TY compute threads, then a whole halo warp); single instances (the
// descriptor in the kernel parameters) or batches (a device array of
// descriptors).
template <class M, class ST, int PASS>
cudaError_t launch19_pass(const LaunchArgs& a, int grid, size_t smem, cudaStream_t st, int* occ) {
    if ((a.ty & 1) || a.ty < 2) return cudaErrorInvalidValue;
    void (*k)(const LaunchArgs);
    const bool w3 = PASS == 0 && !a.plain && a.wind3;
    if (a.use_one)
        k = a.plain ? rd_step19_kernel<M, ST, true, true, PASS>
            : w3    ? rd_step19_kernel<M, ST, true, false, PASS, PASS == 0>
                    : rd_step19_kernel<M, ST, true, false, PASS>;
    else
        k = a.plain ? rd_step19_kernel<M, ST, false, true, PASS>
            : w3    ? rd_step19_kernel<M, ST, false, false, PASS, PASS == 0>
                    : rd_step19_kernel<M, ST, false, false, PASS>;
    static size_t configured[6] = {0, 0, 0, 0, 0, 0};
    size_t& conf = configured[(a.plain ? 1 : w3 ? 2 : 0) + (a.use_one ? 3 : 0)];
    if (smem > conf) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        conf = smem;
    }
    const int threads = Layout19<M, ST, PASS>::threads(a.ty);
    if (threads > kMaxThreads) return cudaErrorInvalidConfiguration;
    if (occ) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k, threads, smem);
    k<<<grid, threads, smem, st>>>(a);
    return cudaGetLastError();
}

template <class M>
cudaError_t launch19_model(int storage, const LaunchArgs& a, int grid, size_t smem,
                           cudaStream_t st, int* occ) {
    if (storage == RD_STORE_F32) return launch19_pass<M, float, 0>(a, grid, smem, st, occ);
    if (storage == RD_STORE_BF16)
        return launch19_pass<M, __nv_bfloat16, 0>(a, grid, smem, st, occ);
    return cudaErrorInvalidValue;
}

// The two launches of a Cahn-Hilliard step: pass 1 (mu), pass 2 (update).
// ``smem`` is pass 2's size; pass 1 takes the smaller ring of its own layout.
template <class M>
cudaError_t launch19_ch_model(int storage, int pass, const LaunchArgs& a, int grid, size_t smem,
                              cudaStream_t st, int* occ) {
    if (storage == RD_STORE_F32)
        return pass == 1 ? launch19_pass<M, float, 1>(a, grid, Layout19<M, float, 1>::total(a.ty),
                                                      st, occ)
                         : launch19_pass<M, float, 2>(a, grid, smem, st, occ);
    if (storage == RD_STORE_BF16)
        return pass == 1 ? launch19_pass<M, __nv_bfloat16, 1>(
                               a, grid, Layout19<M, __nv_bfloat16, 1>::total(a.ty), st, occ)
                         : launch19_pass<M, __nv_bfloat16, 2>(a, grid, smem, st, occ);
    return cudaErrorInvalidValue;
}

}  // namespace rdk
