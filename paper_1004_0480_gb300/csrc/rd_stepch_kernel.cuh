// rd_stepch_kernel.cuh -- the one-step kernel of the models with a
// Cahn-Hilliard species (7-point stencil), included from rd_step_kernel.cuh
// after the helpers it shares with the other step kernels.
#pragma once

namespace rdk {

// -------------------------------------------- one-step Cahn-Hilliard kernel
// The T = 1 path of the models with a Cahn-Hilliard species c (the front
// model a + b -> c, and the phase separation of Table 1, row 3).  Ghost
// cells are copied in by mirror extension to distance two (index -1-i holds
// cell i at a zero-flux face), so mu computed at a ghost cell equals mu at
// the face cell -- the paper's "Laplacian, boundary rule, Laplacian" -- and
// every neighbour sits at a fixed offset.  One thread per 4-cell vector of
// the tile widened by one vector in x and one row in y: at step p each
// computes mu of plane p+1 at its position, and the threads of the tile
// proper (the first warps) the new state of plane p.
// A thread keeps its own mu of planes p-1..p+1 and its own c of planes
// p..p+2 in registers; neighbours' mu of plane p come from a 2-slot shared
// ring (written at step p-1).
// State planes arrive in a 6-slot ring, P = 4 copy groups ahead: at step p
// planes p-1..p+2 are read and p+3, p+4 are in flight.  Slot reuse: step p
// refills the slot of plane p-2, whose neighbour reads (mu of p-2 at step
// p-3, update of p-2 at step p-2) ended a barrier earlier and whose last
// read (own vector, update of p-1) precedes the refill in the owner's
// program order -- every vector is copied by the thread that owns it; the
// two outer rows are only read as neighbours.  The mu slot written at step
// p held mu of p-1, whose last reads were at step p-1.  One barrier per
// plane.
template <class ST> struct LayoutCH {
    static constexpr int S = 3;
    static constexpr int RING = 6;
    static constexpr int P = 4;
    static constexpr int MURING = 2;
    __host__ __device__ static int rows(int ty) { return ty + 4; }
    __host__ __device__ static int plane_elems(int ty) { return rows(ty) * kRW + 2 * kVEC; }
    __host__ __device__ static size_t state_bytes(int ty) {
        return (size_t)RING * S * plane_elems(ty) * sizeof(ST);
    }
    __host__ __device__ static size_t total(int ty) {
        return state_bytes(ty) + (size_t)MURING * plane_elems(ty) * sizeof(float);
    }
    __host__ __device__ static int threads(int ty) { return kNQ * (ty + 2); }
};

// Mirror extension: -1-i for i < 0, 2n-1-i for i >= n; clamped so that
// positions outside the grid by more than n (never stored) stay in bounds.
__device__ __forceinline__ int mirror_index(int i, int n) {
    const int m = i < 0 ? -1 - i : (i >= n ? 2 * n - 1 - i : i);
    return min(max(m, 0), n - 1);
}

// How one vector of the front kernel is fetched: 1 = one async copy, 2 =
// element by element from the precomputed in-row offsets e[] (a vector
// crossing a face: mirror-extended or wrapped elements), 0 = nothing.
struct FetchM {
    int mode;
    int goff;    // element offset of the row (+ x for mode 1) within a plane
    int soff;    // byte offset of the position within a plane buffer
    int e[kVEC]; // mode 2: element offsets within the row
};

// Fetch with mirror-extended (zero-flux) or wrapped (periodic) coordinates.
// Vectors past row ny + 1 or column nx + 1 feed no stored cell: not copied.
// Nor the vectors wholly beyond a zero-flux x face that lies on a vector
// boundary (x = 0, and x = nx when nx is a multiple of 4): their cells are
// the mirror images of the face vector, c(-1) = c(0) and mu(-1) = mu(0) bit
// for bit (mu's x sum adds the same two values in the other order), so the
// face thread reads its own cells instead (see the kernel).
template <class ST>
__device__ __forceinline__ FetchM make_fetch_mirror(int yrow, int xs, int nx, int ny, int pitch,
                                                    bool px, bool py, int soff_elems) {
    FetchM f{0, 0, soff_elems * (int)sizeof(ST), {0, 0, 0, 0}};
    if (yrow > ny + 1 || xs > nx + 1) return f;
    if (!px && (xs + kVEC <= 0 || (xs >= nx && nx % kVEC == 0))) return f;
    const int yw = py ? wrapi(yrow, ny) : mirror_index(yrow, ny);
    const int row = yw * pitch;
    f.goff = row;
    if (xs >= 0 && xs + kVEC <= nx) {
        f.mode = 1;
        f.goff = row + xs;
        return f;
    }
    if (px) {
        const int xw = wrapi(xs, nx);
        if (xw % kVEC == 0 && xw + kVEC <= nx) {
            f.mode = 1;
            f.goff = row + xw;
            return f;
        }
    }
    f.mode = 2;
#pragma unroll
    for (int e = 0; e < kVEC; ++e) f.e[e] = px ? wrapi(xs + e, nx) : mirror_index(xs + e, nx);
    return f;
}

template <class ST, int S>
__device__ __forceinline__ void fetch_all_mirror(const FetchM& f, unsigned char* plane_buf,
                                                 int pe_bytes, const ST* gplane, long long fstride,
                                                 const InstDesc& sd) {
#pragma unroll
    for (int s = 0; s < S; ++s) {
        const ST* src = gplane + s * fstride + f.goff;
        const int ok =
            f.mode == 1 && RD_DBG_GLOBAL(sd, src, 4 * (int)sizeof(ST), kSiteCopySrc);
        Store<ST>::cp_async_if(reinterpret_cast<ST*>(plane_buf + s * pe_bytes + f.soff), src, ok);
    }
    if (f.mode == 2) {
#pragma unroll
        for (int s = 0; s < S; ++s) {
            ST* d = reinterpret_cast<ST*>(plane_buf + s * pe_bytes + f.soff);
            const ST* g = gplane + s * fstride + f.goff;
#pragma unroll
            for (int e = 0; e < kVEC; ++e)
                if (RD_DBG_GLOBAL(sd, g + f.e[e], (int)sizeof(ST), kSiteCopySrc))
                    Store<ST>::cp_async_elem(d + e, g + f.e[e]);
        }
    }
}

// PLAIN: no point source or wind and isotropic D for a and b (held layers
// are still applied); the update of a and b then needs no per-plane tests.
template <class MC, class ST, bool ONE, bool PLAIN>
__global__ void __launch_bounds__(kMaxThreads, 1)
rd_stepch_kernel(const __grid_constant__ LaunchArgs a) {
    using LY = LayoutCH<ST>;
    constexpr int S = 3;
    constexpr int P = LY::P;
    constexpr int RING = LY::RING;
    constexpr int EB = (int)sizeof(ST);
    constexpr int RWB = kRW * EB;

    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ InstDesc sdm;
    __shared__ int s_inst;
    __shared__ long long s_item;

    const int tid = threadIdx.x;
    const int TY = a.ty;
    const int PE = LY::plane_elems(TY);
    const int PEB = PE * EB;
    const int SLOTB = S * PEB;
    unsigned char* const ring = smem + kVEC * EB;
    float* const muring = reinterpret_cast<float*>(smem + LY::state_bytes(TY)) + kVEC;
    // thread -> position (r, v): row r - 1 of the tile (rows -1..TY), vector
    // v - 1 (vectors -1..16).  The 16 x TY inner positions come first, then
    // the halo ring (the row above, the row below, then left/right of each
    // row), so the halo threads fill the last warps and skip the update as
    // whole warps.
    const int ninner = kTileQ * TY;
    const bool inner = tid < ninner;
    int r, v;
    if (inner) {
        r = tid / kTileQ + 1;
        v = tid - (r - 1) * kTileQ + 1;
    } else {
        const int j = tid - ninner;
        if (j < kNQ) {
            r = 0;
            v = j;
        } else if (j < 2 * kNQ) {
            r = TY + 1;
            v = j - kNQ;
        } else {
            r = (j - 2 * kNQ) / 2 + 1;
            v = ((j - 2 * kNQ) & 1) ? kNQ - 1 : 0;
        }
    }
    const int own = (r + 1) * kRW + v * kVEC;       // element offset in a plane
    const int own_b = own * EB;

    int cur_inst = -1;
    if (tid == 0) s_inst = 0;
    for (long long item = first_item<ONE>(a, s_item); item < a.nitems;
         item = next_item<ONE>(a, item, s_item)) {
        if constexpr (!ONE) load_desc(a, item, sdm, s_inst, cur_inst);
        const InstDesc& sd = desc_of<ONE>(a, sdm);
        if (member_done<ONE>(a, sd)) continue;   // block-uniform

        const int nx = sd.nx, ny = sd.ny, nz = sd.nz, pitch = sd.pitch;
        const bool px = sd.per_x, py = sd.per_y, pz = sd.per_z;
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
        const long long fstride = reinterpret_cast<const ST*>(sd.base[lin][1]) - gin;
        const long long plane = sd.plane;

        const int y = y0 - 1 + r;                     // global row of the position
        const int xs = x0 - kVEC + v * kVEC;          // global x of its first element
        const bool stores = inner && y < ny && xs < nx;
        // a zero-flux x face on the vector's edge: the neighbour beyond it is
        // the own face cell, for c and for mu alike
        const bool lface = !px && xs == 0;
        const bool rface = !px && xs + kVEC == nx;
        const unsigned xyf = xy_faces(xs, y, nx, ny);
        const bool src_col = sd.src_s >= 0 && (py ? wrapi(y, ny) : y) == sd.src_y;
        // own state vector, and (first 2 x 18 threads) the outer halo rows
        const FetchM fo = make_fetch_mirror<ST>(y, xs, nx, ny, pitch, px, py, own);
        FetchM fx{0, 0, 0, {0, 0, 0, 0}};
        if (tid < 2 * kNQ) {
            const bool bottom = tid >= kNQ;
            const int vv = tid - (bottom ? kNQ : 0);
            fx = make_fetch_mirror<ST>(bottom ? y0 + TY + 1 : y0 - 2, x0 - kVEC + vv * kVEC, nx, ny,
                                       pitch, px, py, (bottom ? TY + 3 : 0) * kRW + vv * kVEC);
        }

        // planes z0-2 .. z1+1 are copied; plane nld goes to slot sld
        int nld = z0 - 2, sld = 0;
        auto issue = [&]() {
            if (nld <= z1 + 1) {
                const int zs = pz ? wrapi(nld, nz) : mirror_index(nld, nz);
                const ST* g = gin + (long long)zs * plane;
                unsigned char* buf = ring + sld * SLOTB;
                fetch_all_mirror<ST, S>(fo, buf, PEB, g, fstride, sd);
                if (tid < 2 * kNQ) fetch_all_mirror<ST, S>(fx, buf, PEB, g, fstride, sd);
            }
            ++nld;
            sld = (sld == RING - 1) ? 0 : sld + 1;
            cp_async_commit();
        };
#pragma unroll 1
        for (int j = 0; j < P; ++j) issue();

        const float* courant = sd.courant;
        ST* gst = gout + (long long)z0 * plane + (long long)y * pitch + xs;
        float mu_m[kVEC] = {}, mu_0[kVEC] = {};       // own mu of planes p-1, p
        float cz_m[kVEC] = {}, cz_0[kVEC] = {};       // own c of planes p, p+1
        int sc = 0;                                   // ring slot of plane p
        // unrolled by 3: the three-plane windows of mu and c rotate by
        // renaming registers instead of moves
#pragma unroll 3
        for (int p = z0 - 2; p < z1; ++p) {
            // planes through p + 2 must have landed: of the P + (p - z0 + 3)
            // groups issued so far, all but the newest P - 2
            issue();
            cp_async_wait<P - 2>();
            __syncthreads();
            const int sm = sc == 0 ? RING - 1 : sc - 1;
            const int s1 = sc == RING - 1 ? 0 : sc + 1;
            const int s2 = s1 == RING - 1 ? 0 : s1 + 1;
            float mu_p[kVEC];                         // own mu of plane p + 1
            float cz_p[kVEC];                         // own c of plane p + 2
            {
                const unsigned char* Cc = ring + s1 * SLOTB + 2 * PEB + own_b;
                if (p == z0 - 2) {
                    lds_vec<ST>(ring + sc * SLOTB + 2 * PEB + own_b, cz_m);
                    lds_vec<ST>(Cc, cz_0);
                }
                const float(&zm)[kVEC] = cz_m;
                const float(&c)[kVEC] = cz_0;
                float ym[kVEC], yp[kVEC];
                const float(&zp)[kVEC] = cz_p;
                lds_vec<ST>(ring + s2 * SLOTB + 2 * PEB + own_b, cz_p);
                lds_vec<ST>(Cc - RWB, ym);
                lds_vec<ST>(Cc + RWB, yp);
                const float left = lface ? c[0] : lds_one<ST>(Cc - EB);
                const float right = rface ? c[kVEC - 1] : lds_one<ST>(Cc + kVEC * EB);
#pragma unroll
                for (int e = 0; e < kVEC; ++e) {
                    const float xm = e ? c[e - 1] : left;
                    const float xp = (e < kVEC - 1) ? c[e + 1] : right;
                    mu_p[e] = MC::mu(sd, c[e], xm, xp, ym[e], yp[e], zm[e], zp[e]);
                }
                Store<float>::store(muring + ((p + 1) & 1) * PE + own, mu_p);
            }
            if (p >= z0 && inner) {
                // ---- new state of plane p at the inner positions
                const unsigned char* Sc = ring + sc * SLOTB + own_b;
                const unsigned char* Sm = ring + sm * SLOTB + own_b;
                const unsigned char* Sp = ring + s1 * SLOTB + own_b;
                const unsigned faces = xyf | z_faces(p, nz);
                float cen[S][kVEC], inc[S][kVEC];
#pragma unroll
                for (int s = 0; s < 2; ++s) lds_vec<ST>(Sc + s * PEB, cen[s]);
#pragma unroll
                for (int e = 0; e < kVEC; ++e) cen[2][e] = cz_m[e];   // c of plane p, carried
#pragma unroll
                for (int e = 0; e < kVEC; ++e) {
                    float cv[S], iv[S];
#pragma unroll
                    for (int s = 0; s < S; ++s) cv[s] = cen[s][e];
                    MC::react(sd, cv, iv);
#pragma unroll
                    for (int s = 0; s < S; ++s) inc[s][e] = iv[s];
                }
                const float cx = courant_at(sd, courant, p);
                const bool src_here = src_col && p == sd.src_z;
#pragma unroll
                for (int s = 0; s < 2; ++s) {
                    const unsigned char* Ps = Sc + s * PEB;
                    float xm[kVEC], xp[kVEC], ym[kVEC], yp[kVEC], zm[kVEC], zp[kVEC], o[kVEC];
                    lds_vec<ST>(Sm + s * PEB, zm);
                    lds_vec<ST>(Sp + s * PEB, zp);
                    lds_vec<ST>(Ps - RWB, ym);
                    lds_vec<ST>(Ps + RWB, yp);
                    const float left = lface ? cen[s][0] : lds_one<ST>(Ps - EB);
                    const float right = rface ? cen[s][kVEC - 1] : lds_one<ST>(Ps + kVEC * EB);
#pragma unroll
                    for (int e = 0; e < kVEC; ++e) {
                        xm[e] = e ? cen[s][e - 1] : left;
                        xp[e] = (e < kVEC - 1) ? cen[s][e + 1] : right;
                    }
                    if constexpr (PLAIN) {
                        // the same arithmetic species_core takes for this case
                        const float k = sd.kx[s];
#pragma unroll
                        for (int e = 0; e < kVEC; ++e)
                            o[e] = euler_cell_iso(cen[s][e], xm[e], xp[e], ym[e], yp[e], zm[e],
                                                  zp[e], k, inc[s][e]);
                    } else {
                        species_core(sd, s, cen[s], xm, xp, ym, yp, zm, zp, inc[s], cx, src_here,
                                     px, xs, o);
                    }
                    held_layers_at(sd, s, faces, xs, y, p, o);
                    if (stores &&
                        RD_DBG_GLOBAL(sd, gst + s * fstride, 4 * (int)sizeof(ST), kSiteStateStore))
                        Store<ST>::store(gst + s * fstride, o);
                }
                {
                    // c += dt M / h^2 * (7-point Laplacian of mu)
                    const float* Mc = muring + (p & 1) * PE + own;
                    float mym[kVEC], myp[kVEC], o[kVEC];
                    Store<float>::load(Mc - kRW, mym);
                    Store<float>::load(Mc + kRW, myp);
                    const float mleft = lface ? mu_0[0] : Store<float>::get(Mc - 1);
                    const float mright = rface ? mu_0[kVEC - 1] : Store<float>::get(Mc + kVEC);
#pragma unroll
                    for (int e = 0; e < kVEC; ++e) {
                        const float mxm = e ? mu_0[e - 1] : mleft;
                        const float mxp = (e < kVEC - 1) ? mu_0[e + 1] : mright;
                        const float s6 = __fadd_rn(__fadd_rn(__fadd_rn(mxm, mxp), __fadd_rn(mym[e], myp[e])),
                                                   __fadd_rn(mu_m[e], mu_p[e]));
                        const float lap = __fmaf_rn(-6.0f, mu_0[e], s6);
                        o[e] = __fadd_rn(cen[2][e], __fmaf_rn(sd.p[1], lap, inc[2][e]));
                    }
                    held_layers_at(sd, 2, faces, xs, y, p, o);
                    if (stores &&
                        RD_DBG_GLOBAL(sd, gst + 2 * fstride, 4 * (int)sizeof(ST), kSiteStateStore))
                        Store<ST>::store(gst + 2 * fstride, o);
                }
            }
            if (p >= z0) gst += plane;
#pragma unroll
            for (int e = 0; e < kVEC; ++e) {
                mu_m[e] = mu_0[e];
                mu_0[e] = mu_p[e];
                cz_m[e] = cz_0[e];
                cz_0[e] = cz_p[e];
            }
            sc = s1;
        }
        cp_async_wait<0>();
        __syncthreads();
    }
}

}  // namespace rdk
