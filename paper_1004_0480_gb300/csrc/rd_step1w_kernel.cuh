// rd_step1w_kernel.cuh -- the one-step 7-point kernel with 8 cells per
// thread (tile_q = 8 in rd_tuning), for the models without Cahn-Hilliard.
//
// The work items, the 64-cell tile width, the 6-slot cp.async ring of
// planes, the halo warp and the boundary rules are those of rd_step1_kernel
// (rd_step_kernel.cuh); what differs:
//
//  * Each compute thread owns 8 consecutive cells of a row: a tile row is 8
//    threads, a warp 4 rows.  Its plane copies are 16 bytes for bfloat16
//    state (two for float32), and the fixed work of a thread and plane
//    (addresses, the copy loop, the barrier) is spread over twice the cells.
//  * The x neighbours beside the own vector come from the adjacent lanes by
//    warp shuffle (__shfl_up_sync / __shfl_down_sync over whole compute
//    warps: the host admits tile heights that are multiples of 4 only, so
//    no warp holds both compute and halo threads).  The lanes at a tile
//    row's ends read the halo vector in shared memory instead, or at a
//    zero-flux x face their own face cell (the ghost equals it).
//  * Only the own vector of plane q is carried in registers; that of plane
//    q - 1 is re-read from the ring (still resident), which keeps three
//    species within the register budget.
// Every cell is updated by the per-cell functions of rd_step_kernel.cuh in
// the same order, so results equal the 4-cell kernel's bit for bit.
#pragma once

namespace rdk {

constexpr int kW8 = 8;                 // cells per thread
constexpr int kQ8 = 8;                 // threads per tile row (64 cells)
constexpr int kNQ8 = kQ8 + 2;          // vectors per shared row incl. halo
constexpr int kRW8 = kNQ8 * kW8;       // elements per shared row

// 8-cell vectors of either storage type; shared sides checked in the
// debug build as in Store<>.
template <class ST> struct Vec8;

template <> struct Vec8<float> {
    __device__ __forceinline__ static void load(const float* p, float (&v)[8]) {
        Store<float>::load(p, *reinterpret_cast<float(*)[4]>(v));
        Store<float>::load(p + 4, *reinterpret_cast<float(*)[4]>(v + 4));
    }
    __device__ __forceinline__ static void store(float* p, const float (&v)[8]) {
        Store<float>::store(p, *reinterpret_cast<const float(*)[4]>(v));
        Store<float>::store(p + 4, *reinterpret_cast<const float(*)[4]>(v + 4));
    }
    __device__ __forceinline__ static void cp_async_if(float* smem, const float* g, int pred) {
        Store<float>::cp_async_if(smem, g, pred);
        Store<float>::cp_async_if(smem + 4, g + 4, pred);
    }
};

template <> struct Vec8<__nv_bfloat16> {
    __device__ __forceinline__ static void load(const __nv_bfloat16* p, float (&v)[8]) {
        if (!RD_DBG_ANY(p, 16, kSiteSharedLoad)) {
#pragma unroll
            for (int e = 0; e < 8; ++e) v[e] = 0.0f;
            return;
        }
        const uint4 t = *reinterpret_cast<const uint4*>(p);
        const unsigned w[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            v[2 * k] = __uint_as_float(w[k] << 16);
            v[2 * k + 1] = __uint_as_float(w[k] & 0xffff0000u);
        }
    }
    __device__ __forceinline__ static void store(__nv_bfloat16* p, const float (&v)[8]) {
        if (!RD_DBG_ANY(p, 16, kSiteSharedStore)) return;
        unsigned w[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * k], v[2 * k + 1]);
            w[k] = *reinterpret_cast<unsigned*>(&h);
        }
        *reinterpret_cast<uint4*>(p) = make_uint4(w[0], w[1], w[2], w[3]);
    }
    // 16 bytes, where ``pred`` holds
    __device__ __forceinline__ static void cp_async_if(__nv_bfloat16* smem, const __nv_bfloat16* g,
                                                       int pred) {
        if (pred && !RD_DBG_SHARED(smem, 16, kSiteCopyDst)) return;
        const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
        asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %2, 0;\n"
                     " @p cp.async.cg.shared.global [%0], [%1], 16;\n}\n" ::"r"(s), "l"(g),
                     "r"(pred)
                     : "memory");
    }
};

// How one 8-cell vector is fetched (see make_fetch; the same rules).
template <class ST>
__device__ __forceinline__ Fetch make_fetch8(int yrow, int xs, int nx, int ny, int pitch, bool px,
                                             bool py, int soff_elems) {
    Fetch f{0, 0, soff_elems * (int)sizeof(ST), xs};
    int yw = yrow;
    if (py) yw = wrapi(yrow, ny);
    else if (yrow < 0 || yrow >= ny) yw = yrow < 0 ? 0 : ny - 1;    // ghost row = face row
    const int row = yw * pitch;
    if (xs >= 0 && xs + kW8 <= nx) {
        f.mode = 1;
        f.goff = row + xs;
    } else if (px) {
        const int xw = wrapi(xs, nx);
        if (xw % kW8 == 0 && xw + kW8 <= nx) { f.mode = 1; f.goff = row + xw; }
        else { f.mode = 2; f.goff = row; }
    } else if (xs < nx && xs + kW8 > 0) {
        f.mode = 2;                               // straddles a face: clamped ghosts
        f.goff = row;
    }
    return f;
}

template <class ST, int S>
__device__ __forceinline__ void fetch_all8(const Fetch& f, unsigned char* plane_buf, int pe_bytes,
                                           const ST* gplane, long long fstride, int nx, bool px,
                                           const InstDesc& sd) {
#pragma unroll
    for (int s = 0; s < S; ++s) {
        const ST* src = gplane + s * fstride + f.goff;
        const int ok =
            f.mode == 1 && RD_DBG_GLOBAL(sd, src, kW8 * (int)sizeof(ST), kSiteCopySrc);
        Vec8<ST>::cp_async_if(reinterpret_cast<ST*>(plane_buf + s * pe_bytes + f.soff), src, ok);
    }
    if (f.mode == 2) {
#pragma unroll
        for (int s = 0; s < S; ++s) {
            ST* d = reinterpret_cast<ST*>(plane_buf + s * pe_bytes + f.soff);
#pragma unroll
            for (int e = 0; e < kW8; ++e) {
                const int x = f.xs + e;
                const int xi = px ? wrapi(x, nx) : (x < 0 ? 0 : (x >= nx ? nx - 1 : x));
                const ST* src = gplane + s * fstride + f.goff + xi;
                if (RD_DBG_GLOBAL(sd, src, (int)sizeof(ST), kSiteCopySrc))
                    Store<ST>::cp_async_elem(d + e, src);
            }
        }
    }
}

template <class M, class ST> struct Layout1w {
    static constexpr int S = M::S;
    static constexpr int RING = 6;
    static constexpr int P = 5;
    __host__ __device__ static int plane_elems(int ty) { return (ty + 2) * kRW8 + 2 * kW8; }
    __host__ __device__ static size_t total(int ty) {
        return (size_t)RING * S * plane_elems(ty) * sizeof(ST) + 96 * sizeof(int4);
    }
    __host__ __device__ static int threads(int ty) { return kQ8 * ty + 32; }
};

// One half (cells 4h .. 4h + 3) of an 8-cell array, for the 4-cell helpers.
template <class A> __device__ __forceinline__ const float (&chalf4(const A& v, int h))[4] {
    return *reinterpret_cast<const float(*)[4]>(&v[4 * h]);
}

// PLAIN, W3: as rd_step1_kernel.  Tile heights are multiples of 4.
template <class M, class ST, bool ONE, bool PLAIN, bool W3>
__global__ void __launch_bounds__(kMaxThreads, 1)
rd_step1w_kernel(const __grid_constant__ LaunchArgs a) {
    using LY = Layout1w<M, ST>;
    constexpr int S = M::S;
    constexpr int P = LY::P;
    constexpr int RING = LY::RING;
    constexpr int EB = (int)sizeof(ST);
    constexpr int RWB = kRW8 * EB;                           // bytes per shared row
    constexpr unsigned FULL = 0xffffffffu;

    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ InstDesc sdm;
    __shared__ int s_inst;
    __shared__ long long s_item;

    const int tid = threadIdx.x;
    const int TY = a.ty;
    const int PEB = LY::plane_elems(TY) * EB;                // bytes per species plane
    const int SLOTB = S * PEB;                               // bytes per ring slot
    unsigned char* const ring = smem + kW8 * EB;             // slot 0, species 0
    int4* const hfetch = reinterpret_cast<int4*>(smem + RING * SLOTB);
    const int ncomp = kQ8 * TY;
    const bool halo_warp = tid >= ncomp;
    const int r = tid / kQ8;
    const int v = tid - r * kQ8;
    const int own_b = ((r + 1) * kRW8 + (v + 1) * kW8) * EB;

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
        const int x0 = txi * kQ8 * kW8, y0 = tyi * TY;
        const int z0 = zc * sd.zchunk;
        const int z1 = min(z0 + sd.zchunk, nz);
        const int lin = sd.par ^ a.parity;
        const ST* const gin = reinterpret_cast<const ST*>(sd.base[lin][0]);
        ST* const gout = reinterpret_cast<ST*>(sd.base[lin ^ 1][0]);
        const long long fstride = S > 1 ? reinterpret_cast<const ST*>(sd.base[lin][1]) - gin : 0;
        const long long plane = sd.plane;

        // ---- halo lanes: 2 TY side vectors, then 2 x 8 row vectors
        if (halo_warp) {
            const int hl = tid - ncomp;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const int j = hl + 32 * k;
                Fetch f{0, 0, 0, 0};
                if (j < 2 * TY) {
                    const int hr = j >> 1;
                    const bool right = j & 1;
                    const int xh = right ? x0 + kQ8 * kW8 : x0 - kW8;
                    f = make_fetch8<ST>(y0 + hr, xh, nx, ny, pitch, px, py,
                                        (hr + 1) * kRW8 + (right ? kNQ8 - 1 : 0) * kW8);
                } else if (j < 2 * TY + 2 * kQ8) {
                    const int jj = j - 2 * TY;
                    const bool bottom = jj >= kQ8;
                    const int hv = jj - (bottom ? kQ8 : 0);
                    f = make_fetch8<ST>(bottom ? y0 + TY : y0 - 1, x0 + hv * kW8, nx, ny, pitch,
                                        px, py, (bottom ? TY + 1 : 0) * kRW8 + (hv + 1) * kW8);
                }
                if (RD_DBG_SHARED(hfetch + j, 16, kSiteHaloDesc))
                    hfetch[j] = make_int4(f.mode, f.goff, f.soff, f.xs);
            }
        }
        // ---- compute threads: own vector and its neighbours
        const int y = y0 + r;
        const int xs = x0 + v * kW8;
        const bool computes = !halo_warp && y < ny && xs < nx;
        const bool src_col = sd.src_s >= 0 && (py ? wrapi(y, ny) : y) == sd.src_y;
        const unsigned xyf[2] = {xy_faces(xs, y, nx, ny), xy_faces(xs + 4, y, nx, ny)};
        const Fetch fo = halo_warp ? Fetch{0, 0, 0, 0}
                                   : make_fetch8<ST>(y, xs, nx, ny, pitch, px, py, own_b / EB);
        // at a zero-flux x face the neighbour beyond it is the own face cell
        const bool lface = !px && xs == 0;
        const bool rface = !px && xs + kW8 == nx;
        float cy = 0.0f, cz = 0.0f;               // 3-D wind
        if constexpr (W3) wind3d(sd, lin, local, cy, cz);
        __syncthreads();   // halo descriptors written

        // ---- the march (as rd_step1_kernel)
        int nld = z0 - 1;
        int zld = pz ? wrapi(nld, nz) : nld;
        auto issue = [&](int sl) {
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
                        fetch_all8<ST, S>(Fetch{h.x, h.y, h.z, h.w}, buf, PEB, gld, fstride, nx,
                                          px, sd);
                    }
                } else {
                    fetch_all8<ST, S>(fo, buf, PEB, gld, fstride, nx, px, sd);
                }
            }
            ++nld;
            if (!pz) zld = nld;
            else if (++zld == nz) zld = 0;
            cp_async_commit();
        };
#pragma unroll 1
        for (int j = 0; j < P; ++j) issue(j);
        int zq = pz ? wrapi(z0, nz) : z0;
        ST* gst = gout + (long long)z0 * plane + (long long)y * pitch + xs;
        const float* courant = sd.courant;
        int sc = 1;                               // ring slot of plane q
        float own_0[S][kW8];                      // own vector of plane q
#pragma unroll 1
        for (int q = z0; q < z1; ++q) {
            const int sm = sc == 0 ? RING - 1 : sc - 1;
            const int sp = sc == RING - 1 ? 0 : sc + 1;
            issue(sc >= RING - P + 1 ? sc + P - 1 - RING : sc + P - 1);
            cp_async_wait<P - 2>();
            __syncthreads();
            if (!halo_warp) {
                const unsigned char* Pc = ring + sc * SLOTB + own_b;
                const unsigned char* Pm = ring + sm * SLOTB + own_b;
                const unsigned char* Pp = ring + sp * SLOTB + own_b;
                if (q == z0) {
#pragma unroll
                    for (int s = 0; s < S; ++s)
                        Vec8<ST>::load(reinterpret_cast<const ST*>(Pc + s * PEB), own_0[s]);
                }
                float own_p[S][kW8];
#pragma unroll
                for (int s = 0; s < S; ++s)
                    Vec8<ST>::load(reinterpret_cast<const ST*>(Pp + s * PEB), own_p[s]);
                const float cx = PLAIN ? 0.0f : courant_at(sd, courant, zq);
                const bool src_here = src_col && zq == sd.src_z;
                const unsigned zf = z_faces(q, nz);
                // x neighbours beside the own vector, species by species
                float left[S], right[S];
#pragma unroll
                for (int s = 0; s < S; ++s) {
                    const float lsh = __shfl_up_sync(FULL, own_0[s][kW8 - 1], 1);
                    const float rsh = __shfl_down_sync(FULL, own_0[s][0], 1);
                    const unsigned char* Ps = Pc + s * PEB;
                    // a zero-flux face first: it may end a vector inside the
                    // tile row (the lanes beyond it hold no cells)
                    left[s] = lface ? own_0[s][0] : (v != 0 ? lsh : lds_one<ST>(Ps - EB));
                    right[s] = rface ? own_0[s][kW8 - 1]
                                     : (v != kQ8 - 1 ? rsh : lds_one<ST>(Ps + kW8 * EB));
                }
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    // reaction on the half's 4 cells
                    float inc[S][kVEC];
#pragma unroll
                    for (int e = 0; e < kVEC; ++e) {
                        float cv[S], iv[S];
#pragma unroll
                        for (int s = 0; s < S; ++s) cv[s] = own_0[s][4 * h + e];
                        M::react(sd, cv, iv);
#pragma unroll
                        for (int s = 0; s < S; ++s) inc[s][e] = iv[s];
                    }
#pragma unroll
                    for (int s = 0; s < S; ++s) {
                        const unsigned char* Ps = Pc + s * PEB + h * kVEC * EB;
                        float ym[kVEC], yp[kVEC], zm[kVEC], xm[kVEC], xp[kVEC], o[kVEC];
                        lds_vec<ST>(Ps - RWB, ym);
                        lds_vec<ST>(Ps + RWB, yp);
                        lds_vec<ST>(Pm + s * PEB + h * kVEC * EB, zm);
                        const float(&cen)[kVEC] = chalf4(own_0[s], h);
                        const float(&zp)[kVEC] = chalf4(own_p[s], h);
#pragma unroll
                        for (int e = 0; e < kVEC; ++e) {
                            const int c = 4 * h + e;
                            xm[e] = c ? own_0[s][c - 1] : left[s];
                            xp[e] = c < kW8 - 1 ? own_0[s][c + 1] : right[s];
                        }
                        if constexpr (PLAIN) {
                            const float k = sd.kx[s];
#pragma unroll
                            for (int e = 0; e < kVEC; ++e)
                                o[e] = euler_cell_iso(cen[e], xm[e], xp[e], ym[e], yp[e], zm[e],
                                                      zp[e], k, inc[s][e]);
                        } else {
                            species_core(sd, s, cen, xm, xp, ym, yp, zm, zp, inc[s], cx, src_here,
                                         px, xs + 4 * h, o, cy, cz);
                            held_layers_at(sd, s, xyf[h] | zf, xs + 4 * h, y, q, o);
                        }
                        ST* gp = gst + s * fstride + 4 * h;
                        if (computes && RD_DBG_GLOBAL(sd, gp, kVEC * EB, kSiteStateStore))
                            Store<ST>::store(gp, o);
                    }
                }
#pragma unroll
                for (int s = 0; s < S; ++s)
#pragma unroll
                    for (int e = 0; e < kW8; ++e) own_0[s][e] = own_p[s][e];
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
