// rd_api.cu -- host runtime behind the C ABI declared in include/rd.h.
//
// Owns contexts (device state, scratch, stream, CUDA graphs), batches of
// contexts, tuning and the autotuner.  All arithmetic of the step runs in the
// kernels of rd_k_*.cu and rd_aux.cu; this file only validates, lays out
// memory, builds instance descriptors and enqueues launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <utility>
#include <vector>
#include <string>
#include <thread>

#include "rd.h"
#include "rd_internal.h"
#include "rd_ablation.h"
#include "rd_model_turing.h"
#include "rd_resident.h"
#include "rd_step19.h"

using namespace rdk;

namespace {

thread_local char g_err[512] = "";

// Allocation fault injection (rd_debug_fail_alloc): when armed with k > 0,
// the k-th device or pinned-host allocation from then on fails as if the
// memory were exhausted, and the hook disarms.
std::mutex g_fault_mu;
long long g_fail_alloc = 0;

bool injected_failure() {
    std::lock_guard<std::mutex> lk(g_fault_mu);
    if (g_fail_alloc <= 0) return false;
    return --g_fail_alloc == 0;
}

cudaError_t dev_alloc(void** p, size_t n) {
    if (injected_failure()) { *p = nullptr; return cudaErrorMemoryAllocation; }
    return cudaMalloc(p, n);
}

cudaError_t host_alloc(void** p, size_t n) {
    if (injected_failure()) { *p = nullptr; return cudaErrorMemoryAllocation; }
    return cudaMallocHost(p, n);
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

struct Graph {
    cudaGraphExec_t exec = nullptr;
    int launches = 0;        // kernel launches in the graph (even)
    int tsteps = 0;
    long long key = -1;      // tuning/membership signature it was built for
    void reset() {
        if (exec) cudaGraphExecDestroy(exec);
        exec = nullptr;
        launches = 0;
        key = -1;
    }
};

int num_sms() {
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

int max_smem_optin() {
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (n <= 0) n = 48 * 1024;
    }
    return n;
}

int vec_of(int) { return 4; }
int elem_bytes(int storage) { return storage == RD_STORE_BF16 ? 2 : 4; }

// the stencil of a configuration: 7 (7-point, the default) or 19 (eqs. (3)-(4))
int stencil_of(const rd_config& g) { return g.stencil == 19 ? 19 : 7; }

// models with a Cahn-Hilliard species (species 2)
bool is_ch(int model) { return model == RD_MODEL_CH_FRONT || model == RD_MODEL_CH_TABLE1; }

int species_of(int model) {
    switch (model) {
    case RD_MODEL_DIFFUSION: return 1;
    case RD_MODEL_BRUSSELATOR: case RD_MODEL_TURING: return 2;
    default: return 3;
    }
}

// tile width in cells of every kernel (16 vectors of 4 cells, or 8 of 8)
constexpr int kTileW = 64;

// cells per thread of the one-step 7-point kernel for a tile_q
int vw_of(int tile_q) { return tile_q == 8 ? 8 : 4; }

size_t smem_of(int model, int storage, int T, int ty, int stencil = 7, int tq = kTileQ) {
    const int vw = vw_of(tq);
    if (stencil == 19)
        return is_ch(model) ? smem19_ch_bytes(elem_bytes(storage), ty)
                            : smem19_bytes(species_of(model), elem_bytes(storage), ty);
    switch (model) {
    case RD_MODEL_DIFFUSION: return smem_diffusion(storage, T, ty, vw);
    case RD_MODEL_BRUSSELATOR: return smem_brusselator(storage, T, ty, vw);
    case RD_MODEL_CH_FRONT: return smem_ch_front(storage, T, ty, vw);
    case RD_MODEL_CH_TABLE1: return smem_ch_table1(storage, T, ty, vw);
    case RD_MODEL_AIR: return smem_air(storage, T, ty, vw);
    case RD_MODEL_TURING: return smem_turing(storage, T, ty, vw);
    }
    return 0;
}

// CTA size of a step kernel: the one-step kernel has a thread per tile
// vector; the multi-level kernel (tile vectors + 2 halo) x (rows + 2 L)
int threads_of(int model, int T, int ty, int stencil = 7, int tq = kTileQ) {
    if (stencil == 19) return threads19(ty);
    if (T == 1 && !is_ch(model) && vw_of(tq) == 8) return 8 * ty + 32;   // 8 cells per thread
    // the one-step kernel needs an even tile height (16 ty compute threads,
    // then a whole halo warp); an odd height at one step per launch (the
    // last launch of a call whose tuning steps 2 or 3 per launch) runs the
    // multi-level kernel at T = 1
    if (T == 1 && !is_ch(model) && !(ty & 1)) return kTileQ * ty + 32;
    if (T == 1) return (kTileQ + 2) * (ty + 2);   // one-step Cahn-Hilliard kernel
    const int L = (is_ch(model) ? 2 : 1) * T;
    return (kTileQ + 2) * (ty + 2 * L);
}

cudaError_t launch_model(int model, int storage, int T, const LaunchArgs& a, int grid,
                         size_t smem, cudaStream_t st, int* occ, int stencil = 7) {
    if (stencil == 19) {
        if (T != 1) return cudaErrorInvalidValue;
        if (is_ch(model)) {
            // two launches: mu (pass 1), then the update (pass 2); the CTAs
            // per SM reported are those of pass 2, the larger one
            auto pass = model == RD_MODEL_CH_FRONT ? launch19_ch_front : launch19_ch_table1;
            if (occ) return pass(storage, 2, a, grid, smem, st, occ);
            cudaError_t e = pass(storage, 1, a, grid, smem, st, nullptr);
            if (e != cudaSuccess) return e;
            return pass(storage, 2, a, grid, smem, st, nullptr);
        }
        switch (model) {
        case RD_MODEL_DIFFUSION: return launch19_diffusion(storage, a, grid, smem, st, occ);
        case RD_MODEL_BRUSSELATOR: return launch19_brusselator(storage, a, grid, smem, st, occ);
        case RD_MODEL_AIR: return launch19_air(storage, a, grid, smem, st, occ);
        case RD_MODEL_TURING: return launch19_turing(storage, a, grid, smem, st, occ);
        }
        return cudaErrorInvalidValue;
    }
    switch (model) {
    case RD_MODEL_DIFFUSION: return launch_diffusion(storage, T, a, grid, smem, st, occ);
    case RD_MODEL_BRUSSELATOR: return launch_brusselator(storage, T, a, grid, smem, st, occ);
    case RD_MODEL_CH_FRONT: return launch_ch_front(storage, T, a, grid, smem, st, occ);
    case RD_MODEL_CH_TABLE1: return launch_ch_table1(storage, T, a, grid, smem, st, occ);
    case RD_MODEL_AIR: return launch_air(storage, T, a, grid, smem, st, occ);
    case RD_MODEL_TURING: return launch_turing(storage, T, a, grid, smem, st, occ);
    }
    return cudaErrorInvalidValue;
}

// kernel launches per step of a one-step launch sequence: a 19-point
// Cahn-Hilliard step is two (mu, then the update)
int kernels_per_step(const rd_config& g) { return (stencil_of(g) == 19 && is_ch(g.model)) ? 2 : 1; }

// temporal blocking: up to 3 steps per launch (2 with Cahn-Hilliard); the
// 19-point kernel steps once per launch
int max_tsteps(const rd_config& g) {
    if (stencil_of(g) == 19 || g.wind_kind == RD_WIND_3D) return 1;
    return is_ch(g.model) ? 2 : 3;
}

// CTAs per SM for a variant (cached).
bool plain_problem(const rd_config& g);
// kernel variant of a problem: 1 branch-free, 2 with the 3-D wind, else 0
int variant_code(const rd_config& g) {
    return plain_problem(g) ? 1 : g.wind_kind == RD_WIND_3D ? 2 : 0;
}

int occupancy(int model, int storage, int T, int ty, int regcap = 0, int plain = 0,
              int stencil = 7, int tq = kTileQ) {
    static std::mutex mu;
    static std::map<std::tuple<int, int, int, int, int, int, int, int>, int> cache;
    std::lock_guard<std::mutex> g(mu);
    auto key = std::make_tuple(model, storage, T, ty, regcap, plain, stencil, tq);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    int occ = 0;
    LaunchArgs dummy{};
    dummy.use_one = 1;
    dummy.regcap = regcap;
    // plain: 0 the general variant, 1 the branch-free one, 2 the 3-D wind one
    dummy.plain = plain == 1;
    dummy.wind3 = plain == 2;
    dummy.ty = ty;
    dummy.vw = vw_of(tq);
    const size_t smem = smem_of(model, storage, T, ty, stencil, tq);
    if (launch_model(model, storage, T, dummy, 0, smem, nullptr, &occ, stencil) != cudaSuccess)
        occ = 0;
    cudaGetLastError();
    cache[key] = occ;
    return occ;
}

}  // namespace

// ----------------------------------------------------------------- context
struct rd_ctx {
    rd_config cfg{};
    int S = 0, vec = 4, ebytes = 4;
    int pitch = 0;                 // elements per row
    long long plane = 0;           // elements per plane
    size_t field_bytes = 0;        // one species, one level (256-aligned)
    size_t state_bytes = 0, scratch_bytes = 0;
    char* state = nullptr;
    char* scratch = nullptr;
    bool own_mem = false;
    // scratch carve-up
    float* staging = nullptr;      // dense float field for I/O
    double* partials = nullptr;    // reduction partials
    double* result = nullptr;      // reduction result (3 doubles)
    InstDesc* desc_dev = nullptr;  // this context's descriptor
    float* courant = nullptr;      // u(z) dt / h per plane
    float* mu = nullptr;           // 19-point Cahn-Hilliard: the mu field
    long long* stepn = nullptr;    // 3-D wind: step index per time level
    rdk::ResidentBar* bar = nullptr;   // the resident kernel's grid barrier
    int res_phantom = 0;           // rd_debug_resident_stall, next launch only
    rdk::ResidentPlan res_plan{};  // the resident kernel's plan (rd_set_kernel)
    int res_force[3] = {0, 0, 0};  // rd_set_resident_plan: K, ty, tz (0 = planned)
    bool stepn_dirty = true;       // the host's step count is not on the device
    int cur = 0;                   // current time level
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaStream_t capture_stream = nullptr;
    rd_tuning tun{};
    int kernel = RD_KERNEL_MARCH;  // step kernel (rd_set_kernel)
    bool desc_dirty = true;
    InstDesc desc{};
    Graph graph;
    int64_t steps = 0;
    int64_t launches = 0;
    rd_batch* batch = nullptr;
    char err[512] = "";
};

struct rd_batch {
    int model = 0, storage = 0;
    int stencil = 7;                 // of the members (set by the first one)
    std::vector<rd_ctx*> members;
    InstDesc* desc_dev = nullptr;
    size_t desc_cap = 0;
    unsigned long long* work = nullptr;  // work-item counter, after the descriptors
    InstDesc* desc_host = nullptr;   // pinned
    cudaEvent_t upload_done = nullptr;
    cudaStream_t stream = nullptr;       // where work is enqueued
    cudaStream_t own_stream = nullptr;   // created by the batch
    cudaStream_t capture_stream = nullptr;
    rd_tuning tun{};
    bool tun_set = false;
    Graph graph;
    long long members_version = 0;
    int64_t launches = 0;
};

namespace {

rd_status fail(rd_ctx* c, rd_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    std::snprintf(g_err, sizeof(g_err), "%s", buf);
    if (c) std::snprintf(c->err, sizeof(c->err), "%s", buf);
    return st;
}

rd_status cuda_fail(rd_ctx* c, cudaError_t e, const char* what) {
    return fail(c, RD_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define RD_CUDA(c, call)                                   \
    do {                                                   \
        cudaError_t _e = (call);                           \
        if (_e != cudaSuccess) return cuda_fail(c, _e, #call); \
    } while (0)

int periodic_axis(const rd_config& c, int s, int a) {
    return c.bc[s][2 * a] == RD_BC_PERIODIC;
}

rd_status validate(const rd_config* c) {
    if (!c) return fail(nullptr, RD_EINVAL, "null config");
    if (c->nx < 2 || c->ny < 2 || c->nz < 2)
        return fail(nullptr, RD_EINVAL, "grid must be at least 2 cells per axis");
    if ((long long)c->nx * c->ny * c->nz > (1LL << 34))
        return fail(nullptr, RD_EINVAL, "grid too large");
    if (!(c->h > 0) || !(c->dt > 0)) return fail(nullptr, RD_EINVAL, "h and dt must be > 0");
    int want = -1;
    switch (c->model) {
    case RD_MODEL_DIFFUSION: want = 1; break;
    case RD_MODEL_BRUSSELATOR: want = 2; break;
    case RD_MODEL_CH_FRONT: want = 3; break;
    case RD_MODEL_AIR: want = 3; break;
    case RD_MODEL_TURING: want = 2; break;
    case RD_MODEL_CH_TABLE1: want = 3; break;
    default: return fail(nullptr, RD_EINVAL, "unknown model %d", c->model);
    }
    if (c->nspecies != want) {
        if (c->model == RD_MODEL_DIFFUSION && c->nspecies >= 1 && c->nspecies <= RD_MAX_SPECIES)
            return fail(nullptr, RD_EUNSUPPORTED,
                        "the diffusion kernels of this build step one species");
        return fail(nullptr, RD_EINVAL, "model %d needs %d species", c->model, want);
    }
    if (c->storage != RD_STORE_F32 && c->storage != RD_STORE_BF16)
        return fail(nullptr, RD_EINVAL, "unknown storage %d", c->storage);
    for (int s = 0; s < c->nspecies; ++s) {
        for (int f = 0; f < 6; ++f)
            if (c->bc[s][f] < RD_BC_NEUMANN || c->bc[s][f] > RD_BC_DIRICHLET)
                return fail(nullptr, RD_EINVAL, "bad boundary kind");
        for (int a = 0; a < 3; ++a) {
            const bool lo = c->bc[s][2 * a] == RD_BC_PERIODIC;
            const bool hi = c->bc[s][2 * a + 1] == RD_BC_PERIODIC;
            if (lo != hi) return fail(nullptr, RD_EINVAL, "periodic faces must come in pairs");
            if (lo != (c->bc[0][2 * a] == RD_BC_PERIODIC))
                return fail(nullptr, RD_EINVAL, "periodicity must be the same for all species");
            for (int d = 0; d < 3; ++d)
                if (!(c->D[s][d] >= 0) || !std::isfinite(c->D[s][d]))
                    return fail(nullptr, RD_EINVAL, "diffusivities must be finite and >= 0");
        }
    }
    if (is_ch(c->model)) {
        for (int f = 0; f < 6; ++f)
            if (c->bc[2][f] == RD_BC_DIRICHLET)
                return fail(nullptr, RD_EUNSUPPORTED, "no held layer on the Cahn-Hilliard species");
        if (c->D[2][0] != 0 || c->D[2][1] != 0 || c->D[2][2] != 0)
            return fail(nullptr, RD_EUNSUPPORTED, "the Cahn-Hilliard species has no Fickian term");
        // the front problem (Section 4.1, Table 1) has no wind, and the
        // Cahn-Hilliard species moves only by its chemical potential
        if (c->wind_kind != RD_WIND_NONE)
            return fail(nullptr, RD_EUNSUPPORTED, "the front model has no advection");
        if (c->src_species == 2)
            return fail(nullptr, RD_EUNSUPPORTED, "no point source on the Cahn-Hilliard species");
    }
    if (c->stencil != 0 && c->stencil != 7 && c->stencil != 19)
        return fail(nullptr, RD_EINVAL, "stencil must be 7 or 19");
    if (c->stencil == 19) {
        for (int s = 0; s < c->nspecies; ++s)
            if (c->D[s][1] != c->D[s][0] || c->D[s][2] != c->D[s][0])
                return fail(nullptr, RD_EINVAL,
                            "the 19-point Laplacian takes one diffusivity per species");
    }
    if (c->wind_kind < RD_WIND_NONE || c->wind_kind > RD_WIND_3D)
        return fail(nullptr, RD_EINVAL, "unknown wind kind");
    if (c->wind_kind != RD_WIND_NONE && c->wind_kind != RD_WIND_3D && !std::isfinite(c->wind_u0))
        return fail(nullptr, RD_EINVAL, "wind speed must be finite");
    if (c->wind_kind == RD_WIND_3D) {
        for (int a = 0; a < 3; ++a)
            if (!std::isfinite(c->wind_vel[a]))
                return fail(nullptr, RD_EINVAL, "wind speed must be finite");
        if (!(c->wind_tau > 0) || !std::isfinite(c->wind_tau))
            return fail(nullptr, RD_EINVAL, "wind_tau must be finite and > 0");
    }
    if (c->src_species >= 0) {
        if (c->src_species >= c->nspecies || c->src_x < 0 || c->src_x >= c->nx || c->src_y < 0 ||
            c->src_y >= c->ny || c->src_z < 0 || c->src_z >= c->nz)
            return fail(nullptr, RD_EINVAL, "source outside the grid");
    }
    if (!(c->flags & RD_FLAG_FORCE)) {
        double umax = 0.0;
        if (c->wind_kind == RD_WIND_LOG) umax = std::fabs(c->wind_u0) * std::log1p((double)c->nz - 1) / std::log1p((double)c->nz);
        if (c->wind_kind == RD_WIND_CONST) umax = std::fabs(c->wind_u0);
        // upwind along every axis: the centre coefficient loses dt |u_a| / h
        // per axis
        if (c->wind_kind == RD_WIND_3D)
            umax = std::fabs(c->wind_vel[0]) + std::fabs(c->wind_vel[1]) + std::fabs(c->wind_vel[2]);
        // the centre coefficient of the update stays >= 0: it is
        // 1 - dt (w D / h^2 + |u| / h), w = 2 per axis (7-point) or
        // 24 / 6 = 4 (19-point)
        const bool s19 = stencil_of(*c) == 19;
        for (int s = 0; s < c->nspecies; ++s) {
            const double wd = s19 ? 4.0 * c->D[s][0]
                                  : 2.0 * (c->D[s][0] + c->D[s][1] + c->D[s][2]);
            const double g = c->dt * (wd / (c->h * c->h) + umax / c->h);
            if (g > 1.0 + 1e-12)
                return fail(nullptr, RD_EUNSTABLE,
                            "dt too large for species %d: dt*(%s/h^2+|u|/h) = %g > 1", s,
                            s19 ? "4*D" : "2*sum(D)", g);
        }
        if (is_ch(c->model)) {
            // the Cahn-Hilliard term's largest decay rate: dt Mc L (K L + gb)
            // <= 2, L the largest eigenvalue of -Laplacian (12 / h^2 for the
            // 7-point stencil, 16 / (3 h^2) for the 19-point one), Mc the
            // mobility, K the gradient coefficient and gb a bound of -g'(c)
            // over the range of c (front: g = f', f'' >= -1, bounded by 2 as
            // a margin; Table 1 row 3: g = eps c - gamma c^3, -g' <= 3 gamma
            // - eps for |c| <= 1)
            const double L = (stencil_of(*c) == 19 ? 16.0 / 3.0 : 12.0) / (c->h * c->h);
            const bool front = c->model == RD_MODEL_CH_FRONT;
            const double mob = front ? c->params[1] : c->params[2];
            const double kap = front ? c->params[2] : c->params[5];
            const double gb = front ? 2.0 : std::max(0.0, 3.0 * c->params[4] - c->params[3]);
            const double g = c->dt * std::fabs(mob) * L * (std::fabs(kap) * L + gb);
            if (g > 2.0 + 1e-12)
                return fail(nullptr, RD_EUNSTABLE, "dt too large for the Cahn-Hilliard term (%g > 2)", g);
        }
    }
    return RD_OK;
}

// the mu field of a 19-point Cahn-Hilliard context: one float plane stack
// with the state's element pitch
size_t mu_bytes(const rd_ctx* c) {
    if (kernels_per_step(c->cfg) != 2) return 0;
    return align_up((size_t)c->plane * c->cfg.nz * sizeof(float), 256);
}

void layout(rd_ctx* c) {
    const rd_config& g = c->cfg;
    c->S = g.nspecies;
    c->vec = vec_of(g.storage);
    c->ebytes = elem_bytes(g.storage);
    // rows padded to 128 bytes so 16-byte vectors never cross a row end
    const int row_align = 128 / c->ebytes;
    c->pitch = (int)align_up((size_t)g.nx, (size_t)row_align);
    c->plane = (long long)c->pitch * g.ny;
    c->field_bytes = align_up((size_t)c->plane * g.nz * c->ebytes, 256);
    c->state_bytes = c->field_bytes * 2 * c->S;
    const size_t dense = align_up((size_t)g.nx * g.ny * g.nz * sizeof(float), 256);
    const size_t part = align_up((size_t)reduce_blocks() * 3 * sizeof(double), 256);
    const size_t res = 256;
    const size_t desc = align_up(sizeof(InstDesc), 256);
    const size_t cour = align_up((size_t)g.nz * sizeof(float), 256);
    c->scratch_bytes = dense + part + res + desc + cour + 256 + 256 + mu_bytes(c);
}

void carve(rd_ctx* c) {
    const rd_config& g = c->cfg;
    char* p = c->scratch;
    c->staging = reinterpret_cast<float*>(p);
    p += align_up((size_t)g.nx * g.ny * g.nz * sizeof(float), 256);
    c->partials = reinterpret_cast<double*>(p);
    p += align_up((size_t)reduce_blocks() * 3 * sizeof(double), 256);
    c->result = reinterpret_cast<double*>(p);
    p += 256;
    c->desc_dev = reinterpret_cast<InstDesc*>(p);
    p += align_up(sizeof(InstDesc), 256);
    c->courant = reinterpret_cast<float*>(p);
    p += align_up((size_t)g.nz * sizeof(float), 256);
    c->stepn = g.wind_kind == RD_WIND_3D ? reinterpret_cast<long long*>(p) : nullptr;
    p += 256;
    c->bar = reinterpret_cast<rdk::ResidentBar*>(p);
    p += 256;
    c->mu = mu_bytes(c) ? reinterpret_cast<float*>(p) : nullptr;
}

char* field_ptr(rd_ctx* c, int level, int s) {
    return c->state + ((size_t)level * c->S + s) * c->field_bytes;
}


int tiles(int n, int t) { return (n + t - 1) / t; }

// z chunk so one launch has about ``waves`` work items per resident CTA
int auto_zchunk(const rd_config& g, const rd_tuning& t, int occ, int waves) {
    const long long cols = (long long)tiles(g.nx, kTileW) * tiles(g.ny, t.tile_y);
    const long long slots = (long long)std::max(occ, 1) * num_sms() * waves;
    long long nzc = std::max<long long>(1, (slots + cols - 1) / cols);
    int zc = (int)std::max<long long>(1, (g.nz + nzc - 1) / nzc);
    const int L = (is_ch(g.model) ? 2 : 1) * t.tsteps;
    zc = std::max(zc, std::min(g.nz, 4 * L));
    return zc;
}

rd_status check_tuning(const rd_config& g, const rd_tuning& t) {
    if (t.tsteps < 1 || t.tsteps > max_tsteps(g))
        return fail(nullptr, RD_EINVAL, "tsteps out of range");
    if (t.tile_q != kTileQ && t.tile_q != 8)
        return fail(nullptr, RD_EINVAL, "tile_q must be %d or 8 in this build", kTileQ);
    if (t.tile_q == 8) {
        // 8 cells per thread: the one-step 7-point kernel; its compute
        // threads (8 per row) fill whole warps, as its shuffles need
        if (t.tsteps != 1 || is_ch(g.model) || stencil_of(g) != 7)
            return fail(nullptr, RD_EINVAL,
                        "tile_q 8 is the one-step 7-point kernel without Cahn-Hilliard");
        if (t.tile_y % 4 != 0 || t.tile_y > 40)
            return fail(nullptr, RD_EINVAL, "tile_q 8 needs tile_y a multiple of 4, at most 40");
    }
    if (t.tile_y < 1 || t.zchunk < 1) return fail(nullptr, RD_EINVAL, "tile out of range");
    if (t.regcap != 0 && t.regcap != 1) return fail(nullptr, RD_EINVAL, "regcap must be 0 or 1");
    if (t.tsteps == 1 && (!is_ch(g.model) || stencil_of(g) == 19) && (t.tile_y & 1))
        return fail(nullptr, RD_EINVAL, "tile_y must be even for one step per launch");
    if (threads_of(g.model, t.tsteps, t.tile_y, stencil_of(g), t.tile_q) > kMaxThreads)
        return fail(nullptr, RD_EINVAL, "tile_y %d too tall for %d steps per launch", t.tile_y,
                    t.tsteps);
    const size_t sm = smem_of(g.model, g.storage, t.tsteps, t.tile_y, stencil_of(g), t.tile_q);
    if (sm + sizeof(InstDesc) + 64 > (size_t)max_smem_optin())
        return fail(nullptr, RD_EINVAL, "tile needs %zu bytes of shared memory", sm);
    return RD_OK;
}

// z-chunk for problems of (x-y tile columns, nz) sharing ``slots`` resident
// CTAs: the fewest waves of work items times the planes an item marches
// (its chunk plus about three planes of pipeline start), ties to the
// longer chunk.  A wave that is barely filled costs as much as a full one.
int wave_zchunk(const std::vector<std::pair<long long, int>>& cols_nz, long long slots) {
    int maxnz = 1;
    for (auto& p : cols_nz) maxnz = std::max(maxnz, p.second);
    int best = maxnz;
    double best_cost = -1.0;
    for (int zc : {8, 12, 16, 20, 24, 32, 40, 48, 64, 86, 96, 128, 192, 256, 384, 512}) {
        const int z = std::min(zc, maxnz);
        long long items = 0;
        for (auto& p : cols_nz) items += p.first * tiles(p.second, std::min(z, p.second));
        const long long waves = (items + slots - 1) / std::max<long long>(slots, 1);
        const double cost = (double)waves * (z + 3);
        if (best_cost < 0 || cost < best_cost || (cost == best_cost && z > best)) {
            best_cost = cost;
            best = z;
        }
        if (z == maxnz) break;
    }
    return best;
}

// Default tile height of the one-step kernels: 14 rows (12 for the front
// model, whose kernel keeps more planes) fit two CTAs per SM.
int default_tile_y(int model) { return is_ch(model) ? 12 : 14; }

rd_tuning default_tuning(const rd_config& g) {
    rd_tuning t{};
    t.tsteps = 1;
    t.tile_q = kTileQ;
    t.tile_y = default_tile_y(g.model);
    t.graph = 1;
    const int occ = occupancy(g.model, g.storage, t.tsteps, t.tile_y, 0, variant_code(g),
                              stencil_of(g));
    const long long cols = (long long)tiles(g.nx, kTileW) * tiles(g.ny, t.tile_y);
    t.zchunk = wave_zchunk({{cols, g.nz}}, (long long)std::max(occ, 1) * num_sms());
    return t;
}

void fill_desc(rd_ctx* c, InstDesc& d, const rd_tuning& t) {
    const rd_config& g = c->cfg;
    std::memset(&d, 0, sizeof(d));
    for (int l = 0; l < 2; ++l)
        for (int s = 0; s < c->S; ++s) d.base[l][s] = field_ptr(c, l, s);
    d.nx = g.nx; d.ny = g.ny; d.nz = g.nz;
    d.pitch = c->pitch;
    d.plane = c->plane;
    d.par = 0;
    d.per_x = periodic_axis(g, 0, 0);
    d.per_y = periodic_axis(g, 0, 1);
    d.per_z = periodic_axis(g, 0, 2);
    const double ih2 = 1.0 / (g.h * g.h);
    for (int s = 0; s < c->S; ++s) {
        unsigned m = 0;
        for (int f = 0; f < 6; ++f) {
            if (g.bc[s][f] == RD_BC_DIRICHLET) m |= 1u << f;
            d.held_val[s][f] = (float)g.bc_value[s][f];
        }
        d.held_mask[s] = m;
        d.kx[s] = (float)(g.D[s][0] * g.dt * ih2);
        d.ky[s] = (float)(g.D[s][1] * g.dt * ih2);
        d.kz[s] = (float)(g.D[s][2] * g.dt * ih2);
    }
    d.dt = (float)g.dt;
    switch (g.model) {
    case RD_MODEL_BRUSSELATOR:
        d.p[0] = (float)g.params[0];
        d.p[1] = (float)(g.params[1] + 1.0);
        d.p[2] = (float)g.params[1];
        break;
    case RD_MODEL_CH_FRONT:
        d.p[0] = (float)(g.dt * g.params[0]);
        d.p[1] = (float)(g.dt * g.params[1] * ih2);
        d.p[2] = (float)(g.params[2] * ih2);
        break;
    case RD_MODEL_AIR:
        d.p[0] = (float)g.params[0];
        d.p[1] = (float)g.params[1];
        break;
    case RD_MODEL_CH_TABLE1:
        d.p[0] = (float)(g.dt * g.params[0]);
        d.p[1] = (float)(-g.dt * g.params[2] * ih2);
        d.p[2] = (float)(-g.params[5] * ih2);
        d.p[3] = (float)(g.dt * g.params[1]);
        d.p[4] = (float)g.params[3];
        d.p[5] = (float)g.params[4];
        break;
    case RD_MODEL_TURING:
        d.p[0] = (float)g.params[0];
        d.p[1] = (float)g.params[1];
        d.p[2] = (float)g.params[2];
        break;
    default: break;
    }
    d.courant = g.wind_kind != RD_WIND_NONE ? c->courant : nullptr;
    d.mu = c->mu;
    d.mem_lo[0] = c->state;
    d.mem_hi[0] = c->state + c->state_bytes;
    d.mem_lo[1] = c->scratch;
    d.mem_hi[1] = c->scratch + c->scratch_bytes;
    d.stepn = c->stepn;
    if (g.wind_kind == RD_WIND_3D) {
        d.cy = (float)(g.wind_vel[1] * g.dt / g.h);
        d.wz_amp = g.wind_vel[2] * g.dt / g.h;
        d.wz_omega = g.dt / g.wind_tau;
    }
    d.src_s = g.src_species >= 0 ? g.src_species : -1;
    d.src_x = g.src_x; d.src_y = g.src_y; d.src_z = g.src_z;
    d.src_amt = (float)(g.src_rate * g.dt);
    d.ntx = tiles(g.nx, kTileW);
    d.wrap_elems = d.per_x && (g.nx % 4 != 0);
    d.nty = tiles(g.ny, t.tile_y);
    d.zchunk = std::max(1, std::min(t.zchunk, g.nz));
    d.nzc = tiles(g.nz, d.zchunk);
    d.item_begin = 0;
}

long long items_of(const InstDesc& d) { return (long long)d.ntx * d.nty * d.nzc; }

// No point source or wind, every species isotropic and, except for the
// 7-point Cahn-Hilliard models (whose one-step kernel applies held layers on
// this path too), no held layer: the one-step kernels' branch-free update
// applies.
bool plain_problem(const rd_config& g) {
    if (g.wind_kind != RD_WIND_NONE || g.src_species >= 0) return false;
    // the 7-point Cahn-Hilliard kernel's plain path still applies held layers
    const bool held_ok = is_ch(g.model) && stencil_of(g) == 7;
    for (int s = 0; s < g.nspecies; ++s) {
        for (int f = 0; f < 6; ++f)
            if (g.bc[s][f] == RD_BC_DIRICHLET && !held_ok) return false;
        if (g.D[s][0] != g.D[s][1] || g.D[s][0] != g.D[s][2]) return false;
    }
    return true;
}

rd_status upload_desc(rd_ctx* c) {
    if (!c->desc_dirty) return RD_OK;
    fill_desc(c, c->desc, c->tun);
    RD_CUDA(c, cudaMemcpyAsync(c->desc_dev, &c->desc, sizeof(InstDesc), cudaMemcpyHostToDevice,
                               c->stream));
    RD_CUDA(c, cudaStreamSynchronize(c->stream));
    c->desc_dirty = false;
    return RD_OK;
}

rd_status write_courant(rd_ctx* c) {
    const rd_config& g = c->cfg;
    if (g.wind_kind == RD_WIND_NONE) return RD_OK;
    std::vector<float> cz(g.nz);
    for (int z = 0; z < g.nz; ++z) {
        double u = 0.0;
        if (g.wind_kind == RD_WIND_LOG) u = g.wind_u0 * std::log1p((double)z) / std::log1p((double)g.nz);
        else if (g.wind_kind == RD_WIND_3D) u = g.wind_vel[0];
        else u = g.wind_u0;
        cz[z] = (float)(u * g.dt / g.h);
    }
    RD_CUDA(c, cudaMemcpy(c->courant, cz.data(), sizeof(float) * g.nz, cudaMemcpyHostToDevice));
    return RD_OK;
}

rd_status finish_setup(rd_ctx* c) {
    carve(c);
    RD_CUDA(c, cudaMemsetAsync(c->state, 0, c->state_bytes, c->stream));
    if (c->stepn) RD_CUDA(c, cudaMemsetAsync(c->stepn, 0, 2 * sizeof(long long), c->stream));
    RD_CUDA(c, cudaMemsetAsync(c->bar, 0, sizeof(rdk::ResidentBar), c->stream));
    RD_CUDA(c, cudaStreamSynchronize(c->stream));
    rd_status st = write_courant(c);
    if (st != RD_OK) return st;
    c->desc_dirty = true;
    return upload_desc(c);
}

// One fused launch advancing T steps, reading level ``c->cur``.
rd_status launch_ctx(rd_ctx* c, int T, int parity, cudaStream_t st) {
    LaunchArgs a{};
    a.desc = c->desc_dev;
    a.ninst = 1;
    a.parity = parity;
    a.nitems = items_of(c->desc);
    a.use_one = 1;
    a.one = c->desc;
    a.regcap = c->tun.regcap;
    a.plain = plain_problem(c->cfg);
    a.wind3 = c->cfg.wind_kind == RD_WIND_3D;
    a.vw = vw_of(c->tun.tile_q);
    a.ty = c->tun.tile_y;
    if (c->kernel == RD_KERNEL_RESIDENT) {
        // T steps in one cooperative launch (zeroed barrier count and word)
        RD_CUDA(c, cudaMemsetAsync(c->bar, 0, 2 * sizeof(unsigned), st));
        const bool barriers = T > c->res_plan.K;
        const unsigned phantom = barriers ? (unsigned)c->res_phantom : 0u;
        if (barriers) c->res_phantom = 0;
        cudaError_t e = launch_resident(c->cfg.model, c->cfg.storage, a, c->res_plan, T, c->bar,
                                        phantom, st);
        if (e != cudaSuccess) return cuda_fail(c, e, "resident kernel launch");
        c->launches++;
        return RD_OK;
    }
    if (c->kernel != RD_KERNEL_MARCH) {   // the paper's designs, one step each
        if (T != 1) return fail(c, RD_EINVAL, "the ablation kernels step once per launch");
        cudaError_t e = launch_ablation(c->kernel, c->cfg.model, a, st);
        if (e != cudaSuccess) return cuda_fail(c, e, "ablation kernel launch");
        c->launches++;
        return RD_OK;
    }
    const int sten = stencil_of(c->cfg);
    const size_t sm = smem_of(c->cfg.model, c->cfg.storage, T, a.ty, sten, c->tun.tile_q);
    const int occ = std::max(
        1, occupancy(c->cfg.model, c->cfg.storage, T, a.ty, a.regcap,
                     a.plain ? 1 : a.wind3 ? 2 : 0, sten, c->tun.tile_q));
    const long long grid = std::min<long long>(a.nitems, (long long)occ * num_sms());
    cudaError_t e =
        launch_model(c->cfg.model, c->cfg.storage, T, a, (int)grid, sm, st, nullptr, sten);
    if (e != cudaSuccess) return cuda_fail(c, e, "step kernel launch");
    c->launches += kernels_per_step(c->cfg);
    return RD_OK;
}

long long ctx_graph_key(const rd_ctx* c) {
    const rd_tuning& t = c->tun;
    return ((((((long long)t.tsteps * 64 + t.tile_q) * 64 + t.tile_y) * 100000 + t.zchunk) * 2 +
             t.regcap) * 4 + c->kernel);
}

constexpr int kGraphLaunches = 16;

rd_status build_ctx_graph(rd_ctx* c) {
    const long long key = ctx_graph_key(c);
    if (c->graph.exec && c->graph.key == key) return RD_OK;
    c->graph.reset();
    if (!c->capture_stream)
        RD_CUDA(c, cudaStreamCreateWithFlags(&c->capture_stream, cudaStreamNonBlocking));
    RD_CUDA(c, cudaStreamBeginCapture(c->capture_stream, cudaStreamCaptureModeThreadLocal));
    const int64_t before = c->launches;
    rd_status st = RD_OK;
    for (int i = 0; i < kGraphLaunches && st == RD_OK; ++i)
        st = launch_ctx(c, c->tun.tsteps, i & 1, c->capture_stream);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(c->capture_stream, &g);
    if (st != RD_OK) { if (g) cudaGraphDestroy(g); return st; }
    if (e != cudaSuccess) return cuda_fail(c, e, "graph capture");
    e = cudaGraphInstantiate(&c->graph.exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(c, e, "graph instantiate");
    c->graph.launches = (int)(c->launches - before);   // kernels in the graph
    c->launches = before;                               // captured, not run
    c->graph.tsteps = c->tun.tsteps;
    c->graph.key = key;
    return RD_OK;
}

// Put the host's step count on the device as the step index of the current
// level (3-D wind), after creation or rd_set_step_count.  The copy is from
// pageable memory, so the value is taken before the call returns.
rd_status sync_stepn(rd_ctx* c, cudaStream_t st) {
    if (!c->stepn || !c->stepn_dirty) return RD_OK;
    const long long n = c->steps;
    RD_CUDA(c, cudaMemcpyAsync(c->stepn + c->cur, &n, sizeof(n), cudaMemcpyHostToDevice, st));
    RD_CUDA(c, cudaStreamSynchronize(st));
    c->stepn_dirty = false;
    return RD_OK;
}

rd_status step_ctx(rd_ctx* c, int64_t n) {
    rd_status st = upload_desc(c);
    if (st != RD_OK) return st;
    if ((st = sync_stepn(c, c->stream)) != RD_OK) return st;
    if (c->kernel == RD_KERNEL_RESIDENT) {   // many steps per launch, no graph
        for (int64_t left = n; left > 0;) {
            const int k = (int)std::min<int64_t>(left, rdk::kResidentMaxSteps);
            if ((st = launch_ctx(c, k, c->cur, c->stream)) != RD_OK) return st;
            // each round of K steps is one transition between the levels
            const int rounds = (k + c->res_plan.K - 1) / c->res_plan.K;
            c->cur ^= rounds & 1;
            left -= k;
        }
        c->steps += n;
        return RD_OK;
    }
    const int T = c->tun.tsteps;
    int64_t full = n / T;
    const int rem = (int)(n % T);
    if (c->tun.graph && full >= kGraphLaunches) {
        st = build_ctx_graph(c);
        if (st != RD_OK) return st;
        if (c->cur == 1) {   // the graph starts from level 0
            if ((st = launch_ctx(c, T, 1, c->stream)) != RD_OK) return st;
            c->cur = 0;
            --full;
        }
        while (full >= kGraphLaunches) {
            cudaError_t e = cudaGraphLaunch(c->graph.exec, c->stream);
            if (e != cudaSuccess) return cuda_fail(c, e, "graph launch");
            c->launches += c->graph.launches;
            full -= kGraphLaunches;
        }
    }
    for (int64_t i = 0; i < full; ++i) {
        if ((st = launch_ctx(c, T, c->cur, c->stream)) != RD_OK) return st;
        c->cur ^= 1;
    }
    if (rem) {
        if ((st = launch_ctx(c, rem, c->cur, c->stream)) != RD_OK) return st;
        c->cur ^= 1;
    }
    c->steps += n;
    return RD_OK;
}

// Work of a batch member may still be queued on the batch's stream.
void drain_batch(rd_ctx* c) {
    if (c->batch) cudaStreamSynchronize(c->batch->stream);
}

bool is_device_ptr(const void* p) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

std::mutex g_tune_mu;
std::map<std::string, rd_tuning> g_tune_cache;
bool g_tune_file_loaded = false;

std::string tune_key(const rd_config& g) {
    char buf[256];
    std::snprintf(buf, sizeof(buf), "m%d_s%d_%dx%dx%d_p%d%d%d_w%d_sm%d%s", g.model, g.storage,
                  g.nx, g.ny, g.nz, periodic_axis(g, 0, 0), periodic_axis(g, 0, 1),
                  periodic_axis(g, 0, 2), g.wind_kind != RD_WIND_NONE, num_sms(),
                  stencil_of(g) == 19 ? "_st19" : "");
    return buf;
}

void load_tune_file() {
    if (g_tune_file_loaded) return;
    g_tune_file_loaded = true;
    const char* path = std::getenv("RD_AUTOTUNE_CACHE");
    if (!path) return;
    FILE* f = std::fopen(path, "r");
    if (!f) return;
    char line[512];
    while (std::fgets(line, sizeof(line), f)) {
        char key[256];
        rd_tuning t{};
        if (std::sscanf(line,
                        " {\"key\": \"%255[^\"]\", \"tsteps\": %d, \"tile_q\": %d, \"tile_y\": %d, "
                        "\"zchunk\": %d, \"graph\": %d, \"regcap\": %d",
                        key, &t.tsteps, &t.tile_q, &t.tile_y, &t.zchunk, &t.graph, &t.regcap) == 7)
            g_tune_cache[key] = t;
    }
    std::fclose(f);
}

void save_tune(const std::string& key, const rd_tuning& t, double gcups) {
    const char* path = std::getenv("RD_AUTOTUNE_CACHE");
    if (!path) return;
    FILE* f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f,
                 "{\"key\": \"%s\", \"tsteps\": %d, \"tile_q\": %d, \"tile_y\": %d, \"zchunk\": %d, "
                 "\"graph\": %d, \"regcap\": %d, \"gcups\": %.3f}\n",
                 key.c_str(), t.tsteps, t.tile_q, t.tile_y, t.zchunk, t.graph, t.regcap, gcups);
    std::fclose(f);
}

}  // namespace

// ================================================================ C ABI
extern "C" {

rd_status rd_config_init(rd_config* cfg) {
    if (!cfg) return RD_EINVAL;
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->h = 1.0;
    cfg->src_species = -1;
    return RD_OK;
}

rd_status rd_query_sizes(const rd_config* cfg, size_t* state_bytes, size_t* scratch_bytes) {
    rd_status st = validate(cfg);
    if (st != RD_OK) return st;
    rd_ctx tmp;
    tmp.cfg = *cfg;
    layout(&tmp);
    if (state_bytes) *state_bytes = tmp.state_bytes;
    if (scratch_bytes) *scratch_bytes = tmp.scratch_bytes;
    return RD_OK;
}

rd_status rd_create(const rd_config* cfg, rd_ctx** out) {
    if (!out) return fail(nullptr, RD_EINVAL, "null output pointer");
    *out = nullptr;
    rd_status st = validate(cfg);
    if (st != RD_OK) return st;
    rd_ctx* c = new (std::nothrow) rd_ctx();
    if (!c) return fail(nullptr, RD_ENOMEM, "host allocation failed");
    c->cfg = *cfg;
    layout(c);
    cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) { delete c; return cuda_fail(nullptr, e, "cudaStreamCreate"); }
    c->own_stream = true;
    c->tun = default_tuning(c->cfg);
    if (!(cfg->flags & RD_FLAG_NO_ALLOC)) {
        // owned from the first allocation on, so rd_destroy frees whatever
        // was obtained when a later one fails
        c->own_mem = true;
        e = dev_alloc(reinterpret_cast<void**>(&c->state), c->state_bytes);
        if (e == cudaSuccess) e = dev_alloc(reinterpret_cast<void**>(&c->scratch), c->scratch_bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            const size_t sb = c->state_bytes, xb = c->scratch_bytes;
            rd_destroy(c);
            return fail(nullptr, RD_ENOMEM, "cudaMalloc of %zu + %zu bytes failed", sb, xb);
        }
        st = finish_setup(c);
        if (st != RD_OK) { rd_destroy(c); return st; }
    }
    *out = c;
    return RD_OK;
}

rd_status rd_attach(rd_ctx* c, void* state, void* scratch) {
    if (!c || !state || !scratch) return fail(c, RD_EINVAL, "null argument");
    if (!(c->cfg.flags & RD_FLAG_NO_ALLOC) || c->state)
        return fail(c, RD_EINVAL, "context already has memory");
    if ((reinterpret_cast<uintptr_t>(state) | reinterpret_cast<uintptr_t>(scratch)) & 255)
        return fail(c, RD_EINVAL, "attached memory must be 256-byte aligned");
    c->state = static_cast<char*>(state);
    c->scratch = static_cast<char*>(scratch);
    c->own_mem = false;
    return finish_setup(c);
}

rd_status rd_destroy(rd_ctx* c) {
    if (!c) return RD_EINVAL;
    if (c->batch) rd_batch_remove(c->batch, c);
    if (c->stream) cudaStreamSynchronize(c->stream);
    c->graph.reset();
    if (c->own_mem) {
        cudaFree(c->state);
        cudaFree(c->scratch);
    }
    if (c->capture_stream) cudaStreamDestroy(c->capture_stream);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
    return RD_OK;
}

rd_status rd_set_stream(rd_ctx* c, void* stream) {
    if (!c) return RD_EINVAL;
    if (c->stream) cudaStreamSynchronize(c->stream);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    c->stream = static_cast<cudaStream_t>(stream);
    c->own_stream = false;
    return RD_OK;
}

rd_status rd_set_field(rd_ctx* c, int s, const float* src, size_t count) {
    if (!c || !src) return fail(c, RD_EINVAL, "null argument");
    if (!c->state) return fail(c, RD_EINVAL, "no memory attached");
    if (s < 0 || s >= c->S) return fail(c, RD_EINVAL, "species %d out of range", s);
    drain_batch(c);
    const rd_config& g = c->cfg;
    const size_t n = (size_t)g.nx * g.ny * g.nz;
    if (count != n) return fail(c, RD_EINVAL, "count %zu != nx*ny*nz = %zu", count, n);
    const bool dev = is_device_ptr(src);
    RD_CUDA(c, cudaMemcpyAsync(c->staging, src, n * sizeof(float),
                               dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
    float hv[6];
    unsigned m = 0;
    for (int f = 0; f < 6; ++f) {
        hv[f] = (float)g.bc_value[s][f];
        if (g.bc[s][f] == RD_BC_DIRICHLET) m |= 1u << f;
    }
    cudaError_t e = launch_pack(c->staging, field_ptr(c, c->cur, s), g.storage, g.nx, g.ny, g.nz,
                                c->pitch, m, hv, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "pack kernel");
    c->launches++;
    RD_CUDA(c, cudaStreamSynchronize(c->stream));
    return RD_OK;
}

rd_status rd_get_field(rd_ctx* c, int s, float* dst, size_t count) {
    if (!c || !dst) return fail(c, RD_EINVAL, "null argument");
    if (!c->state) return fail(c, RD_EINVAL, "no memory attached");
    if (s < 0 || s >= c->S) return fail(c, RD_EINVAL, "species %d out of range", s);
    drain_batch(c);
    const rd_config& g = c->cfg;
    const size_t n = (size_t)g.nx * g.ny * g.nz;
    if (count != n) return fail(c, RD_EINVAL, "count %zu != nx*ny*nz = %zu", count, n);
    cudaError_t e = launch_unpack(field_ptr(c, c->cur, s), c->staging, g.storage, g.nx, g.ny,
                                  g.nz, c->pitch, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "unpack kernel");
    c->launches++;
    const bool dev = is_device_ptr(dst);
    RD_CUDA(c, cudaMemcpyAsync(dst, c->staging, n * sizeof(float),
                               dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
    RD_CUDA(c, cudaStreamSynchronize(c->stream));
    return RD_OK;
}

size_t rd_plane_bytes(const rd_ctx* c) {
    return c ? (size_t)c->plane * c->ebytes : 0;
}

rd_status rd_copy_planes(rd_ctx* c, int s, int z0, int k, void* buf, size_t bytes,
                         int32_t to_buf) {
    if (!c || !buf) return fail(c, RD_EINVAL, "null argument");
    if (!c->state) return fail(c, RD_EINVAL, "no memory attached");
    if (s < 0 || s >= c->S) return fail(c, RD_EINVAL, "species %d out of range", s);
    if (k < 0 || z0 < 0 || (long long)z0 + k > c->cfg.nz)
        return fail(c, RD_EINVAL, "planes %d..%d outside 0..%d", z0, z0 + k - 1, c->cfg.nz - 1);
    const size_t pb = rd_plane_bytes(c);
    if (bytes != pb * (size_t)k)
        return fail(c, RD_EINVAL, "buffer of %zu bytes for %d planes of %zu bytes", bytes, k, pb);
    if (!is_device_ptr(buf)) return fail(c, RD_EINVAL, "the buffer must be device memory");
    if (k == 0) return RD_OK;
    drain_batch(c);
    // the planes of one species are contiguous: one copy
    char* field = field_ptr(c, c->cur, s) + (size_t)z0 * pb;
    if (to_buf)
        RD_CUDA(c, cudaMemcpyAsync(buf, field, bytes, cudaMemcpyDeviceToDevice, c->stream));
    else
        RD_CUDA(c, cudaMemcpyAsync(field, buf, bytes, cudaMemcpyDeviceToDevice, c->stream));
    return RD_OK;
}

rd_status rd_step(rd_ctx* c, int64_t nsteps) {
    if (!c || nsteps < 0) return fail(c, RD_EINVAL, "bad argument");
    if (!c->state) return fail(c, RD_EINVAL, "no memory attached");
    if (c->batch) return fail(c, RD_EINVAL, "context is in a batch; step the batch");
    if (nsteps == 0) return RD_OK;
    return step_ctx(c, nsteps);
}

rd_status rd_mass(rd_ctx* c, int s, double out[3]) {
    if (!c || !out) return fail(c, RD_EINVAL, "null argument");
    if (!c->state) return fail(c, RD_EINVAL, "no memory attached");
    if (s < 0 || s >= c->S) return fail(c, RD_EINVAL, "species %d out of range", s);
    drain_batch(c);
    const rd_config& g = c->cfg;
    cudaError_t e = launch_reduce(field_ptr(c, c->cur, s), g.storage, g.nx, g.ny, g.nz, c->pitch,
                                  c->partials, c->result, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "reduce kernel");
    c->launches += 2;
    RD_CUDA(c, cudaMemcpyAsync(out, c->result, 3 * sizeof(double), cudaMemcpyDeviceToHost,
                               c->stream));
    RD_CUDA(c, cudaStreamSynchronize(c->stream));
    return out[2] > 0 ? RD_ENONFINITE : RD_OK;
}

// The debug build's bounds report after a synchronisation (RD_OK in the
// normal build, whose word is always 0).
static rd_status bounds_status(rd_ctx* c) {
    unsigned long long w = 0;
    RD_CUDA(c, debug_word(&w, false));
    if (!w) return RD_OK;
    RD_CUDA(c, debug_word(&w, true));
    const long long off = (long long)(w << 24) >> 24;   // sign-extend 40 bits
    return fail(c, RD_EBOUNDS, "bounds check: out-of-range access at site %d, byte offset %lld",
                (int)((w >> 40) & 0xFFFF), off);
}

// A resident launch whose grid barrier timed out since the last check
// (RD_ETIMEOUT; the flag is cleared).  Only contexts that use the kernel
// pay the read.
static rd_status resident_status(rd_ctx* c, cudaStream_t st) {
    if (c->kernel != RD_KERNEL_RESIDENT || !c->bar) return RD_OK;
    unsigned failed = 0;
    RD_CUDA(c, cudaMemcpyAsync(&failed, &c->bar->failed, sizeof(failed), cudaMemcpyDeviceToHost,
                               st));
    RD_CUDA(c, cudaStreamSynchronize(st));
    if (!failed) return RD_OK;
    RD_CUDA(c, cudaMemsetAsync(&c->bar->failed, 0, sizeof(unsigned), st));
    RD_CUDA(c, cudaStreamSynchronize(st));
    return fail(c, RD_ETIMEOUT, "resident kernel: a grid barrier wait ran out; the steps of "
                                "that launch are incomplete");
}

rd_status rd_sync(rd_ctx* c) {
    if (!c) return RD_EINVAL;
    drain_batch(c);
    RD_CUDA(c, cudaStreamSynchronize(c->stream));
    rd_status st = resident_status(c, c->stream);
    if (st != RD_OK) return st;
    return bounds_status(c);
}

rd_status rd_wait(rd_ctx* c, int64_t timeout_ms) {
    if (!c) return RD_EINVAL;
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        cudaError_t e = cudaStreamQuery(c->stream);
        if (e == cudaSuccess) return RD_OK;
        if (e != cudaErrorNotReady) return cuda_fail(c, e, "cudaStreamQuery");
        const auto ms = std::chrono::duration_cast<std::chrono::milliseconds>(
                            std::chrono::steady_clock::now() - t0).count();
        if (ms >= timeout_ms) return fail(c, RD_ETIMEOUT, "stream still busy after %lld ms", (long long)ms);
        std::this_thread::sleep_for(std::chrono::microseconds(200));
    }
}

int64_t rd_step_count(const rd_ctx* c) { return c ? c->steps : -1; }

rd_status rd_set_step_count(rd_ctx* c, int64_t n) {
    if (!c) return RD_EINVAL;
    c->steps = n;
    c->stepn_dirty = true;
    return RD_OK;
}

int64_t rd_launch_count(const rd_ctx* c) { return c ? c->launches : -1; }

rd_status rd_get_tuning(const rd_ctx* c, rd_tuning* out) {
    if (!c || !out) return RD_EINVAL;
    *out = c->tun;
    return RD_OK;
}

rd_status rd_set_kernel(rd_ctx* c, int32_t kernel) {
    if (!c) return fail(nullptr, RD_EINVAL, "null context");
    if (kernel < RD_KERNEL_MARCH || kernel > RD_KERNEL_RESIDENT)
        return fail(c, RD_EINVAL, "unknown kernel %d", kernel);
    if (kernel == RD_KERNEL_RESIDENT) {
        const rd_config& g = c->cfg;
        if (stencil_of(g) != 7 || is_ch(g.model) || g.wind_kind == RD_WIND_3D)
            return fail(c, RD_EUNSUPPORTED,
                        "the resident kernel needs the 7-point stencil, a model without "
                        "Cahn-Hilliard and no 3-D wind");
        rdk::ResidentPlan plan{};
        const cudaError_t e = rdk::plan_resident(
            g.model, g.storage, plain_problem(g), !periodic_axis(g, 0, 1) && !periodic_axis(g, 0, 2),
            g.nx, g.ny, g.nz, c->res_force[0], c->res_force[1], c->res_force[2], &plan);
        if (e == cudaErrorInvalidValue)
            return fail(c, RD_EUNSUPPORTED,
                        "the resident kernel's rows do not fit shared memory (nx = %d)", g.nx);
        if (e != cudaSuccess) return cuda_fail(c, e, "resident plan");
        c->res_plan = plan;
    } else if (kernel != RD_KERNEL_MARCH) {
        const rd_config& g = c->cfg;
        if (stencil_of(g) != 19 || g.storage != RD_STORE_F32 || is_ch(g.model) ||
            !plain_problem(g))
            return fail(c, RD_EUNSUPPORTED,
                        "the Shared and Moving Tiles kernels need the 19-point stencil, FP32 "
                        "state, no Cahn-Hilliard and no held layer, source or wind");
        if (c->tun.tsteps != 1) return fail(c, RD_EINVAL, "tsteps must be 1");
    }
    c->kernel = kernel;
    return RD_OK;
}

int32_t rd_get_kernel(const rd_ctx* c) { return c ? c->kernel : -1; }

rd_status rd_set_tuning(rd_ctx* c, const rd_tuning* t) {
    if (!c || !t) return fail(c, RD_EINVAL, "null argument");
    rd_status st = check_tuning(c->cfg, *t);
    if (st != RD_OK) return fail(c, st, "%s", g_err);
    c->tun = *t;
    c->tun.zchunk = std::min(c->tun.zchunk, c->cfg.nz);
    c->desc_dirty = true;
    return RD_OK;
}

rd_status rd_autotune(rd_ctx* c, rd_tuning* best_out) {
    if (!c) return RD_EINVAL;
    if (!c->state) return fail(c, RD_EINVAL, "no memory attached");
    if (c->kernel != RD_KERNEL_MARCH)
        return fail(c, RD_EUNSUPPORTED, "the autotuner tunes the march kernel only");
    const rd_config& g = c->cfg;
    const std::string key = tune_key(g);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        load_tune_file();
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end() && check_tuning(g, it->second) == RD_OK) {
            c->tun = it->second;
            c->desc_dirty = true;
            if (best_out) *best_out = c->tun;
            return RD_OK;
        }
    }
    {
        rd_status st = sync_stepn(c, c->stream);
        if (st != RD_OK) return st;
    }
    const rd_tuning saved = c->tun;
    std::vector<rd_tuning> cands;
    const int sten = stencil_of(g);
    for (int T = 1; T <= max_tsteps(g); ++T)
      for (int tq : {kTileQ, 8}) {
        // 8 cells per thread: the one-step 7-point kernel (heights 4k)
        if (tq == 8 && (T != 1 || is_ch(g.model) || sten != 7)) continue;
        for (int ty : {4, 8, 10, 12, 14, 16, 20, 24, 28, 32}) {
          // the register cap is a variant of the 7-point 4-cell one-step kernel
          const bool rc_variant = T == 1 && !is_ch(g.model) && sten == 7 && tq == kTileQ;
          for (int rc = 0; rc <= (rc_variant ? 1 : 0); ++rc) {
            rd_tuning t{};
            t.tsteps = T; t.tile_q = tq; t.tile_y = ty; t.graph = 1; t.zchunk = 1;
            t.regcap = rc;
            if (check_tuning(g, t) != RD_OK) continue;
            const int occ = occupancy(g.model, g.storage, T, ty, rc, variant_code(g), sten, tq);
            if (occ < 1) continue;
            // z-chunks for 1, 2, 4, 8 waves of CTAs; for one step per launch
            // also every split of z into 1..16 chunks, since how evenly the
            // items fill the CTA slots decides as much as the tile does
            std::vector<int> zcs;
            for (int waves : {1, 2, 4, 8}) zcs.push_back(auto_zchunk(g, t, occ, waves));
            if (T == 1)
                for (int k = 1; k <= 16; ++k) zcs.push_back((g.nz + k - 1) / k);
            for (int zc : zcs) {
                t.zchunk = zc;
                bool dup = false;
                for (auto& o : cands)
                    dup |= (o.tsteps == t.tsteps && o.tile_q == t.tile_q && o.tile_y == t.tile_y &&
                            o.zchunk == t.zchunk && o.regcap == t.regcap);
                if (!dup) cands.push_back(t);
            }
          }
        }
      }
    cudaEvent_t e0, e1;
    RD_CUDA(c, cudaEventCreate(&e0));
    RD_CUDA(c, cudaEventCreate(&e1));
    const double cells = (double)g.nx * g.ny * g.nz;
    // GLUPS of tuning t: the median of ``samples`` timings of ``reps``
    // launches after one warm-up launch, all reading the current level
    // (negative if the tuning cannot run)
    auto time_tuning = [&](const rd_tuning& t, int reps, int samples) -> double {
        c->tun = t;
        c->desc_dirty = true;
        if (upload_desc(c) != RD_OK) return -1.0;
        rd_status st = launch_ctx(c, t.tsteps, c->cur, c->stream);
        if (st != RD_OK) { cudaGetLastError(); return -1.0; }
        std::vector<double> rates;
        for (int k = 0; k < samples; ++k) {
            cudaEventRecord(e0, c->stream);
            for (int i = 0; i < reps && st == RD_OK; ++i)
                st = launch_ctx(c, t.tsteps, c->cur, c->stream);
            cudaEventRecord(e1, c->stream);
            if (cudaEventSynchronize(e1) != cudaSuccess || st != RD_OK) {
                cudaGetLastError();
                return -1.0;
            }
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            rates.push_back(cells * t.tsteps * reps / (ms * 1e-3) / 1e9);
        }
        std::sort(rates.begin(), rates.end());
        return rates[rates.size() / 2];
    };
    // pass 1: every candidate, briefly; pass 2: the best few, median of
    // several longer timings (one short timing is too noisy to rank tilings
    // a few percent apart)
    std::vector<std::pair<double, rd_tuning>> ranked;
    for (const rd_tuning& t : cands) {
        const double rate = time_tuning(t, 4, 1);
        if (std::getenv("RD_AUTOTUNE_VERBOSE"))
            std::fprintf(stderr, "rd_autotune %s T=%d tile_y=%d zchunk=%d regcap=%d: %.2f GLUPS\n",
                         key.c_str(), t.tsteps, t.tile_y, t.zchunk, t.regcap, rate);
        if (rate > 0) ranked.push_back({rate, t});
    }
    std::stable_sort(ranked.begin(), ranked.end(),
                     [](const auto& x, const auto& y) { return x.first > y.first; });
    double best = -1.0;
    rd_tuning bt = saved;
    const size_t finalists = std::min<size_t>(ranked.size(), 8);
    for (size_t i = 0; i < finalists; ++i) {
        const rd_tuning& t = ranked[i].second;
        const double rate = time_tuning(t, 8, 5);
        if (std::getenv("RD_AUTOTUNE_VERBOSE"))
            std::fprintf(stderr, "rd_autotune %s final T=%d tile_y=%d zchunk=%d regcap=%d: %.2f GLUPS\n",
                         key.c_str(), t.tsteps, t.tile_y, t.zchunk, t.regcap, rate);
        if (rate > best) { best = rate; bt = t; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->tun = best > 0 ? bt : saved;
    c->desc_dirty = true;
    if (best > 0) {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache[key] = c->tun;
        save_tune(key, c->tun, best);
    }
    if (best_out) *best_out = c->tun;
    return upload_desc(c);
}

const char* rd_status_str(rd_status st) {
    switch (st) {
    case RD_OK: return "ok";
    case RD_EINVAL: return "invalid argument";
    case RD_ENOMEM: return "out of memory";
    case RD_ECUDA: return "CUDA error";
    case RD_EUNSTABLE: return "time step above the stability bound";
    case RD_ENONFINITE: return "non-finite values in the state";
    case RD_ETIMEOUT: return "timed out";
    case RD_EBUDGET: return "memory budget exceeded";
    case RD_EUNSUPPORTED: return "not supported by this build";
    case RD_EBOUNDS: return "out-of-range access found by the bounds-checked build";
    }
    return "unknown status";
}

const char* rd_last_error(const rd_ctx* c) { return c ? c->err : g_err; }

rd_status rd_set_resident_plan(rd_ctx* c, int32_t K, int32_t tile_y, int32_t tile_z) {
    if (!c) return fail(nullptr, RD_EINVAL, "null context");
    if (c->kernel != RD_KERNEL_RESIDENT)
        return fail(c, RD_EUNSUPPORTED, "the context's kernel is not the resident kernel");
    if (K < 0 || K > rdk::kResidentMaxK || tile_y < 0 || tile_z < 0)
        return fail(c, RD_EINVAL, "plan out of range: K %d, tile %d x %d", K, tile_y, tile_z);
    const rd_config& g = c->cfg;
    rdk::ResidentPlan plan{};
    const cudaError_t e = rdk::plan_resident(
        g.model, g.storage, plain_problem(g), !periodic_axis(g, 0, 1) && !periodic_axis(g, 0, 2),
        g.nx, g.ny, g.nz, K, tile_y, tile_z, &plan);
    if (e == cudaErrorInvalidValue)
        return fail(c, RD_EINVAL, "K %d with a %d x %d tile does not fit shared memory", K,
                    tile_y, tile_z);
    if (e != cudaSuccess) return cuda_fail(c, e, "resident plan");
    c->res_force[0] = K;
    c->res_force[1] = tile_y;
    c->res_force[2] = tile_z;
    c->res_plan = plan;
    return RD_OK;
}

rd_status rd_get_resident_plan(const rd_ctx* c, int32_t out[8]) {
    if (!c || !out) return RD_EINVAL;
    if (c->kernel != RD_KERNEL_RESIDENT) return RD_EUNSUPPORTED;
    const rdk::ResidentPlan& p = c->res_plan;
    out[0] = p.K;
    out[1] = p.ty;
    out[2] = p.tz;
    out[3] = p.nty * p.ntz;
    out[4] = p.grid;
    out[5] = p.threads;
    out[6] = p.smem;
    out[7] = p.tma;
    return RD_OK;
}

rd_status rd_debug_resident_stall(rd_ctx* c, int32_t phantom) {
    if (!c || phantom < 0) return fail(c, RD_EINVAL, "bad argument");
    if (c->kernel != RD_KERNEL_RESIDENT)
        return fail(c, RD_EUNSUPPORTED, "the context's kernel is not the resident kernel");
    c->res_phantom = phantom;
    return RD_OK;
}

rd_status rd_debug_fail_alloc(int64_t k) {
    if (k < 0) return RD_EINVAL;
    std::lock_guard<std::mutex> lk(g_fault_mu);
    g_fail_alloc = k;
    return RD_OK;
}

// ================================================================ batches
rd_status rd_batch_create(int32_t model, int32_t storage, rd_batch** out) {
    if (!out) return RD_EINVAL;
    *out = nullptr;
    if (model < RD_MODEL_DIFFUSION || model > RD_MODEL_CH_TABLE1)
        return fail(nullptr, RD_EINVAL, "bad model");
    if (storage != RD_STORE_F32 && storage != RD_STORE_BF16) return fail(nullptr, RD_EINVAL, "bad storage");
    rd_batch* b = new (std::nothrow) rd_batch();
    if (!b) return RD_ENOMEM;
    b->model = model;
    b->storage = storage;
    if (cudaStreamCreateWithFlags(&b->own_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->upload_done, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        delete b;
        return fail(nullptr, RD_ECUDA, "batch stream/event creation failed");
    }
    b->stream = b->own_stream;
    *out = b;
    return RD_OK;
}

rd_status rd_batch_add(rd_batch* b, rd_ctx* c) {
    if (!b || !c) return RD_EINVAL;
    if (c->batch) return fail(c, RD_EINVAL, "context already in a batch");
    if (c->cfg.model != b->model || c->cfg.storage != b->storage)
        return fail(c, RD_EINVAL, "model/storage differ from the batch");
    if (!b->members.empty() && stencil_of(c->cfg) != b->stencil)
        return fail(c, RD_EINVAL, "the members of a batch share one stencil");
    if (!c->state) return fail(c, RD_EINVAL, "no memory attached");
    cudaStreamSynchronize(c->stream);
    if (b->members.empty()) b->stencil = stencil_of(c->cfg);
    b->members.push_back(c);
    c->batch = b;
    b->members_version++;
    return RD_OK;
}

rd_status rd_batch_remove(rd_batch* b, rd_ctx* c) {
    if (!b || !c) return RD_EINVAL;
    auto it = std::find(b->members.begin(), b->members.end(), c);
    if (it == b->members.end()) return fail(c, RD_EINVAL, "not a member");
    cudaStreamSynchronize(b->stream);
    b->members.erase(it);
    c->batch = nullptr;
    c->desc_dirty = true;
    b->members_version++;
    return RD_OK;
}

int32_t rd_batch_size(const rd_batch* b) { return b ? (int32_t)b->members.size() : -1; }

rd_status rd_batch_set_stream(rd_batch* b, void* stream) {
    if (!b) return RD_EINVAL;
    cudaStreamSynchronize(b->stream);
    b->stream = static_cast<cudaStream_t>(stream);
    return RD_OK;
}

rd_status rd_batch_set_tuning(rd_batch* b, const rd_tuning* t) {
    if (!b || !t) return RD_EINVAL;
    b->tun = *t;
    b->tun_set = true;
    b->graph.reset();
    return RD_OK;
}

namespace {

// The batch's tuning: the one set by rd_batch_set_tuning, else one step per
// launch at the default tile height with a z-chunk that fills the CTA slots
// over all current members.
rd_tuning batch_tuning(rd_batch* b) {
    if (b->tun_set) return b->tun;
    rd_tuning t{};
    t.tsteps = 1;
    t.tile_q = kTileQ;
    t.tile_y = default_tile_y(b->model);
    t.graph = 1;
    const int occ = occupancy(b->model, b->storage, 1, t.tile_y, 0, 0, b->stencil);
    std::vector<std::pair<long long, int>> cols_nz;
    for (rd_ctx* c : b->members)
        cols_nz.push_back({(long long)tiles(c->cfg.nx, kTileW) *
                               tiles(c->cfg.ny, t.tile_y),
                           c->cfg.nz});
    t.zchunk = cols_nz.empty() ? 32 : wave_zchunk(cols_nz, (long long)std::max(occ, 1) * num_sms());
    return t;
}

// Rebuild and upload the descriptor array: member i reads level cur_i at
// parity 0.
// ``caps``: launches each member takes part in (rd_batch_step_each), or
// nullptr for every launch.
rd_status batch_upload(rd_batch* b, const rd_tuning& t, long long* nitems,
                       const long long* caps = nullptr) {
    const size_t n = b->members.size();
    if (n > b->desc_cap) {
        if (b->desc_dev) cudaFree(b->desc_dev);
        if (b->desc_host) cudaFreeHost(b->desc_host);
        b->desc_dev = nullptr;
        b->desc_host = nullptr;
        b->work = nullptr;
        size_t cap = std::max<size_t>(16, n * 2);
        // the descriptors, then the work-item counter (InstDesc is a
        // multiple of 16 bytes, so the counter is aligned)
        if (dev_alloc(reinterpret_cast<void**>(&b->desc_dev),
                      cap * sizeof(InstDesc) + 256) != cudaSuccess ||
            host_alloc(reinterpret_cast<void**>(&b->desc_host), cap * sizeof(InstDesc)) != cudaSuccess) {
            cudaGetLastError();
            // keep nothing of a half-made pair
            if (b->desc_dev) cudaFree(b->desc_dev);
            if (b->desc_host) cudaFreeHost(b->desc_host);
            b->desc_dev = nullptr;
            b->desc_host = nullptr;
            b->desc_cap = 0;
            return fail(nullptr, RD_ENOMEM, "batch descriptor allocation failed");
        }
        b->desc_cap = cap;
        b->work = reinterpret_cast<unsigned long long*>(b->desc_dev + cap);
        cudaError_t e = cudaMemsetAsync(b->work, 0, 2 * sizeof(unsigned long long), b->stream);
        if (e != cudaSuccess) return cuda_fail(nullptr, e, "batch work counter");
        b->graph.reset();
    }
    // the previous upload must have left the pinned buffer
    cudaEventSynchronize(b->upload_done);
    long long begin = 0;
    for (size_t i = 0; i < n; ++i) {
        rd_ctx* c = b->members[i];
        rd_tuning ti = t;
        ti.zchunk = std::min(t.zchunk, c->cfg.nz);
        fill_desc(c, b->desc_host[i], ti);
        b->desc_host[i].par = c->cur;
        b->desc_host[i].item_begin = begin;
        b->desc_host[i].launch_cap = caps ? caps[i] : -1;
        begin += items_of(b->desc_host[i]);
    }
    *nitems = begin;
    if (n) {
        cudaError_t e = cudaMemcpyAsync(b->desc_dev, b->desc_host, n * sizeof(InstDesc),
                                        cudaMemcpyHostToDevice, b->stream);
        if (e != cudaSuccess) return cuda_fail(nullptr, e, "batch descriptor upload");
        cudaEventRecord(b->upload_done, b->stream);
    }
    return RD_OK;
}

static_assert(sizeof(InstDesc) % alignof(unsigned long long) == 0,
              "the batch's work counter follows its descriptor array");

// launches (of T steps each, alternating parity) captured in a batch's graph
constexpr int kBatchGraphLaunches = 16;

// ``caps``: the launch counts members' launches (rd_batch_step_each), so its
// CTAs pull their items from the batch's counter, whose last pull counts the
// launch.  Otherwise they pull only when the items fill four or more waves
// of the grid (uneven items then balance; with fewer, the pulls' round
// trips cost more than they balance: a served mix of small requests measured
// a longer tail with them).
rd_status batch_launch(rd_batch* b, const rd_tuning& t, int T, int parity, long long nitems,
                       cudaStream_t st, bool caps) {
    LaunchArgs a{};
    a.desc = b->desc_dev;
    a.ninst = (int)b->members.size();
    a.parity = parity;
    a.nitems = nitems;
    a.regcap = t.regcap;
    a.plain = 1;
    for (rd_ctx* m : b->members) {
        a.plain = a.plain && plain_problem(m->cfg);
        a.wind3 = a.wind3 || m->cfg.wind_kind == RD_WIND_3D;
    }
    a.ty = t.tile_y;
    a.vw = vw_of(t.tile_q);
    const size_t sm = smem_of(b->model, b->storage, T, a.ty, b->stencil, t.tile_q);
    const int occ = std::max(
        1, occupancy(b->model, b->storage, T, a.ty, a.regcap, a.plain ? 1 : a.wind3 ? 2 : 0,
                     b->stencil, t.tile_q));
    const long long grid = std::min<long long>(nitems, (long long)occ * num_sms());
    a.work = (caps || nitems >= 4 * grid) ? b->work : nullptr;
    cudaError_t e = launch_model(b->model, b->storage, T, a, (int)grid, sm, st, nullptr, b->stencil);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "batch step launch");
    b->launches += kernels_per_step(b->members[0]->cfg);
    return RD_OK;
}

}  // namespace

// ``steps``: per-member step counts (each at most nsteps), or nullptr for
// nsteps steps of every member.
rd_status batch_step_impl(rd_batch* b, int64_t nsteps, const int64_t* steps) {
    if (b->members.size() == 1) {
        // a batch of one steps its member as a single context does (its own
        // tuning, descriptor in the kernel parameters), on the batch's stream
        rd_ctx* c = b->members[0];
        cudaStream_t own = c->stream;
        const int64_t before = c->launches;
        c->stream = b->stream;
        rd_status st = step_ctx(c, nsteps);
        c->stream = own;
        b->launches += c->launches - before;
        return st;
    }
    const rd_tuning t = batch_tuning(b);
    rd_status st = check_tuning(b->members[0]->cfg, t);
    if (st != RD_OK) return st;
    if (steps && t.tsteps != 1)
        return fail(nullptr, RD_EINVAL, "per-member step counts need one step per launch");
    long long nitems = 0;
    for (rd_ctx* c : b->members)
        if ((st = sync_stepn(c, b->stream)) != RD_OK) return st;
    std::vector<long long> caps;
    if (steps) {
        const int kps = kernels_per_step(b->members[0]->cfg);
        for (size_t i = 0; i < b->members.size(); ++i) caps.push_back(steps[i] * kps);
    }
    if ((st = batch_upload(b, t, &nitems, steps ? caps.data() : nullptr)) != RD_OK) return st;
    // launches completed in this call: the members' caps count from zero
    cudaError_t ew = cudaMemsetAsync(b->work + 1, 0, sizeof(unsigned long long), b->stream);
    if (ew != cudaSuccess) return cuda_fail(nullptr, ew, "batch launch count");
    const int T = t.tsteps;
    int64_t full = nsteps / T;
    const int rem = (int)(nsteps % T);
    int parity = 0;
    const long long key = (b->members_version * 1000003LL + nitems) * 2 + (steps ? 1 : 0);
    if (t.graph && full >= kBatchGraphLaunches) {
        if (!b->graph.exec || b->graph.key != key) {
            b->graph.reset();
            if (!b->capture_stream &&
                cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking) != cudaSuccess)
                return fail(nullptr, RD_ECUDA, "capture stream");
            cudaError_t e = cudaStreamBeginCapture(b->capture_stream, cudaStreamCaptureModeThreadLocal);
            if (e != cudaSuccess) return cuda_fail(nullptr, e, "begin capture");
            const int64_t before = b->launches;
            for (int i = 0; i < kBatchGraphLaunches && st == RD_OK; ++i)
                st = batch_launch(b, t, T, i & 1, nitems, b->capture_stream, steps != nullptr);
            cudaGraph_t g = nullptr;
            e = cudaStreamEndCapture(b->capture_stream, &g);
            if (st != RD_OK) { if (g) cudaGraphDestroy(g); return st; }
            if (e != cudaSuccess) return cuda_fail(nullptr, e, "end capture");
            e = cudaGraphInstantiate(&b->graph.exec, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) return cuda_fail(nullptr, e, "instantiate");
            b->graph.launches = (int)(b->launches - before);   // kernels in the graph
            b->launches = before;                               // captured, not run
            b->graph.key = key;
        }
        while (full >= kBatchGraphLaunches) {
            cudaError_t e = cudaGraphLaunch(b->graph.exec, b->stream);
            if (e != cudaSuccess) return cuda_fail(nullptr, e, "graph launch");
            b->launches += b->graph.launches;
            full -= kBatchGraphLaunches;
        }
    }
    for (int64_t i = 0; i < full; ++i) {
        if ((st = batch_launch(b, t, T, parity, nitems, b->stream, steps != nullptr)) != RD_OK)
            return st;
        parity ^= 1;
    }
    if (rem) {
        if ((st = batch_launch(b, t, rem, parity, nitems, b->stream, steps != nullptr)) != RD_OK)
            return st;
        parity ^= 1;
    }
    const int64_t launches = nsteps / T + (rem ? 1 : 0);
    for (size_t i = 0; i < b->members.size(); ++i) {
        rd_ctx* c = b->members[i];
        // one transition between the levels per step (per launch of T steps)
        const int64_t n = steps ? steps[i] : nsteps;
        c->cur ^= (int)((steps ? n : launches) & 1);
        c->steps += n;
        if (steps && n < nsteps) c->stepn_dirty = true;   // its counter stopped early
    }
    return RD_OK;
}

rd_status rd_batch_step(rd_batch* b, int64_t nsteps) {
    if (!b || nsteps < 0) return RD_EINVAL;
    if (b->members.empty() || nsteps == 0) return RD_OK;
    return batch_step_impl(b, nsteps, nullptr);
}

rd_status rd_batch_step_each(rd_batch* b, const int64_t* steps) {
    if (!b || (!steps && !b->members.empty())) return RD_EINVAL;
    int64_t n = 0;
    for (size_t i = 0; i < b->members.size(); ++i) {
        if (steps[i] < 0) return fail(nullptr, RD_EINVAL, "negative step count");
        n = std::max(n, steps[i]);
    }
    if (n == 0) return RD_OK;
    return batch_step_impl(b, n, steps);
}

rd_status rd_batch_sync(rd_batch* b) {
    if (!b) return RD_EINVAL;
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "batch sync");
    if (b->members.size() == 1) {   // a batch of one steps with its member's kernel
        rd_status st = resident_status(b->members[0], b->stream);
        if (st != RD_OK) return st;
    }
    return bounds_status(nullptr);
}

rd_status rd_batch_destroy(rd_batch* b) {
    if (!b) return RD_EINVAL;
    cudaStreamSynchronize(b->stream);
    for (rd_ctx* c : b->members) { c->batch = nullptr; c->desc_dirty = true; }
    b->graph.reset();
    if (b->desc_dev) cudaFree(b->desc_dev);
    if (b->desc_host) cudaFreeHost(b->desc_host);
    if (b->upload_done) cudaEventDestroy(b->upload_done);
    if (b->capture_stream) cudaStreamDestroy(b->capture_stream);
    if (b->own_stream) cudaStreamDestroy(b->own_stream);
    delete b;
    return RD_OK;
}

int64_t rd_batch_launch_count(const rd_batch* b) { return b ? b->launches : -1; }

}  // extern "C"
