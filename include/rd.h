/*
 * rd.h -- C ABI of the GB300 (sm_103a) reaction-diffusion stepper.
 *
 * The library advances reaction-diffusion systems with the method of lines
 * of the paper's Section 2: a 7-point finite-difference Laplacian per
 * species and axis (or the paper's isotropic 19-point Laplacian, eqs.
 * (3)-(4)), the pointwise reaction term R(c) of eq. (1), optional
 * first-order upwind advection and a point emission term (Section 4.1 and
 * Table 1), and the forward-Euler update of eq. (5).  Every species is
 * stored as its own array, x fastest, as in the paper's kernels (Tables
 * 4-5), two time levels per species (the "first"/"second" arrays of the
 * paper's host loop, Table 3).
 *
 * Conventions shared by every entry point
 *   - Every call returns rd_status; nothing is thrown across the ABI.
 *   - Grid fields exchanged with the caller are DENSE float32 arrays of
 *     nz*ny*nx values, index ((z*ny)+y)*nx+x, i.e. C order (z, y, x).
 *     Pointers may be host or device memory (detected per call).
 *   - Host arrays always belong to the caller.  Device state belongs to the
 *     context unless the caller attached its own memory (RD_FLAG_NO_ALLOC +
 *     rd_attach), in which case rd_destroy does not free it.
 *   - Work is enqueued on the context's CUDA stream (its own non-blocking
 *     stream unless rd_set_stream gave another).  rd_step is asynchronous;
 *     rd_get_field, rd_mass and rd_sync synchronise that stream.
 *   - A context is not thread-safe: one host thread at a time.
 */
#ifndef RD_H
#define RD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RD_MAX_SPECIES 4

typedef enum rd_status {
    RD_OK = 0,
    RD_EINVAL = 1,        /* bad argument or configuration                  */
    RD_ENOMEM = 2,        /* device or host allocation failed               */
    RD_ECUDA = 3,         /* a CUDA call failed; see rd_last_error          */
    RD_EUNSTABLE = 4,     /* dt violates the explicit stability bound       */
    RD_ENONFINITE = 5,    /* a reduction found NaN/Inf in the state         */
    RD_ETIMEOUT = 6,      /* rd_wait gave up before the stream finished     */
    RD_EBUDGET = 7,       /* a batch or server memory budget was exceeded   */
    RD_EUNSUPPORTED = 8,  /* valid request this build does not implement    */
    RD_EBOUNDS = 9        /* bounds-checked debug build: a kernel met an
                             out-of-range index (see rd_debug_bounds)       */
} rd_status;

/* Boundary rule of one face of one species (faces -x,+x,-y,+y,-z,+z). */
typedef enum rd_bc_kind {
    RD_BC_NEUMANN = 0,    /* zero flux: the ghost value equals the face cell */
    RD_BC_PERIODIC = 1,   /* wrap-around; both faces of the axis, every
                             species the same                                */
    RD_BC_DIRICHLET = 2   /* the outermost cell layer on that face is held at
                             bc_value and never updated (the paper keeps its
                             boundary points in the outermost layer,
                             Section 4.1)                                    */
} rd_bc_kind;

/* Model families (paper Table 1 rows, in the benchmark parameterisation). */
typedef enum rd_model {
    RD_MODEL_DIFFUSION = 0,   /* R = 0, any species count 1..4              */
    RD_MODEL_BRUSSELATOR = 1, /* 2 species u, v:  R_u = a-(b+1)u+u^2 v,
                                 R_v = b u - u^2 v;  params[0]=a, [1]=b      */
    RD_MODEL_CH_FRONT = 2,    /* 3 species a, b, c: a+b->c at rate k a b;
                                 c also moves by M Lap(f'(c) - kappa Lap c),
                                 f'(c) = 2c(c-1)(2c-1) (Cahn-Hilliard, the
                                 biharmonic as two chained Laplacians,
                                 Section 4.1); params[0]=k, [1]=M, [2]=kappa;
                                 species c has no Fickian term (D[2] = 0)    */
    RD_MODEL_AIR = 3,         /* 3 species NO, NO2, O3: NO2 -> NO + O3 at
                                 j NO2, NO + O3 -> NO2 at k NO O3;
                                 params[0]=j, [1]=k                          */
    RD_MODEL_TURING = 4,      /* 2 species, the activator-inhibitor system of
                                 Table 1 (row 2): R_1 = c1 - c1^3 - c2,
                                 R_2 = gamma (c1 - alpha c2 - beta);
                                 params[0]=alpha, [1]=beta, [2]=gamma        */
    RD_MODEL_CH_TABLE1 = 5    /* 3 species c1, c2, c3, the phase separation
                                 behind a front of Table 1 (row 3):
                                 c1 + c2 -> c3 at k1 c1 c2, the sink k2 c1 c3
                                 of c1 and c3, and c3 also moves by
                                 -lambda Lap(eps c3 - gamma c3^3 + sigma Lap c3)
                                 (Cahn-Hilliard, as RD_MODEL_CH_FRONT);
                                 params[0]=k1, [1]=k2, [2]=lambda, [3]=eps,
                                 [4]=gamma, [5]=sigma; c3 has no Fickian term
                                 (D[2] = 0)                                  */
} rd_model;

typedef enum rd_storage {
    RD_STORE_F32 = 0,     /* float32 state                                  */
    RD_STORE_BF16 = 1     /* bfloat16 state, float32 arithmetic, each new
                             value rounded to nearest-even when stored      */
} rd_storage;

/* Advection velocity along +x (first-order upwind, Section 4.1). */
typedef enum rd_wind {
    RD_WIND_NONE = 0,
    RD_WIND_LOG = 1,      /* u_x(z) = wind_u0 * ln(1+z) / ln(1+nz), z the
                             cell index 0..nz-1                              */
    RD_WIND_CONST = 2,    /* u_x = wind_u0 everywhere                       */
    RD_WIND_3D = 3        /* the plume wind of Table 1 (row 4): first-order
                             upwind along all three axes with
                             u = (wind_vel[0], wind_vel[1],
                                  wind_vel[2] * sin(t / wind_tau)),
                             t = n dt at the start of step n (every term of
                             the explicit step is taken at level n); the
                             step index is kept on the device per context,
                             so captured launch sequences stay valid.  One
                             step per launch (tsteps = 1); wind_tau > 0     */
} rd_wind;

enum {
    RD_FLAG_NO_ALLOC = 1, /* rd_create allocates no device memory; the
                             caller must rd_attach state and scratch        */
    RD_FLAG_FORCE = 2     /* skip the stability check                       */
};

/*
 * Problem statement.  Units are the caller's; cells are cubes of edge h.
 *   nx, ny, nz   cells per axis, each >= 2
 *   nspecies     species count (fixed by the model except for diffusion)
 *   h, dt        grid spacing and time step of eq. (5)
 *   D[s][a]      diffusivity of species s along axis a (x, y, z): eq. (1)
 *                with D diagonal, per axis where a problem needs it
 *   bc, bc_value per species and face (-x,+x,-y,+y,-z,+z)
 *   params       model constants (see rd_model)
 *   wind_*       advection (see rd_wind); applies to every species; the
 *                time of RD_WIND_3D is rd_step_count() * dt
 *   src_*        point emission: species src_species gains src_rate per
 *                unit time at cell (src_x, src_y, src_z); src_species < 0
 *                means none
 *   stencil      Laplacian: 0 or 7 = the 7-point stencil, per axis;
 *                19 = the isotropic 19-point stencil of eqs. (3)-(4),
 *                (1/6h^2) (-24 c + 2 x 6 face + 1 x 12 edge neighbours),
 *                edge ghosts taking both crossed faces' rules.  It needs
 *                one diffusivity per species (D[s][0] = D[s][1] = D[s][2],
 *                else RD_EINVAL), steps once per launch (tsteps = 1), and
 *                its stability check uses the centre weight 4 D / h^2 in
 *                place of 2 sum(D) / h^2.  With a Cahn-Hilliard model a
 *                step is two kernel launches, the paper's "Laplacian,
 *                boundary rule, Laplacian" (Section 4.1): the first writes
 *                mu of every cell to a float field in the context's scratch
 *                (rd_query_sizes counts it), the second updates the state
 *                with the 19-point Laplacian of mu, whose ghost cells take
 *                species 2's face rules.
 */
typedef struct rd_config {
    int32_t nx, ny, nz, nspecies;
    int32_t model, storage;
    double h, dt;
    double D[RD_MAX_SPECIES][3];
    int32_t bc[RD_MAX_SPECIES][6];
    double bc_value[RD_MAX_SPECIES][6];
    double params[8];
    int32_t wind_kind, stencil;
    double wind_u0;
    int32_t src_x, src_y, src_z, src_species;
    double src_rate;
    int32_t flags, reserved1;
    double wind_vel[3];   /* RD_WIND_3D: velocity scales along x, y, z      */
    double wind_tau;      /* RD_WIND_3D: time scale of u_z                  */
} rd_config;

typedef struct rd_ctx rd_ctx;

/* Zero the config and set neutral defaults (h = 1, no source, no wind). */
rd_status rd_config_init(rd_config* cfg);

/* Bytes of device memory a context for ``cfg`` needs: the two time levels of
 * all species (pitched rows) and the scratch area (staging for field I/O,
 * reduction partials, instance descriptor, wind table).  Either output
 * pointer may be NULL. */
rd_status rd_query_sizes(const rd_config* cfg, size_t* state_bytes,
                         size_t* scratch_bytes);

/* Validate ``cfg`` and create a context on the current CUDA device for the
 * problem of eq. (1), discretised by the method of lines (Section 2).
 * Checks: sizes >= 2, species count for the model, periodic faces paired
 * and the same for every species, Dirichlet only on non-periodic faces and
 * not on the Cahn-Hilliard species, and the explicit stability bound
 *   dt * (sum_a 2 D[s][a] / h^2 + |u|max / h) <= 1 for every species
 * (isotropic diffusion: dt <= h^2 / (6 D); the 19-point stencil counts
 * 4 D / h^2 instead), plus, for the Cahn-Hilliard species,
 * dt * Mc * L (K L + gb) <= 2 with L the largest eigenvalue of -Laplacian
 * (12 / h^2 for the 7-point stencil, 16 / (3 h^2) for the 19-point one),
 * Mc, K the mobility and gradient coefficient (M, kappa of
 * RD_MODEL_CH_FRONT with gb = 2; lambda, sigma of RD_MODEL_CH_TABLE1 with
 * gb = max(0, 3 gamma - eps)); RD_EUNSTABLE otherwise unless
 * RD_FLAG_FORCE.
 * Allocates both levels and scratch unless RD_FLAG_NO_ALLOC.  The state is
 * zero until rd_set_field.  *out receives the context. */
rd_status rd_create(const rd_config* cfg, rd_ctx** out);

/* Attach caller-owned device memory (RD_FLAG_NO_ALLOC contexts only):
 * ``state`` of state_bytes and ``scratch`` of scratch_bytes as reported by
 * rd_query_sizes, both 256-byte aligned.  The caller keeps ownership and
 * must keep both alive until rd_destroy.
 * State layout: species s of time level l starts at byte
 * (l * nspecies + s) * (state_bytes / (2 * nspecies)); each field is nz
 * planes of ny rows of ``pitch`` elements (float32 or bfloat16), pitch = nx
 * rounded up to a multiple of 128 bytes, x fastest.  Level 0 is current
 * after rd_set_field and after every even number of kernel launches. */
rd_status rd_attach(rd_ctx* ctx, void* state, void* scratch);

/* Free what the context owns (device memory, stream, graphs). */
rd_status rd_destroy(rd_ctx* ctx);

/* Enqueue subsequent work on ``stream`` (a cudaStream_t; NULL = the legacy
 * default stream).  The context does not take ownership. */
rd_status rd_set_stream(rd_ctx* ctx, void* stream);

/* Copy ``count`` = nx*ny*nz dense float32 values (host or device pointer)
 * into species ``s`` of the current level, converting to the storage type
 * (the host loop's copy of the initial state to the GPU, Table 3).
 * Cells of held (Dirichlet) layers are set to their bc_value.  Returns
 * after the source buffer may be reused. */
rd_status rd_set_field(rd_ctx* ctx, int s, const float* src, size_t count);

/* Advance every species by ``nsteps`` forward-Euler steps (eq. (5)).
 * Asynchronous: enqueued on the context's stream.  Internally the steps
 * run as fused kernels advancing T steps per launch (temporal blocking),
 * replayed from a captured CUDA graph when enabled. */
rd_status rd_step(rd_ctx* ctx, int64_t nsteps);

/* Copy species ``s`` of the current level out as ``count`` = nx*ny*nz dense
 * float32 values (host or device pointer), the copy back of Table 3's host
 * loop.  Synchronises the stream. */
rd_status rd_get_field(rd_ctx* ctx, int s, float* dst, size_t count);

/* Bytes of one plane of one species: ny rows of the row pitch in elements of
 * the storage type (see rd_attach).  0 for a NULL context. */
size_t rd_plane_bytes(const rd_ctx* ctx);

/* Copy planes z0 .. z0 + k - 1 of species ``s`` of the current level
 * between the context and the caller's device buffer ``buf`` of ``bytes`` =
 * k * rd_plane_bytes(ctx) bytes (the planes back to back in the context's
 * layout, storage type and row pitch kept): to_buf = 1 reads the context
 * into buf, 0 writes buf into the context.  The ghost-plane exchange of a
 * z-slab decomposition of one problem over several GPUs, as the paper's
 * host loop moves whole arrays between host and device (Table 3).  One
 * device-to-device copy, asynchronous on the context's stream; the caller
 * keeps buf alive until that stream has passed it.  RD_EINVAL for planes
 * outside the grid, a wrong size or a host pointer. */
rd_status rd_copy_planes(rd_ctx* ctx, int s, int z0, int k, void* buf, size_t bytes,
                         int32_t to_buf);

/* FP64 reduction of species ``s`` of the current level: out[0] = sum,
 * out[1] = sum of squares, out[2] = count of non-finite values.  The sums
 * are accumulated in double precision in a fixed order, so repeated calls
 * on the same state give bitwise identical results.  Synchronises the
 * stream; returns RD_ENONFINITE (with out filled) if out[2] > 0. */
rd_status rd_mass(rd_ctx* ctx, int s, double out[3]);

/* Wait for all work enqueued on the context's stream (and, for a batch
 * member, on the batch's stream). */
rd_status rd_sync(rd_ctx* ctx);

/* Like rd_sync, but give up after timeout_ms milliseconds of polling and
 * return RD_ETIMEOUT (the work keeps running; the context stays usable).
 * RD_OK says only that the stream is idle: a resident barrier that ran out
 * or a recorded bounds violation stays flagged for the next rd_sync. */
rd_status rd_wait(rd_ctx* ctx, int64_t timeout_ms);

/* Time steps taken since creation (or the last rd_set_step_count). */
int64_t rd_step_count(const rd_ctx* ctx);
rd_status rd_set_step_count(rd_ctx* ctx, int64_t n);

/* Kernel tuning of a context.
 *   tsteps  steps per launch (temporal blocking depth), 1..3 (1..2 for
 *           the Cahn-Hilliard models, 1 for the 19-point stencil)
 *   tile_q  tile width in vectors, a tile being 64 cells wide: 16 (4 cells
 *           per thread, every kernel) or 8 (8 cells per thread: the
 *           one-step 7-point kernel of a model without Cahn-Hilliard, so
 *           tsteps 1 and tile_y a multiple of 4, at most 40; its CTA is
 *           8 tile_y compute threads, whose x neighbours come by warp
 *           shuffle, plus one halo warp); else RD_EINVAL
 *   tile_y  tile height in rows, >= 1 (even for tsteps = 1 with the
 *           19-point stencil or without Cahn-Hilliard, where the CTA is 16
 *           tile_y compute threads plus one halo warp); otherwise the CTA
 *           has (tile_q + 2) x (tile_y + 2 L) threads (L = tsteps, 2 tsteps
 *           for Cahn-Hilliard); at most 512 threads
 *   zchunk  z planes per work item, >= 1
 *   graph   1: replay rd_step launches from a captured CUDA graph
 * rd_set_tuning validates; RD_EINVAL if the CTA or its shared memory does
 * not fit one SM.  A new context starts with tsteps 1, tile_y 14 (12 for
 * the Cahn-Hilliard models), graph 1, regcap 0 and the z-chunk whose work
 * items fill the resident CTA slots in the fewest waves. */
typedef struct rd_tuning {
    int32_t tsteps, tile_q, tile_y, zchunk, graph;
    int32_t regcap;   /* 1: cap the 7-point one-step kernel at 64 registers
                         per thread (more resident warps), 0: let it use up
                         to 128; the 19-point kernel ignores it              */
} rd_tuning;
rd_status rd_get_tuning(const rd_ctx* ctx, rd_tuning* out);
rd_status rd_set_tuning(rd_ctx* ctx, const rd_tuning* t);

/* Time a built-in list of tunings on this context's problem (launches read
 * the current level and write the spare level, so the state is unchanged)
 * and keep the fastest.  Results are cached per (model, storage, grid, BC,
 * stencil) in-process and, if the environment variable RD_AUTOTUNE_CACHE names a
 * file, in that file (one JSON object per line).  *best may be NULL. */
rd_status rd_autotune(rd_ctx* ctx, rd_tuning* best);

/* Step kernel of a context.  RD_KERNEL_MARCH (the default) is this
 * library's z-marching kernel for the context's stencil.  The other two are
 * the paper's own designs (Section 4.1, Tables 4-5), restated for this GPU
 * as ablation baselines:
 *   RD_KERNEL_SHARED  3-D blocks of 32 x 8 x 4 threads, one cell each, over
 *                     x-y tiles overlapping by one cell; the rim loads but
 *                     does not update; the block walks up z keeping two
 *                     planes in shared memory ("Shared" method);
 *   RD_KERNEL_TILES   blocks of 32 x 8 x 4 threads over overlapping y-z
 *                     tiles, walking along x in 32-cell windows with the
 *                     next window preloaded ("Moving Tiles").
 * Both need the 19-point stencil, FP32 storage, a model without
 * Cahn-Hilliard and no held layer, point source or wind (else
 * RD_EUNSUPPORTED); they ignore rd_tuning except `graph`, and rd_autotune
 * refuses them (RD_EUNSUPPORTED).  Results agree with the march kernel to
 * rounding (other summation order), not bit for bit.
 *   RD_KERNEL_RESIDENT  for small grids whose state stays in L2 (the 64^3
 *                     problems): one cooperative launch advances up to
 *                     65536 steps (rd_step splits longer runs).  Each CTA
 *                     owns tiles of full x rows; a round copies a tile with
 *                     a halo of K rows and planes into shared memory (one
 *                     tensor-memory box per tile where y and z are not
 *                     periodic),
 *                     advances it K steps there (K <= 4, see
 *                     rd_set_resident_plan) and writes the tile's rows; a
 *                     grid-wide barrier separates rounds.  Every level is
 *                     eq. (5) with the march kernel's per-cell arithmetic
 *                     and neighbour values, rounded to the state's type, so
 *                     results equal the march kernel's bit for bit.  Needs
 *                     the 7-point stencil, a model without Cahn-Hilliard, no
 *                     3-D wind, and rows that fit shared memory with a
 *                     one-row tile (else RD_EUNSUPPORTED); FP32 or BF16
 *                     state; rd_tuning is ignored and rd_autotune refuses
 *                     it.  Every barrier wait is bounded (about 0.2 s): a
 *                     wait that runs out stops the launch, and the next
 *                     rd_sync (or rd_batch_sync of a batch of one) returns
 *                     RD_ETIMEOUT.  After rd_step the current level holds
 *                     the result; the other level need not hold the step
 *                     before it.
 * A batch of two or more members steps them with the march kernel whatever
 * their own kernel. */
typedef enum rd_kernel {
    RD_KERNEL_MARCH = 0,
    RD_KERNEL_SHARED = 1,
    RD_KERNEL_TILES = 2,
    RD_KERNEL_RESIDENT = 3
} rd_kernel;
rd_status rd_set_kernel(rd_ctx* ctx, int32_t kernel);
int32_t rd_get_kernel(const rd_ctx* ctx);   /* -1 for a NULL context */

/* Plan of the resident kernel: K steps per round (1..4) and tiles of
 * tile_y rows by tile_z planes (clamped to the grid); 0 leaves a choice to
 * the library's cost model (the default for all three).  The choice is kept
 * for later rd_set_kernel(RD_KERNEL_RESIDENT) calls.  RD_EUNSUPPORTED
 * unless the context's kernel is RD_KERNEL_RESIDENT; RD_EINVAL for values
 * out of range or a tile whose rows and halo do not fit shared memory (the
 * previous plan stays).  rd_get_resident_plan writes out[0..7] = K, tile_y,
 * tile_z, tiles, CTAs, threads per CTA, shared memory bytes per CTA, and 1
 * if tiles arrive as tensor-memory (TMA) boxes (y and z not periodic, rows
 * of at most 256 elements; else per-thread copies, 0). */
rd_status rd_set_resident_plan(rd_ctx* ctx, int32_t K, int32_t tile_y, int32_t tile_z);
rd_status rd_get_resident_plan(const rd_ctx* ctx, int32_t out[8]);

/* Launch statistics: kernels this context enqueued since creation. */
int64_t rd_launch_count(const rd_ctx* ctx);

/* Text of a status code, and of the last error seen by a context. */
const char* rd_status_str(rd_status st);
const char* rd_last_error(const rd_ctx* ctx);

/* The bounds-checked debug build (the paper has no counterpart; a stand-in
 * for a memory checker).  That variant of this library checks every
 * shared-memory access the step kernels make through their load, store and
 * copy helpers against the launch's dynamic shared memory, and every global
 * access against the instance's state and scratch allocations; an access
 * out of range is skipped (a load yields 0), never made, and the first one
 * is recorded in a device word: bit 63 set, bits 40..55 a site code (1
 * shared load, 2 shared store, 3 copy destination, 4 copy source, 5 state
 * store, 6 Courant table or step counter, 7 mu field, 8 halo descriptors,
 * 9 state load of the resident kernel, 0xFFFF the self-test), bits 0..39
 * the byte offset from the start of the window missed.  rd_sync and
 * rd_batch_sync then return RD_EBOUNDS (and clear the word), with the site
 * and offset in rd_last_error.
 *   op 0: *word = the word; 1: the same, then clear it; 2: launch a
 *   self-test kernel that records a violation at site 0xFFFF without
 *   touching memory, then as 1.
 * The normal build returns RD_EUNSUPPORTED. */
rd_status rd_debug_bounds(uint64_t* word, int32_t op);

/* Testing hook for the failure paths (the paper has no counterpart): with
 * k > 0, the k-th device or pinned-host allocation this library makes from
 * now on (rd_create's state and scratch, a batch's descriptor arrays) fails
 * as if memory were exhausted, and the hook disarms; k = 0 disarms it.
 * The call that meets the failure returns RD_ENOMEM and frees what it had
 * obtained.  RD_EINVAL for k < 0. */
rd_status rd_debug_fail_alloc(int64_t k);

/* Testing hook for the resident kernel's bounded barrier waits (the paper
 * has no counterpart): the context's next resident launch of more than one
 * round (more steps than the plan's K) counts `phantom` (> 0) CTAs that
 * never arrive, so its first grid barrier wait runs out after about 0.2 s;
 * every CTA then leaves after the launch's first round, so the state is not
 * the one asked for, and the next rd_sync returns RD_ETIMEOUT.  Only that
 * launch is affected; 0 disarms.
 * RD_EINVAL for a null context or phantom < 0, RD_EUNSUPPORTED unless the
 * context's kernel is RD_KERNEL_RESIDENT. */
rd_status rd_debug_resident_stall(rd_ctx* ctx, int32_t phantom);

/* FP64 moments of one field held anywhere in device memory, for callers
 * that must not allocate device memory at that point: code that is
 * capturing a CUDA graph (cudaMalloc / cudaFree are not allowed during a
 * stream capture), serving loops held to a memory budget fixed at start-up,
 * and monitors that must not trigger the device-wide synchronisation that
 * cudaMalloc / cudaFree can cause.  The paper has no counterpart; it is the
 * reduction of rd_mass without a context.
 *   field    device pointer to nz planes of ny rows of ``pitch`` elements of
 *            the given storage kind (RD_STORE_F32 / RD_STORE_BF16), x fastest
 *   out      device pointer to 3 doubles: sum, sum of squares, count of
 *            non-finite values (same fixed-order FP64 sums as rd_mass)
 *   stream   cudaStream_t to run on (NULL = legacy default stream)
 * Limits: nx, ny, nz >= 1, nx <= pitch <= 2^31 - 1, ny * nz <= 2^31 - 1;
 * RD_EINVAL beyond them.  Asynchronous; allocates nothing.  The partial
 * sums live in one file-scope device array of 608 x 3 doubles (14,592
 * bytes) that every GPU loading this library keeps until the process exits.
 * The first call on a device looks up that array's address (with the device
 * current), so make a first call before any stream capture.  The address is
 * then kept for the life of the process: after cudaDeviceReset, or after
 * the device's primary context is released and created again, the library's
 * module is loaded anew and the kept address is stale, so do not call this
 * entry point on that device again in the same process.  Calls share
 * the array: two calls that overlap on the GPU (unordered streams) race and
 * may return wrong sums. */
rd_status rd_moments_noalloc(const void* field, int32_t storage, int32_t nx, int32_t ny,
                             int32_t nz, int64_t pitch, double* out, void* stream);

/*
 * Batches: many independent instances (contexts) of the same model and
 * storage stepped together by one persistent kernel launch per T steps.
 * The launch walks a work list of (instance, x-tile, y-tile, z-chunk) items
 * across all members, so uneven grids share the GPU in one launch.  Members
 * remain ordinary contexts: rd_get_field / rd_mass work on them between
 * batch steps.
 */
typedef struct rd_batch rd_batch;

/* Create an empty batch for one model and storage kind. */
rd_status rd_batch_create(int32_t model, int32_t storage, rd_batch** out);
/* Add ``ctx`` (same model, storage and stencil as the members already in
 * the batch, else RD_EINVAL; at most one batch at a time). */
rd_status rd_batch_add(rd_batch* b, rd_ctx* ctx);
/* Remove ``ctx``; it becomes a standalone context again. */
rd_status rd_batch_remove(rd_batch* b, rd_ctx* ctx);
/* Number of members. */
int32_t rd_batch_size(const rd_batch* b);
/* Enqueue on ``stream`` (NULL = legacy default stream). */
rd_status rd_batch_set_stream(rd_batch* b, void* stream);
/* Tuning shared by all members (tile_q, tile_y, zchunk, tsteps, graph,
 * regcap).  Without it a batch uses one step per launch, the default tile
 * height and the z-chunk that fills the CTA slots in the fewest waves over
 * its current members. */
rd_status rd_batch_set_tuning(rd_batch* b, const rd_tuning* t);
/* Advance every member by nsteps (asynchronous).  A batch with a single
 * member steps it exactly as rd_step would (the member's own tuning), on
 * the batch's stream. */
rd_status rd_batch_step(rd_batch* b, int64_t nsteps);
/* Advance member i (in the order of rd_batch_add) by steps[i] >= 0 steps in
 * one batched launch sequence of max(steps) steps (asynchronous): a member
 * whose count is used up is left alone for the rest of the sequence (its
 * work items are skipped), so members with different counts need not be
 * stepped in separate calls.  Results equal rd_batch_step of each member
 * alone bit for bit.  Needs one step per launch in the batch's tuning
 * (RD_EINVAL otherwise, and for a negative count or a NULL array). */
rd_status rd_batch_step_each(rd_batch* b, const int64_t* steps);
/* Wait for the batch's stream. */
rd_status rd_batch_sync(rd_batch* b);
/* Destroy the batch (members are left intact and detached). */
rd_status rd_batch_destroy(rd_batch* b);
int64_t rd_batch_launch_count(const rd_batch* b);

#ifdef __cplusplus
}
#endif
#endif /* RD_H */
