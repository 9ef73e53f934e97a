/*
 * pplbm.h -- C ABI of the GB300 (sm_103a) pseudopotential lattice Boltzmann
 * library: the per-time-step update of a D2Q9 lattice with the
 * nearest-neighbour "force approach" of Czelusniak et al., arXiv 2003.07968.
 *
 * One time step (Eq. TLBE) on a periodic nx x ny lattice:
 *   rho   = sum_i f_i                                   Eq. (FD)
 *   psi   = sqrt((P_EOS(rho) - c_s^2 rho) / G)          Eqs. (DED), (CSEOS)
 *   M1,M2 = psi moments over the 3x3 neighbourhood      Eqs. (FOMED), (SOMED)
 *   F     = F^SC - 3/4 eps c_s^2 G F1 + (sigma-1) c_s^2 G F2
 *                                                       Eqs. (SCF), (DFTCCC),
 *                                                       (DFTCST), (IFT)
 *   u     = (sum_i f_i c_i + F/2) / rho                 Eq. (FMD)
 *   f_i(x + c_i, t + 1) = f_i - (f_i - f_i^eq)/tau + (1 - 1/(2 tau)) S_i
 *                                                       Eqs. (BGKCO), (SEDF),
 *                                                       (GFS), (GFSBGK)
 * D2Q9 velocities and weights: Eq. (VelocitySet) and the text after Eq. (SEDF).
 *
 * Conventions for every entry point:
 *   - All functions return an int status: LBM_OK (0), LBM_PENDING (1), or a
 *     negative LBM_ERR_* code.  No C++ exception crosses this boundary: a
 *     host allocation that fails inside a call returns LBM_ERR_OOM, any other
 *     internal exception LBM_ERR_STATE.  If the server's worker thread meets
 *     one, every request fails with LBM_ERR_STATE and lbm_submit refuses
 *     new ones.
 *   - Host arrays are owned by the caller and only borrowed for the call.
 *     Fields are row-major [ny][nx] FP64 (x fastest).
 *   - Device memory and streams are owned by the handle.  Device memory comes
 *     from the allocator in lbm_runtime_opts (e.g. a PyTorch caching
 *     allocator), else from cudaMalloc.
 *   - Work is queued on the handle's stream (the caller's, if given).
 *     lbm_step returns once the work is queued.  lbm_moments, lbm_sync and
 *     lbm_destroy wait for it.  A numeric fault found on the device
 *     (psi undefined: rho <= 0, b rho >= 1 or a negative radicand in Eq. DED)
 *     is reported as LBM_ERR_NUMERIC by the next lbm_sync / lbm_moments /
 *     lbm_step, with the lattice index available from lbm_status_detail.
 *   - A handle is used by one host thread at a time.
 */
#ifndef PPLBM_H
#define PPLBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes -------------------------------------------------------- */
#define LBM_OK 0
#define LBM_PENDING 1
#define LBM_ERR_ARG (-1)            /* invalid argument                         */
#define LBM_ERR_OOM (-2)            /* device or host allocation failed         */
#define LBM_ERR_CUDA (-3)           /* CUDA runtime error (see lbm_last_error)  */
#define LBM_ERR_NUMERIC (-4)        /* psi undefined somewhere (see above)      */
#define LBM_ERR_TIMEOUT (-5)        /* a bounded device wait ran out            */
#define LBM_ERR_STATE (-6)          /* call not valid in the handle's state     */
#define LBM_ERR_UNKNOWN_TICKET (-7) /* lbm_poll of a ticket never issued        */
#define LBM_ERR_CAPACITY (-8)       /* request larger than the server can hold  */

/* ---- population storage (precision forms) -------------------------------- */
/* Every form stores rest-referenced deviations: per site, plane 0 holds
 * R = f_0 - w_0 rho0 and plane i (1..8) holds (f_i - w_i rho0) - (w_i/w_0) R
 * plus a share of R's rounding, so that eight of the nine stored numbers are
 * small and a site's stored mass, rho0 + 9/4 R + sum_i (plane i), is exact
 * to roundings of small numbers.  The forms differ in element type and rho0. */
#define LBM_STORE_F32 0     /* FP32, rho0 = 0                                    */
#define LBM_STORE_F32_DEV 1 /* FP32, rho0 from the descriptor or automatic       */
#define LBM_STORE_F16_DEV 2 /* FP16 (IEEE binary16), rho0 as LBM_STORE_F32_DEV   */

/* ---- arithmetic of psi / Eq. (CSEOS) ------------------------------------- */
#define LBM_EOS_F64 0 /* native FP64                                             */
#define LBM_EOS_DF 1  /* float-float pairs (about 43 significant bits on the
                          radicand), FP32 psi                                  */
#define LBM_EOS_F32 2 /* FP32                                                    */

/* ---- equation of state behind psi, Eq. (DED) ----------------------------- */
#define LBM_EOS_KIND_CS 0  /* Carnahan-Starling, Eq. (CSEOS):
                              P = k [c rho T (1 + b rho + (b rho)^2 - (b rho)^3)
                                     / (1 - b rho)^3 - a rho^2]              */
#define LBM_EOS_KIND_VDW 1 /* van der Waals in the same constants:
                              P = k [c rho T / (1 - b rho) - a rho^2]; with
                              a = 3, b = 1/3, c = 8/3 the reduced equation,
                              critical point rho = T = 1, P = k              */

/* ---- collision operator -------------------------------------------------- */
#define LBM_COLL_BGK 0 /* Eq. (BGKCO) with Guo forcing Eq. (GFSBGK)            */
#define LBM_COLL_MRT 1 /* Eq. (MRTCO), Gram-Schmidt M of Appendix A, Eq. (GFSMRT) */

/* ---- kernel variant ------------------------------------------------------ */
#define LBM_KERNEL_AUTO 0  /* per pass, the variant and tile measured fastest
                              on GB300 (or found by lbm_autotune): the single
                              pass uses the TMA kernel with 32x16 tiles where
                              the population arena can be one tensor (one
                              lattice, or a batch in one row space), else
                              plain loads with 32x8 tiles                    */
#define LBM_KERNEL_PLAIN 1 /* plain global loads, 1, 2 or 4 sites per thread
                              (with 2 or 4, site pairs share the paired FP32
                              instructions); tile_x a multiple of 32,
                              tile_y a multiple of the sites per thread,
                              tile_x*tile_y/sites_per_thread <= 512          */
#define LBM_KERNEL_TMA 2   /* tiles staged in shared memory by TMA bulk copies
                              through a warp-specialised mbarrier pipeline
                              (one producer warp, eight consumer warps);
                              single pass: tiles 64x8, 32x16, 64x16, 128x8;
                              two-pass: 64x8, 64x16, 128x4, 128x8, 32x16   */

/* ---- step schedule ------------------------------------------------------- */
#define LBM_SCHED_AUTO 0     /* the faster schedule on GB300: LBM_SCHED_FUSED
                                (two-pass for TMA tiles of a two-pass-only
                                shape)                                         */
#define LBM_SCHED_TWO_PASS 1 /* psi pass, then fused force+collide+pull pass    */
#define LBM_SCHED_FUSED 2    /* one pass per step: each tile rebuilds psi on a
                                one-site ring from populations pulled up to two
                                sites out; 72 instead of 116 bytes per FP32 site */

/* One lattice.  Defaults (lbm_desc_default): tau = 1, G = -1, eps = 1.73,
 * sigma = 1, T = 0.8, a/b/c/k = 3.852462257 / 0.1304438842 / 2.785855166 /
 * 0.01 (Sec. IV.A), rho0 = -1 (automatic), LBM_STORE_F32_DEV, LBM_EOS_DF,
 * direct trace, BGK, MRT rates diag(1,1,1,1,1,1,1,1/tau,1/tau) (Eq. RM),
 * LBM_EOS_KIND_CS.  For LBM_EOS_KIND_VDW set a, b, c as well (3, 1/3, 8/3
 * for the reduced van der Waals equation). */
typedef struct {
    int32_t nx, ny;           /* lattice size, each >= 2                        */
    double tau;               /* relaxation time, > 0.5                         */
    double G;                 /* interaction parameter (sign keeps psi real)    */
    double eps, sigma;        /* Eq. (IFT)                                       */
    double T;                 /* reduced temperature in Eq. (CSEOS)             */
    double eos_a, eos_b, eos_c, eos_k;
    double rho0;              /* reference density of deviation storage; < 0:
                                 automatic, the smallest density of the field
                                 given to lbm_init (ignored by LBM_STORE_F32)   */
    int32_t storage;          /* LBM_STORE_*                                     */
    int32_t eos_precision;    /* LBM_EOS_*                                       */
    int32_t m2_trace_variant; /* 0: M2_bb direct trace (Eq. SOMED);
                                 1: 2 c_s^2 (M0 - psi) (text after Eq. DFTCST)  */
    int32_t collision;        /* LBM_COLL_*                                      */
    double mrt_rates[9];      /* diagonal of Lambda (Eq. RelaxationMatrix)      */
    int32_t eos_kind;         /* LBM_EOS_KIND_*; may differ between lattices    */
} lbm_lattice_desc;

/* Optional runtime settings; pass NULL for defaults. */
typedef struct {
    /* Device allocator: alloc returns a device pointer aligned to >= 256 bytes,
       or NULL on failure; free releases it.  Both NULL: cudaMalloc/cudaFree. */
    void* (*alloc)(size_t bytes, void* ctx);
    void (*free)(void* ptr, size_t bytes, void* ctx);
    void* alloc_ctx;
    void* stream;      /* cudaStream_t to queue work on; NULL: a private stream */
    int32_t tile_x;    /* tile width in sites (0: tuned/default)               */
    int32_t tile_y;    /* tile height in sites (0: tuned/default)              */
    int32_t grid_ctas; /* CTAs of the persistent launches (0: SMs x occupancy) */
    int32_t schedule;  /* LBM_SCHED_*                                          */
    int32_t graph_steps; /* steps per captured CUDA graph (0: default, <0: off) */
    int32_t kernel_variant; /* LBM_KERNEL_*                                   */
    int32_t sites_per_thread; /* with tile_x/tile_y: 1, 2 or 4 (0: 1)          */
} lbm_runtime_opts;

typedef struct lbm_handle lbm_handle;

/* Fill *d with the defaults listed above for an nx x ny lattice. */
void lbm_desc_default(lbm_lattice_desc* d, int32_t nx, int32_t ny);

/* Create a handle over n_lattices independent lattices (n_lattices = 1: one
 * lattice; > 1: a batch stepped together in persistent launches over one tile
 * list).  All lattices of a handle share storage, eos_precision, collision
 * and m2_trace_variant; tau, G, eps, sigma, T, EOS constants, rho0 and the
 * MRT rates may differ per lattice.  MRT runs in the plain-load kernels and
 * in the single-pass TMA kernel (the two-pass schedule with
 * kernel_variant LBM_KERNEL_TMA and MRT is refused).  Allocates all device
 * memory now.
 * Errors: LBM_ERR_ARG (bad sizes/params, mixed storage), LBM_ERR_OOM,
 * LBM_ERR_CUDA.  *out is NULL on error. */
int lbm_create(const lbm_lattice_desc* descs, int32_t n_lattices,
               const lbm_runtime_opts* opts, lbm_handle** out);

/* Initialise one lattice at equilibrium, f_i = f_i^eq(rho, u) (the
 * initialisation described after Eq. ISD).  rho, ux, uy: host [ny][nx] FP64,
 * ux/uy may be NULL (zero velocity).  Copies the fields in, then returns
 * with the work queued.  Errors: LBM_ERR_ARG (also for a density that is not
 * finite), LBM_ERR_CUDA. */
int lbm_init(lbm_handle* h, int32_t lattice, const double* rho, const double* ux,
             const double* uy);

/* Advance every lattice of the handle by nsteps >= 0 time steps.  Queues the
 * work and returns.  Reports an earlier numeric fault if one is already
 * known.  Errors: LBM_ERR_ARG, LBM_ERR_CUDA, LBM_ERR_NUMERIC. */
int lbm_step(lbm_handle* h, int64_t nsteps);

/* Macroscopic fields of one lattice at the current time: rho (Eq. FD), the
 * force-shifted velocity (Eq. FMD) and the total mass sum_x rho.  Each
 * site's nine stored values are summed as a float-float pair and the
 * result is FP64 (within 2^-42 of the largest partial sum of the exact sum
 * of the stored values); the mass is an FP64 sum of those site sums.  Host outputs are
 * row-major [ny][nx]; any output may be NULL.  Velocities need psi and the
 * force (one extra pass); rho and the mass alone do not.  Waits for queued
 * work.  Errors: LBM_ERR_ARG, LBM_ERR_CUDA, LBM_ERR_NUMERIC. */
int lbm_moments(lbm_handle* h, int32_t lattice, double* rho, double* ux, double* uy,
                double* mass);

/* Total mass of one lattice (FP64 sum of the stored populations) into *mass.
 * Waits.  Errors: LBM_ERR_ARG, LBM_ERR_CUDA. */
int lbm_mass(lbm_handle* h, int32_t lattice, double* mass);

/* Wait for all queued work; returns LBM_ERR_NUMERIC if a numeric fault was
 * flagged, LBM_ERR_CUDA on a CUDA error, else LBM_OK. */
int lbm_sync(lbm_handle* h);

/* Index of the first lattice with a numeric fault, or -1. */
int lbm_status_detail(lbm_handle* h, int32_t* lattice);

/* Release everything (waits for queued work first).  NULL is ignored. */
void lbm_destroy(lbm_handle* h);

/* Static text for a status code. */
const char* lbm_strerror(int code);

/* Text of the handle's last CUDA or argument error ("" if none).  The string
 * belongs to the handle and lives until the next call on it. */
const char* lbm_last_error(lbm_handle* h);

/* ---- measurement and tuning --------------------------------------------- */

/* Record CUDA events around every kernel launch from now on (on = 1) or stop
 * (on = 0).  Launches are not captured into graphs while recording. */
int lbm_profile(lbm_handle* h, int32_t on);

typedef struct {
    char name[32];      /* kernel name                                         */
    int64_t launches;   /* launches recorded                                   */
    double total_ms;    /* summed event time                                   */
    double bytes_per_launch; /* algorithmic bytes one launch moves            */
} lbm_kernel_stat;

/* Waits, then reads the per-kernel records since lbm_profile(h, 1) into
 * out[0..max), returning the number of kernels in *n. */
int lbm_profile_read(lbm_handle* h, lbm_kernel_stat* out, int32_t max, int32_t* n);

/* Number of kernels this handle has launched so far (graph replays count
 * each contained kernel). */
int64_t lbm_launch_count(lbm_handle* h);

/* Handle facts: sites, device bytes held, and per pass (psi pass, collision
 * pass) the kernel variant, tile shape, tile count and grid. */
typedef struct {
    int64_t sites;
    int64_t device_bytes;
    int32_t tile_x, tile_y, n_tiles, grid_ctas;                 /* collision pass */
    int32_t psi_tile_x, psi_tile_y, psi_n_tiles, psi_grid_ctas; /* psi pass       */
    int32_t psi_variant, collide_variant;                       /* LBM_KERNEL_*   */
    int32_t schedule;
    int32_t n_lattices;
    int32_t spt, psi_spt;     /* sites per thread, collision / psi pass         */
    int32_t tensor_map;       /* 1: the single-pass TMA kernel fills each stage
                                 with one tensor copy per tile (else row copies) */
} lbm_info_t;
int lbm_info(lbm_handle* h, lbm_info_t* out);

/* Autotune each pass on this handle's lattices: kernel variant (unless the
 * handle was created with a fixed one), tile shape and grid (persistent or
 * one CTA per tile), timed with CUDA events over repeated trial launches
 * that leave the state unchanged.  Keeps the fastest per pass; results are
 * cached per device, storage, EOS arithmetic and size class for the life of
 * the process and used by later lbm_create calls.  Errors: LBM_ERR_CUDA. */
int lbm_autotune(lbm_handle* h, int32_t repeats);

/* ---- serving: continuous batching --------------------------------------- */
/* A server keeps many independent lattices (requests) resident in one
 * device arena and steps all of them together: every chunk of steps is one
 * pair of launches per step over a tile list that spans every resident
 * lattice (the same kernels as a batch handle).  Requests are admitted at
 * chunk boundaries, first come first served but skipping any that do not
 * fit yet, whenever a slot and arena space (HBM footprint: both population
 * buffers at the arena's common pitch, plus psi) are free and the resident
 * sites stay below a target; a
 * chunk runs each lattice for min(k, its remaining steps), where k is the
 * number of steps that fills about chunk_ms of GPU time at the throughput
 * measured on earlier chunks (CUDA event timings), capped at chunk_steps.
 * Short chunks keep admission and completion close to the request's own
 * work when the GPU is lightly loaded.  The
 * worker keeps two chunks in flight: new requests' fields are uploaded
 * from pinned memory on their own stream while a chunk runs, the next
 * chunk is queued before the previous one is retired, and a finished
 * lattice's moments are copied out to pinned memory while the next chunk
 * runs; its space is then reused.  lbm_submit copies the field into a
 * pinned slot (on the caller's thread) when one is free, and lbm_poll
 * copies the result from its pinned slot, so the worker thread that drives
 * the GPU does no large host copies.  The submit and poll calls are
 * thread-safe and never wait for the GPU.  The numerics of a request do not
 * depend on what else is resident. */
typedef struct lbm_server lbm_server;

typedef struct {
    size_t arena_bytes;       /* device bytes for resident lattices (0: 8 GiB)    */
    int32_t max_resident;     /* resident lattices at most (0: 1024)              */
    int32_t chunk_steps;      /* most steps between admission points (0: 100)     */
    int64_t max_request_sites;/* largest nx*ny accepted (0: 2048*2048)            */
    int64_t target_resident_sites; /* admit while resident sites stay below this
                                 (0: 16 Mi); enough to keep the GPU busy,
                                 small enough to keep latency close to FIFO      */
    int32_t storage;          /* LBM_STORE_* of every request                     */
    int32_t eos_precision;    /* LBM_EOS_* of every request                       */
    int32_t kernel_variant;   /* LBM_KERNEL_AUTO (single pass: the TMA kernel,
                                 32x16 tiles), LBM_KERNEL_TMA or LBM_KERNEL_PLAIN */
    int32_t schedule;         /* LBM_SCHED_* (AUTO: single pass)                  */
    int32_t tile_x, tile_y;   /* 0: defaults; else both passes                    */
    int32_t sites_per_thread; /* with tile_x/tile_y: 1, 2 or 4 (0: 1)              */
    int32_t with_velocity;    /* 1 (default): results carry ux, uy; 0: rho only
                                 (lbm_poll then fills ux, uy with NaN)           */
    int32_t max_width;        /* widest nx accepted (0: 2048).  The arena holds
                                 every resident lattice at the pitch of this
                                 width (its ny + 4 rows in each of 18 planes, a
                                 ninth of the arena for psi), so that one tensor
                                 map covers them all for the TMA single pass    */
    double chunk_ms;          /* GPU time a chunk aims at (0: 4 ms; < 0: every
                                 chunk runs chunk_steps steps)                   */
    /* Device allocator for the arena, staging and tables, as in
       lbm_runtime_opts: alloc returns a device pointer aligned to >= 256
       bytes, or NULL on failure (lbm_server_create then fails with
       LBM_ERR_OOM after freeing what it took; a table that grows later fails
       the requests of that chunk); free releases it.  Both NULL:
       cudaMalloc/cudaFree.  Called from the creating thread and from the
       server's worker thread; it must outlive the server.  Pinned host
       buffers always come from cudaMallocHost. */
    void* (*alloc)(size_t bytes, void* ctx);
    void (*free)(void* ptr, size_t bytes, void* ctx);
    void* alloc_ctx;
} lbm_server_opts;

typedef struct {
    int64_t submitted, completed, failed;
    int32_t queued, resident;
    int64_t site_steps;       /* lattice-site updates done                       */
    double busy_s;            /* GPU time of the chunks (CUDA event timings)     */
    int64_t arena_bytes, arena_in_use;
    int64_t launches;         /* kernels launched by the worker                  */
} lbm_server_stats;

/* Fill *o with the defaults above (FP32 deviation storage, float-float EOS). */
void lbm_server_opts_default(lbm_server_opts* o);

/* Create a server on the current device: allocates the arena, staging and
 * tables with cudaMalloc and starts the worker thread.
 * Errors: LBM_ERR_ARG, LBM_ERR_OOM, LBM_ERR_CUDA. */
int lbm_server_create(const lbm_server_opts* opts, lbm_server** out);

/* Queue one solve: a BGK lattice `d` (its storage and eos_precision are
 * replaced by the server's), initial density rho (host [ny][nx] FP64, copied before
 * return, u = 0), nsteps >= 1 time steps.  Thread-safe; never waits for the
 * GPU.  *ticket identifies the request.  Errors: LBM_ERR_ARG (bad desc or
 * nsteps), LBM_ERR_CAPACITY (the lattice can never fit: larger than the
 * arena or than max_request_sites), LBM_ERR_STATE (server shutting down). */
int lbm_submit(lbm_server* s, const lbm_lattice_desc* d, const double* rho, int64_t nsteps,
               uint64_t* ticket);

/* Result of a request: LBM_PENDING while queued or running; once done,
 * copies rho, ux, uy (host [ny][nx] FP64, any may be NULL) of the final state
 * (Eqs. FD, FMD) and the submit-to-done time in seconds, forgets the ticket
 * and returns LBM_OK, or the request's error (LBM_ERR_NUMERIC if psi became
 * undefined).  Thread-safe.  Errors: LBM_ERR_UNKNOWN_TICKET. */
int lbm_poll(lbm_server* s, uint64_t ticket, double* rho, double* ux, double* uy,
             double* latency_s);

/* Counters of the server so far.  Thread-safe. */
int lbm_server_get_stats(lbm_server* s, lbm_server_stats* out);

/* Stop the worker (finishing the chunk in flight), free everything.  Pending
 * requests are dropped.  No other call on this server may be in progress or
 * follow (submit and poll are thread-safe among themselves, not against
 * destroy).  NULL is ignored. */
void lbm_server_destroy(lbm_server* s);

/* ---- mass without allocation ------------------------------------------- */
/* The paper has no counterpart to this entry point.  It serves callers that
 * may not allocate device memory at the moment they want a mass check:
 * applications that reserve all device memory up front through their own
 * allocator and forbid later allocations, and real-time loops that must not
 * take an allocator's locks or wait for it.
 *
 * Writes to *mass_out (device pointer, caller-owned) the FP64 sum of
 * `count` FP32 values at `values` (device pointer, caller-owned, dense: every
 * value in [values, values + count) is added, so a pitched array would add
 * its padding too) plus `offset`, e.g. a density field the caller holds in
 * FP32.  A handle's stored population planes are not such values: they hold
 * rest-referenced deviations whose mass needs weights (lbm_mass gives it).
 * Queued on `stream` (cudaStream_t, NULL = the legacy default stream);
 * returns once queued.
 * Allocates nothing: its partial sums live in a fixed array in the
 * library's own device memory, 2 MiB on every GPU that loads the library,
 * held until the process exits.  That array limits `count` to
 * LBM_NOALLOC_MAX_COUNT values (4 GiB of FP32); larger requests fail with
 * LBM_ERR_CAPACITY before any GPU work.  The first call on a device looks up
 * the array's device address (the host only sees a stand-in for the
 * symbol) and keeps it for the life of the process: do not use the entry
 * point on a device after a reset of it (cudaDeviceReset), whose new
 * context would not hold that address.  Every call uses the same array, so calls whose kernels
 * overlap on the GPU race; order them on one stream.  Errors: LBM_ERR_ARG
 * (NULL pointer, count < 1), LBM_ERR_CAPACITY, LBM_ERR_CUDA. */
#define LBM_NOALLOC_MAX_COUNT 1073741824LL
int lbm_mass_noalloc(const float* values, int64_t count, double offset, double* mass_out,
                     void* stream);

/* Failure-detection test of the single pass (schedule LBM_SCHED_FUSED on the
 * TMA kernel): the next time step skips the shared-memory staging copy of
 * tile `tile` (0 <= tile < the pass's tile count, lbm_info n_tiles), so the
 * consumers' bounded wait for it runs out (that launch's waits are limited
 * to 2e8 SM cycles, about 0.1 s at 2 GHz; other launches wait up to 4e9
 * cycles, about 2 s), every consumer of that CTA leaves together and the producer drains
 * its copies (bounded too).  No kernel traps or hangs; the step's results
 * are garbage and the next lbm_sync reports LBM_ERR_TIMEOUT with the lattice
 * in lbm_status_detail.  lbm_init of that lattice clears the fault, and the
 * handle goes on.  Arms one launch; no CUDA graph replays it.
 * Errors: LBM_ERR_ARG (no handle, another schedule or kernel, tile out of
 * range). */
int lbm_inject_copy_timeout(lbm_handle* h, int32_t tile);

/* The reciprocal and square root of the step kernels (the hardware
 * approximations, each refined by one Newton-Raphson step on the paired FP32
 * pipe; used by the float-float EOS, Eqs. DED and CSEOS, and by the velocity of
 * Eq. FMD), applied on the current device to n host values x (1 <= n <= 2^24):
 * rcp[i] = the kernels' 1/x[i], sq[i] = their sqrt(x[i]) (meaningful for
 * normal x[i] > 0, resp. finite x[i] >= 0).  Caller-owned host arrays of n
 * floats.  For tests of their error bounds against correctly rounded
 * results.  Also runs each value through the one-value (scalar) lane and
 * returns LBM_ERR_STATE if any result differs in a bit from the paired lane.
 * Errors: LBM_ERR_ARG, LBM_ERR_OOM, LBM_ERR_CUDA, LBM_ERR_STATE. */
int lbm_selfcheck_arith(const float* x, int64_t n, float* rcp, float* sq);

/* psi of Eq. (DED) (with Eq. CSEOS or the van der Waals equation, as
 * d->eos_kind says) exactly as the step kernels evaluate it, in the
 * arithmetic d->eos_precision names and with the lattice constants that
 * lbm_create derives from *d, for n host densities rho (1 <= n <= 2^24,
 * FP32, the type the kernels hold rho in): psi[i] (NaN where psi is not
 * defined: rho <= 0, b rho >= 1 or a negative radicand) and, for
 * LBM_EOS_DF, radicand[i] = psi^2 before its one rounding to FP32, in FP64
 * (NaN for the other arithmetics).  Caller-owned host arrays of n values.
 * For tests of the EOS arithmetic against an FP64 evaluation.  Also runs
 * each value through the one-value (scalar) lane and returns LBM_ERR_STATE
 * if any psi differs in a bit from the paired lane.
 * Errors: LBM_ERR_ARG (bad descriptor or sizes), LBM_ERR_OOM, LBM_ERR_CUDA,
 * LBM_ERR_STATE. */
int lbm_selfcheck_psi(const lbm_lattice_desc* d, const float* rho, int64_t n, float* psi,
                      double* radicand);

/* Host-only consistency proof of the shared-memory staging used by the
 * LBM_KERNEL_TMA passes (two-pass and single-pass plans): for a set of
 * lattice shapes, every tile shape, both storages and both population
 * buffers, each bulk copy is 16-byte aligned
 * on both sides, has a size that is a multiple of 16 bytes, stays inside
 * its lattice's allocation and its shared-memory box, and the copies cover
 * every value an active site (and, single pass, a ring cell) reads.  Writes a one-line report.  Needs no GPU.
 * Returns LBM_OK, or LBM_ERR_STATE with the first violation in the report. */
int lbm_selfcheck(char* report, int32_t report_len);

#ifdef __cplusplus
}
#endif
#endif /* PPLBM_H */
