/*
 * lbm_gb300.h -- C ABI of the GB300 fused D3Q19 lattice Boltzmann library for
 * pressure-driven flow through periodic sphere packs (Fattahi et al., "Pore-scale
 * lattice Boltzmann simulation of laminar and turbulent flow through a sphere pack",
 * arXiv:1508.02960).
 *
 * One time step (Sec. 2, Eqs. collision and streaming, streamed first then collided)
 * is one fused kernel: pull streaming with the periodic pressure-drop shift (Sec.
 * 2.2.2, Eqs. Periodicfunkown and PeriodicfunkownRight), solid-wall handling by simple
 * bounce-back (Eq. noslip) or central linear interpolation (Eq. CLI), moments (Eq.
 * Macro), incompressible equilibrium (Eq. equilibrium) and SRT, TRT or MRT relaxation
 * (Eqs. SRT, TRT, MRT).  An FP64 reduction of the volume-averaged velocity follows;
 * the host turns it into permeability (Eq. Darcy), Forchheimer coefficient (Eq.
 * Forchheimer) and friction factor (Eq. frictionFactor).
 *
 * Conventions
 *  - Lattice units.  Box nx * ny * nz, periodic in all three directions, flow along +x
 *    from the high-density left boundary (rho_L = rho_R + delta_rho, Eq.
 *    generalPeriodicRho).  Cell (i, j, k) has centre (i + 1/2, j + 1/2, k + 1/2).
 *  - Cell index: x + nx * (y + ny * z).  Scalar host fields are [nz][ny][nx]; population
 *    host fields are [19][nz][ny][nx] in this direction order (opposites adjacent):
 *      0:(0,0,0)  1:(1,0,0) 2:(-1,0,0) 3:(0,1,0) 4:(0,-1,0) 5:(0,0,1) 6:(0,0,-1)
 *      7:(1,1,0) 8:(-1,-1,0) 9:(1,-1,0) 10:(-1,1,0) 11:(1,0,1) 12:(-1,0,-1)
 *      13:(1,0,-1) 14:(-1,0,1) 15:(0,1,1) 16:(0,-1,-1) 17:(0,1,-1) 18:(0,-1,1)
 *    Weights 1/3 (rest), 1/18 (axis), 1/36 (diagonal).
 *  - Ownership.  Every input array is copied during the call that receives it.  The
 *    library owns all device memory of a context, a batch and a server; host output
 *    buffers are allocated by the caller.  Device work is queued on the CUDA stream
 *    given at creation (NULL = the legacy default stream).
 *  - Errors.  Every call returns an lbm_status; nothing throws or aborts across the
 *    ABI.  lbm_last_error() returns a thread-local message for the last failure.
 *  - Threading.  A context or batch is used by one thread at a time.  A server is
 *    internally synchronised.
 */
#ifndef LBM_GB300_H
#define LBM_GB300_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define LBM_API __attribute__((visibility("default")))
#else
#define LBM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LBM_OK = 0,
    LBM_ERR_ARG = -1,           /* invalid argument or descriptor */
    LBM_ERR_NO_MEMORY = -2,     /* device or host allocation failed, or over budget */
    LBM_ERR_CUDA = -3,          /* a CUDA runtime call failed */
    LBM_ERR_DIVERGED = -4,      /* non-finite moments or |u| > 1 seen by a reduction */
    LBM_ERR_NOT_CONVERGED = -5, /* max_steps reached before the convergence test passed */
    LBM_ERR_TIMEOUT = -6,       /* a bounded wait ran out */
    LBM_ERR_STATE = -7,         /* call not valid in the object's current state */
    LBM_ERR_IO = -8,            /* checkpoint file could not be read or written */
    LBM_ERR_CANCELLED = -9,     /* a served request was cancelled (lbm_server_cancel) */
    LBM_ERR_BOUNDS = -10        /* checked build: a kernel met an index outside its arrays */
} lbm_status;

/* Collision operator (Sec. 2.1). */
enum { LBM_SRT = 0, LBM_TRT = 1, LBM_MRT = 2 };
/* Solid-wall rule (Sec. 2.2.1): simple bounce-back, central linear interpolation. */
/* Wall rules of Sec. 2.2.1: simple bounce-back (Eq. noslip), central linear interpolation
 * (Eq. CLI), linear and quadratic interpolation bounce-back (Eqs. LIBB, QIBB),
 * interpolation/extrapolation bounce-back (Eqs. fstar, IEBB) and multi-reflection (Eq. MR).
 * LIBB, QIBB, IEBB and MR need the A-B layout; IEBB needs tau != 2.  Where a node a rule
 * reads is solid it falls back: to SBB when x_f2 is solid, QIBB to LIBB and MR to CLI when
 * only x_f3 is. */
enum { LBM_SBB = 0, LBM_CLI = 1, LBM_LIBB = 2, LBM_QIBB = 3, LBM_IEBB = 4, LBM_MR = 5 };
/* Population storage.  All formats store the deviation f_k - w_k rho0; FP64 and FP32
 * compute in their own precision, FP16/BF16 compute in FP32.  FP16DEV stores the
 * deviation times 2^dev_scale_log2. */
enum { LBM_F64 = 0, LBM_F32 = 1, LBM_F16DEV = 2, LBM_BF16DEV = 3 };
/* Memory layout: two buffers (A-B), or one buffer updated in place (AA pattern). */
enum { LBM_LAYOUT_AB = 0, LBM_LAYOUT_AA = 1 };

#define LBM_DEV_SCALE_AUTO (-1000)
#define LBM_BLOCK_AUTO (-1)

typedef struct {
    double cx, cy, cz, r; /* centre and radius in lattice units */
} lbm_sphere;

/* Problem description (Sec. 2 and 3: geometry, viscosity, pressure drop, collision
 * operator, wall rule).  Zero-initialise it and set what is needed. */
typedef struct {
    int32_t nx, ny, nz;         /* periodic box, each >= 1 */
    int32_t n_spheres;          /* number of entries of spheres */
    const lbm_sphere *spheres;  /* sphere pack (minimum-image periodic); or NULL */
    const uint8_t *flags;       /* used when spheres == NULL: [nz][ny][nx], 1 = solid */
    const double *q;            /* with flags and CLI: [19][nz][ny][nx] wall distance of the
                                   link from a fluid cell along e_k into a solid cell, in
                                   (0, 1]; other entries ignored.  NULL = 1/2 everywhere */
    double tau;                 /* relaxation time, > 1/2; nu = (tau - 1/2)/3 */
    double delta_rho;           /* periodic density drop across the box in x */
    double rho0;                /* mean density; 0 means 1 */
    double magic_lambda;        /* TRT magic parameter Lambda; 0 means 3/16 */
    double mrt_energy_ratio;    /* MRT: (1/s_nu - 1/2)/(1/s_e - 1/2); 0 means 4.6 */
    const double *mrt_rates;    /* MRT: optional 19 explicit rates s_0..s_18 (copied) */
    int32_t collision;          /* LBM_SRT / LBM_TRT / LBM_MRT */
    int32_t wall;               /* LBM_SBB, LBM_CLI, LBM_LIBB, LBM_QIBB, LBM_IEBB, LBM_MR */
    int32_t storage;            /* LBM_F64 / LBM_F32 / LBM_F16DEV / LBM_BF16DEV */
    int32_t layout;             /* LBM_LAYOUT_AB / LBM_LAYOUT_AA */
    int32_t dev_scale_log2;     /* FP16DEV scale exponent; LBM_DEV_SCALE_AUTO = from delta_rho */
    int32_t block_cells;        /* step kernel: 0 or 128 = tiles of 128 fluid cells (default);
                                   256 = bricks of 32 x 2 x 4 cells staged by TMA (single A-B
                                   instance; nx, ny, nz multiples of 32, 2, 4);
                                   LBM_BLOCK_AUTO = the faster of the two, measured at
                                   creation (see lbm_create) */
    double d_p;                 /* particle diameter of Re_p; 0 = volume-mean sphere diameter */
    double perturb_u;           /* lbm_init_equilibrium: amplitude of a seeded random initial
                                   velocity (0 = fluid at rest) */
    uint64_t seed;              /* seed of that perturbation */
} lbm_desc;

/* Observables after the last completed step (Secs. 1 and 4), lattice units. */
typedef struct {
    double U_sup;     /* sum over fluid cells of u_x / (nx ny nz): volume-averaged velocity */
    double U_int;     /* sum over fluid cells of u_x / n_fluid: intrinsic average */
    double mass;      /* sum over fluid cells of rho */
    double porosity;  /* n_fluid / (nx ny nz) */
    double K;         /* permeability mu U_sup / (delta_p / L_x), delta_p = delta_rho / 3 */
    double K_app;     /* apparent permeability (= K, Eq. AppPer measured with Eq. Darcy) */
    double Re_p;      /* U_sup d_p / nu */
    double Re_K;      /* rho U sqrt(K_D) / mu (needs K_D) */
    double beta;      /* Forchheimer beta (needs K_D) */
    double C_F;       /* beta sqrt(K_D) */
    double F_K;       /* (delta_p / L) sqrt(K_D) / (rho U^2) */
    double u_max;     /* largest |u| seen by the last reduction (0 when not tracked) */
    double F_x, F_y, F_z; /* drag force F_D on all solids: momentum handed to the solid
                             through the cut links in the last reducing step, by momentum
                             exchange (Sec. 3); NaN when the moments came from a stored state
                             rather than a step */
    double C_D;       /* F_x / (6 pi mu U_sup r), Eq. AnalyticForce; r = sum of the sphere
                         radii (NaN for a flag-field geometry) */
    double C_D_A;     /* F_x / (rho0 A U_sup^2), A = sum of pi r^2 (Sec. 4 resolution study) */
    double K_star;    /* K_app / K_D (Eq. normalizedPermeability; needs K_D) */
    int64_t steps;    /* time steps completed */
    int64_t n_fluid;  /* fluid cells */
} lbm_obs;

/* Static facts about a context. */
typedef struct {
    int64_t n_cells, n_fluid, n_boundary, n_links, n_links_cli;
    int64_t bytes_populations; /* device bytes of population storage */
    int64_t bytes_geometry;    /* device bytes of segment, boundary and link tables */
    int64_t kernel_launches;   /* library kernels launched so far (graph nodes counted) */
    int32_t block_cells, storage, layout, collision, wall, dev_scale_log2;
    int64_t steps;
    int32_t autotune;          /* how block_cells was chosen: 0 given, 1 measured at creation,
                                  2 taken from the autotuner cache */
    int32_t pad_;
    double tune_ms_tiles;      /* autotuner: ms per step of the tile kernel (0 = not timed) */
    double tune_ms_bricks;     /* autotuner: ms per step of the brick kernel (0 = not timed) */
    /* block shape of the non-reducing SBB/CLI step of the tile kernel, tuned online by the
     * first lbm_step / lbm_batch_step call of more than 48 steps (all shapes give the same
     * state bit for bit): warps per block (4, 2 or 8; 0 = brick kernel), how it was chosen
     * (0 default, 1 timed, 2 cached for the same storage, collision, layout, instance count,
     * fluid cells and device), and ms per step of the candidates 4, 2, 8 (0 = not timed) */
    int32_t step_warps, shape_source;
    double shape_ms[3];
} lbm_info;

typedef struct lbm_ctx lbm_ctx;
typedef struct lbm_batch lbm_batch;
typedef struct lbm_server lbm_server;

/* Thread-local text of the last error ("" if none). */
LBM_API const char *lbm_last_error(void);
/* Library version string. */
LBM_API const char *lbm_version(void);

/* Create a context: validates the descriptor, copies the geometry, builds on the
 * device the solid flags (Sec. 3 voxelisation), the fluid/boundary cell tables and,
 * for every cut link, the wall distance q of Sec. 2.2.1 (computed once, as in Sec. 3),
 * and allocates the populations.  The populations are left uninitialised: call
 * lbm_init_equilibrium or lbm_set_populations_f64 next.  cuda_stream: a cudaStream_t
 * or NULL.  On failure *out is NULL.
 * With desc.block_cells = LBM_BLOCK_AUTO the step kernel is chosen by measurement. The
 * tile and brick kernels each run a few hundred steps on a temporary copy of the
 * instance, which takes as much device memory again for the duration.  The choice is
 * cached per box, fluid-cell count, storage, collision, wall, layout and device.  The
 * cache lives for the process, and also in the file named by the environment variable
 * LBM_AUTOTUNE_CACHE when it is set.  lbm_get_info reports the choice and the times. */
LBM_API lbm_status lbm_create(const lbm_desc *desc, void *cuda_stream, lbm_ctx **out);
LBM_API void lbm_destroy(lbm_ctx *ctx);

/* Set every fluid cell to f^eq(rho0, u) (Eq. equilibrium) with u = 0, or with the
 * seeded perturbation of desc.perturb_u, as the post-collision state at step 0. */
LBM_API lbm_status lbm_init_equilibrium(lbm_ctx *ctx);

/* Advance n_steps >= 0 time steps (queued on the stream; returns without waiting).
 * The last step also reduces the moments for lbm_observables. */
LBM_API lbm_status lbm_step(lbm_ctx *ctx, int64_t n_steps);

/* Step in chunks of check_interval until |U_n - U_{n-1}| / |U_n| < tol (U = U_sup after
 * each chunk), a divergence is detected, or max_steps is reached.  *steps_done (may be
 * NULL) receives the steps taken.  Returns LBM_OK, LBM_ERR_DIVERGED or
 * LBM_ERR_NOT_CONVERGED. */
LBM_API lbm_status lbm_run_to_convergence(lbm_ctx *ctx, double tol, int64_t check_interval,
                                  int64_t max_steps, int64_t *steps_done);

/* Time average (Sec. 4: volume-averaged velocity averaged over a period of the developed
 * flow, and the time-averaged drag of the resolution study): advance n_samples *
 * sample_interval steps, reduce the moments and the drag after every sample_interval steps
 * and average them in FP64; *out receives the observables of the averaged U_sup and F_D
 * (K_darcy as in lbm_observables), u_max unused, steps = steps done so far.
 * Returns LBM_ERR_DIVERGED (with the average so far) when a sample diverged. */
LBM_API lbm_status lbm_average(lbm_ctx *ctx, int64_t n_samples, int64_t sample_interval, double K_darcy,
                               lbm_obs *out);

/* Developed-flow time average (Sec. 4: the averaging starts once the drag on the spheres
 * has converged and runs over 100-150 flow-through times).  A flow-through time is
 * T = nx / U_sup steps, U_sup the volume-averaged velocity of the latest sample.
 * Spin-up: windows of one flow-through time, sampled samples_per_ft times, until the
 * window-averaged drag F_x changes by less than drag_tol (relative) from the previous
 * window, after at least min_spinup_ft and at most max_spinup_ft flow-through times.
 * Averaging: average_ft flow-through times sampled samples_per_ft times each; the moments
 * and the drag are averaged in FP64.  max_steps caps the whole run. */
typedef struct {
    double min_spinup_ft, max_spinup_ft;
    double drag_tol;
    double average_ft;
    int32_t samples_per_ft;
    int32_t reserved;
    int64_t max_steps;
} lbm_develop_opts;

typedef struct {
    lbm_obs avg;               /* observables of the averaged U and F_D (K_darcy as given) */
    double flow_through_steps; /* T at the averaged U */
    double spinup_ft;          /* flow-through times of the spin-up */
    double average_ft;         /* flow-through times averaged */
    double drag_change;        /* relative change of the window drag when spin-up ended */
    int64_t spinup_steps, average_steps;
    int32_t developed;         /* 1: the drag converged within max_spinup_ft */
    int32_t reserved;
} lbm_develop_result;

/* Returns LBM_OK (also when the drag did not converge: see developed), LBM_ERR_DIVERGED,
 * LBM_ERR_NOT_CONVERGED when max_steps ran out before the averaging ended (out holds the
 * average so far), LBM_ERR_ARG for bad options or a flow at rest (no flow-through time). */
LBM_API lbm_status lbm_run_developed(lbm_ctx *ctx, const lbm_develop_opts *opts, double K_darcy,
                                     lbm_develop_result *out);

/* Least-squares fit of the Barree-Conway apparent permeability (Eq. AppPer), normalised
 * by K_D (Eq. normalizedPermeability): K*(Re) = m + (1 - m) / (1 + (a Re)^F)^E, with
 * m = K_min / K_D in (0, 1), a = l_T / d_p (so that a Re_p = Re_T), E, F > 0, over n >= 4
 * points (re[i] > 0, kstar[i]).  init: starting guess [m, a, E, F] or NULL.  params_out[4]
 * receives [m, a, E, F], rms_out (may be NULL) the RMS residual in K*.  Host code (no GPU);
 * Levenberg-Marquardt on (logit m, ln a, ln E, ln F), deterministic. */
LBM_API lbm_status lbm_fit_barree_conway(const double *re, const double *kstar, int32_t n, const double *init,
                                         double *params_out, double *rms_out);

/* Observables of the last step (synchronises the stream).  K_darcy > 0 enables beta,
 * C_F, F_K and Re_K; K_darcy = 0 leaves them NaN.  Returns LBM_ERR_DIVERGED (with *out
 * filled) when the last reduction saw a diverged cell. */
LBM_API lbm_status lbm_observables(lbm_ctx *ctx, double K_darcy, lbm_obs *out);

/* Host-side fault injection for tests (there is no device-side fault injection): after
 * the next n device allocations made by the library succeed, the following ones fail as if
 * the device were out of memory (cudaErrorMemoryAllocation), so that every out-of-memory
 * path can be exercised without touching the GPU's state.  n < 0 (the default) disables it.
 * Process-wide; not for production use. */
LBM_API void lbm_debug_fail_alloc_after(int64_t n);

/* Features the library was compiled with.  LBM_BUILD_CHECKED: the bounds-checked build
 * (compiled with LBM_CHECKED).  There every index the step kernels use is tested against
 * the extent of its array. A failing test skips the access and sets a sticky error word,
 * and the next call that reads the reductions returns LBM_ERR_BOUNDS.  The default
 * build returns 0. */
#define LBM_BUILD_CHECKED 1u
LBM_API unsigned lbm_build_flags(void);

/* Checked build only, for tests of the checks: overwrites the first entry of the
 * context's fluid-cell work list with the index one past the last cell.  The next
 * reduction then reports LBM_ERR_BOUNDS.  The context's results are meaningless
 * afterwards; destroy it.  The default build returns LBM_ERR_STATE and changes nothing,
 * since its kernels would use such an index. */
LBM_API lbm_status lbm_debug_corrupt_worklist(lbm_ctx *ctx);

/* Host code (no GPU), for tests of the step kernels' work list: packs the fluid cells
 * cells[0 .. n_cells) (strictly increasing linear indices below 2^28, as the library lists
 * a geometry's fluid cells) into work items of 32 entries, one warp each, as a context
 * does.  A 32-cell segment of the box (cells 32s .. 32s+31) that is all fluid is an item of
 * its own; the fluid cells of the other segments are packed up to 32 to an item in cell
 * order, an item spanning at most 449 consecutive cells.  A padding entry is 0xFFFFFFFF
 * and follows the item's cells.  Writes *n_items always.  If out_cap >= 32 * *n_items it
 * also writes the 32 * *n_items entries to out (caller-owned). Otherwise it returns
 * LBM_ERR_ARG, as it does for NULL or unordered input. */
LBM_API lbm_status lbm_debug_pack_work_items(const uint32_t *cells, int64_t n_cells, uint32_t *out, int64_t out_cap,
                                             int64_t *n_items);

/* FP64 sums over fluid cells of (rho - rho0, u_x, u_y, u_z), computed now from the
 * stored post-collision populations (synchronises).  sums: host array of 4. */
LBM_API lbm_status lbm_moment_sums(lbm_ctx *ctx, double *sums);

/* Copy out / in the post-collision populations f_k (not deviations) as FP64
 * [19][nz][ny][nx].  Export writes 0 for solid cells; import ignores them.  In AA
 * layout the in-place storage is unswapped on export.  Both synchronise. */
LBM_API lbm_status lbm_get_populations_f64(lbm_ctx *ctx, double *host_out);
LBM_API lbm_status lbm_set_populations_f64(lbm_ctx *ctx, const double *host_in);

/* The stored state of the fluid cells, bit for bit, in the context's storage type.
 * Layout: host[k * n_fluid + j] is the post-collision deviation g~_k = f_k - w_k rho0 of
 * the j-th fluid cell in cell order (x fastest; n_fluid from lbm_get_info).  The values are
 * as stored: double (LBM_F64), float (LBM_F32), or the 16-bit pattern of an IEEE half
 * times 2^dev_scale_log2 (LBM_F16DEV) or of a bfloat16 (LBM_BF16DEV).
 * bytes must equal 19 * n_fluid * element size, else LBM_ERR_ARG.  The host buffer stays
 * the caller's; pinned memory transfers faster, and pageable memory also works.  The copy
 * of one direction overlaps the device-side gather or scatter of the other.
 * A state read with lbm_get_state and written back with lbm_set_state continues bit for bit
 * as the original would (the wall terms of the A-B layout are rebuilt from it, as by
 * lbm_set_populations_f64).  It carries 19 values per fluid cell in the storage type.
 * lbm_set_populations_f64 carries 19 FP64 values per cell of the box.  Both synchronise. */
LBM_API lbm_status lbm_get_state(lbm_ctx *ctx, void *host_out, size_t bytes);
LBM_API lbm_status lbm_set_state(lbm_ctx *ctx, const void *host_in, size_t bytes);

/* Prefetched state input, for streams of states: lbm_stage_state starts the copy of
 * host_in (lbm_set_state's layout and size) into one of two device staging buffers, on a
 * copy stream of the context's own, and returns at once.  The copy can then overlap the
 * steps queued meanwhile.  host_in must stay unchanged until the lbm_apply_staged_state
 * that consumes it has returned (pinned memory, or the copy is not asynchronous).  At most
 * two states are staged: a third call returns LBM_ERR_STATE.  Wrong bytes: LBM_ERR_ARG.
 * lbm_apply_staged_state makes the oldest staged state the current state, as
 * lbm_set_state does.  It is queued on the context's stream after that state's copy and
 * returns without waiting.  With nothing staged it returns LBM_ERR_STATE. */
LBM_API lbm_status lbm_stage_state(lbm_ctx *ctx, const void *host_in, size_t bytes);
LBM_API lbm_status lbm_apply_staged_state(lbm_ctx *ctx);

/* Velocity u = rho0^-1 sum e_k f_k of the stored state, FP64 [3][nz][ny][nx] (0 in solid). */
LBM_API lbm_status lbm_get_velocity_f64(lbm_ctx *ctx, double *host_out);
/* Solid flags [nz][ny][nx] (1 = solid) as built on the device. */
LBM_API lbm_status lbm_get_flags(lbm_ctx *ctx, uint8_t *host_out);
/* Wall distance q of every cut link as [19][nz][ny][nx] FP64, indexed by the link
 * direction from the fluid cell into the wall; NaN where no link is cut. */
LBM_API lbm_status lbm_get_wall_distances(lbm_ctx *ctx, double *host_out);
LBM_API lbm_status lbm_get_info(lbm_ctx *ctx, lbm_info *out);
/* Wait for all queued work of the context. */
LBM_API lbm_status lbm_synchronize(lbm_ctx *ctx);

/* Moment sums without any allocation, for callers that cannot let a library allocate
 * device memory (every byte owned by a memory pool, no allocation allowed after start-up,
 * or work about to be captured into a CUDA graph).  The paper has no counterpart; it is
 * lbm_moment_sums for a caller-owned field and needs no context.
 *   f_dev     device, FP64 populations f_k (not deviations), [19][n_cells] in the
 *             direction order above; entries of solid cells are ignored
 *   solid_dev device, n_cells flags (1 = solid), or NULL when every cell is fluid
 *   sums_dev  device, 4 doubles out: sums over fluid cells of (rho - rho0, u_x, u_y, u_z),
 *             u = rho0^-1 sum e_k f_k, reduced in a fixed order
 *   cuda_stream  stream the two kernels are queued on (NULL = legacy default stream)
 * Calls no cudaMalloc or cudaFree: block sums go to a fixed 256 KiB scratch array inside
 * the library, held by every GPU that loads it.  n_cells is limited to 268,435,456
 * (8192 blocks of 32768 cells); larger fields return LBM_ERR_ARG.  The first call on
 * each device looks up the scratch address (cudaGetSymbolAddress) and should come before
 * any stream capture.  The address is kept, per device ordinal, for the life of the
 * process: after cudaDeviceReset on a device it is stale, so a process that resets a
 * device must not call this entry point on it again.  Calls share the scratch: calls that
 * overlap on the GPU race.  Returns without waiting for the kernels. */
LBM_API lbm_status lbm_moment_sums_f64_noalloc(const double *f_dev, const uint8_t *solid_dev, int64_t n_cells,
                                               double rho0, double *sums_dev, void *cuda_stream);

/* Checkpoint: header, parameters, step count, AA parity and the stored populations in
 * their native format.  lbm_load needs a context created from the same descriptor. */
LBM_API lbm_status lbm_save(lbm_ctx *ctx, const char *path);
LBM_API lbm_status lbm_load(lbm_ctx *ctx, const char *path);

/* Pressure drop that gives a target Re_p = U d_p / nu, from the Forchheimer relation
 * delta_p / L = mu U / K_D + C_F / sqrt(K_D) rho U^2 (Eq. Forchheimer with beta =
 * C_F K_D^-1/2), delta_rho = 3 L delta_p / L.  Pure host arithmetic. */
LBM_API double lbm_delta_rho_for_re_p(double re_p, double tau, double d_p, int32_t lx, double K_D,
                              double C_F, double rho0);

/* ---------------------------------------------------------------------------------
 * Batched sweep: many independent periodic cells advanced together by one persistent
 * kernel launch per step (all instances must share collision, storage; layout A-B).
 * ------------------------------------------------------------------------------- */
LBM_API lbm_status lbm_batch_create(const lbm_desc *descs, int32_t n, void *cuda_stream,
                            lbm_batch **out);
LBM_API void lbm_batch_destroy(lbm_batch *b);
LBM_API lbm_status lbm_batch_init_equilibrium(lbm_batch *b);
LBM_API lbm_status lbm_batch_step(lbm_batch *b, int64_t n_steps);
LBM_API lbm_status lbm_batch_observables(lbm_batch *b, int32_t i, double K_darcy, lbm_obs *out);
LBM_API lbm_status lbm_batch_get_populations_f64(lbm_batch *b, int32_t i, double *host_out);
LBM_API lbm_status lbm_batch_set_populations_f64(lbm_batch *b, int32_t i, const double *host_in);
LBM_API lbm_status lbm_batch_get_info(lbm_batch *b, lbm_info *out); /* totals over instances */

/* ---------------------------------------------------------------------------------
 * Serving: a request loop that admits sweep points by their device-memory footprint,
 * advances all admitted points together (continuous batching: points arriving while
 * others run join at the next chunk boundary), retires converged points and reports
 * the submit-to-converged latency.
 * ------------------------------------------------------------------------------- */
typedef struct {
    size_t hbm_budget_bytes; /* device bytes the resident points may use */
    int32_t check_interval;  /* steps between convergence checks (0 = 200) */
    int32_t max_resident;    /* cap on simultaneously resident points (0 = 256) */
} lbm_server_opts;

typedef struct {
    int64_t submitted, completed, failed, resident, queued, cancelled;
    double fluid_updates;    /* total fluid-cell updates performed */
    double busy_seconds;     /* wall time with at least one resident point */
    double mlups;            /* fluid_updates / busy_seconds / 1e6 */
    int64_t kernel_launches;
} lbm_server_stats;

LBM_API lbm_status lbm_server_create(const lbm_server_opts *opts, lbm_server **out);
/* Queue a point; it converges when |U_n - U_{n-1}| / |U_n| < tol over check_interval
 * steps or stops at max_steps.  Fails with LBM_ERR_NO_MEMORY if the point alone exceeds
 * the budget. */
LBM_API lbm_status lbm_server_submit(lbm_server *s, const lbm_desc *desc, double tol,
                             int64_t max_steps, int64_t *req_id);
/* LBM_ERR_STATE while the request is queued or running; LBM_OK with the result once it
 * converged; LBM_ERR_NOT_CONVERGED / LBM_ERR_DIVERGED with the last result otherwise.
 * latency_s (may be NULL): submit-to-finish wall time. */
LBM_API lbm_status lbm_server_poll(lbm_server *s, int64_t req_id, lbm_obs *out, double *latency_s);
/* Block until every submitted request has finished (bounded by timeout_s; <= 0: none). */
LBM_API lbm_status lbm_server_drain(lbm_server *s, double timeout_s);
/* Cancel a request: a queued one is dropped at once, a resident one is retired at the next
 * chunk boundary; its poll then returns LBM_ERR_CANCELLED (with the observables of its
 * last chunk when it was resident).  LBM_ERR_STATE if it has already finished. */
LBM_API lbm_status lbm_server_cancel(lbm_server *s, int64_t req_id);
LBM_API lbm_status lbm_server_get_stats(lbm_server *s, lbm_server_stats *out);
LBM_API void lbm_server_destroy(lbm_server *s);

#ifdef __cplusplus
}
#endif
#endif /* LBM_GB300_H */
