/*
 * swe.h -- C ABI of the GB300 shallow-water MacCormack library.
 *
 * The library advances the 2D shallow-water equations with the explicit
 * predictor-corrector MacCormack scheme of Seitz et al., "A GPU
 * Implementation for Two-Dimensional Shallow Water Modeling" (2013): the
 * unknowns are the free-surface elevation eta and the two depth-averaged
 * velocities u, v of every cell of a structured grid (Sec. 1); one time step
 * is the chain of 16 dependent sub-steps of Sec. 1, each independent per
 * cell; the step size is variable (Sec. 3.1); drying, which the paper's code
 * lacked (Sec. 6.2), is handled.  The sub-steps and every reading of what the
 * paper leaves to Ransom's thesis are:
 *   S1  h = eta - z, wet iff h > h_dry
 *   S2  dt = min(cfl / max_wet[(|u|+sqrt(g h))/dx + (|v|+sqrt(g h))/dy], dt_max)
 *       (dt_max when nothing is wet), reduced on the GPU in FP64
 *   S3  ghost ring from the boundary conditions (below)
 *   S4  fluxes h u, h v; face flux = flux of the downwind cell of the
 *       predictor's one-sided difference; boundary faces: wall 0, inflow
 *       q_in, outflow the adjacent cell's flux
 *   S5  eta* = eta - dt (dFx/dx + dFy/dy)
 *   S6  C = g n^2 |U| / h^(4/3) on wet cells, else 0
 *   S7  u* = (u - dt (u u_x + v u_y + g eta_x)) / (1 + dt C), v* alike;
 *       a dry neighbour whose bed is above the cell's surface is seen at the
 *       cell's own elevation (a wall)
 *   S8  h* < 0: eta* = z (tallied as clamp volume); h* <= h_dry: u* = v* = 0
 *   S9-S13  the same on the predicted state with the opposite one-sided
 *       differences, always updating from the level-n eta, u, v
 *   S14 average of the predicted and corrected states
 *   S15 artificial dissipation kappa * (eps (phi_{i+1}-phi_i) - eps (phi_i-phi_{i-1}))
 *       per axis on eta, u, v of level n, eps = max of the two cells'
 *       |h_{i-1}+h_{i+1}-2h_i| / (|h_{i-1}|+|h_{i+1}|+2|h_i|+1e-12), on
 *       interior faces between two wet cells only
 *   S16 the S8 fix on the new level, tallies.
 * The predictor direction alternates every step (forward/forward, then
 * backward/backward) unless dir_cycle says otherwise.
 *
 * Boundary conditions, per side W (x = 0), E, S (y = 0), N: WALL reflects the
 * normal velocity (free slip); INFLOW prescribes the discharge per unit width
 * q_in entering the domain; OUTFLOW is transmissive (zero gradient).
 *
 * Arrays.  Host arrays are ny*nx doubles, row-major, x fastest (cell (i,j)
 * at j*nx+i), owned by the caller and copied.  Device-array calls take
 * dense ny*nx arrays of the context's real type (double for SWE_FP64, float
 * for SWE_FP32) on the context's device, ordered on the context's stream, and
 * never keep the pointer.  The context owns every device buffer it uses.
 *
 * Errors.  Every call returns a swe_status; nothing throws or exits across
 * the ABI.  swe_last_error gives a text for the last failure of a context.
 * Calls on one context are not thread-safe; distinct contexts are
 * independent.  A CUDA error poisons the context (SWE_ERR_STATE after it).
 */
#ifndef SWE_H
#define SWE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SWE_OK = 0,
    SWE_ERR_ARG = 1,        /* invalid argument, size or pointer */
    SWE_ERR_CUDA = 2,       /* a CUDA call failed; text in swe_last_error */
    SWE_ERR_NONFINITE = 3,  /* the state holds NaN or Inf after the call */
    SWE_ERR_NEGDEPTH = 4,   /* input depth below -1e-12 m */
    SWE_ERR_TIMEOUT = 5,    /* a bounded device-side wait gave up */
    SWE_ERR_STATE = 6,      /* call out of order, or context poisoned */
    SWE_ERR_UNSUPPORTED = 7, /* configuration the called entry point does not handle */
    SWE_ERR_CHECK = 8       /* a device-side index or alignment check failed (checked builds only) */
} swe_status;

typedef enum { SWE_BC_WALL = 0, SWE_BC_INFLOW = 1, SWE_BC_OUTFLOW = 2 } swe_bc;
typedef enum { SWE_SIDE_W = 0, SWE_SIDE_E = 1, SWE_SIDE_S = 2, SWE_SIDE_N = 3 } swe_side;
typedef enum { SWE_FP64 = 0, SWE_FP32 = 1 } swe_precision;
typedef enum {
    SWE_KERNEL_FUSED = 0,   /* one sweep per step (default) */
    SWE_KERNEL_PLAIN = 1,   /* one thread per cell, predictor and corrector as two kernels */
    /* The paper's own GPU layout (Sec. 3.1), kept to measure it beside the
     * fused sweep: one kernel per sub-step, every intermediate in global
     * memory, one-dimensional blocks along a row.  SWE_KERNEL_PAPER computes
     * each step size on the host from a device-to-host copy of the state
     * (the call waits for the GPU every step); SWE_KERNEL_PAPER_DEVDT reduces
     * it on the GPU.  With the same step sizes the state equals the other
     * kernels' bit for bit.  No adjoint (SWE_ERR_UNSUPPORTED). */
    SWE_KERNEL_PAPER = 2,
    SWE_KERNEL_PAPER_DEVDT = 3,
    /* The paper's shared-memory design (Sec. 3.2): as SWE_KERNEL_PAPER(_DEVDT),
     * but the sub-steps that read neighbours run in 16 x 16 thread blocks with
     * the block's cells and halo staged in shared memory.  Same results bit
     * for bit. */
    SWE_KERNEL_PAPER_SHARED = 4,
    SWE_KERNEL_PAPER_SHARED_DEVDT = 5
} swe_kernel;

/* Step-info flag bits */
#define SWE_FLAG_NONFINITE 1u
#define SWE_FLAG_TIMEOUT 2u
#define SWE_FLAG_CLAMPED 4u
#define SWE_FLAG_CHECK 8u      /* checked builds: a shared-memory read, global store or TMA
                                  coordinate of the fused or batched row step was out of range
                                  or misaligned; the access was skipped */

typedef struct {
    int32_t nx, ny;         /* cells in x and y, >= 1 */
    double dx, dy;          /* cell sizes, m, > 0 */
    double g;               /* gravity, m/s^2 (9.81) */
    double cfl;             /* Courant number of S2 (0.5) */
    double h_dry;           /* wet/dry threshold, m (1e-3) */
    double dt_max;          /* time-step cap, s (10) */
    double kappa;           /* S15 coefficient, 0 = off, at most 0.25 */
    double manning_n;       /* uniform Manning n, used without a per-cell field */
    int32_t bc[4];          /* swe_bc per side, order W, E, S, N */
    double q_in[4];         /* inflow discharge per unit width into the domain, m^2/s */
    int32_t precision;      /* swe_precision */
    int32_t dir_cycle;      /* bit 0: alternate directions per step; bit 1: x starts
                               backward; bit 2: y starts backward (default 1) */
    int32_t device;         /* CUDA device ordinal */
    int32_t kernel;         /* swe_kernel */
    void* stream;           /* cudaStream_t to order all work on; NULL: context-owned */
    int32_t seg_rows;       /* fused kernel: rows per work item, 0 = automatic */
    int32_t cta_warps;      /* fused kernel: warps per CTA, 0 = automatic */
    int32_t use_graph;      /* capture multi-step calls in CUDA graphs (default 1) */
    int32_t dry_skip;       /* skip all-dry work items (default 1) */
    /* Ablation forms (0 = the readings of the header comment, the default).
     * friction 1: explicit friction, u* = u - dt (A + C u) with C and u of the
     * stage's differenced state, in place of the point-implicit update.
     * dissipation 1: the TVD-MacCormack term (Davis; Garcia-Navarro, Alcrudo
     * and Saviron for shallow water) in place of S15's switch form, kappa
     * ignored.  Only the plain and paper-layout kernels run them; the fused,
     * batched, adjoint and no-allocation paths answer SWE_ERR_UNSUPPORTED. */
    int32_t friction;
    int32_t dissipation;
    /* reserved[0], reserved[1]: test hooks of the batched step (ignored
     * elsewhere; 0 = off).  reserved[0]: the grid-barrier wait limit in
     * microseconds (default about 2 s, at most 10 s).  reserved[1]: the CTA
     * of index reserved[1] - 1 withholds its arrival at the first grid
     * barrier of the next swe_batch_step call (that call only), so that the
     * other CTAs' bounded waits run out and the call returns
     * SWE_ERR_TIMEOUT. */
    int32_t reserved[2];
} swe_params;

typedef struct {
    double t;               /* simulated time, s */
    double dt_last;         /* last step size, s */
    double dt_min;          /* smallest step size of the call */
    double dt_max_seen;     /* largest step size of the call */
    double volume;          /* sum of h dx dy, m^3, summed in FP64 */
    double clamp_volume;    /* water added by the negative-depth fix since creation, m^3 */
    double bflux[4];        /* water entered through each side since creation, m^3 */
    int64_t step;           /* global step index */
    int64_t n_wet;          /* wet cells of the current state */
    int32_t flags;          /* SWE_FLAG_* seen during the call */
    int32_t pad;
} swe_step_info;

typedef struct swe_ctx swe_ctx;

/* Fills p with the defaults named above (walls, FP64, fused kernel, alternating
 * directions, device 0, own stream); nx, ny, dx, dy still need setting. */
void swe_params_default(swe_params* p);

/* The grid and scheme settings of one problem (paper Sec. 1: a structured
 * grid carrying eta, u, v; Sec. 3.1: the variable step's Courant number).
 * Validates p (SWE_ERR_ARG on a bad size, cell size, constant, boundary code
 * or kernel; SWE_ERR_CUDA when the device or an allocation fails) and
 * allocates the context and its device buffers (state ping-pong, bed,
 * friction field, reduction scratch); the context owns them.  *out receives
 * the context, or NULL on failure.  Bed and state start at zero until set. */
swe_status swe_create(const swe_params* p, swe_ctx** out);

/* The domain's topography (paper Sec. 4: each workload gives the domain
 * topology and initial conditions): bed elevation z (m) and, optionally, a
 * per-cell Manning n field (NULL: the uniform manning_n) for the friction
 * sub-steps S6/S12.  Host arrays, ny*nx doubles, row-major, copied; the
 * caller keeps ownership.  SWE_ERR_ARG for a NULL z or a non-finite or
 * negative n; SWE_ERR_STATE on a poisoned context. */
swe_status swe_set_bed(swe_ctx* ctx, const double* z, const double* n_field);

/* Initial conditions (paper Sec. 4) of the unknowns eta, u, v (Sec. 1): host
 * arrays, ny*nx doubles, row-major, copied.  A depth below -1e-12 m is
 * SWE_ERR_NEGDEPTH and a non-finite value SWE_ERR_ARG; after either the
 * context holds no valid state (swe_step returns SWE_ERR_STATE until a state
 * is set again).  A smaller negative depth is
 * clamped (eta = z); dry cells get zero velocity (the drying rule read from
 * Sec. 6.2).  Computes the first step's
 * CFL reduction (S2, Sec. 3.1).  Keeps the step index and time. */
swe_status swe_set_state(swe_ctx* ctx, const double* eta, const double* u, const double* v);

/* Sets the step index (direction parity) and the simulated time. */
swe_status swe_set_clock(swe_ctx* ctx, int64_t step, double t);

/* Advances nsteps explicit MacCormack steps, each the 16 sub-steps of paper
 * Sec. 1 with the variable step size of Sec. 3.1 (computed on the GPU, not
 * copied to the host as the paper's code did).  dt_fixed (nullable, host,
 * nsteps values) replaces S2 by the given step sizes; dt_out (nullable, host,
 * nsteps values) receives the step sizes used; info (nullable) receives the
 * diagnostics at the end of the call (reading it synchronises the stream).
 * SWE_ERR_STATE before a state is set or on a poisoned context;
 * SWE_ERR_NONFINITE when the state holds NaN/Inf at the end (Sec. 4 reports
 * NaNs in one Fortran run); SWE_ERR_TIMEOUT when a bounded device wait gave
 * up.  After either the context still accepts calls: the step index has
 * advanced, the state is what the steps left (set a new one to go on). */
swe_status swe_step(swe_ctx* ctx, int32_t nsteps, const double* dt_fixed, double* dt_out,
                    swe_step_info* info);

/* The unknowns of the current level (paper Sec. 1: elevation and the two
 * velocities per cell) to host arrays, ny*nx doubles each, caller-owned
 * (synchronises the stream).  SWE_ERR_ARG for a NULL array. */
swe_status swe_get_state(swe_ctx* ctx, double* eta, double* u, double* v);

/* Diagnostics of the current state (synchronises the stream). */
swe_status swe_get_info(swe_ctx* ctx, swe_step_info* info);

/* Device-array variants of set_state / get_state / set_bed (context real
 * type, dense ny*nx, asynchronous on the context stream). */
swe_status swe_set_state_device(swe_ctx* ctx, const void* eta, const void* u, const void* v);
swe_status swe_get_state_device(swe_ctx* ctx, void* eta, void* u, void* v);
swe_status swe_set_bed_device(swe_ctx* ctx, const void* z, const void* n_field);

/* The context's CUDA stream (cudaStream_t). */
void* swe_stream(const swe_ctx* ctx);

/* Frees the context and every buffer it owns (the paper has no counterpart;
 * it ends the problem created by swe_create).  NULL is ignored. */
void swe_destroy(swe_ctx* ctx);

/* Discrete adjoint (reverse mode) of nsteps steps from the current state: the
 * loss L = 1/2 sum_{k=1..nsteps} sum_g (eta_g^k - obs[(k-1)*ngauges + g])^2 at
 * the gauge cells gauges[g] (index j*nx+i), and its gradient with respect to
 * the per-cell Manning n (grad_n, host, ny*nx; the uniform manning_n counts
 * as a field), to the initial elevation (grad_eta0, host, ny*nx) and to the
 * bed elevation (grad_z, host, ny*nx, with the initial elevation held, so
 * that a bed change is a depth change); all three nullable.  The paper has no
 * adjoint: this differentiates the step of Sec. 1 with the step sizes of
 * Sec. 3.1 held at the forward run's.  The step sizes are those of the forward run and are held fixed
 * (the CFL minimum is not differentiated).  Requires kappa = 0
 * (SWE_ERR_UNSUPPORTED otherwise); the derivative is that of the smooth,
 * fully wet branch of the wet/dry fixes.  The forward states are kept every
 * checkpoint_every steps (0: ceil(sqrt(nsteps))) and recomputed per segment.
 * Advances the context by nsteps steps (the forward run) and allocates its
 * working buffers for the duration of the call. */
swe_status swe_adjoint(swe_ctx* ctx, int32_t nsteps, const int64_t* gauges, int32_t ngauges, const double* obs,
                       int32_t checkpoint_every, double* loss, double* grad_n, double* grad_eta0, double* grad_z);

/* Work-item autotuner of the fused step (the kernel's only shape parameter is
 * the number of rows per work item, seg_rows; an item is one warp's column
 * strip of 62 cells by that many rows).  swe_autotune_candidates writes the
 * built-in candidate list (heights giving about 1 to 8 items per resident
 * warp, and 32 and 64 rows) into rows[0..cap) and returns its length, or
 * minus a status.  swe_autotune times each candidate (rows[0..nrows), or the
 * built-in list when rows is NULL) on the context's current state: one
 * warm-up step, then probe_steps steps timed with CUDA events on the
 * context's stream; ms_per_step (nullable; needs rows) receives the time per
 * step of each candidate.  It keeps the fastest (written to *chosen,
 * nullable, and to the context's seg_rows) and restores the state, clock
 * and tallies, so the call does not advance the simulation; results of later
 * steps do not depend on the choice (bitwise).  Needs the fused kernel
 * (SWE_ERR_UNSUPPORTED otherwise) and a set state (SWE_ERR_STATE); allocates
 * three state planes for the duration of the call. */
int32_t swe_autotune_candidates(swe_ctx* ctx, int32_t* rows, int32_t cap);
swe_status swe_autotune(swe_ctx* ctx, int32_t probe_steps, const int32_t* rows, int32_t nrows, double* ms_per_step,
                        int32_t* chosen);

/* ---------------------------------------------------------------- strips
 * Row-strip decomposition of one domain over several contexts (Sec. 6.1 of
 * the paper proposes it for several GPUs): each strip context holds its own
 * rows plus two halo rows on every side that faces another strip.  One step
 * of the decomposed domain is: swe_step(strip, 1, ...) on every strip, then
 * swe_copy_rows for every halo (from the neighbour's current level), then
 * swe_cfl_combine over all strips.  Call swe_cfl_combine once after the
 * states are set, too.  The own rows then equal the undecomposed domain's
 * bit for bit, step sizes included.
 *
 * swe_set_own_rows marks rows [lo, hi) as the context's own (default: all
 * rows): halo rows are stepped like the others but enter no tally, no CFL
 * maximum and no diagnostic of swe_get_info.  swe_copy_rows copies nrows rows
 * of the current level (eta, u, v) of src from its row src_row into dst from
 * row dst_row (same nx, precision and device), ordered after the work queued
 * on both contexts, and clears dst's dry-skip flags.  swe_cfl_combine
 * replaces the CFL maximum of every context's current level by the maximum
 * over the n contexts (same step index, same device; n <= 64).  The sides
 * that face another strip may have any boundary condition: it only touches
 * halo rows. */
swe_status swe_set_own_rows(swe_ctx* ctx, int32_t lo, int32_t hi);
swe_status swe_copy_rows(swe_ctx* dst, int32_t dst_row, const swe_ctx* src, int32_t src_row, int32_t nrows);
swe_status swe_cfl_combine(swe_ctx* const* ctxs, int32_t n);

/* ---------------------------------------------------------------- batches
 * Many independent scenarios of uneven grid size advanced together (FP32),
 * each with its own CFL step: one persistent cooperative launch per
 * swe_batch_step call, captured in a CUDA graph when use_graph is set.  The
 * shared settings come from p (g, cfl, h_dry, dt_max, kappa, bc, q_in,
 * dir_cycle 0 or 1, device, stream, seg_rows, use_graph, dry_skip; nx, ny
 * and manning_n are ignored); count scenarios have sizes nx[i] x ny[i] and
 * Manning n manning_n[i].  Host arrays per scenario are ny[i]*nx[i] doubles.
 * Scenario i's results are bitwise those of a single-grid FP32 context with
 * the same inputs.  An item of cells whose 3x3 neighbourhood of items is dry
 * (and away from inflow sides) is skipped when dry_skip is set; dry cells of
 * such a neighbourhood would not change.  infos (nullable) receives count
 * step-info records.  precision must be SWE_FP32 (else SWE_ERR_UNSUPPORTED). */
typedef struct swe_batch swe_batch;
swe_status swe_batch_create(const swe_params* p, int32_t count, const int32_t* nx, const int32_t* ny,
                            const double* manning_n, swe_batch** out);
swe_status swe_batch_set_bed(swe_batch* b, int32_t idx, const double* z);
/* Same normalisation and errors as swe_set_state; the bed must be set first. */
swe_status swe_batch_set_state(swe_batch* b, int32_t idx, const double* eta, const double* u, const double* v);
swe_status swe_batch_step(swe_batch* b, int32_t nsteps, swe_step_info* infos);
swe_status swe_batch_get_state(swe_batch* b, int32_t idx, double* eta, double* u, double* v);
/* Work-item autotuner of the batched step, as swe_autotune: the built-in
 * candidates are 32 to 512 rows per item (default 192); the probes run on the batch's
 * current states, which are restored with their clocks and tallies (the
 * dry-skip flags are cleared).  The items are rebuilt for the chosen height,
 * which also becomes the batch's seg_rows. */
int32_t swe_batch_autotune_candidates(swe_batch* b, int32_t* rows, int32_t cap);
swe_status swe_batch_autotune(swe_batch* b, int32_t probe_steps, const int32_t* rows, int32_t nrows,
                              double* ms_per_step, int32_t* chosen);
void swe_batch_destroy(swe_batch* b);
const char* swe_batch_last_error(const swe_batch* b);

/* No-allocation FP32 step.  The paper has no counterpart to this entry point.
 * It serves callers that cannot allocate device memory: engines whose device
 * memory is all handed out by their own pool (a cudaMalloc behind the pool's
 * back breaks its budget), plug-ins running inside a host application that
 * owns the device memory, and loops with hard latency limits that cannot wait
 * on the allocator (cudaMalloc and cudaFree may synchronise the device).  The
 * caller passes device arrays (float, dense ny*nx, row-major) of the bed and
 * the input state, and separate output arrays: an output sharing any byte
 * with an input or another output is SWE_ERR_ARG.  The call queues one plain
 * step (predictor and corrector kernels, the scheme of the header comment,
 * uniform Manning n) on `stream` (NULL: the default stream) of the current
 * device and allocates nothing.  Its scratch -- the predicted planes, the
 * reduction control block and the step size -- is one static device array of
 * SWE_NOALLOC_MAX_CELLS cells (12 MB) that every GPU loading this library
 * holds until the process exits; grids above that size are rejected with
 * SWE_ERR_ARG.  dt_fixed > 0 gives the step size (passed to the GPU by
 * value), 0 computes it from the CFL rule.  dt_out (host, nullable) receives
 * the step size used; with it the call waits for the stream and returns
 * SWE_ERR_NONFINITE if the new state holds NaN or Inf.  Without dt_out the
 * call does not wait and does not check for non-finite values.  The predictor
 * direction is that of step 0 of dir_cycle.  The first call on a device looks
 * up the scratch's device address (once per device, kept until the process
 * exits; do not call this entry point on a device after cudaDeviceReset).
 * Every call shares the one array, whose control block each call clears
 * first: calls that overlap on the GPU (other streams, other threads) race. */
#define SWE_NOALLOC_MAX_CELLS (1 << 20)
swe_status swe_step_plain_f32_noalloc(const swe_params* p, const float* z, const float* eta, const float* u,
                                      const float* v, float* eta_out, float* u_out, float* v_out, double dt_fixed,
                                      double* dt_out, void* stream);

/* Text of the last failure on ctx (static text when ctx is NULL). */
const char* swe_last_error(const swe_ctx* ctx);
const char* swe_status_string(swe_status s);

#ifdef __cplusplus
}
#endif
#endif /* SWE_H */
