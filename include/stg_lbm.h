/*
 * stg_lbm.h -- C ABI of the GB300 STG-LBM library (libstglbm.so).
 *
 * One handle = one channel lattice resident on one GPU.  Each time step runs
 * the synthetic turbulence generator on the inlet plane and then one fused
 * stream + boundary + regularized-collision pass over every cell, following
 * Algorithm 1 of Xue, Yao & Davidson, "Synthetic turbulence generator for
 * lattice Boltzmann method at the interface between RANS and LES":
 *   - STG inlet velocity: Sec. III.A eqs. (u_couple), (v_fluc), (cholesky),
 *     (aux_vec), (dn), (qn), (psu), (Nmode), (lcut); Sec. III.C eqs.
 *     (u_phys), (u_transfer); plus a first-order temporal filter of the
 *     fluctuation (not in the paper; see stg_params.T_filter).
 *   - Inlet populations: Sec. III.B eqs. (f_i), (f_i_neq), (pi_neq),
 *     (unknown_neq), (density_bc), (density_bc_sub), (bc_eq).
 *   - Bulk: Sec. II eqs. (density), (momentum), (tensor), (lbe), (local_eq),
 *     (lbe-nu), (bodyforce), (smogrinsky_model), (tau_eff).
 *   - Walls, periodic span and the regularized pressure outlet: Sec. IV.
 *
 * Conventions
 *   - D3Q19 population order (every population array crossing this ABI):
 *       0:(0,0,0)  1:(1,0,0)  2:(-1,0,0)  3:(0,1,0)  4:(0,-1,0)  5:(0,0,1)
 *       6:(0,0,-1) 7:(1,1,0)  8:(-1,-1,0) 9:(1,-1,0) 10:(-1,1,0) 11:(1,0,1)
 *       12:(-1,0,-1) 13:(1,0,-1) 14:(-1,0,1) 15:(0,1,1) 16:(0,-1,-1)
 *       17:(0,1,-1) 18:(0,-1,1)
 *   - Population layout f[i][z][y][x], x fastest.  Both storage formats hold
 *     the shifted population g_i = f_i - w_i (w_i the D3Q19 weight): as float
 *     for STG_FP32, as IEEE binary16 for STG_FP16_SHIFTED.
 *   - Populations held by a handle between steps are post-collision.
 *   - Inlet plane layout u[c][z][y] (y fastest), lattice units.
 *   - Statistics layout s[k][y][x] (x fastest).
 *   - Lattice units: dx = dt = 1, c_s^2 = 1/3.  Node (x,y,z) sits at
 *     y + 1/2 from the lower wall; walls are half-way between nodes.
 *   - Every function returns STG_OK or an error code and records a message
 *     retrievable with stg_lbm_last_error().  No function aborts the process
 *     or traps the device.
 *   - Device memory is owned by the handle (through the caller's allocator
 *     when one is given) and released by stg_lbm_destroy().  Host arrays
 *     passed in are copied; the caller keeps ownership.
 */
#ifndef STG_LBM_H
#define STG_LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define STG_OK 0
#define STG_ERR_INVALID 1   /* bad argument or unphysical setup (Ma >= 0.1, ...) */
#define STG_ERR_NOMEM 2     /* device allocation failed or exceeds the budget */
#define STG_ERR_UNSTABLE 3  /* NaN/Inf or mass drift found by the periodic check */
#define STG_ERR_TIMEOUT 4   /* a bounded host wait expired */
#define STG_ERR_CUDA 5      /* a CUDA runtime call failed */

/* stg_domain.storage */
#define STG_FP32 0
#define STG_FP16_SHIFTED 1     /* binary16 of f_i - w_i, round to nearest even */
#define STG_FP16_SHIFTED_SR 2  /* binary16 of f_i - w_i, stochastic rounding (unbiased: updates
                                * smaller than half a binary16 spacing are kept on average; the
                                * random bits are a fixed function of cell, step and population) */
/* stg_domain.collision */
#define STG_REGULARIZED 0   /* BGK relaxation of the regularized non-equilibrium part */
#define STG_BGK 1           /* plain BGK, eq. (lbe) */
/* stg_domain.bc_x */
/* STG inlet at x = 0 (regularized Zou-He reconstruction of the inlet plane's velocity); pressure
 * outlet at x = nx-1 (rho = 1, velocity of the neighbour x = nx-2 at the same step, regularized) */
#define STG_BC_X_INLET_OUTLET 0
#define STG_BC_X_PERIODIC 1
/* stg_domain.bc_y */
#define STG_BC_Y_WALLS 0    /* half-way bounce-back at y = -1/2 and y = ny - 1/2 */
#define STG_BC_Y_PERIODIC 1
/* stg_domain.streaming: how the pull of eq. (lbe), f_i(x) <- f*_i(x - c_i), is laid out in memory.
 * Both give the same populations, statistics and mass; they differ in memory and in layout. */
#define STG_STREAM_PULL 0   /* two lattices: each step reads the previous one and writes the next
                             * (2 x 19 populations per cell) */
#define STG_STREAM_AA 1     /* one lattice updated in place (AA pattern, 19 populations per cell):
                             * steps of even index read slot opp(i) of cell x - c_i and write slot i
                             * of cell x + c_i, steps of odd index read slot i and write slot opp(i)
                             * of the same cell.  Needs an even nx >= 4 and 19 nx ny nz < 2^32. */

/* Lattice, physics and cadence of one channel.  z is always periodic. */
typedef struct {
    int32_t nx, ny, nz;   /* lattice size; nx >= 3 with the inlet/outlet */
    int32_t storage;      /* STG_FP32 | STG_FP16_SHIFTED | STG_FP16_SHIFTED_SR */
    int32_t collision;    /* STG_REGULARIZED | STG_BGK */
    int32_t bc_x;         /* STG_BC_X_* */
    int32_t bc_y;         /* STG_BC_Y_* */
    int32_t stats_every;  /* accumulate u and u u over z and time after every k-th step; 0 = off */
    int32_t check_every;  /* FP64 mass / NaN check after every k-th step; 0 = off */
    int32_t streaming;    /* STG_STREAM_PULL (0) | STG_STREAM_AA */
    double tau0;          /* molecular relaxation time, nu0 = (tau0 - 1/2)/3, eq. (lbe-nu) */
    double c_smag;        /* C in nu_t = C delta^2 |S| (C = Cs^2), eq. (smogrinsky_model) */
    double force[3];      /* body-force density, Guo forcing, eq. (bodyforce) */
    double mass_tol;      /* |M/M0 - 1| above this fails the check; <= 0: NaN/Inf only */
    /* Sponge zone before the outlet, eq. (sponge_visco) (Sec. IV): in the last
     * sponge_len lattice spacings before x_end = nx - 1 (x_start = x_end -
     * sponge_len) the viscosity is nu_eff [K xi^p + 1], xi = (x - x_start) /
     * sponge_len, i.e. tau = 1/2 + [K xi^p + 1] (tau_eff - 1/2).  sponge_len = 0
     * switches it off (the paper: 0.4 half-heights, K = 1000, p = 3).  The
     * factor depends on x only; a sponge needs force = 0. */
    double sponge_len, sponge_K, sponge_p;
} stg_domain;

/* RANS interface profile on wall-normal finite-volume cells (Algorithm 1,
 * RANS section, step 2).  Physical units.  Required when bc_x is
 * STG_BC_X_INLET_OUTLET, ignored otherwise. */
typedef struct {
    int32_t n_fv, pad0;
    const double *y_c;    /* n_fv cell centres, strictly increasing inside (0, 2 h_phys) */
    const double *U;      /* n_fv streamwise mean velocity */
    const double *k;      /* n_fv turbulent kinetic energy */
    const double *eps;    /* n_fv dissipation rate (omega = eps / (0.09 k)) */
    const double *R;      /* n_fv x 6 Reynolds stresses, components 11,22,33,12,13,23 */
    double U_bulk;        /* bulk velocity U_b of eq. (psu) */
    double nu_phys;       /* kinematic viscosity */
    double h_phys;        /* channel half height; the lattice spans 2 h_phys in y */
    double mach_target;   /* > 0: map max(U) to mach_target * c_s; 0: c_t from nu (Sec. IV) */
} stg_rans_profile;

/* Synthetic turbulence generator parameters (Sec. III.A). */
typedef struct {
    int32_t n_modes, pad0; /* Fourier modes N; 0 = eq. (Nmode) */
    double C_l;            /* l_e = min(2 d_w, C_l l_t); paper: 3.0 */
    double alpha;          /* mode spacing for eq. (Nmode); paper: 0.01 */
    double T_filter;       /* time constant (steps) of u_f <- a u_f + (1-a) u', a = exp(-1/T); 0 = off */
} stg_params;

/* Optional device allocator (e.g. a framework's caching allocator).  alloc
 * returns a 256-byte aligned device pointer or NULL; free releases it. */
typedef struct {
    void *(*alloc)(size_t bytes, void *ctx);
    void (*free)(void *ptr, size_t bytes, void *ctx);
    void *ctx;
} stg_allocator;

/* Results read back by stg_lbm_stats.  mean_sum / rey_sum are caller-owned
 * host buffers of 3*nx*ny and 6*nx*ny doubles (or NULL to skip): sums over z
 * and over the sampled steps of u_a and u_a u_b (11,22,33,12,13,23), where u
 * is the macroscopic velocity of eq. (momentum) in the sampled step.  The
 * per-(x,y) sample count is n_samples * nz. */
typedef struct {
    int64_t step;       /* steps completed */
    int64_t n_samples;  /* statistics samples taken */
    double mass;        /* FP64 sum of rho at the last check (0 if none) */
    double mass0;       /* mass of the initial state */
    double *mean_sum;
    double *rey_sum;
} stg_stats;

/* Derived setup scalars, in lattice units unless noted. */
typedef struct {
    double c_x, c_t;        /* eq. (c_factor): m per lattice unit, s per step */
    double U_b;             /* bulk velocity, lattice units */
    double max_le;          /* max l_e over the inlet, eq. (psu) */
    double k_min, k_max;    /* mode range, eq. (Nmode) */
    double a_filter;        /* filter coefficient a */
    int64_t n_modes;
    int64_t device_bytes;   /* device memory held by the handle */
} stg_info;

typedef struct stg_lbm stg_lbm;

/* Create a lattice on the current CUDA device.  Validates the inputs, builds
 * the inlet tables (interpolation of the RANS profile onto the lattice nodes,
 * unit conversion, length scales, mode wavenumbers and random directions
 * drawn from `seed` with SplitMix64, FP64 Cholesky of R and FP64 spectrum
 * weights q^n on the device; Algorithm 1, LBM section steps 1-4), allocates
 * the device state and sets every node to f^eq(1, u_int(y)) (periodic x:
 * f = w_i).  `stream` is the cudaStream_t on which every later call is
 * ordered (NULL: the handle creates and owns a non-blocking stream; the
 * legacy default stream cannot be captured into CUDA graphs).  On success
 * *out holds the handle.
 * Errors: STG_ERR_INVALID, STG_ERR_NOMEM, STG_ERR_CUDA (*out = NULL). */
int stg_lbm_create(const stg_domain *domain, const stg_rans_profile *rans, const stg_params *stg,
                   uint64_t seed, const stg_allocator *alloc, void *stream, stg_lbm **out);

/* Enqueue n >= 0 time steps on the handle's stream (asynchronous; replays
 * captured CUDA graphs).  Returns STG_ERR_UNSTABLE if a completed earlier
 * check saw NaN/Inf or mass drift, else STG_OK or STG_ERR_CUDA. */
int stg_lbm_step(stg_lbm *h, int64_t n);

/* Enqueue n steps as individual launches and report mean device times,
 * measured with CUDA events on the handle's stream (ms_step: one step pass,
 * i.e. the fused stream/collide launches of a step and, on sampling steps,
 * the statistics reduction; ms_inlet: the STG inlet kernel; either pointer may
 * be NULL).  Synchronises the stream.  Same physics as stg_lbm_step.
 * Errors: those of stg_lbm_step and stg_lbm_stats. */
int stg_lbm_step_timed(stg_lbm *h, int64_t n, double *ms_step, double *ms_inlet);

/* Wait for the handle's stream (bounded by timeout_s seconds, polling) and
 * copy statistics and the last mass check into *out.  STG_ERR_TIMEOUT if the
 * wait expires, STG_ERR_UNSTABLE if a check failed. */
int stg_lbm_stats(stg_lbm *h, stg_stats *out);

/* Restart the running statistics (the FP64 sums of u and u u behind eqs.
 * y_plus and v_rms, Sec. V) at the current step, e.g. to leave the inflow's
 * start-up transient out of the time averages: waits for the handle's stream,
 * zeroes the sums and makes the current step the origin of the sample count.
 * The populations, the step counter and the inlet filter are untouched.
 * Errors: STG_ERR_INVALID (NULL, a lattice in a batch), STG_ERR_TIMEOUT,
 * STG_ERR_CUDA. */
int stg_lbm_reset_stats(stg_lbm *h);

/* Copy the populations (storage format g_i = f_i - w_i, 19*nx*ny*nz elements
 * of 4 or 2 bytes, layout f[i][z][y][x]) to or from host memory owned by the
 * caller; both wait for the handle's stream.  The host copy is always the
 * canonical state: the post-collision populations f*_i of the last step, not
 * yet streamed, population i of cell x in slot i of x (what the two-lattice
 * scheme stores); for an in-place lattice the library converts from and to
 * its arrangement of the current step parity on the host.  set_state also sets the step
 * counter to `step` (>= 0), restarts the temporal filter and takes the state's
 * mass as the reference of the mass check.  `bytes` must equal the state
 * size.  Errors: STG_ERR_INVALID (NULL, size mismatch, negative step, a
 * lattice in a batch for set_state), STG_ERR_TIMEOUT, STG_ERR_CUDA. */
int stg_lbm_get_state(stg_lbm *h, void *host, size_t bytes);
int stg_lbm_set_state(stg_lbm *h, const void *host, size_t bytes, int64_t step);

/* Checkpoint / resume: the whole evolving state (current populations, step
 * counter, inlet filter state, the current step's inlet plane and the filter's
 * restart step, FP64 statistics sums and
 * sample origin, reference mass) as one host image of stg_lbm_checkpoint_bytes
 * bytes.  Loading it into a lattice created with the same domain and inputs
 * continues the run bit-identically.  load() refuses an image of another
 * lattice size or storage.  Errors: STG_ERR_INVALID, STG_ERR_CUDA. */
int stg_lbm_checkpoint_bytes(const stg_lbm *h, size_t *bytes);
int stg_lbm_save(stg_lbm *h, void *host, size_t bytes);
int stg_lbm_load(stg_lbm *h, const void *host, size_t bytes);

/* Copy a sub-block of the current populations (storage format, canonical
 * arrangement as for stg_lbm_get_state) to host memory: cells x0..x0+bx-1,
 * y0.., z0.., layout [19][bz][by][bx].  The block must lie inside the lattice.
 * An in-place lattice gathers the block on the device into a temporary buffer
 * (cudaMalloc'ed and freed by the call).  Errors: STG_ERR_INVALID,
 * STG_ERR_CUDA. */
int stg_lbm_get_block(stg_lbm *h, int32_t x0, int32_t y0, int32_t z0, int32_t bx, int32_t by, int32_t bz,
                      void *host);

/* Copy the inlet velocity of the last completed step (3*nz*ny floats, lattice
 * units, layout u[c][z][y]) to host memory owned by the caller (waits for the
 * handle's stream).  Errors: STG_ERR_INVALID (NULL), STG_ERR_TIMEOUT,
 * STG_ERR_CUDA. */
int stg_lbm_get_inlet(stg_lbm *h, float *host_u);

/* Device pointer of the current populations and the inlet plane of the last
 * completed step (valid until the next step / destroy; owned by the library,
 * never freed by the caller); for zero-copy inspection, ordered on the
 * handle's stream.  Either output may be NULL.  Two lattices: the canonical
 * arrangement f[i][z][y][x].  In place: the lattice's own arrangement after t
 * completed steps -- t even: f*_i of cell x in slot opp(i) of x; t odd: in slot
 * i of cell x + c_i, or in slot opp(i) of x when x + c_i lies outside the
 * lattice (a wall in y, the open ends in x); any order-free reduction (such as
 * the mass) is the same in every arrangement.  Errors: STG_ERR_INVALID. */
int stg_lbm_device_state(stg_lbm *h, void **pops, float **inlet_u);

/* Derived setup scalars and the device memory held (stg_info).
 * Errors: STG_ERR_INVALID (NULL). */
int stg_lbm_info(const stg_lbm *h, stg_info *out);

/* Launch tile of the plain (non-sampling) steps of the vector step kernels
 * (lattices with even nx; other lattices ignore it).  The paper fixes no
 * kernel decomposition: the tile changes only how the lattice is cut into
 * thread blocks, never the arithmetic of a cell, so every tile gives
 * bit-identical populations and statistics (the FP64 mass of a check can
 * differ in its last bits, its block partials being summed in another order).
 *   interior_layout  0: 8 warps on one x chunk, warps interleaved in z;
 *                    1: 4 warps on 4 consecutive x chunks walking z together
 *                    (x chunks of 64 cells, two per lane; binary16 regularized
 *                    unforced lattices with nx a multiple of 4 take 128-cell
 *                    chunks, four cells per lane, and layout 1 then puts one
 *                    warp in a block)
 *   interior_zc      z planes per block of the rows 1..ny-2 (0: the whole z column,
 *                    else >= 4)
 *   wall_zc          z planes per block of the wall rows y = 0, ny-1 (0 or >= 4)
 * Default {1, 8, 24}. */
typedef struct {
    int32_t interior_layout;
    int32_t interior_zc;
    int32_t wall_zc;
    int32_t pad0;
} stg_tile;

/* Set the tile (re-captures the step graphs; synchronises the stream).
 * Errors: STG_ERR_INVALID (bad field; the tile is unchanged), STG_ERR_CUDA. */
int stg_lbm_set_tile(stg_lbm *h, const stg_tile *tile);
int stg_lbm_get_tile(const stg_lbm *h, stg_tile *tile);

/* Velocity probes for time series (the auto-correlation B_uu and the
 * integral time scale of Sec. V, eq. (time-integral)).  set_probes stores n
 * cells (xyz: 3 n host int32, x y z each inside the lattice; n = 0 clears).
 * step_probed advances n >= 1 steps like stg_lbm_step and after every step
 * samples the velocity u = (sum_i c_i f_i - F/2)/rho of each probe cell from
 * the stored populations; u_host receives n x n_probes x 3 floats (step-major)
 * and the call returns after the copy.  Errors: STG_ERR_INVALID (no probes,
 * bad sizes), STG_ERR_NOMEM, and those of stg_lbm_step. */
int stg_lbm_set_probes(stg_lbm *h, int32_t n, const int32_t *xyz);
int stg_lbm_step_probed(stg_lbm *h, int64_t n, float *u_host);

/* Autotuner: time every candidate tile on this lattice (`trial_passes` >= 1
 * plain step passes each, CUDA events on the handle's stream, after one
 * warm-up pass), keep the fastest and store it in *chosen (may be NULL).
 * The trial passes recompute the next state from the current one without
 * advancing the step counter, the inlet filter or the statistics, so tuning
 * leaves the simulation's results unchanged.  An in-place lattice's trial
 * passes update the lattice itself: its populations and step counters are
 * copied to host memory first and put back afterwards.  Synchronises the
 * stream. */
int stg_lbm_autotune(stg_lbm *h, int32_t trial_passes, stg_tile *chosen);

/* Release everything the handle owns (NULL-safe).  Synchronises its stream. */
void stg_lbm_destroy(stg_lbm *h);

/* Message of the last error on h (h may be NULL: last create() error). */
const char *stg_lbm_last_error(const stg_lbm *h);

/* The 4*n uniform draws in [0,1) used for n modes (per mode: Phi, gamma, eta,
 * phi), SplitMix64 of `seed` (Steele, Lea & Flood 2014), top 53 bits. */
int stg_mode_draws(uint64_t seed, int32_t n, double *out);

/* Device bytes that stg_lbm_create would take for this domain (an upper
 * bound: with n_modes = 0 the mode count is bounded by its largest value for
 * this ny).  `stg` may be NULL for periodic-x domains.  Used for admission by
 * memory budget.  Errors: STG_ERR_INVALID. */
int stg_lbm_estimate_bytes(const stg_domain *domain, const stg_params *stg, int64_t *bytes);

/* ---------------------------------------------------------------------------
 * Batch executor.  The paper runs one channel; the batch runs an ensemble of
 * independent lattices together.  Each block of B steps is one CUDA-graph
 * launch in which every member's chain of B steps (inlet kernel, then the
 * step pass with its boundary branch) is its own branch, so small lattices
 * fill the GPU together and no member waits for another between steps.  B is
 * the smallest multiple of 2 and of every member's sampling period that is at
 * least 16 (members whose periods have no common multiple <= 256 are
 * refused).  A member runs exactly the kernels and arguments it runs alone:
 * its populations and statistics are bit-identical to a solo run.  Members
 * keep their own state, statistics and mass checks; stg_lbm_stats,
 * get_state, get_inlet, device_state and info work on a member as usual and
 * are ordered after the batch's work; stg_lbm_step, step_timed, set_state,
 * set_tile and autotune return STG_ERR_INVALID while it is a member.
 * Destroying a member takes it out of its batch first. */
typedef struct stg_batch stg_batch;

/* Empty batch ordered on `stream` (NULL: the batch creates a non-blocking
 * stream of its own).  Errors: STG_ERR_INVALID, STG_ERR_CUDA. */
int stg_batch_create(void *stream, stg_batch **out);
/* Add / remove a member (same device).  remove() leaves the lattice usable on
 * its own.  Errors: STG_ERR_INVALID, STG_ERR_CUDA. */
int stg_batch_add(stg_batch *b, stg_lbm *h);
int stg_batch_remove(stg_batch *b, stg_lbm *h);
int stg_batch_size(const stg_batch *b);
/* Steps per block graph (B above). */
int stg_batch_block_steps(const stg_batch *b);
/* Advance every member by n >= 0 steps (asynchronous): whole blocks replay
 * the block graph, the rest runs as each member's single-step graphs.
 * Returns the first member error a completed check reported
 * (STG_ERR_UNSTABLE; the message names the member's index), else STG_OK or
 * STG_ERR_CUDA. */
int stg_batch_step(stg_batch *b, int64_t n);
/* Wait for the batch's work (bounded; STG_ERR_TIMEOUT). */
int stg_batch_sync(stg_batch *b);
/* Autotuner for the batch: every candidate tile is timed over `trial_passes`
 * concurrent plain passes of all members (no state advance, as in
 * stg_lbm_autotune); the fastest is set on every member. */
int stg_batch_autotune(stg_batch *b, int32_t trial_passes, stg_tile *chosen);
/* Release the members (they stay alive) and the batch (NULL-safe). */
void stg_batch_destroy(stg_batch *b);
/* Message of the last error on b (b may be NULL: last create() error). */
const char *stg_batch_last_error(const stg_batch *b);

/* ---------------------------------------------------------------------------
 * Serving loop (no counterpart in the paper): a stream of channel jobs with
 * arrival times is run with continuous batching.  In arrival order, a job is
 * admitted once it has arrived, a slot is free (max_active) and its device
 * memory (stg_lbm_estimate_bytes) fits the budget next to the running jobs; it
 * joins the running batch at the next block boundary, so its work overlaps
 * with the jobs already on the GPU.  A job whose remaining steps are fewer
 * than one block leaves the batch and finishes on its own stream; its FP64
 * statistics are copied to the caller's buffers, its memory is freed and the
 * next job can be admitted.  Jobs are independent: each result equals that
 * of the same job run alone.  A job larger than the budget fails with
 * STG_ERR_NOMEM; a job that fails its checks gets that status and the others
 * continue. */
typedef struct {
    double arrival_s;              /* seconds after the start of the run */
    const stg_domain *domain;      /* as for stg_lbm_create */
    const stg_rans_profile *rans;
    const stg_params *stg;
    uint64_t seed;
    int64_t steps;                 /* >= 1 */
    double *mean_sum;              /* optional outputs, caller-owned: 3*nx*ny and */
    double *rey_sum;               /* 6*nx*ny doubles as in stg_stats (NULL: skipped) */
} stg_job;

typedef struct {
    int32_t status;                /* STG_OK or the job's error */
    int32_t pad0;
    double admit_s, finish_s;      /* seconds after the start of the run */
    double latency_s;              /* finish_s - arrival_s */
    int64_t n_samples;             /* statistics samples accumulated */
    int64_t device_bytes;          /* admission estimate */
    double mass, mass0;            /* FP64 mass at the end / after create */
} stg_job_result;

typedef struct {
    double hbm_budget_bytes;       /* device memory the admitted jobs may hold together */
    int32_t max_active;            /* jobs running at once (<= 0: no limit) */
    int32_t pad0;
} stg_serve_config;

typedef struct {
    double wall_s;                 /* start of the run to the last completion */
    double jobs_per_s;             /* completed jobs / wall_s */
    double aggregate_mlups;        /* cell updates of the completed jobs / wall_s / 1e6 */
    double p50_latency_s, p99_latency_s, mean_latency_s;
    int64_t completed, failed;
    int64_t cell_updates;
    int64_t peak_device_bytes;     /* largest admitted estimate total */
    int32_t peak_active;
    int32_t pad0;
} stg_serve_report;

/* Run the jobs (arrival times relative to the call) and return when all
 * have completed or failed.  `stream` orders the batch's work (NULL: own).
 * results[i] belongs to jobs[i].  Errors: STG_ERR_INVALID (arguments),
 * STG_ERR_CUDA / STG_ERR_TIMEOUT (the run itself). */
int stg_serve_run(const stg_job *jobs, int32_t n_jobs, const stg_serve_config *cfg, void *stream,
                  stg_job_result *results, stg_serve_report *report);
/* Message of the last stg_serve_run error on this thread. */
const char *stg_serve_last_error(void);

/* Library version string. */
const char *stg_lbm_version(void);

/* FP64 mass (sum over cells and populations of f_i) of a stored population
 * field, for callers that cannot allocate device memory: code running where
 * cudaMalloc is forbidden or too costly (a fixed device-memory budget that is
 * already committed, a latency-critical loop where an allocation would
 * synchronise the device, or a host framework that owns every allocation).
 * The paper has no counterpart; this is the same reduction kernel that
 * stg_lbm_stats uses, with its scratch in a file-scope device array instead
 * of handle memory.
 *   pops      device pointer to 19*nx*ny*nz elements in the storage format
 *             (g_i = f_i - w_i as float for STG_FP32, as binary16 for
 *             STG_FP16_SHIFTED), layout f[i][z][y][x];
 *   mass_out  device pointer to one double, written when the kernel finishes;
 *   stream    cudaStream_t the work is ordered on (NULL: legacy stream).
 * Allocates nothing (no cudaMalloc/cudaFree, no allocating library routine).
 * The scratch is 8 KB per GPU that loads the library, held until process
 * exit, shared by every call on that GPU: calls that overlap on the GPU race,
 * and each call clears the counter it needs before launching.  The first call
 * on a device (with that device current) looks up the scratch address with
 * cudaGetSymbolAddress: make that first call before any stream capture.
 * Every later call made outside stream capture looks the address up again, so
 * a device reset (cudaDeviceReset, which invalidates the array's old address)
 * is picked up by the next such call; a call made during stream capture uses
 * the address found by the last call outside capture on that device.
 * At most 2^31-1 cells; larger sizes, NULL pointers or a bad storage code
 * return STG_ERR_INVALID, CUDA failures STG_ERR_CUDA (message via
 * stg_lbm_last_error(NULL)).  Asynchronous: returns after enqueueing. */
int stg_lattice_mass_noalloc(const void *pops, int32_t storage, int32_t nx, int32_t ny, int32_t nz,
                             double *mass_out, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* STG_LBM_H */
