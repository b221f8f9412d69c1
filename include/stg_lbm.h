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
#define STG_FP16_SHIFTED 1
/* stg_domain.collision */
#define STG_REGULARIZED 0   /* BGK relaxation of the regularized non-equilibrium part */
#define STG_BGK 1           /* plain BGK, eq. (lbe) */
/* stg_domain.bc_x */
#define STG_BC_X_INLET_OUTLET 0 /* STG inlet at x = 0, pressure outlet at x = nx-1 */
#define STG_BC_X_PERIODIC 1
/* stg_domain.bc_y */
#define STG_BC_Y_WALLS 0    /* half-way bounce-back at y = -1/2 and y = ny - 1/2 */
#define STG_BC_Y_PERIODIC 1

/* Lattice, physics and cadence of one channel.  z is always periodic. */
typedef struct {
    int32_t nx, ny, nz;   /* lattice size; nx >= 3 with the inlet/outlet */
    int32_t storage;      /* STG_FP32 | STG_FP16_SHIFTED */
    int32_t collision;    /* STG_REGULARIZED | STG_BGK */
    int32_t bc_x;         /* STG_BC_X_* */
    int32_t bc_y;         /* STG_BC_Y_* */
    int32_t stats_every;  /* accumulate u and u u over z and time after every k-th step; 0 = off */
    int32_t check_every;  /* FP64 mass / NaN check after every k-th step; 0 = off */
    int32_t pad0;
    double tau0;          /* molecular relaxation time, nu0 = (tau0 - 1/2)/3, eq. (lbe-nu) */
    double c_smag;        /* C in nu_t = C delta^2 |S| (C = Cs^2), eq. (smogrinsky_model) */
    double force[3];      /* body-force density, Guo forcing, eq. (bodyforce) */
    double mass_tol;      /* |M/M0 - 1| above this fails the check; <= 0: NaN/Inf only */
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

/* Enqueue n steps as individual launches and report the mean device time of
 * one launch of each kernel, measured with CUDA events on the handle's stream
 * (ms_step: fused step kernel, ms_inlet: STG inlet kernel; either may be
 * NULL).  Synchronises the stream.  Same physics as stg_lbm_step. */
int stg_lbm_step_timed(stg_lbm *h, int64_t n, double *ms_step, double *ms_inlet);

/* Wait for the handle's stream (bounded by timeout_s seconds, polling) and
 * copy statistics and the last mass check into *out.  STG_ERR_TIMEOUT if the
 * wait expires, STG_ERR_UNSTABLE if a check failed. */
int stg_lbm_stats(stg_lbm *h, stg_stats *out);

/* Copy the populations (storage format g_i = f_i - w_i, 19*nx*ny*nz elements
 * of 4 or 2 bytes)
 * to or from host memory.  set_state also sets the step counter to `step` and
 * restarts the temporal filter.  `bytes` must equal the state size. */
int stg_lbm_get_state(stg_lbm *h, void *host, size_t bytes);
int stg_lbm_set_state(stg_lbm *h, const void *host, size_t bytes, int64_t step);

/* Copy the inlet velocity of the last completed step (3*nz*ny floats, lattice
 * units, layout u[c][z][y]) to host memory. */
int stg_lbm_get_inlet(stg_lbm *h, float *host_u);

/* Device pointer of the current populations and the inlet plane (valid until
 * the next step / destroy); for zero-copy inspection by the caller. */
int stg_lbm_device_state(stg_lbm *h, void **pops, float **inlet_u);

int stg_lbm_info(const stg_lbm *h, stg_info *out);

/* Launch tile of the plain (non-sampling) steps of the vector step kernels
 * (lattices with even nx; other lattices ignore it).  The paper fixes no
 * kernel decomposition: the tile changes only how the lattice is cut into
 * thread blocks, never the arithmetic of a cell, so every tile gives
 * bit-identical populations and statistics (the FP64 mass of a check can
 * differ in its last bits, its block partials being summed in another order).
 *   interior_layout  0: 8 warps on one 64-cell x chunk, warps interleaved in z;
 *                    1: 4 warps on 4 consecutive 64-cell x chunks walking z together
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

/* Autotuner: time every candidate tile on this lattice (`trial_passes` >= 1
 * plain step passes each, CUDA events on the handle's stream, after one
 * warm-up pass), keep the fastest and store it in *chosen (may be NULL).
 * The trial passes recompute the next state from the current one without
 * advancing the step counter, the inlet filter or the statistics, so tuning
 * leaves the simulation's results unchanged.  Synchronises the stream. */
int stg_lbm_autotune(stg_lbm *h, int32_t trial_passes, stg_tile *chosen);

/* Release everything the handle owns (NULL-safe).  Synchronises its stream. */
void stg_lbm_destroy(stg_lbm *h);

/* Message of the last error on h (h may be NULL: last create() error). */
const char *stg_lbm_last_error(const stg_lbm *h);

/* The 4*n uniform draws in [0,1) used for n modes (per mode: Phi, gamma, eta,
 * phi), SplitMix64 of `seed` (Steele, Lea & Flood 2014), top 53 bits. */
int stg_mode_draws(uint64_t seed, int32_t n, double *out);

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
 * At most 2^31-1 cells; larger sizes, NULL pointers or a bad storage code
 * return STG_ERR_INVALID, CUDA failures STG_ERR_CUDA (message via
 * stg_lbm_last_error(NULL)).  Asynchronous: returns after enqueueing. */
int stg_lattice_mass_noalloc(const void *pops, int32_t storage, int32_t nx, int32_t ny, int32_t nz,
                             double *mass_out, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* STG_LBM_H */
