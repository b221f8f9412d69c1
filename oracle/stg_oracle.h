/*
 * CPU FP64 oracle for the STG-LBM hot path (Xue, Yao & Davidson, "Synthetic
 * turbulence generator for lattice Boltzmann method at the interface between
 * RANS and LES").
 *
 * TEST INFRASTRUCTURE ONLY.  This header and stg_oracle.c are a plain, slow,
 * step-by-step restatement of the paper's equations used to check the CUDA
 * library.  Only the test suite, the smoke check and the benchmark's CPU
 * baseline may build, load or call it.  It shares no code, header, table or
 * constant generator with the CUDA library.
 *
 * Lattice: D3Q19 in the order rest, +x, -x, +y, -y, +z, -z, (1,1,0),
 * (-1,-1,0), (1,-1,0), (-1,1,0), (1,0,1), (-1,0,-1), (1,0,-1), (-1,0,1),
 * (0,1,1), (0,-1,-1), (0,1,-1), (0,-1,1).  Population arrays are
 * f[i][z][y][x] (x fastest).  The inlet velocity plane is u[c][z][y].
 */
#ifndef STG_ORACLE_H
#define STG_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int32_t nx, ny, nz;
    int32_t bc_x;        /* 0: STG inlet at x=0 + pressure outlet at x=nx-1; 1: periodic */
    int32_t bc_y;        /* 0: half-way bounce-back walls below y=0 and above y=ny-1; 1: periodic */
    int32_t collision;   /* 0: BGK on regularized non-equilibrium; 1: plain BGK */
    int32_t stats_every; /* accumulate velocity statistics after every k-th step; 0: off */
    int32_t pad0;
    double tau0;         /* molecular relaxation time */
    double c_smag;       /* C of nu_t = C delta^2 |S| */
    double force[3];     /* body-force density (Guo forcing) */
    double sponge_len;   /* sponge zone length before x = nx-1 (lattice units); 0: off */
    double sponge_K, sponge_p;  /* eq. (sponge_visco) constants */
} orc_domain;

typedef struct {
    int32_t n_fv, pad0;
    const double *y_c, *U, *k, *eps;
    const double *R;     /* n_fv x 6, components 11,22,33,12,13,23 */
    double U_bulk, nu_phys, h_phys, mach_target;
} orc_rans;

typedef struct {
    int32_t n_modes, pad0; /* 0: mode count from the paper's formula */
    double C_l, alpha, T_filter;
} orc_stg_params;

typedef struct orc_sim orc_sim;

/* ---- pointwise primitives ---- */
void   orc_d3q19(int32_t *c57, double *w19, int32_t *opp19);
void   orc_splitmix64(uint64_t seed, int32_t n, uint64_t *out);
void   orc_uniform_draws(uint64_t seed, int32_t n, double *out);
void   orc_equilibrium(double rho, const double *u3, double *feq19);
void   orc_moments(const double *f19, const double *F3, double *rho, double *u3, double *pi_neq9);
double orc_tau_eff(double tau0, double C, double rho, double Q_half);
void   orc_regularized_neq(const double *pi_neq9, double *fneq19);
void   orc_collide(const orc_domain *d, const double *f19, double *out19, double *rho, double *u3);
double orc_sponge_factor(const orc_domain *d, int32_t x);
double orc_zou_he_density(const double *f19, double ux);
void   orc_inlet_reconstruct(const double *f19, const double *u_bc3, double *out19);
void   orc_outlet_reconstruct(const double *f19, const double *u_out3, double *out19);
void   orc_cholesky(const double *R6, double *a6);
double orc_spectrum(double k, double l_e, double l_eta, double l_cut);
void   orc_unit_scales(const orc_rans *r, double tau0, int32_t ny, double *c_x, double *c_t);
void   orc_filter_update(int32_t first, double a, const double *u_raw, double *u_f, int32_t n);
double orc_f16_to_double(uint16_t h);

/* ---- one cell of one step, read from an arbitrary stored lattice ----
 * src_type 0: double f[19][nz][ny][nx]; 1: float f; 2: binary16 bits of
 * (f_i - w_i); 3: float (f_i - w_i).  u_bc3 is the inlet velocity of node
 * (y,z) (used at x=0).                                                      */
void orc_cell_update(const orc_domain *d, int32_t src_type, const void *src,
                     int32_t x, int32_t y, int32_t z, const double *u_bc3, double *out19);

/* ---- whole simulation ---- */
int32_t orc_sim_create(const orc_domain *d, const orc_rans *r, const orc_stg_params *p,
                       uint64_t seed, orc_sim **out);
void    orc_sim_destroy(orc_sim *s);
void    orc_sim_set_pops(orc_sim *s, const double *f);
void    orc_sim_get_pops(const orc_sim *s, double *f);
void    orc_sim_step(orc_sim *s, int32_t n);
int64_t orc_sim_time(const orc_sim *s);
double  orc_sim_mass(const orc_sim *s);
void    orc_sim_get_inlet(const orc_sim *s, double *u_bc);
void    orc_sim_get_stats(const orc_sim *s, double *mean_sum, double *rey_sum, int64_t *n_samples);
int32_t orc_sim_n_modes(const orc_sim *s);
void    orc_sim_scalars(const orc_sim *s, double *out8);
void    orc_sim_tables(const orc_sim *s, double *u_int, double *a6, double *l_e,
                       double *q, double *kn, double *d3, double *sigma3, double *phi);
void    orc_sim_stg_raw(const orc_sim *s, double t, int32_t j, int32_t k, double *u3);
int32_t orc_threads(void);

#ifdef __cplusplus
}
#endif
#endif
