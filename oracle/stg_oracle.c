/*
 * CPU FP64 oracle for the STG-LBM hot path.  TEST INFRASTRUCTURE ONLY: only
 * the test suite, the smoke check and the benchmark's CPU baseline may build,
 * load or call this file.  It is a plain, slow restatement of the paper's
 * equations, one step at a time, in double precision; it shares nothing with
 * the CUDA library.
 *
 * Paper: Xue, Yao & Davidson, "Synthetic turbulence generator for lattice
 * Boltzmann method at the interface between RANS and LES".  Sections cited:
 *   Sec. II.A  eqs. (density), (momentum), (tensor), (lbe), (local_eq),
 *              (lbe-nu), (bodyforce)          -- LBM, BGK, Guo forcing
 *   Sec. II.B  eqs. (smogrinsky_model), (strain), (tau_eff) -- Smagorinsky SGS
 *   Sec. III.A eqs. (u_couple), (v_fluc), (cholesky), (aux_vec), (dn), (qn),
 *              (psu), (Nmode), (lcut)         -- synthetic turbulence generator
 *   Sec. III.B eqs. (f_i), (f_i_neq), (pi_neq), (unknown_neq), (density_bc),
 *              (density_bc_sub), (bc_eq)      -- regularized inlet reconstruction
 *   Sec. III.C eqs. (u_phys), (u_transfer), (c_factor); Sec. IV eqs. (ma-eq),
 *              (sponge_visco)                -- unit conversion, sponge zone
 *   Algorithm 1                               -- order of the steps
 *
 * Where the paper is silent or garbled the reading taken is stated at the
 * point of use (marked READING).
 */
#include "stg_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define Q19 19
static const double PI = 3.14159265358979323846;

/* ---------------------------------------------------------------------------
 * D3Q19 lattice (Sec. II.A).  c_s^2 = 1/3; weights 1/3 (rest), 1/18 (axis),
 * 1/36 (edge diagonals).
 * ------------------------------------------------------------------------- */
static const int CV[Q19][3] = {
    {0, 0, 0},
    {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1},
    {1, 1, 0}, {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},
    {1, 0, 1}, {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
    {0, 1, 1}, {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
static const double CS2 = 1.0 / 3.0;

static double weight(int i)
{
    int s = CV[i][0] * CV[i][0] + CV[i][1] * CV[i][1] + CV[i][2] * CV[i][2];
    return s == 0 ? 1.0 / 3.0 : (s == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
}

static int opposite(int i)
{
    for (int j = 0; j < Q19; ++j)
        if (CV[j][0] == -CV[i][0] && CV[j][1] == -CV[i][1] && CV[j][2] == -CV[i][2]) return j;
    return -1;
}

void orc_d3q19(int32_t *c57, double *w19, int32_t *opp19)
{
    for (int i = 0; i < Q19; ++i) {
        for (int a = 0; a < 3; ++a) c57[3 * i + a] = CV[i][a];
        w19[i] = weight(i);
        opp19[i] = opposite(i);
    }
}

/* ---------------------------------------------------------------------------
 * Seeded uniform draws: SplitMix64 (Steele, Lea & Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014): the state advances by the
 * golden-ratio increment and each output is the state passed through the
 * published 64-bit finaliser.  Doubles in [0,1) take the top 53 bits.
 * ------------------------------------------------------------------------- */
void orc_splitmix64(uint64_t seed, int32_t n, uint64_t *out)
{
    uint64_t s = seed;
    for (int32_t i = 0; i < n; ++i) {
        s += 0x9E3779B97F4A7C15ULL;
        uint64_t z = s;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
        out[i] = z ^ (z >> 31);
    }
}

void orc_uniform_draws(uint64_t seed, int32_t n, double *out)
{
    uint64_t *tmp = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(n > 0 ? n : 1));
    orc_splitmix64(seed, n, tmp);
    for (int32_t i = 0; i < n; ++i) out[i] = (double)(tmp[i] >> 11) * (1.0 / 9007199254740992.0);
    free(tmp);
}

/* ---------------------------------------------------------------------------
 * Equilibrium, eq. (local_eq):
 *   f_i^eq = w_i rho [1 + c.u/cs^2 + (c.u)^2/(2 cs^4) - u.u/(2 cs^2)]
 * ------------------------------------------------------------------------- */
void orc_equilibrium(double rho, const double *u, double *feq)
{
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int i = 0; i < Q19; ++i) {
        double cu = CV[i][0] * u[0] + CV[i][1] * u[1] + CV[i][2] * u[2];
        feq[i] = weight(i) * rho * (1.0 + cu / CS2 + cu * cu / (2.0 * CS2 * CS2) - uu / (2.0 * CS2));
    }
}

/* Moments, eqs. (density), (momentum), (tensor); Pi_neq = Pi - Pi_eq with
 * Pi_eq the second moment of f^eq(rho, u) (Sec. II.A, split below (tensor)).
 * READING: no force correction is added to Pi_neq. */
void orc_moments(const double *f, const double *F, double *rho_o, double *u, double *pi_neq)
{
    double rho = 0.0, j[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < Q19; ++i) {
        rho += f[i];
        for (int a = 0; a < 3; ++a) j[a] += f[i] * CV[i][a];
    }
    for (int a = 0; a < 3; ++a) u[a] = (j[a] + 0.5 * (F ? F[a] : 0.0)) / rho;
    double feq[Q19];
    orc_equilibrium(rho, u, feq);
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double s = 0.0;
            for (int i = 0; i < Q19; ++i) s += CV[i][a] * CV[i][b] * (f[i] - feq[i]);
            pi_neq[3 * a + b] = s;
        }
    *rho_o = rho;
}

/* Eq. (tau_eff) with c = dx/dt = 1:
 *   tau_eff = tau0/2 + sqrt((tau0 rho)^2 + 18 sqrt(2) C Q^{1/2}) / (2 rho)
 * READING: used as printed (rho^2 multiplies tau0^2 only). */
double orc_tau_eff(double tau0, double C, double rho, double Q_half)
{
    return 0.5 * tau0 + sqrt((tau0 * rho) * (tau0 * rho) + 18.0 * sqrt(2.0) * C * Q_half) / (2.0 * rho);
}

/* Regularized non-equilibrium part, eq. (f_i_neq) with Q_i = c_i c_i - cs^2 I.
 * READING: the prefactor is w_i / (2 cs^4); only with the 1/2 does the
 * second moment of the rebuilt part return Pi_neq. */
void orc_regularized_neq(const double *pi, double *fneq)
{
    for (int i = 0; i < Q19; ++i) {
        double s = 0.0;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                double Qab = CV[i][a] * CV[i][b] - (a == b ? CS2 : 0.0);
                s += Qab * pi[3 * a + b];
            }
        fneq[i] = weight(i) / (2.0 * CS2 * CS2) * s;
    }
}

/* Guo forcing term, eq. (bodyforce):
 *   F_i = (1 - 1/(2 tau)) w_i [(c_i - u)/cs^2 + (c_i.u) c_i / cs^4] . F */
static void guo_term(double tau, const double *u, const double *F, double *Fi)
{
    for (int i = 0; i < Q19; ++i) {
        double cu = CV[i][0] * u[0] + CV[i][1] * u[1] + CV[i][2] * u[2];
        double s = 0.0;
        for (int a = 0; a < 3; ++a) s += ((CV[i][a] - u[a]) / CS2 + cu * CV[i][a] / (CS2 * CS2)) * F[a];
        Fi[i] = (1.0 - 1.0 / (2.0 * tau)) * weight(i) * s;
    }
}

/* Collision, eq. (lbe) with Omega = dt/tau_eff (Sec. II.B, last sentence).
 * READING: the relaxation is f - (f - f^eq)/tau (the printed '+' sign is a
 * typo).  collision 0 relaxes only the regularized non-equilibrium part,
 * i.e. the projection of f - f^eq on the Hermite polynomials of order <= 2:
 *   f^neq_reg,i = w_i c_i.a1/cs^2 + w_i/(2 cs^4) Q_i : Pi_neq,
 *   a1 = sum_i c_i (f_i - f_i^eq)   (= -F/2, because u carries F/2),
 *   f* = f^eq + (1 - 1/tau_eff) f^neq_reg + F_i;
 * keeping a1 makes the momentum gain per step exactly F, as in BGK.
 * collision 1 is plain BGK:  f* = f - (f - f^eq)/tau_eff + F_i. */
/* Sponge zone, eq. (sponge_visco): nu_sponge = nu_eff [K xi^p + 1] with
 * xi = (x - x_start)/(x_end - x_start) inside the zone.
 * READING: lattice units; the zone is the last sponge_len lattice spacings
 * before the outlet column, x_end = nx - 1, x_start = x_end - sponge_len;
 * outside it the factor is 1.  Since nu = c_s^2 (tau - 1/2) (eq. lbe-nu),
 * the zone's relaxation time is tau = 1/2 + F(x) (tau_eff - 1/2), used for
 * the whole collision (forcing included).  The factor depends on x only, so
 * it is defined whatever the x boundary. */
double orc_sponge_factor(const orc_domain *d, int32_t x)
{
    if (!(d->sponge_len > 0.0)) return 1.0;
    const double xe = (double)(d->nx - 1), xs = xe - d->sponge_len;
    if ((double)x < xs) return 1.0;
    const double xi = ((double)x - xs) / (xe - xs);
    return d->sponge_K * pow(xi, d->sponge_p) + 1.0;
}

static void collide_nu(const orc_domain *d, const double *f, double *out, double *rho_o, double *u_o,
                       double nu_factor)
{
    double rho, u[3], pi[9], feq[Q19], Fi[Q19], fneq[Q19];
    orc_moments(f, d->force, &rho, u, pi);
    orc_equilibrium(rho, u, feq);
    double q2 = 0.0;
    for (int k = 0; k < 9; ++k) q2 += pi[k] * pi[k];
    double tau = orc_tau_eff(d->tau0, d->c_smag, rho, sqrt(q2));
    if (nu_factor != 1.0) tau = 0.5 + nu_factor * (tau - 0.5);
    guo_term(tau, u, d->force, Fi);
    if (d->collision == 0) {
        double a1[3] = {0.0, 0.0, 0.0};
        for (int i = 0; i < Q19; ++i)
            for (int a = 0; a < 3; ++a) a1[a] += CV[i][a] * (f[i] - feq[i]);
        orc_regularized_neq(pi, fneq);
        for (int i = 0; i < Q19; ++i) {
            double ca = CV[i][0] * a1[0] + CV[i][1] * a1[1] + CV[i][2] * a1[2];
            fneq[i] += weight(i) * ca / CS2;
            out[i] = feq[i] + (1.0 - 1.0 / tau) * fneq[i] + Fi[i];
        }
    } else {
        for (int i = 0; i < Q19; ++i) out[i] = f[i] - (f[i] - feq[i]) / tau + Fi[i];
    }
    if (rho_o) *rho_o = rho;
    if (u_o) for (int a = 0; a < 3; ++a) u_o[a] = u[a];
}

void orc_collide(const orc_domain *d, const double *f, double *out, double *rho_o, double *u_o)
{
    collide_nu(d, f, out, rho_o, u_o, 1.0);
}

/* Zou-He density at the x = 0 inlet, eqs. (density_bc), (density_bc_sub).
 * READING: the standard Zou-He form.  With the outward normal n = -x,
 * u.n = -u_x, and
 *   rho_bc = (sum_{c_x = 0} f + 2 sum_{c_x < 0} f) / (1 - u_x),
 * i.e. the factor 2 belongs to the populations leaving through the boundary
 * (their mirror images are the unknowns). */
double orc_zou_he_density(const double *f, double ux)
{
    double par = 0.0, out = 0.0;
    for (int i = 0; i < Q19; ++i) {
        if (CV[i][0] == 0) par += f[i];
        else if (CV[i][0] < 0) out += f[i];
    }
    return (par + 2.0 * out) / (1.0 - ux);
}

/* Regularized rebuild of all 19 populations from a known set, eqs. (f_i),
 * (f_i_neq), (pi_neq), (unknown_neq), (bc_eq): the unknown set's
 * non-equilibrium parts are copied from the opposite (known) directions,
 * Pi_neq = sum_i Q_i f_i^neq, and f_i = f_i^eq + w_i/(2 cs^4) Q_i : Pi_neq. */
static void regularized_rebuild(const double *f, double rho, const double *u, int unknown_sign, double *out)
{
    double feq[Q19], fneq[Q19], pi[9];
    orc_equilibrium(rho, u, feq);
    for (int i = 0; i < Q19; ++i) {
        int unknown = (unknown_sign > 0) ? (CV[i][0] > 0) : (CV[i][0] < 0);
        if (!unknown) fneq[i] = f[i] - feq[i];
    }
    for (int i = 0; i < Q19; ++i) {
        int unknown = (unknown_sign > 0) ? (CV[i][0] > 0) : (CV[i][0] < 0);
        if (unknown) {
            int o = opposite(i);
            fneq[i] = f[o] - feq[o];
        }
    }
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double s = 0.0;
            for (int i = 0; i < Q19; ++i) s += (CV[i][a] * CV[i][b] - (a == b ? CS2 : 0.0)) * fneq[i];
            pi[3 * a + b] = s;
        }
    double reg[Q19];
    orc_regularized_neq(pi, reg);
    for (int i = 0; i < Q19; ++i) out[i] = feq[i] + reg[i];
}

/* Inlet (x = 0): unknowns are c_x > 0; density by Zou-He; Algorithm 1 steps 9-10. */
void orc_inlet_reconstruct(const double *f, const double *u_bc, double *out)
{
    double rho = orc_zou_he_density(f, u_bc[0]);
    double tmp[Q19];
    regularized_rebuild(f, rho, u_bc, +1, tmp);
    memcpy(out, tmp, sizeof(tmp));
}

/* Outlet (x = nx-1), "regularized pressure-free" (Sec. IV).  READING: density
 * fixed to 1, velocity copied from the neighbour column (zero gradient), the
 * unknowns c_x < 0 rebuilt as at the inlet. */
void orc_outlet_reconstruct(const double *f, const double *u_out, double *out)
{
    double tmp[Q19];
    regularized_rebuild(f, 1.0, u_out, -1, tmp);
    memcpy(out, tmp, sizeof(tmp));
}

/* Cholesky factor of the Reynolds stress, eq. (cholesky).  R6 = 11,22,33,12,13,23.
 * a6 = a11, a21, a22, a31, a32, a33.  READING: a negative radicand is taken as
 * zero and a zero pivot zeroes the column below it (walls, where R -> 0). */
void orc_cholesky(const double *R, double *a)
{
    double R11 = R[0], R22 = R[1], R33 = R[2], R21 = R[3], R31 = R[4], R32 = R[5];
    double a11 = sqrt(fmax(R11, 0.0));
    double a21 = a11 > 0.0 ? R21 / a11 : 0.0;
    double a31 = a11 > 0.0 ? R31 / a11 : 0.0;
    double a22 = sqrt(fmax(R22 - a21 * a21, 0.0));
    double a32 = a22 > 0.0 ? (R32 - a21 * a31) / a22 : 0.0;
    double a33 = sqrt(fmax(R33 - a31 * a31 - a32 * a32, 0.0));
    a[0] = a11; a[1] = a21; a[2] = a22; a[3] = a31; a[4] = a32; a[5] = a33;
}

/* Modified von Karman spectrum used in eq. (qn).  The paper cites it without
 * printing it.  READING (Shur et al. 2014, the cited source):
 *   E(k) = (k/k_e)^4 / [1 + 2.4 (k/k_e)^2]^(17/6) * f_eta * f_cut,
 *   f_eta = exp(-(12 k/k_eta)^2), f_cut = exp(-(4 max(k - 0.9 k_cut, 0)/k_cut)^3),
 *   k_e = 2 pi/l_e, k_eta = 2 pi/l_eta, k_cut = 2 pi/l_cut.
 * l_eta <= 0 means no viscous cut-off; l_e <= 0 gives E = 0. */
double orc_spectrum(double k, double l_e, double l_eta, double l_cut)
{
    if (l_e <= 0.0) return 0.0;
    double ke = 2.0 * PI / l_e;
    double x = k / ke;
    double E = pow(x, 4.0) / pow(1.0 + 2.4 * x * x, 17.0 / 6.0);
    if (l_eta > 0.0) {
        double keta = 2.0 * PI / l_eta;
        E *= exp(-pow(12.0 * k / keta, 2.0));
    }
    if (l_cut > 0.0) {
        double kcut = 2.0 * PI / l_cut;
        E *= exp(-pow(4.0 * fmax(k - 0.9 * kcut, 0.0) / kcut, 3.0));
    }
    return E;
}

/* Unit conversion, eqs. (c_factor), (u_transfer), (lbe-nu), (ma-eq).
 * c_x: the channel height 2h over ny lattice cells.  c_t: READING: if the
 * profile carries a Mach target, the RANS maximum velocity is mapped to
 * mach_target * c_s; otherwise the paper's route nu_LB = cs^2 (tau0 - 1/2),
 * c_t = nu_LB c_x^2 / nu_phys (Sec. IV). */
void orc_unit_scales(const orc_rans *r, double tau0, int32_t ny, double *c_x, double *c_t)
{
    double cx = 2.0 * r->h_phys / (double)ny;
    double ct;
    if (r->mach_target > 0.0) {
        double umax = 0.0;
        for (int i = 0; i < r->n_fv; ++i) umax = fmax(umax, r->U[i]);
        ct = r->mach_target * sqrt(CS2) * cx / umax;
    } else {
        ct = CS2 * (tau0 - 0.5) * cx * cx / r->nu_phys;
    }
    *c_x = cx;
    *c_t = ct;
}

/* Temporal filter of the fluctuations.  READING (the paper has no filter):
 * first-order recursive low-pass with unit gain at zero frequency,
 *   u_f(t) = a u_f(t-1) + (1 - a) u'(t),  a = exp(-1/T_filter),
 * started from u_f = u' on the first step; a = 0 is the identity. */
void orc_filter_update(int32_t first, double a, const double *u_raw, double *u_f, int32_t n)
{
    for (int32_t i = 0; i < n; ++i) u_f[i] = first ? u_raw[i] : a * u_f[i] + (1.0 - a) * u_raw[i];
}

double orc_f16_to_double(uint16_t h)
{
    int s = (h >> 15) & 1, e = (h >> 10) & 31, m = h & 1023;
    double v;
    if (e == 0) v = ldexp((double)m, -24);
    else if (e == 31) v = m ? NAN : INFINITY;
    else v = ldexp((double)(1024 + m), e - 25);
    return s ? -v : v;
}

/* ---------------------------------------------------------------------------
 * One cell of one time step (Algorithm 1 steps 9-12 for that cell).
 * READING of the step order: pull the post-collision populations of the
 * previous step along -c_i (eq. (lbe), left side), apply the boundaries,
 * rebuild inlet/outlet nodes, then collide.  Walls: half-way bounce-back of
 * resting walls at y = -1/2 and y = ny - 1/2 (f_i <- f*_opp(i) of the same
 * cell).  Unknown inlet/outlet populations are NaN until rebuilt, so any
 * accidental use poisons the result.
 * ------------------------------------------------------------------------- */
static double load(int32_t type, const void *src, size_t ncell, int i, size_t cell)
{
    size_t idx = (size_t)i * ncell + cell;
    if (type == 0) return ((const double *)src)[idx];
    if (type == 1) return (double)((const float *)src)[idx];
    if (type == 3) return weight(i) + (double)((const float *)src)[idx];
    return weight(i) + orc_f16_to_double(((const uint16_t *)src)[idx]);
}

static int wrap(int a, int n) { a %= n; return a < 0 ? a + n : a; }

/* Pull streaming into cell (x, y, z), eq. (lbe) left side: f_i(x) =
 * f*_i(x - c_i); half-way bounce-back at the y walls, periodic z (and x, y
 * when so configured); a source outside an open x end is unknown (NaN). */
static void pull_cell(const orc_domain *d, int32_t type, const void *src, int x, int y, int z, double *f)
{
    const int nx = d->nx, ny = d->ny, nz = d->nz;
    const size_t ncell = (size_t)nx * ny * nz;
    size_t here = ((size_t)z * ny + y) * nx + x;
    for (int i = 0; i < Q19; ++i) {
        int xs = x - CV[i][0], ys = y - CV[i][1], zs = wrap(z - CV[i][2], nz);
        if (d->bc_y == 0 && (ys < 0 || ys >= ny)) {
            f[i] = load(type, src, ncell, opposite(i), here);
            continue;
        }
        ys = wrap(ys, ny);
        if (d->bc_x == 1) xs = wrap(xs, nx);
        else if (xs < 0 || xs >= nx) { f[i] = NAN; continue; }
        f[i] = load(type, src, ncell, i, ((size_t)zs * ny + ys) * nx + xs);
    }
}

static void cell_update(const orc_domain *d, int32_t type, const void *src, int x, int y, int z,
                        const double *u_bc, double *out, double *rho_o, double *u_o)
{
    const int nx = d->nx;
    double f[Q19];
    pull_cell(d, type, src, x, y, z, f);
    if (d->bc_x == 0 && x == 0) {
        orc_inlet_reconstruct(f, u_bc, f);
    } else if (d->bc_x == 0 && x == nx - 1) {
        /* READING (zero gradient): the outlet takes the velocity of its
         * neighbour x = nx-2 at this step, i.e. the moments of the neighbour's
         * streamed populations, with the same definition as the collision's
         * velocity, u = (sum c f + F/2)/rho (eq. momentum). */
        double g[Q19], rho = 0.0, j[3] = {0.0, 0.0, 0.0}, uo[3];
        pull_cell(d, type, src, nx - 2, y, z, g);
        for (int i = 0; i < Q19; ++i) {
            rho += g[i];
            for (int a = 0; a < 3; ++a) j[a] += g[i] * CV[i][a];
        }
        for (int a = 0; a < 3; ++a) uo[a] = (j[a] + 0.5 * d->force[a]) / rho;
        orc_outlet_reconstruct(f, uo, f);
    }
    collide_nu(d, f, out, rho_o, u_o, orc_sponge_factor(d, x));
}

void orc_cell_update(const orc_domain *d, int32_t src_type, const void *src,
                     int32_t x, int32_t y, int32_t z, const double *u_bc3, double *out19)
{
    cell_update(d, src_type, src, x, y, z, u_bc3, out19, NULL, NULL);
}

/* ---------------------------------------------------------------------------
 * Whole simulation.
 * ------------------------------------------------------------------------- */
struct orc_sim {
    orc_domain d;
    orc_stg_params p;
    int has_stg;
    size_t ncell;
    double *f, *g;
    int64_t t;
    double c_x, c_t, U_b, max_le, k_min, k_max, a_filter;
    int N;
    double *u_int, *a6, *le, *leta, *lcut, *q, *kn, *d3, *sig3, *phi;
    double *u_f, *u_bc, *u_raw;
    int filt_init;
    double *rho_cell, *u_cell;
    double *mean_sum, *rey_sum;
    int64_t n_samples;
    double mass;
};

int32_t orc_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* piecewise-linear interpolation on the FV cell centres augmented with the
 * two wall points (Sec. III.C, "numerical interpolation"; READING: linear,
 * U = k = R = 0 at the walls, eps constant-extrapolated to the walls). */
static double interp(const orc_rans *r, const double *v, int stride, int comp, double wall_val_lo,
                     double wall_val_hi, double y)
{
    int n = r->n_fv;
    double y0 = 0.0, v0 = wall_val_lo;
    for (int i = 0; i <= n; ++i) {
        double y1 = (i < n) ? r->y_c[i] : 2.0 * r->h_phys;
        double v1 = (i < n) ? v[(size_t)i * stride + comp] : wall_val_hi;
        if (y <= y1 || i == n) {
            double t = (y1 > y0) ? (y - y0) / (y1 - y0) : 0.0;
            return v0 + t * (v1 - v0);
        }
        y0 = y1;
        v0 = v1;
    }
    return v0;
}

static int setup_stg(orc_sim *s, const orc_rans *r, uint64_t seed)
{
    const int ny = s->d.ny, nz = s->d.nz;
    orc_unit_scales(r, s->d.tau0, ny, &s->c_x, &s->c_t);
    const double cx = s->c_x, su = s->c_t / s->c_x; /* velocity scale, eq. (u_transfer) */
    s->U_b = r->U_bulk * su;
    s->u_int = calloc(ny, sizeof(double));
    s->a6 = calloc((size_t)6 * ny, sizeof(double));
    s->le = calloc(ny, sizeof(double));
    s->leta = calloc(ny, sizeof(double));
    s->lcut = calloc(ny, sizeof(double));
    double Umax = 0.0;
    for (int i = 0; i < r->n_fv; ++i) Umax = fmax(Umax, r->U[i]);
    if (Umax * su / sqrt(CS2) >= 0.1) return 1; /* Mach limit, Sec. IV */
    for (int j = 0; j < ny; ++j) {
        double y = (j + 0.5) * cx; /* physical wall distance of node j */
        double U = interp(r, r->U, 1, 0, 0.0, 0.0, y);
        double k = interp(r, r->k, 1, 0, 0.0, 0.0, y);
        double eps = interp(r, r->eps, 1, 0, r->eps[0], r->eps[r->n_fv - 1], y);
        double R[6];
        for (int c = 0; c < 6; ++c) R[c] = interp(r, r->R, 6, c, 0.0, 0.0, y) * su * su;
        s->u_int[j] = U * su;
        orc_cholesky(R, s->a6 + 6 * j);
        /* length scales, Sec. III.A below eq. (psu): l_t = sqrt(k)/(0.09 omega)
         * with omega = eps/(0.09 k) (READING: k-eps input) = k^{3/2}/eps;
         * l_e = min(2 d_w, C_l l_t).  Converted to lattice units by c_x. */
        double dw = fmin(y, 2.0 * r->h_phys - y);
        double lt = (eps > 0.0) ? pow(fmax(k, 0.0), 1.5) / eps : 0.0;
        s->le[j] = fmin(2.0 * dw, s->p.C_l * lt) / cx;
        s->leta[j] = (eps > 0.0) ? pow(r->nu_phys * r->nu_phys * r->nu_phys / eps, 0.25) / cx : 0.0;
        /* eq. (lcut) with the LES spacings (all one lattice unit).  READING. */
        double dxl = 1.0, dyl = 1.0, dzl = 1.0;
        double dmax = fmax(dxl, fmax(dyl, dzl));
        s->lcut[j] = 2.0 * fmin(fmax(fmax(dxl, dyl), 0.3 * dmax) + 0.1 * dw / cx, dmax);
    }
    double maxle = 0.0, maxkc = 0.0;
    for (int j = 0; j < ny; ++j) {
        maxle = fmax(maxle, s->le[j]);
        maxkc = fmax(maxkc, 2.0 * PI / s->lcut[j]);
    }
    s->max_le = maxle;
    /* degenerate profile with no turbulence anywhere (k = 0 or eps = 0 at
     * every node): l_e = 0, no wavenumber range, and the fluctuation is zero */
    if (maxle <= 0.0) maxle = 1.0;
    s->k_min = PI / maxle;
    s->k_max = 1.5 * maxkc;
    /* eq. (Nmode); READING: a configured mode count takes precedence */
    int N = s->p.n_modes;
    if (N <= 0) N = (int)ceil(log(s->k_max / s->k_min) / log(1.0 + s->p.alpha) + 1.0);
    s->N = N;
    s->kn = calloc(N, sizeof(double));
    s->d3 = calloc((size_t)3 * N, sizeof(double));
    s->sig3 = calloc((size_t)3 * N, sizeof(double));
    s->phi = calloc(N, sizeof(double));
    s->q = calloc((size_t)ny * N, sizeof(double));
    /* READING: geometric spacing k^n = k_min r^(n-1) from k_min to k_max,
     * dk^n = k^n - k^(n-1) with k^0 = k^1/r. */
    double ratio = (N > 1) ? pow(s->k_max / s->k_min, 1.0 / (N - 1)) : 1.0;
    for (int n = 0; n < N; ++n) s->kn[n] = s->k_min * pow(ratio, (double)n);
    /* random directions, eq. (dn): Phi, Theta, eta, phi per mode, drawn in the
     * order Phi, gamma, eta, phi.  READING: gamma uniform in [0,1), Theta =
     * arccos(1 - 2 gamma) (uniform on the sphere). */
    double *u = calloc((size_t)4 * N, sizeof(double));
    orc_uniform_draws(seed, 4 * N, u);
    for (int n = 0; n < N; ++n) {
        double Phi = 2.0 * PI * u[4 * n], gam = u[4 * n + 1], eta = 2.0 * PI * u[4 * n + 2];
        double Th = acos(1.0 - gam / 0.5);
        s->phi[n] = 2.0 * PI * u[4 * n + 3];
        s->d3[3 * n + 0] = sin(Th) * cos(Phi);
        s->d3[3 * n + 1] = sin(Th) * sin(Phi);
        s->d3[3 * n + 2] = cos(Th);
        s->sig3[3 * n + 0] = cos(Phi) * cos(Th) * cos(eta) - sin(Phi) * sin(eta);
        s->sig3[3 * n + 1] = sin(Phi) * cos(Th) * cos(eta) + cos(Phi) * sin(eta);
        s->sig3[3 * n + 2] = -sin(Th) * cos(eta);
    }
    free(u);
    /* normalised amplitudes, eq. (qn), per inlet node */
    for (int j = 0; j < ny; ++j) {
        double sum = 0.0;
        for (int n = 0; n < N; ++n) {
            double dk = s->kn[n] - s->kn[n] / ratio;
            if (N == 1) dk = 1.0;
            double e = orc_spectrum(s->kn[n], s->le[j], s->leta[j], s->lcut[j]) * dk;
            s->q[(size_t)j * N + n] = e;
            sum += e;
        }
        for (int n = 0; n < N; ++n) s->q[(size_t)j * N + n] = sum > 0.0 ? s->q[(size_t)j * N + n] / sum : 0.0;
    }
    s->a_filter = (s->p.T_filter > 0.0) ? exp(-1.0 / s->p.T_filter) : 0.0;
    s->u_f = calloc((size_t)3 * ny * nz, sizeof(double));
    s->u_bc = calloc((size_t)3 * ny * nz, sizeof(double));
    s->u_raw = calloc((size_t)3 * ny * nz, sizeof(double));
    return 0;
}

/* Synthetic fluctuation at inlet node (j,k) at time t: eqs. (aux_vec),
 * (psu), (v_fluc).  x = 0 at the inlet, y = j + 1/2, z = k (lattice units). */
void orc_sim_stg_raw(const orc_sim *s, double t, int32_t j, int32_t k, double *u3)
{
    double v[3] = {0.0, 0.0, 0.0};
    const double y = j + 0.5, z = (double)k, x = 0.0;
    if (s->max_le <= 0.0) { u3[0] = u3[1] = u3[2] = 0.0; return; }
    for (int n = 0; n < s->N; ++n) {
        double kn = s->kn[n];
        double xp = 2.0 * PI / (kn * s->max_le) * (x - s->U_b * t); /* eq. (psu) */
        double arg = kn * (s->d3[3 * n] * xp + s->d3[3 * n + 1] * y + s->d3[3 * n + 2] * z) + s->phi[n];
        double amp = sqrt(s->q[(size_t)j * s->N + n]) * cos(arg);
        for (int a = 0; a < 3; ++a) v[a] += amp * s->sig3[3 * n + a];
    }
    for (int a = 0; a < 3; ++a) v[a] *= sqrt(6.0);
    const double *a6 = s->a6 + 6 * j;
    u3[0] = a6[0] * v[0];
    u3[1] = a6[1] * v[0] + a6[2] * v[1];
    u3[2] = a6[3] * v[0] + a6[4] * v[1] + a6[5] * v[2];
}

int32_t orc_sim_create(const orc_domain *d, const orc_rans *r, const orc_stg_params *p,
                       uint64_t seed, orc_sim **out)
{
    *out = NULL;
    if (d->nx < 1 || d->ny < 1 || d->nz < 1) return 1;
    if (d->bc_x == 0 && (d->nx < 3 || r == NULL || p == NULL)) return 1;
    orc_sim *s = calloc(1, sizeof(orc_sim));
    s->d = *d;
    if (p) s->p = *p;
    s->ncell = (size_t)d->nx * d->ny * d->nz;
    s->f = calloc(Q19 * s->ncell, sizeof(double));
    s->g = calloc(Q19 * s->ncell, sizeof(double));
    s->rho_cell = calloc(s->ncell, sizeof(double));
    s->u_cell = calloc(3 * s->ncell, sizeof(double));
    s->mean_sum = calloc((size_t)3 * d->nx * d->ny, sizeof(double));
    s->rey_sum = calloc((size_t)6 * d->nx * d->ny, sizeof(double));
    if (!s->f || !s->g || !s->rho_cell || !s->u_cell) { orc_sim_destroy(s); return 2; }
    s->has_stg = (d->bc_x == 0);
    if (s->has_stg) {
        if (setup_stg(s, r, seed)) { orc_sim_destroy(s); return 1; }
        /* initial state: f^eq(1, u_int(y)) */
        for (int z = 0; z < d->nz; ++z)
            for (int y = 0; y < d->ny; ++y)
                for (int x = 0; x < d->nx; ++x) {
                    double u[3] = {s->u_int[y], 0.0, 0.0}, feq[Q19];
                    orc_equilibrium(1.0, u, feq);
                    size_t c = ((size_t)z * d->ny + y) * d->nx + x;
                    for (int i = 0; i < Q19; ++i) s->f[(size_t)i * s->ncell + c] = feq[i];
                }
    } else {
        for (int i = 0; i < Q19; ++i)
            for (size_t c = 0; c < s->ncell; ++c) s->f[(size_t)i * s->ncell + c] = weight(i);
    }
    *out = s;
    return 0;
}

void orc_sim_destroy(orc_sim *s)
{
    if (!s) return;
    free(s->f); free(s->g); free(s->rho_cell); free(s->u_cell);
    free(s->mean_sum); free(s->rey_sum);
    free(s->u_int); free(s->a6); free(s->le); free(s->leta); free(s->lcut); free(s->q);
    free(s->kn); free(s->d3); free(s->sig3); free(s->phi);
    free(s->u_f); free(s->u_bc); free(s->u_raw);
    free(s);
}

void orc_sim_set_pops(orc_sim *s, const double *f) { memcpy(s->f, f, sizeof(double) * Q19 * s->ncell); }
void orc_sim_get_pops(const orc_sim *s, double *f) { memcpy(f, s->f, sizeof(double) * Q19 * s->ncell); }
int64_t orc_sim_time(const orc_sim *s) { return s->t; }
double orc_sim_mass(const orc_sim *s) { return s->mass; }
int32_t orc_sim_n_modes(const orc_sim *s) { return s->N; }

void orc_sim_get_inlet(const orc_sim *s, double *u_bc)
{
    if (s->has_stg) memcpy(u_bc, s->u_bc, sizeof(double) * 3 * s->d.ny * s->d.nz);
}

void orc_sim_get_stats(const orc_sim *s, double *mean_sum, double *rey_sum, int64_t *n_samples)
{
    size_t m = (size_t)s->d.nx * s->d.ny;
    memcpy(mean_sum, s->mean_sum, sizeof(double) * 3 * m);
    memcpy(rey_sum, s->rey_sum, sizeof(double) * 6 * m);
    *n_samples = s->n_samples;
}

void orc_sim_scalars(const orc_sim *s, double *o)
{
    o[0] = s->c_x; o[1] = s->c_t; o[2] = s->U_b; o[3] = s->max_le;
    o[4] = s->k_min; o[5] = s->k_max; o[6] = (double)s->N; o[7] = s->a_filter;
}

void orc_sim_tables(const orc_sim *s, double *u_int, double *a6, double *l_e, double *q,
                    double *kn, double *d3, double *sigma3, double *phi)
{
    int ny = s->d.ny, N = s->N;
    if (!s->has_stg) return;
    memcpy(u_int, s->u_int, sizeof(double) * ny);
    memcpy(a6, s->a6, sizeof(double) * 6 * ny);
    memcpy(l_e, s->le, sizeof(double) * ny);
    memcpy(q, s->q, sizeof(double) * (size_t)ny * N);
    memcpy(kn, s->kn, sizeof(double) * N);
    memcpy(d3, s->d3, sizeof(double) * 3 * N);
    memcpy(sigma3, s->sig3, sizeof(double) * 3 * N);
    memcpy(phi, s->phi, sizeof(double) * N);
}

/* Inlet velocity for step t: Algorithm 1 steps 5-8, eqs. (u_phys),
 * (u_transfer); the fluctuation is filtered in time before it is added. */
static void stg_plane(orc_sim *s)
{
    const int ny = s->d.ny, nz = s->d.nz;
    const size_t plane = (size_t)ny * nz;
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j) {
            double u3[3];
            orc_sim_stg_raw(s, (double)s->t, j, k, u3);
            for (int a = 0; a < 3; ++a) s->u_raw[a * plane + (size_t)k * ny + j] = u3[a];
        }
    orc_filter_update(!s->filt_init, s->a_filter, s->u_raw, s->u_f, (int32_t)(3 * plane));
    s->filt_init = 1;
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j) {
            size_t c = (size_t)k * ny + j;
            s->u_bc[c] = s->u_int[j] + s->u_f[c];
            s->u_bc[plane + c] = s->u_f[plane + c];
            s->u_bc[2 * plane + c] = s->u_f[2 * plane + c];
        }
}

void orc_sim_step(orc_sim *s, int32_t n)
{
    const orc_domain *d = &s->d;
    const int nx = d->nx, ny = d->ny, nz = d->nz;
    const size_t plane = (size_t)ny * nz;
    for (int32_t step = 0; step < n; ++step) {
        if (s->has_stg) stg_plane(s);
#pragma omp parallel for schedule(static)
        for (int z = 0; z < nz; ++z)
            for (int y = 0; y < ny; ++y)
                for (int x = 0; x < nx; ++x) {
                    double out[Q19], rho, u[3], ub[3] = {0.0, 0.0, 0.0};
                    if (s->has_stg && x == 0)
                        for (int a = 0; a < 3; ++a) ub[a] = s->u_bc[a * plane + (size_t)z * ny + y];
                    cell_update(d, 0, s->f, x, y, z, ub, out, &rho, u);
                    size_t c = ((size_t)z * ny + y) * nx + x;
                    for (int i = 0; i < Q19; ++i) s->g[(size_t)i * s->ncell + c] = out[i];
                    s->rho_cell[c] = rho;
                    for (int a = 0; a < 3; ++a) s->u_cell[3 * c + a] = u[a];
                }
        double *tmp = s->f; s->f = s->g; s->g = tmp;
        /* mass of the step, summed in cell order */
        double m = 0.0;
        for (size_t c = 0; c < s->ncell; ++c) m += s->rho_cell[c];
        s->mass = m;
        /* running statistics (sums over z and time of u and u u, per (x, y)) */
        if (d->stats_every > 0 && (s->t + 1) % d->stats_every == 0) {
            for (int y = 0; y < ny; ++y)
                for (int x = 0; x < nx; ++x) {
                    size_t xy = (size_t)y * nx + x, m2 = (size_t)nx * ny;
                    for (int z = 0; z < nz; ++z) {
                        const double *u = s->u_cell + 3 * (((size_t)z * ny + y) * nx + x);
                        s->mean_sum[0 * m2 + xy] += u[0];
                        s->mean_sum[1 * m2 + xy] += u[1];
                        s->mean_sum[2 * m2 + xy] += u[2];
                        s->rey_sum[0 * m2 + xy] += u[0] * u[0];
                        s->rey_sum[1 * m2 + xy] += u[1] * u[1];
                        s->rey_sum[2 * m2 + xy] += u[2] * u[2];
                        s->rey_sum[3 * m2 + xy] += u[0] * u[1];
                        s->rey_sum[4 * m2 + xy] += u[0] * u[2];
                        s->rey_sum[5 * m2 + xy] += u[1] * u[2];
                    }
                }
            s->n_samples += 1;
        }
        s->t += 1;
    }
}
