// Fused LES-LBM time step for one channel lattice (Algorithm 1, step 12, with
// steps 9-11 for the inlet nodes and the outlet rebuild folded in).
//
// One pass per cell: pull the 19 post-collision populations of the previous
// step along -c_i (eq. lbe, left side) with half-way bounce-back at the y
// walls, periodic z (and optionally x, y); rebuild the inlet node (x = 0) by
// the regularized Zou-He reconstruction (Sec. III.B) and the outlet node
// (x = nx-1) by the regularized pressure outlet (Sec. IV); take the moments
// (eqs. density, momentum, tensor); set the Smagorinsky relaxation time
// (eq. tau_eff); collide (regularized or plain BGK, eqs. lbe, local_eq,
// bodyforce) and store.  On sampling steps the same pass accumulates the FP64
// velocity statistics and the FP64 mass.
//
// Layout: SoA f[i][z][y][x].  A block is 32 consecutive x (one warp row) by 8
// z-lanes at one y; each thread walks z with stride 8, so a block owns all z
// of its (x, y) column and the statistics need no atomics.
#include <cuda_fp16.h>

#include "d3q19.cuh"
#include "internal.h"

namespace stg {

constexpr int BX = 32;
constexpr int BZ = 8;

// Both storage formats hold the shifted population g_i = f_i - w_i, and all
// arithmetic below works on g: the rest weights never enter a sum, so FP32
// rounding acts on the small fluctuating part only (no weight-rounding bias
// in the mass, no loss of the low-order bits of slow flows).
template <typename S>
struct Pop;

template <>
struct Pop<float> {
    static __device__ __forceinline__ float ld(const float *p) { return __ldg(p); }
    static __device__ __forceinline__ void st(float *p, float g) { __stcs(p, g); }
};

template <>
struct Pop<__half> {
    static __device__ __forceinline__ float ld(const __half *p) { return __half2float(__ldg(p)); }
    static __device__ __forceinline__ void st(__half *p, float g) { __stcs(p, __float2half_rn(g)); }
};

// shifted equilibrium g^eq_i = f^eq_i - w_i = w_i [drho + rho (3 c.u + 4.5 (c.u)^2 - 1.5 u.u)]
__device__ __forceinline__ float geq(float w, float drho, float rho, float cu, float uu)
{
    return w * (drho + rho * (3.0f * cu + 4.5f * cu * cu - 1.5f * uu));
}

// Regularized rebuild of a boundary node (eqs. f_i, f_i_neq, pi_neq,
// unknown_neq, bc_eq): the unknown directions (sign(c_x) == SGN) take the
// non-equilibrium part of their opposite; all 19 are then replaced by
// f^eq + w_i/(2 cs^4) Q_i : Pi_neq.
template <int SGN>
__device__ __forceinline__ void rebuild(float (&g)[Q], float drho, float ux, float uy, float uz)
{
    const float rho = 1.0f + drho;
    const float uu = ux * ux + uy * uy + uz * uz;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int cx = cx_of(i), cy = cy_of(i), cz = cz_of(i);
        if (cx != SGN) g[i] = g[i] - geq(w_of(i), drho, rho, cx * ux + cy * uy + cz * uz, uu);
    }
#pragma unroll
    for (int i = 0; i < Q; ++i)
        if (cx_of(i) == SGN) g[i] = g[opp_of(i)];
    float s = 0.f, pxx = 0.f, pyy = 0.f, pzz = 0.f, pxy = 0.f, pxz = 0.f, pyz = 0.f;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int cx = cx_of(i), cy = cy_of(i), cz = cz_of(i);
        const float v = g[i];
        s += v;
        if (cx * cx) pxx += v;
        if (cy * cy) pyy += v;
        if (cz * cz) pzz += v;
        if (cx * cy) pxy += cx * cy * v;
        if (cx * cz) pxz += cx * cz * v;
        if (cy * cz) pyz += cy * cz * v;
    }
    // Pi_neq = sum_i Q_i f_i^neq with Q_i = c_i c_i - I/3
    pxx -= s * (1.0f / 3.0f);
    pyy -= s * (1.0f / 3.0f);
    pzz -= s * (1.0f / 3.0f);
    const float tr3 = (pxx + pyy + pzz) * (1.0f / 3.0f);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int cx = cx_of(i), cy = cy_of(i), cz = cz_of(i);
        const float cpc = cx * cx * pxx + cy * cy * pyy + cz * cz * pzz
                        + 2.0f * (cx * cy * pxy + cx * cz * pxz + cy * cz * pyz);
        g[i] = geq(w_of(i), drho, rho, cx * ux + cy * uy + cz * uz, uu) + 4.5f * w_of(i) * (cpc - tr3);
    }
}

// Pull of the 19 populations of cell `here` for a warp whose cells and all
// their x/y neighbours are inside the lattice (no wall, no inlet/outlet lane,
// no x/y wrap): the source of population i is srci[i] + (cell index of the
// source z row), srci[i] already carrying the -(c_x + c_y nx) shift; hzm /
// hzp are `here` moved to the z-1 / z+1 row (periodic wrap at the ends).
template <typename S>
__device__ __forceinline__ void gather_interior(const StepArgs &a, unsigned here, unsigned hzm, unsigned hzp,
                                                float (&g)[Q])
{
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int cz = cz_of(i);
        const unsigned h = cz > 0 ? hzm : (cz < 0 ? hzp : here);
        g[i] = Pop<S>::ld(static_cast<const S *>(a.srci[i]) + h);
    }
}

// General pull: half-way bounce-back at y walls, periodic wraps, unknown
// (c_x pointing in from outside) populations at the inlet/outlet set to 0.
template <typename S>
__device__ __forceinline__ void gather_general(const S *__restrict__ src, unsigned P, int nx, int ny, int x, int y,
                                               int z, int xm, int xp, bool xm_ok, bool xp_ok, int ym, int yp,
                                               bool ym_w, bool yp_w, int zm, int zp, unsigned here, float (&g)[Q])
{
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int cx = cx_of(i), cy = cy_of(i), cz = cz_of(i);
        const int xs = cx == 0 ? x : (cx > 0 ? xm : xp);
        const bool xok = cx == 0 ? true : (cx > 0 ? xm_ok : xp_ok);
        const int ys = cy == 0 ? y : (cy > 0 ? ym : yp);
        const bool yw = cy == 0 ? false : (cy > 0 ? ym_w : yp_w);
        const int zs = cz == 0 ? z : (cz > 0 ? zm : zp);
        const unsigned cell = ((unsigned)zs * ny + ys) * nx + xs;
        const unsigned pl = yw ? (unsigned)opp_of(i) : (unsigned)i;
        const unsigned c2 = yw ? here : cell;
        g[i] = (yw || xok) ? Pop<S>::ld(src + (size_t)pl * P + c2) : 0.0f;
    }
}

// Moments, Smagorinsky relaxation and collision of one cell, in shifted
// variables, written over opposite pairs (i, i+1), c_{i+1} = -c_i: every
// term of the update is either even in c (equilibrium second order,
// regularized non-equilibrium, force x velocity) or odd (first order), so
// each pair costs one even and one odd part.
template <bool REG, bool FORCE>
__device__ __forceinline__ void collide(float (&g)[Q], float tau0, float kq, float Fx, float Fy, float Fz,
                                        float &rho_o, float &ux_o, float &uy_o, float &uz_o)
{
    float s[9], d[9];
#pragma unroll
    for (int p = 0; p < 9; ++p) {
        s[p] = g[2 * p + 1] + g[2 * p + 2];
        d[p] = g[2 * p + 1] - g[2 * p + 2];
    }
    float drho = g[0], jx = 0.f, jy = 0.f, jz = 0.f;
    float pxx = 0.f, pyy = 0.f, pzz = 0.f, pxy = 0.f, pxz = 0.f, pyz = 0.f;
#pragma unroll
    for (int p = 0; p < 9; ++p) {
        const int i = 2 * p + 1;
        const int cx = cx_of(i), cy = cy_of(i), cz = cz_of(i);
        drho += s[p];
        if (cx) jx += cx * d[p];
        if (cy) jy += cy * d[p];
        if (cz) jz += cz * d[p];
        if (cx) pxx += s[p];
        if (cy) pyy += s[p];
        if (cz) pzz += s[p];
        if (cx * cy) pxy += cx * cy * s[p];
        if (cx * cz) pxz += cx * cz * s[p];
        if (cy * cz) pyz += cy * cz * s[p];
    }
    const float rho = 1.0f + drho;
    const float irho = 1.0f / rho;
    const float ux = (FORCE ? jx + 0.5f * Fx : jx) * irho;
    const float uy = (FORCE ? jy + 0.5f * Fy : jy) * irho;
    const float uz = (FORCE ? jz + 0.5f * Fz : jz) * irho;
    // Pi_neq = Pi - rho (cs^2 I + u u) = sum c c g - drho/3 I - rho u u
    const float rux = rho * ux, ruy = rho * uy, ruz = rho * uz;
    const float nxx = pxx - drho * (1.0f / 3.0f) - rux * ux;
    const float nyy = pyy - drho * (1.0f / 3.0f) - ruy * uy;
    const float nzz = pzz - drho * (1.0f / 3.0f) - ruz * uz;
    const float nxy = pxy - rux * uy;
    const float nxz = pxz - rux * uz;
    const float nyz = pyz - ruy * uz;
    const float qh = sqrtf(nxx * nxx + nyy * nyy + nzz * nzz + 2.0f * (nxy * nxy + nxz * nxz + nyz * nyz));
    // eq. (tau_eff), c = 1: tau = tau0/2 + sqrt((tau0 rho)^2 + 18 sqrt2 C Q^1/2)/(2 rho)
    const float tau = 0.5f * tau0 + 0.5f * sqrtf(tau0 * tau0 + kq * qh * irho * irho);
    const float om = 1.0f / tau;
    const float uu = ux * ux + uy * uy + uz * uz;
    const float tr3 = (nxx + nyy + nzz) * (1.0f / 3.0f);
    const float uF = FORCE ? ux * Fx + uy * Fy + uz * Fz : 0.f;
    const float kneq = REG ? 4.5f * (1.0f - om) : 0.f;   // (1 - 1/tau) w_i/(2 cs^4) / w_i
    const float kf = FORCE ? (1.0f - 0.5f * om) : 0.f;   // Guo prefactor
    // base of the even part shared by all directions: drho - 1.5 rho u.u
    const float e0 = drho - 1.5f * rho * uu;
    // rest population
    {
        const float w = w_of(0);
        float ge = w * e0;
        if (REG) {
            float go = ge - w * kneq * tr3;
            if (FORCE) go += kf * w * (-3.0f * uF);
            g[0] = go;
        } else {
            float go = g[0] - om * (g[0] - ge);
            if (FORCE) go += kf * w * (-3.0f * uF);
            g[0] = go;
        }
    }
#pragma unroll
    for (int p = 0; p < 9; ++p) {
        const int i = 2 * p + 1;
        const int cx = cx_of(i), cy = cy_of(i), cz = cz_of(i);
        const float w = w_of(i);
        const float cu = cx * ux + cy * uy + cz * uz;
        // even and odd parts of the shifted equilibrium: w [e0 + 4.5 rho cu^2] +- w 3 rho cu
        float ev = w * (e0 + 4.5f * rho * cu * cu);
        float od = w * 3.0f * rho * cu;
        if (REG) {
            const float cpc = cx * cx * nxx + cy * cy * nyy + cz * cz * nzz
                            + 2.0f * (cx * cy * nxy + cx * cz * nxz + cy * cz * nyz);
            ev += w * kneq * (cpc - tr3);
        }
        if (FORCE) {
            const float cF = cx * Fx + cy * Fy + cz * Fz;
            // Guo term, eq. (bodyforce): even part 9 (c.u)(c.F) - 3 u.F, odd part 3 c.F
            ev += kf * w * (9.0f * cu * cF - 3.0f * uF);
            od += kf * w * 3.0f * cF;
            // regularized: keep the first-order neq part a1 = -F/2
            if (REG) od -= (1.0f - om) * 1.5f * w * cF;
        }
        if (REG) {
            g[i] = ev + od;
            g[i + 1] = ev - od;
        } else {
            g[i] = g[i] - om * (g[i] - (ev + od));
            g[i + 1] = g[i + 1] - om * (g[i + 1] - (ev - od));
            if (FORCE) {
                // the Guo parts were folded into ev/od above; undo the relaxation on them
                const float cF = cx * Fx + cy * Fy + cz * Fz;
                const float fe = kf * w * (9.0f * cu * cF - 3.0f * uF), fo = kf * w * 3.0f * cF;
                g[i] += (1.0f - om) * (fe + fo);
                g[i + 1] += (1.0f - om) * (fe - fo);
            }
        }
    }
    rho_o = rho;
    ux_o = ux;
    uy_o = uy;
    uz_o = uz;
}

// One block = one (x chunk, y) column over all z.  EDGE selects the general
// pull (walls, wraps, inlet/outlet rebuild); the interior variant only sees
// columns whose x chunk is neither the first nor the last and whose y has
// both neighbours inside the lattice.
template <typename S, bool REG, bool FORCE, bool EDGE>
__device__ __forceinline__ void step_column(const StepArgs &a, int bx, int y)
{
    const S *__restrict__ src = static_cast<const S *>(a.src);
    S *__restrict__ dst = static_cast<S *>(a.dst);
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int nxy = nx * ny;
    const unsigned P = a.P;
    const int x = bx * BX + threadIdx.x;
    const int tz = threadIdx.y;
    const long long t = a.ctl->t[a.parity];
    const bool do_stats = a.stats_every > 0 && ((t + 1) % a.stats_every) == 0;
    const bool do_check = a.check_every > 0 && ((t + 1) % a.check_every) == 0;

    float su0 = 0.f, su1 = 0.f, su2 = 0.f;
    float s00 = 0.f, s11 = 0.f, s22 = 0.f, s01 = 0.f, s02 = 0.f, s12 = 0.f;
    float sdr = 0.f;

    if (x < nx) {
        const float tau0 = a.tau0, kq = a.kq;
        const float Fx = a.Fx, Fy = a.Fy, Fz = a.Fz;
        int xm = 0, xp = 0, ym = 0, yp = 0;
        bool xm_ok = true, xp_ok = true, ym_w = false, yp_w = false;
        const bool inout = (a.bc_x == 0);
        if (EDGE) {
            xm = x - 1;
            xp = x + 1;
            if (inout) {
                xm_ok = xm >= 0;
                xp_ok = xp < nx;
                xm = max(xm, 0);
                xp = min(xp, nx - 1);
            } else {
                if (xm < 0) xm += nx;
                if (xp >= nx) xp -= nx;
            }
            ym = y - 1;
            yp = y + 1;
            if (a.bc_y == 0) {
                ym_w = ym < 0;
                yp_w = yp >= ny;
                ym = max(ym, 0);
                yp = min(yp, ny - 1);
            } else {
                if (ym < 0) ym += ny;
                if (yp >= ny) yp -= ny;
            }
        }
        for (int z = tz; z < nz; z += BZ) {
            const unsigned here = ((unsigned)z * ny + y) * nx + x;
            float g[Q];
            if (!EDGE) {
                const int dzm = (z == 0) ? -(nz - 1) * nxy : nxy;
                const int dzp = (z == nz - 1) ? (nz - 1) * nxy : -nxy;
                gather_interior<S>(a, here, here - dzm, here - dzp, g);
            } else {
                const int zm = (z == 0) ? nz - 1 : z - 1;
                const int zp = (z == nz - 1) ? 0 : z + 1;
                gather_general<S>(src, P, nx, ny, x, y, z, xm, xp, xm_ok, xp_ok, ym, yp, ym_w, yp_w, zm, zp, here, g);
                if (inout && (x == 0 || x == nx - 1)) {
                    if (x == 0) {
                        const size_t pc = (size_t)z * ny + y, pl3 = (size_t)ny * nz;
                        const float ubx = a.ubc[pc], uby = a.ubc[pl3 + pc], ubz = a.ubc[2 * pl3 + pc];
                        // Zou-He density, eq. (density_bc): parallel set + 2 x leaving set.
                        // The weights of that combination sum to 1 (2/3 + 2 x 1/6), so
                        // rho_bc - 1 = (S_g + u_x)/(1 - u_x) with S_g the same sum of g.
                        float par = 0.f, lv = 0.f;
#pragma unroll
                        for (int i = 0; i < Q; ++i) {
                            if (cx_of(i) == 0) par += g[i];
                            if (cx_of(i) < 0) lv += g[i];
                        }
                        const float drb = (par + 2.0f * lv + ubx) / (1.0f - ubx);
                        rebuild<1>(g, drb, ubx, uby, ubz);
                    } else {
                        // zero-gradient velocity from the stored column x = nx-2, rho = 1
                        const unsigned nb = ((unsigned)z * ny + y) * nx + (nx - 2);
                        float r = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
                        for (int i = 0; i < Q; ++i) {
                            const float v = Pop<S>::ld(src + (size_t)i * P + nb);
                            r += v;
                            jx += cx_of(i) * v;
                            jy += cy_of(i) * v;
                            jz += cz_of(i) * v;
                        }
                        const float ir = 1.0f / (1.0f + r);
                        rebuild<-1>(g, 0.0f, jx * ir, jy * ir, jz * ir);
                    }
                }
            }
            float rho, ux, uy, uz;
            collide<REG, FORCE>(g, tau0, kq, Fx, Fy, Fz, rho, ux, uy, uz);
#pragma unroll
            for (int i = 0; i < Q; ++i) Pop<S>::st(static_cast<S *>(a.dstp[i]) + here, g[i]);
            if (do_stats) {
                su0 += ux; su1 += uy; su2 += uz;
                s00 += ux * ux; s11 += uy * uy; s22 += uz * uz;
                s01 += ux * uy; s02 += ux * uz; s12 += uy * uz;
            }
            if (do_check) sdr += rho - 1.0f;
        }
    }

    if (do_stats) {
        __shared__ float red[9][BZ][BX];
        const int tx = threadIdx.x;
        red[0][tz][tx] = su0; red[1][tz][tx] = su1; red[2][tz][tx] = su2;
        red[3][tz][tx] = s00; red[4][tz][tx] = s11; red[5][tz][tx] = s22;
        red[6][tz][tx] = s01; red[7][tz][tx] = s02; red[8][tz][tx] = s12;
        __syncthreads();
        if (tz == 0 && x < nx) {
            const size_t xy = (size_t)y * nx + x, m = (size_t)nx * ny;
#pragma unroll
            for (int q = 0; q < 9; ++q) {
                double sacc = 0.0;
                for (int k = 0; k < BZ; ++k) sacc += (double)red[q][k][tx];
                if (q < 3) a.stat_mean[q * m + xy] += sacc;
                else a.stat_rey[(q - 3) * m + xy] += sacc;
            }
        }
    }

    if (do_check) {
        // block partial, then the last of all nxc*ny blocks (both kernels)
        // adds the partials in index order: deterministic FP64 mass
        __shared__ double rd[BZ * BX];
        __shared__ int s_last;
        const int tid = threadIdx.y * BX + threadIdx.x;
        rd[tid] = (double)sdr;
        __syncthreads();
        for (int off = BZ * BX / 2; off > 0; off >>= 1) {
            if (tid < off) rd[tid] += rd[tid + off];
            __syncthreads();
        }
        const int nxc = (nx + BX - 1) / BX;
        const unsigned nblocks = (unsigned)nxc * ny;
        if (tid == 0) {
            a.mass_partial[(size_t)y * nxc + bx] = rd[0];
            __threadfence();
            const unsigned prev = atomicAdd(a.mass_counter, 1u);
            s_last = (prev == nblocks - 1);
        }
        __syncthreads();
        if (s_last) {
            __threadfence();
            double acc = 0.0;
            for (unsigned k = tid; k < nblocks; k += BZ * BX) acc += __ldcg(a.mass_partial + k);
            rd[tid] = acc;
            __syncthreads();
            for (int off = BZ * BX / 2; off > 0; off >>= 1) {
                if (tid < off) rd[tid] += rd[tid + off];
                __syncthreads();
            }
            if (tid == 0) {
                a.mass_out[0] = rd[0] + (double)P;
                *a.mass_counter = 0u;
            }
        }
    }
}

// Interior columns: x chunks 1..nxc-2, y = 1..ny-2.
template <typename S, bool REG, bool FORCE>
__global__ void __launch_bounds__(BX *BZ, 4) lbm_step_kernel(const StepArgs a)
{
    step_column<S, REG, FORCE, false>(a, blockIdx.x + 1, blockIdx.y + 1);
}

// Edge columns: x chunks 0 and nxc-1 for every y, then y = 0 and y = ny-1
// for the interior x chunks.  It also advances the device step counter
// (read by the next step's kernels only).
template <typename S, bool REG, bool FORCE>
__global__ void __launch_bounds__(BX *BZ, 2) lbm_edge_kernel(const StepArgs a)
{
    const int nxc = (a.nx + BX - 1) / BX;
    const int b = blockIdx.x;
    const int nedge_x = (nxc > 1 ? 2 : 1) * a.ny;
    int bx, y;
    if (b < nedge_x) {
        bx = (nxc > 1 && b >= a.ny) ? nxc - 1 : 0;
        y = (nxc > 1 && b >= a.ny) ? b - a.ny : b;
    } else {
        const int r = b - nedge_x;       // interior x chunks, rows y = 0 and y = ny-1
        const int nin = nxc - 2;
        bx = 1 + (r % nin);
        y = (r / nin == 0) ? 0 : a.ny - 1;
    }
    const long long t = a.ctl->t[a.parity];
    step_column<S, REG, FORCE, true>(a, bx, y);
    if (b == 0 && threadIdx.x == 0 && threadIdx.y == 0) a.ctl->t[a.parity ^ 1] = t + 1;
}

int step_grid_blocks(int nx, int ny) { return ((nx + BX - 1) / BX) * ny; }

// interior grid (x chunks 1..nxc-2) x (y 1..ny-2) and the number of edge
// columns; interior + edge = nxc * ny, each column exactly once.
static void edge_counts(int nx, int ny, int &n_interior_x, int &n_interior_y, int &n_edge)
{
    const int nxc = (nx + BX - 1) / BX;
    n_interior_x = nxc > 2 ? nxc - 2 : 0;
    n_interior_y = ny > 2 ? ny - 2 : 0;
    n_edge = (nxc > 1 ? 2 : 1) * ny + (ny >= 2 ? 2 : 1) * n_interior_x;
}

template <typename S, bool REG>
static void launch_typed(const StepArgs &a, cudaStream_t s, cudaStream_t side)
{
    int nix, niy, ne;
    edge_counts(a.nx, a.ny, nix, niy, ne);
    const dim3 block(BX, BZ);
    if (a.has_force) {
        lbm_edge_kernel<S, REG, true><<<ne, block, 0, side>>>(a);
        if (nix > 0 && niy > 0) lbm_step_kernel<S, REG, true><<<dim3(nix, niy), block, 0, s>>>(a);
    } else {
        lbm_edge_kernel<S, REG, false><<<ne, block, 0, side>>>(a);
        if (nix > 0 && niy > 0) lbm_step_kernel<S, REG, false><<<dim3(nix, niy), block, 0, s>>>(a);
    }
}

// One fused step pass.  With a side stream and two events the edge columns
// run on a forked branch concurrently with the interior columns (both read
// only the previous lattice and write disjoint cells); `s` waits for both.
cudaError_t launch_step(const StepArgs &a, int storage, int collision, cudaStream_t s, cudaStream_t side,
                        cudaEvent_t fork, cudaEvent_t join)
{
    cudaError_t e = cudaSuccess;
    const bool forked = side != nullptr && fork != nullptr && join != nullptr;
    if (forked) {
        if ((e = cudaEventRecord(fork, s)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(side, fork, 0)) != cudaSuccess) return e;
    }
    cudaStream_t es = forked ? side : s;
    if (storage == 0) {
        if (collision == 0) launch_typed<float, true>(a, s, es);
        else launch_typed<float, false>(a, s, es);
    } else {
        if (collision == 0) launch_typed<__half, true>(a, s, es);
        else launch_typed<__half, false>(a, s, es);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (forked) {
        if ((e = cudaEventRecord(join, side)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(s, join, 0)) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// ---------------------------------------------------------------------------
// Initial state f^eq(1, (u_int(y), 0, 0)) (u_int == nullptr: rest state),
// stored shifted.
template <typename S>
__global__ void init_eq_kernel(S *dst, int nx, int ny, int nz, const float *u_int)
{
    const size_t P = (size_t)nx * ny * nz;
    for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < P; c += (size_t)gridDim.x * blockDim.x) {
        const int y = (int)((c / nx) % ny);
        const float ux = u_int ? u_int[y] : 0.0f;
#pragma unroll
        for (int i = 0; i < Q; ++i) Pop<S>::st(dst + (size_t)i * P + c, geq(w_of(i), 0.0f, 1.0f, cx_of(i) * ux, ux * ux));
    }
}

cudaError_t launch_init_equilibrium(void *dst, int storage, int nx, int ny, int nz, const float *u_int, cudaStream_t s)
{
    const int blocks = 152 * 8;
    if (storage == 0) init_eq_kernel<float><<<blocks, 256, 0, s>>>(static_cast<float *>(dst), nx, ny, nz, u_int);
    else init_eq_kernel<__half><<<blocks, 256, 0, s>>>(static_cast<__half *>(dst), nx, ny, nz, u_int);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// FP64 mass of a stored lattice, sum over cells and populations, in a fixed
// reduction order (block partials, then the last block to finish adds them
// in index order).
constexpr int MASS_BLOCKS = 152 * 4;
constexpr int MASS_THREADS = 256;

template <typename S>
__global__ void __launch_bounds__(MASS_THREADS) mass_kernel(const MassArgs a)
{
    const S *src = static_cast<const S *>(a.src);
    __shared__ double rd[MASS_THREADS];
    __shared__ int s_last;
    double acc = 0.0;
    for (size_t c = blockIdx.x * (size_t)MASS_THREADS + threadIdx.x; c < a.P; c += (size_t)gridDim.x * MASS_THREADS) {
        float r = 0.f;
#pragma unroll
        for (int i = 0; i < Q; ++i) r += Pop<S>::ld(src + (size_t)i * a.P + c);
        acc += (double)r;
    }
    const int tid = threadIdx.x;
    rd[tid] = acc;
    __syncthreads();
    for (int off = MASS_THREADS / 2; off > 0; off >>= 1) {
        if (tid < off) rd[tid] += rd[tid + off];
        __syncthreads();
    }
    if (tid == 0) {
        a.partial[blockIdx.x] = rd[0];
        __threadfence();
        s_last = (atomicAdd(a.counter, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (s_last) {
        double v = 0.0;
        for (unsigned k = tid; k < gridDim.x; k += MASS_THREADS) v += __ldcg(a.partial + k);
        rd[tid] = v;
        __syncthreads();
        for (int off = MASS_THREADS / 2; off > 0; off >>= 1) {
            if (tid < off) rd[tid] += rd[tid + off];
            __syncthreads();
        }
        if (tid == 0) {
            a.out[0] = rd[0] + (double)a.P;
            *a.counter = 0u;
        }
    }
}

int mass_grid_blocks() { return MASS_BLOCKS; }

cudaError_t launch_mass(const MassArgs &a, cudaStream_t s)
{
    if (a.storage == 0) mass_kernel<float><<<MASS_BLOCKS, MASS_THREADS, 0, s>>>(a);
    else mass_kernel<__half><<<MASS_BLOCKS, MASS_THREADS, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace stg
