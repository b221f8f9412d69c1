// Per-cell pieces of the fused LES-LBM step shared by the scalar and the
// two-cells-per-thread kernels: storage access, shifted equilibrium,
// regularized boundary rebuild and the regularized/BGK collision.
#pragma once

#include <cuda_fp16.h>

#include "d3q19.cuh"

namespace stg {

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

// Moments, Smagorinsky relaxation and collision of one cell, in shifted
// variables.  Both collisions are written as
//     g*_i = K g_i + w_i [a0 + c_i.B + c_i.A.c_i]
// with K = 0 for the regularized collision (eq. f_i_neq applied in the bulk)
// and K = 1 - 1/tau for plain BGK (eq. lbe); the scalar a0, vector B and
// symmetric tensor A gather the shifted equilibrium (eq. local_eq), the
// regularized non-equilibrium part and the Guo force term (eq. bodyforce):
//   regularized: a0 = drho - 1.5 rho u.u - 1.5 (1-w) tr Pi_neq - 3 kf u.F
//                B  = 3 rho u + (3 kf - 1.5 (1-w)) F
//                A  = 4.5 rho u u + 4.5 (1-w) Pi_neq + 9 kf sym(u F)
//   BGK:         a0 = w (drho - 1.5 rho u.u) - 3 kf u.F
//                B  = 3 w rho u + 3 kf F
//                A  = 4.5 w rho u u + 9 kf sym(u F)
// (w = 1/tau_eff here, kf = 1 - w/2).  Outputs: the density excess
// drho = rho - 1 (the sum of the shifted populations, before rho is rounded)
// and the velocity u.  The 18 moving populations come in
// opposite pairs, and the edge pairs (a, b, +-) share A_aa + A_bb, so the
// whole update is a few dozen fused multiply-adds.
// SP: sponge zone, eq. (sponge_visco): the cell's viscosity is nu_eff times
// nuf, i.e. tau = 1/2 + nuf (tau_eff - 1/2).
// collide_sd is the same from the pair sums s_p = g_a + g_b and differences
// d_p = g_a - g_b of the 9 opposite pairs (a = 2p+1, b = 2p+2) and
// drho0 = g_0 + s_0, which the caller may form without converting every
// population; g then only carries the input of the BGK term K g_i and
// receives the result.
template <bool REG, bool FORCE, bool SP = false>
__device__ __forceinline__ void collide_sd(float (&g)[Q], const float (&s)[9], const float (&d)[9], float drho0,
                                           float tau0, float kq, float Fx, float Fy, float Fz, float &drho_o,
                                           float &ux_o, float &uy_o, float &uz_o, float nuf = 1.0f)
{
    // moments, eqs. (density), (momentum), (tensor): rho = 1 + sum g,
    // rho u = sum c g (+ F/2), Pi = sum c c g + I/3
    float drho = drho0, jx = 0.f, jy = 0.f, jz = 0.f;
    float pxx = 0.f, pyy = 0.f, pzz = 0.f, pxy = 0.f, pxz = 0.f, pyz = 0.f;
#pragma unroll
    for (int p = 0; p < 9; ++p) {
        const int i = 2 * p + 1;
        const int cx = cx_of(i), cy = cy_of(i), cz = cz_of(i);
        if (p) drho += s[p];
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
    const float d3 = drho * (1.0f / 3.0f);
    const float nxx = pxx - d3 - rux * ux;
    const float nyy = pyy - d3 - ruy * uy;
    const float nzz = pzz - d3 - ruz * uz;
    const float nxy = pxy - rux * uy;
    const float nxz = pxz - rux * uz;
    const float nyz = pyz - ruy * uz;
    const float q2 = nxx * nxx + nyy * nyy + nzz * nzz + 2.0f * (nxy * nxy + nxz * nxz + nyz * nyz);
    const float qh = q2 > 0.f ? sqrtf(q2) : 0.f;
    // eq. (tau_eff), c = 1: tau = tau0/2 + sqrt((tau0 rho)^2 + 18 sqrt2 C Q^1/2)/(2 rho)
    float tau = 0.5f * (tau0 + sqrtf(tau0 * tau0 + kq * qh * irho * irho));
    if (SP) tau = fmaf(nuf, tau - 0.5f, 0.5f);
    const float om = 1.0f / tau;
    const float uu = ux * ux + uy * uy + uz * uz;
    const float kf = FORCE ? (1.0f - 0.5f * om) : 0.f;  // Guo prefactor
    const float uF = FORCE ? ux * Fx + uy * Fy + uz * Fz : 0.f;
    float a0, Bx, By, Bz, Axx, Ayy, Azz, Axy, Axz, Ayz, K;
    if (REG) {
        const float km = 1.0f - om;
        const float k45 = 4.5f * km;
        a0 = drho - 1.5f * rho * uu - 1.5f * km * (nxx + nyy + nzz);
        Bx = 3.0f * rux;
        By = 3.0f * ruy;
        Bz = 3.0f * ruz;
        Axx = 4.5f * rux * ux + k45 * nxx;
        Ayy = 4.5f * ruy * uy + k45 * nyy;
        Azz = 4.5f * ruz * uz + k45 * nzz;
        Axy = 4.5f * rux * uy + k45 * nxy;
        Axz = 4.5f * rux * uz + k45 * nxz;
        Ayz = 4.5f * ruy * uz + k45 * nyz;
        K = 0.f;
        if (FORCE) {
            // regularized: the first-order neq part a1 = -F/2 is kept
            const float kb = 3.0f * kf - 1.5f * km;
            Bx += kb * Fx;
            By += kb * Fy;
            Bz += kb * Fz;
        }
    } else {
        a0 = om * (drho - 1.5f * rho * uu);
        const float r3 = 3.0f * om, r45 = 4.5f * om;
        Bx = r3 * rux;
        By = r3 * ruy;
        Bz = r3 * ruz;
        Axx = r45 * rux * ux;
        Ayy = r45 * ruy * uy;
        Azz = r45 * ruz * uz;
        Axy = r45 * rux * uy;
        Axz = r45 * rux * uz;
        Ayz = r45 * ruy * uz;
        K = 1.0f - om;
        if (FORCE) {
            Bx += 3.0f * kf * Fx;
            By += 3.0f * kf * Fy;
            Bz += 3.0f * kf * Fz;
        }
    }
    if (FORCE) {
        const float k9 = 9.0f * kf;
        a0 -= 3.0f * kf * uF;
        Axx += k9 * ux * Fx;
        Ayy += k9 * uy * Fy;
        Azz += k9 * uz * Fz;
        Axy += 0.5f * k9 * (ux * Fy + uy * Fx);
        Axz += 0.5f * k9 * (ux * Fz + uz * Fx);
        Ayz += 0.5f * k9 * (uy * Fz + uz * Fy);
    }
    constexpr float W0 = 1.0f / 3.0f, W1 = 1.0f / 18.0f, W2 = 1.0f / 36.0f;
    // rest population
    g[0] = REG ? W0 * a0 : fmaf(K, g[0], W0 * a0);
    // axis pairs (1,2) +-x, (3,4) +-y, (5,6) +-z
    {
        const float w1a0 = W1 * a0;
        const float ex = fmaf(W1, Axx, w1a0), ey = fmaf(W1, Ayy, w1a0), ez = fmaf(W1, Azz, w1a0);
        const float ox = W1 * Bx, oy = W1 * By, oz = W1 * Bz;
        if (REG) {
            g[1] = ex + ox; g[2] = ex - ox;
            g[3] = ey + oy; g[4] = ey - oy;
            g[5] = ez + oz; g[6] = ez - oz;
        } else {
            g[1] = fmaf(K, g[1], ex + ox); g[2] = fmaf(K, g[2], ex - ox);
            g[3] = fmaf(K, g[3], ey + oy); g[4] = fmaf(K, g[4], ey - oy);
            g[5] = fmaf(K, g[5], ez + oz); g[6] = fmaf(K, g[6], ez - oz);
        }
    }
    // edge pairs: (7,8) +-(1,1,0), (9,10) +-(1,-1,0), (11,12) +-(1,0,1), (13,14) +-(1,0,-1),
    //             (15,16) +-(0,1,1), (17,18) +-(0,1,-1)
    {
        const float w2a0 = W2 * a0;
        const float bx = W2 * Bx, by = W2 * By, bz = W2 * Bz;
        const float sxy = fmaf(W2, Axx + Ayy, w2a0), txy = (2.0f * W2) * Axy;
        const float sxz = fmaf(W2, Axx + Azz, w2a0), txz = (2.0f * W2) * Axz;
        const float syz = fmaf(W2, Ayy + Azz, w2a0), tyz = (2.0f * W2) * Ayz;
        const float e7 = sxy + txy, e9 = sxy - txy, e11 = sxz + txz, e13 = sxz - txz, e15 = syz + tyz, e17 = syz - tyz;
        const float o7 = bx + by, o9 = bx - by, o11 = bx + bz, o13 = bx - bz, o15 = by + bz, o17 = by - bz;
        if (REG) {
            g[7] = e7 + o7; g[8] = e7 - o7;
            g[9] = e9 + o9; g[10] = e9 - o9;
            g[11] = e11 + o11; g[12] = e11 - o11;
            g[13] = e13 + o13; g[14] = e13 - o13;
            g[15] = e15 + o15; g[16] = e15 - o15;
            g[17] = e17 + o17; g[18] = e17 - o17;
        } else {
            g[7] = fmaf(K, g[7], e7 + o7); g[8] = fmaf(K, g[8], e7 - o7);
            g[9] = fmaf(K, g[9], e9 + o9); g[10] = fmaf(K, g[10], e9 - o9);
            g[11] = fmaf(K, g[11], e11 + o11); g[12] = fmaf(K, g[12], e11 - o11);
            g[13] = fmaf(K, g[13], e13 + o13); g[14] = fmaf(K, g[14], e13 - o13);
            g[15] = fmaf(K, g[15], e15 + o15); g[16] = fmaf(K, g[16], e15 - o15);
            g[17] = fmaf(K, g[17], e17 + o17); g[18] = fmaf(K, g[18], e17 - o17);
        }
    }
    drho_o = drho;
    ux_o = ux;
    uy_o = uy;
    uz_o = uz;
}

// collide: from the 19 shifted populations g of the cell
template <bool REG, bool FORCE, bool SP = false>
__device__ __forceinline__ void collide(float (&g)[Q], float tau0, float kq, float Fx, float Fy, float Fz,
                                        float &drho_o, float &ux_o, float &uy_o, float &uz_o, float nuf = 1.0f)
{
    float s[9], d[9];
#pragma unroll
    for (int p = 0; p < 9; ++p) {
        s[p] = g[2 * p + 1] + g[2 * p + 2];
        d[p] = g[2 * p + 1] - g[2 * p + 2];
    }
    collide_sd<REG, FORCE, SP>(g, s, d, g[0] + s[0], tau0, kq, Fx, Fy, Fz, drho_o, ux_o, uy_o, uz_o, nuf);
}

}  // namespace stg
