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

// Every multiply-add below is written out: a product that feeds an addition
// is either fused by an explicit fmaf or formed by __fmul_rn, which the
// compiler may not fuse.  Left to itself the compiler contracts such pairs
// differently in different kernel instances, and the instances that share
// this code (tiles, sampling and plain steps, both streaming schemes) must
// round every cell alike.

// c_i . u for a lattice direction (components in {-1, 0, 1}), no products
__device__ __forceinline__ float cdot(int cx, int cy, int cz, float ux, float uy, float uz)
{
    float r = cx > 0 ? ux : (cx < 0 ? -ux : 0.f);
    if (cy) r = cx ? (cy > 0 ? r + uy : r - uy) : (cy > 0 ? uy : -uy);
    if (cz) r = (cx || cy) ? (cz > 0 ? r + uz : r - uz) : (cz > 0 ? uz : -uz);
    return r;
}

// shifted equilibrium g^eq_i = f^eq_i - w_i = w_i [drho + rho (3 c.u + 4.5 (c.u)^2 - 1.5 u.u)]
__device__ __forceinline__ float geq(float w, float drho, float rho, float cu, float uu)
{
    return __fmul_rn(w, fmaf(rho, fmaf(cu, fmaf(4.5f, cu, 3.0f), -1.5f * uu), drho));
}

// Regularized rebuild of a boundary node (eqs. f_i, f_i_neq, pi_neq,
// unknown_neq, bc_eq): the unknown directions (sign(c_x) == SGN) take the
// non-equilibrium part of their opposite; all 19 are then replaced by
// f^eq + w_i/(2 cs^4) Q_i : Pi_neq.
template <int SGN>
__device__ __forceinline__ void rebuild(float (&g)[Q], float drho, float ux, float uy, float uz)
{
    const float rho = 1.0f + drho;
    const float uu = fmaf(uz, uz, fmaf(uy, uy, ux * ux));
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int cx = cx_of(i), cy = cy_of(i), cz = cz_of(i);
        if (cx != SGN) g[i] = g[i] - geq(w_of(i), drho, rho, cdot(cx, cy, cz, ux, uy, uz), uu);
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
    pxx = fmaf(-1.0f / 3.0f, s, pxx);
    pyy = fmaf(-1.0f / 3.0f, s, pyy);
    pzz = fmaf(-1.0f / 3.0f, s, pzz);
    const float tsum = (pxx + pyy) + pzz;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int cx = cx_of(i), cy = cy_of(i), cz = cz_of(i);
        // c.Pi.c = diagonal part + 2 x off-diagonal part (the terms with c_a c_b != 0)
        float dg = 0.f, od = 0.f;
        if (cx) dg = pxx;
        if (cy) dg = cx ? dg + pyy : pyy;
        if (cz) dg = (cx || cy) ? dg + pzz : pzz;
        if (cx * cy) od = cx * cy > 0 ? pxy : -pxy;
        if (cx * cz) od = cx * cz > 0 ? pxz : -pxz;
        if (cy * cz) od = cy * cz > 0 ? pyz : -pyz;
        const float cpc = (cx * cy || cx * cz || cy * cz) ? fmaf(2.0f, od, dg) : dg;
        g[i] = fmaf(4.5f * w_of(i), fmaf(-1.0f / 3.0f, tsum, cpc),
                    geq(w_of(i), drho, rho, cdot(cx, cy, cz, ux, uy, uz), uu));
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
    const float ux = (FORCE ? fmaf(0.5f, Fx, jx) : jx) * irho;
    const float uy = (FORCE ? fmaf(0.5f, Fy, jy) : jy) * irho;
    const float uz = (FORCE ? fmaf(0.5f, Fz, jz) : jz) * irho;
    // Pi_neq = Pi - rho (cs^2 I + u u) = sum c c g - drho/3 I - rho u u
    const float rux = rho * ux, ruy = rho * uy, ruz = rho * uz;
    const float nxx = fmaf(-rux, ux, fmaf(-1.0f / 3.0f, drho, pxx));
    const float nyy = fmaf(-ruy, uy, fmaf(-1.0f / 3.0f, drho, pyy));
    const float nzz = fmaf(-ruz, uz, fmaf(-1.0f / 3.0f, drho, pzz));
    const float nxy = fmaf(-rux, uy, pxy);
    const float nxz = fmaf(-rux, uz, pxz);
    const float nyz = fmaf(-ruy, uz, pyz);
    const float q2 = fmaf(2.0f, fmaf(nyz, nyz, fmaf(nxz, nxz, nxy * nxy)), fmaf(nzz, nzz, fmaf(nyy, nyy, nxx * nxx)));
    const float qh = q2 > 0.f ? sqrtf(q2) : 0.f;
    // eq. (tau_eff), c = 1: tau = tau0/2 + sqrt((tau0 rho)^2 + 18 sqrt2 C Q^1/2)/(2 rho)
    float tau = 0.5f * (tau0 + sqrtf(fmaf(kq * qh, irho * irho, tau0 * tau0)));
    if (SP) tau = fmaf(nuf, tau - 0.5f, 0.5f);
    const float om = 1.0f / tau;
    const float uu = fmaf(uz, uz, fmaf(uy, uy, ux * ux));
    const float kf = FORCE ? fmaf(-0.5f, om, 1.0f) : 0.f;  // Guo prefactor
    const float uF = FORCE ? fmaf(uz, Fz, fmaf(uy, Fy, ux * Fx)) : 0.f;
    float a0, Bx, By, Bz, Axx, Ayy, Azz, Axy, Axz, Ayz, K;
    if (REG) {
        const float km = 1.0f - om;
        const float k45 = 4.5f * km;
        a0 = fmaf(-1.5f, fmaf(km, (nxx + nyy) + nzz, rho * uu), drho);
        Bx = 3.0f * rux;
        By = 3.0f * ruy;
        Bz = 3.0f * ruz;
        Axx = fmaf(k45, nxx, (4.5f * rux) * ux);
        Ayy = fmaf(k45, nyy, (4.5f * ruy) * uy);
        Azz = fmaf(k45, nzz, (4.5f * ruz) * uz);
        Axy = fmaf(k45, nxy, (4.5f * rux) * uy);
        Axz = fmaf(k45, nxz, (4.5f * rux) * uz);
        Ayz = fmaf(k45, nyz, (4.5f * ruy) * uz);
        K = 0.f;
        if (FORCE) {
            // regularized: the first-order neq part a1 = -F/2 is kept
            const float kb = fmaf(3.0f, kf, -1.5f * km);
            Bx = fmaf(kb, Fx, Bx);
            By = fmaf(kb, Fy, By);
            Bz = fmaf(kb, Fz, Bz);
        }
    } else {
        a0 = om * fmaf(-1.5f * rho, uu, drho);
        const float r3 = 3.0f * om, r45 = 4.5f * om;
        Bx = r3 * rux;
        By = r3 * ruy;
        Bz = r3 * ruz;
        Axx = __fmul_rn(r45 * rux, ux);
        Ayy = __fmul_rn(r45 * ruy, uy);
        Azz = __fmul_rn(r45 * ruz, uz);
        Axy = __fmul_rn(r45 * rux, uy);
        Axz = __fmul_rn(r45 * rux, uz);
        Ayz = __fmul_rn(r45 * ruy, uz);
        K = 1.0f - om;
        if (FORCE) {
            Bx = fmaf(3.0f * kf, Fx, Bx);
            By = fmaf(3.0f * kf, Fy, By);
            Bz = fmaf(3.0f * kf, Fz, Bz);
        }
    }
    if (FORCE) {
        const float k9 = 9.0f * kf, k45 = 4.5f * kf;
        a0 = fmaf(-3.0f * kf, uF, a0);
        Axx = fmaf(k9 * ux, Fx, Axx);
        Ayy = fmaf(k9 * uy, Fy, Ayy);
        Azz = fmaf(k9 * uz, Fz, Azz);
        Axy = fmaf(k45, fmaf(ux, Fy, uy * Fx), Axy);
        Axz = fmaf(k45, fmaf(ux, Fz, uz * Fx), Axz);
        Ayz = fmaf(k45, fmaf(uy, Fz, uz * Fy), Ayz);
    }
    constexpr float W0 = 1.0f / 3.0f, W1 = 1.0f / 18.0f, W2 = 1.0f / 36.0f;
    // rest population
    g[0] = REG ? W0 * a0 : fmaf(K, g[0], W0 * a0);
    // axis pairs (1,2) +-x, (3,4) +-y, (5,6) +-z
    {
        const float w1a0 = W1 * a0;
        const float ex = fmaf(W1, Axx, w1a0), ey = fmaf(W1, Ayy, w1a0), ez = fmaf(W1, Azz, w1a0);
        const float px = fmaf(W1, Bx, ex), mx = fmaf(-W1, Bx, ex);
        const float py = fmaf(W1, By, ey), my = fmaf(-W1, By, ey);
        const float pz = fmaf(W1, Bz, ez), mz = fmaf(-W1, Bz, ez);
        if (REG) {
            g[1] = px; g[2] = mx;
            g[3] = py; g[4] = my;
            g[5] = pz; g[6] = mz;
        } else {
            g[1] = fmaf(K, g[1], px); g[2] = fmaf(K, g[2], mx);
            g[3] = fmaf(K, g[3], py); g[4] = fmaf(K, g[4], my);
            g[5] = fmaf(K, g[5], pz); g[6] = fmaf(K, g[6], mz);
        }
    }
    // edge pairs: (7,8) +-(1,1,0), (9,10) +-(1,-1,0), (11,12) +-(1,0,1), (13,14) +-(1,0,-1),
    //             (15,16) +-(0,1,1), (17,18) +-(0,1,-1)
    {
        const float w2a0 = W2 * a0;
        const float bx = __fmul_rn(W2, Bx), by = __fmul_rn(W2, By), bz = __fmul_rn(W2, Bz);
        const float sxy = fmaf(W2, Axx + Ayy, w2a0), sxz = fmaf(W2, Axx + Azz, w2a0), syz = fmaf(W2, Ayy + Azz, w2a0);
        const float e7 = fmaf(2.0f * W2, Axy, sxy), e9 = fmaf(-2.0f * W2, Axy, sxy);
        const float e11 = fmaf(2.0f * W2, Axz, sxz), e13 = fmaf(-2.0f * W2, Axz, sxz);
        const float e15 = fmaf(2.0f * W2, Ayz, syz), e17 = fmaf(-2.0f * W2, Ayz, syz);
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
