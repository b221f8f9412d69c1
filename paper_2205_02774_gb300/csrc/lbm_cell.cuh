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

}  // namespace stg
