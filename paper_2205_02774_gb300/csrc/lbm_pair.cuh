// The regularized collision of lbm_cell.cuh (collide_sd, unforced) for the
// two cells a lane of the vector kernels holds, computed together: every
// float2 operation below acts on both cells (.x the lane's first cell, .y its
// second) through the packed FP32 instructions of sm_100 and later
// (add/sub/mul/fma .f32x2: one instruction, two roundings, each the IEEE
// result of the scalar operation).  Only the reciprocals and square roots go
// cell by cell.  The update is collide_sd's
//     g*_i = w_i [a0 + c_i.B + c_i.A.c_i]
// written with B = 3 b and A = 4.5 A' so that the factors 3 and 4.5 join the
// weights in the output stage:
//     a0 = drho - 1.5 (rho u.u + km tr Pi_neq),  b = rho u,
//     A' = rho u u + km Pi_neq,                  km = 1 - 1/tau_eff.
#pragma once

#include "d3q19.cuh"

namespace stg {

__device__ __forceinline__ float2 p_add(float2 a, float2 b)
{
    float2 r;
    asm("{.reg .b64 a, b, d; mov.b64 a, {%2, %3}; mov.b64 b, {%4, %5}; add.rn.ftz.f32x2 d, a, b; mov.b64 {%0, %1}, d;}"
        : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}
__device__ __forceinline__ float2 p_sub(float2 a, float2 b)
{
    float2 r;
    asm("{.reg .b64 a, b, d; mov.b64 a, {%2, %3}; mov.b64 b, {%4, %5}; sub.rn.ftz.f32x2 d, a, b; mov.b64 {%0, %1}, d;}"
        : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}
__device__ __forceinline__ float2 p_mul(float2 a, float2 b)
{
    float2 r;
    asm("{.reg .b64 a, b, d; mov.b64 a, {%2, %3}; mov.b64 b, {%4, %5}; mul.rn.ftz.f32x2 d, a, b; mov.b64 {%0, %1}, d;}"
        : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}
// a b + c
__device__ __forceinline__ float2 p_fma(float2 a, float2 b, float2 c)
{
    float2 r;
    asm("{.reg .b64 a, b, c, d; mov.b64 a, {%2, %3}; mov.b64 b, {%4, %5}; mov.b64 c, {%6, %7};"
        " fma.rn.ftz.f32x2 d, a, b, c; mov.b64 {%0, %1}, d;}"
        : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return r;
}
__device__ __forceinline__ float2 p_k(float k) { return make_float2(k, k); }

// Moments of the pair, eqs. (density), (momentum), (tensor) in shifted
// variables: drho = sum g, j = sum c g, p_ab = sum c_a c_b g.  They are
// accumulated from the pair sums s_p = g_a + g_b and differences
// d_p = g_a - g_b of the 9 opposite pairs (a = 2p + 1, b = 2p + 2) as each
// pair is read, so no sum outlives its pair.  pop(i) gives population i of
// both cells.  The first member a of the pairs has c = (1,0,0), (0,1,0),
// (0,0,1), (1,1,0), (1,-1,0), (1,0,1), (1,0,-1), (0,1,1), (0,1,-1).
struct PairMoments {
    float2 drho, jx, jy, jz, pxx, pyy, pzz, pxy, pxz, pyz;
};

template <typename Pop2>
__device__ __forceinline__ PairMoments pair_moments(Pop2 pop)
{
    static_assert(cx_of(1) == 1 && cy_of(3) == 1 && cz_of(5) == 1, "axis pairs");
    static_assert(cx_of(7) == 1 && cy_of(7) == 1 && cx_of(9) == 1 && cy_of(9) == -1, "xy edge pairs");
    static_assert(cx_of(11) == 1 && cz_of(11) == 1 && cx_of(13) == 1 && cz_of(13) == -1, "xz edge pairs");
    static_assert(cy_of(15) == 1 && cz_of(15) == 1 && cy_of(17) == 1 && cz_of(17) == -1, "yz edge pairs");
    PairMoments m;
    float2 a, b, s, d;
    auto pair = [&](int p) {
        a = pop(2 * p + 1);
        b = pop(2 * p + 2);
        s = p_add(a, b);
        d = p_sub(a, b);
    };
    pair(0);  // +-x
    m.drho = p_add(pop(0), s);
    m.jx = d;
    m.pxx = s;
    pair(1);  // +-y
    m.drho = p_add(m.drho, s);
    m.jy = d;
    m.pyy = s;
    pair(2);  // +-z
    m.drho = p_add(m.drho, s);
    m.jz = d;
    m.pzz = s;
    pair(3);  // +-(1,1,0)
    m.drho = p_add(m.drho, s);
    m.jx = p_add(m.jx, d);
    m.jy = p_add(m.jy, d);
    m.pxx = p_add(m.pxx, s);
    m.pyy = p_add(m.pyy, s);
    m.pxy = s;
    pair(4);  // +-(1,-1,0)
    m.drho = p_add(m.drho, s);
    m.jx = p_add(m.jx, d);
    m.jy = p_sub(m.jy, d);
    m.pxx = p_add(m.pxx, s);
    m.pyy = p_add(m.pyy, s);
    m.pxy = p_sub(m.pxy, s);
    pair(5);  // +-(1,0,1)
    m.drho = p_add(m.drho, s);
    m.jx = p_add(m.jx, d);
    m.jz = p_add(m.jz, d);
    m.pxx = p_add(m.pxx, s);
    m.pzz = p_add(m.pzz, s);
    m.pxz = s;
    pair(6);  // +-(1,0,-1)
    m.drho = p_add(m.drho, s);
    m.jx = p_add(m.jx, d);
    m.jz = p_sub(m.jz, d);
    m.pxx = p_add(m.pxx, s);
    m.pzz = p_add(m.pzz, s);
    m.pxz = p_sub(m.pxz, s);
    pair(7);  // +-(0,1,1)
    m.drho = p_add(m.drho, s);
    m.jy = p_add(m.jy, d);
    m.jz = p_add(m.jz, d);
    m.pyy = p_add(m.pyy, s);
    m.pzz = p_add(m.pzz, s);
    m.pyz = s;
    pair(8);  // +-(0,1,-1)
    m.drho = p_add(m.drho, s);
    m.jy = p_add(m.jy, d);
    m.jz = p_sub(m.jz, d);
    m.pyy = p_add(m.pyy, s);
    m.pzz = p_add(m.pzz, s);
    m.pyz = p_sub(m.pyz, s);
    return m;
}

// Smagorinsky relaxation (eq. tau_eff, with the sponge factor nuf of eq.
// sponge_visco when SP) and regularized collision of the pair; out(i, r)
// receives the result r of population i (both cells) in the order
// i = 0, 1, ..., 18.  Returns the density excess and velocity per cell.
template <bool SP, typename Out>
__device__ __forceinline__ void collide_pair(const PairMoments &m, float tau0, float kq, float2 nuf, Out out,
                                             float2 &drho_o, float2 &ux_o, float2 &uy_o, float2 &uz_o)
{
    const float2 drho = m.drho;
    const float2 rho = p_add(drho, p_k(1.0f));
    const float2 irho = make_float2(1.0f / rho.x, 1.0f / rho.y);
    const float2 ux = p_mul(m.jx, irho), uy = p_mul(m.jy, irho), uz = p_mul(m.jz, irho);
    // rho u u and Pi_neq = sum c c g - drho/3 I - rho u u
    const float2 rux = p_mul(rho, ux), ruy = p_mul(rho, uy), ruz = p_mul(rho, uz);
    const float2 Pxx = p_mul(rux, ux), Pyy = p_mul(ruy, uy), Pzz = p_mul(ruz, uz);
    const float2 Pxy = p_mul(rux, uy), Pxz = p_mul(rux, uz), Pyz = p_mul(ruy, uz);
    const float2 d3 = p_mul(drho, p_k(1.0f / 3.0f));
    const float2 nxx = p_sub(m.pxx, p_add(d3, Pxx));
    const float2 nyy = p_sub(m.pyy, p_add(d3, Pyy));
    const float2 nzz = p_sub(m.pzz, p_add(d3, Pzz));
    const float2 nxy = p_sub(m.pxy, Pxy), nxz = p_sub(m.pxz, Pxz), nyz = p_sub(m.pyz, Pyz);
    const float2 qd = p_fma(nzz, nzz, p_fma(nyy, nyy, p_mul(nxx, nxx)));
    const float2 qo = p_fma(nyz, nyz, p_fma(nxz, nxz, p_mul(nxy, nxy)));
    const float2 q2 = p_fma(qo, p_k(2.0f), qd);
    const float2 qh = make_float2(q2.x > 0.f ? sqrtf(q2.x) : 0.f, q2.y > 0.f ? sqrtf(q2.y) : 0.f);
    // eq. (tau_eff), c = 1: tau = tau0/2 + sqrt((tau0 rho)^2 + 18 sqrt2 C Q^1/2)/(2 rho)
    const float2 rad = p_fma(p_k(kq), p_mul(qh, p_mul(irho, irho)), p_k(tau0 * tau0));
    float2 tau = p_fma(p_k(0.5f), make_float2(sqrtf(rad.x), sqrtf(rad.y)), p_k(0.5f * tau0));
    if (SP) tau = p_fma(nuf, p_sub(tau, p_k(0.5f)), p_k(0.5f));
    const float2 km = p_sub(p_k(1.0f), make_float2(1.0f / tau.x, 1.0f / tau.y));
    const float2 uu = p_fma(uz, uz, p_fma(uy, uy, p_mul(ux, ux)));
    const float2 a0 = p_fma(p_k(-1.5f), p_fma(km, p_add(p_add(nxx, nyy), nzz), p_mul(rho, uu)), drho);
    const float2 Axx = p_fma(km, nxx, Pxx), Ayy = p_fma(km, nyy, Pyy), Azz = p_fma(km, nzz, Pzz);
    const float2 Axy = p_fma(km, nxy, Pxy), Axz = p_fma(km, nxz, Pxz), Ayz = p_fma(km, nyz, Pyz);
    constexpr float W0 = 1.0f / 3.0f, W1 = 1.0f / 18.0f, W2 = 1.0f / 36.0f;
    // rest population
    out(0, p_mul(p_k(W0), a0));
    // axis pairs (1,2) +-x, (3,4) +-y, (5,6) +-z
    {
        const float2 w1a0 = p_mul(p_k(W1), a0);
        const float2 ex = p_fma(p_k(4.5f * W1), Axx, w1a0), ox = p_mul(p_k(3.0f * W1), rux);
        out(1, p_add(ex, ox));
        out(2, p_sub(ex, ox));
        const float2 ey = p_fma(p_k(4.5f * W1), Ayy, w1a0), oy = p_mul(p_k(3.0f * W1), ruy);
        out(3, p_add(ey, oy));
        out(4, p_sub(ey, oy));
        const float2 ez = p_fma(p_k(4.5f * W1), Azz, w1a0), oz = p_mul(p_k(3.0f * W1), ruz);
        out(5, p_add(ez, oz));
        out(6, p_sub(ez, oz));
    }
    // edge pairs: (7,8) +-(1,1,0), (9,10) +-(1,-1,0), (11,12) +-(1,0,1), (13,14) +-(1,0,-1),
    //             (15,16) +-(0,1,1), (17,18) +-(0,1,-1)
    {
        const float2 w2a0 = p_mul(p_k(W2), a0);
        const float2 bx = p_mul(p_k(3.0f * W2), rux), by = p_mul(p_k(3.0f * W2), ruy), bz = p_mul(p_k(3.0f * W2), ruz);
        const float2 sxy = p_fma(p_k(4.5f * W2), p_add(Axx, Ayy), w2a0), txy = p_mul(p_k(9.0f * W2), Axy);
        const float2 e7 = p_add(sxy, txy), o7 = p_add(bx, by);
        out(7, p_add(e7, o7));
        out(8, p_sub(e7, o7));
        const float2 e9 = p_sub(sxy, txy), o9 = p_sub(bx, by);
        out(9, p_add(e9, o9));
        out(10, p_sub(e9, o9));
        const float2 sxz = p_fma(p_k(4.5f * W2), p_add(Axx, Azz), w2a0), txz = p_mul(p_k(9.0f * W2), Axz);
        const float2 e11 = p_add(sxz, txz), o11 = p_add(bx, bz);
        out(11, p_add(e11, o11));
        out(12, p_sub(e11, o11));
        const float2 e13 = p_sub(sxz, txz), o13 = p_sub(bx, bz);
        out(13, p_add(e13, o13));
        out(14, p_sub(e13, o13));
        const float2 syz = p_fma(p_k(4.5f * W2), p_add(Ayy, Azz), w2a0), tyz = p_mul(p_k(9.0f * W2), Ayz);
        const float2 e15 = p_add(syz, tyz), o15 = p_add(by, bz);
        out(15, p_add(e15, o15));
        out(16, p_sub(e15, o15));
        const float2 e17 = p_sub(syz, tyz), o17 = p_sub(by, bz);
        out(17, p_add(e17, o17));
        out(18, p_sub(e17, o17));
    }
    drho_o = drho;
    ux_o = ux;
    uy_o = uy;
    uz_o = uz;
}

}  // namespace stg
