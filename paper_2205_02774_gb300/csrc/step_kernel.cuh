// Fused LES-LBM time step for one channel lattice (Algorithm 1, step 12, with
// steps 9-11 for the inlet nodes and the outlet rebuild folded in): the device
// templates, instantiated per storage and collision by step_f32_reg.cu,
// step_f32_bgk.cu, step_f16_reg.cu and step_f16_bgk.cu.
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
// Layout: SoA f[i][z][y][x].  The even-nx path (vector kernels) gives each
// lane two consecutive x cells; plain steps cut the lattice into blocks of
// (x chunk, row, z chunk) chosen by the launch tile, sampling steps into
// fixed groups of z planes whose per-(x, y) sums are added in order.  The
// odd-nx path (one cell per thread) keeps a block per (x chunk, row) column.
//
// Streaming schemes (vector kernels, MODE):
//  PULL      two lattices: read src[i] at x - c_i, write dst[i] at x;
//  AA_SHIFT  one lattice, steps with even index: read slot opp(i) at x - c_i,
//            write the result of population i to slot i at x + c_i;
//  AA_LOCAL  one lattice, steps with odd index: read slot i at x, write the
//            result of population i to slot opp(i) at x.
// In the one-lattice (AA-pattern) scheme a cell reads and writes the same 19
// slots, so the update is in place and race-free: a slot read across a wall
// (source outside in y) is the cell's own slot i, which the previous local
// step left holding f*_opp(i); a result whose target lies outside the
// lattice (a wall in y, the open ends in x) goes to the cell's own slot
// opp(i), where the next local step reads it as the bounced-back (wall) or
// unknown (inlet/outlet, rebuilt) population.  Every value a thread uses is
// read before any thread writes its slot, so the read-only load path and the
// non-aliasing qualifiers stay valid in place.
#pragma once

#include <cuda_fp16.h>

#include "d3q19.cuh"
#include "internal.h"
#include "lbm_cell.cuh"
#include "lbm_pair.cuh"
#include "reduce.cuh"

namespace stg {

constexpr int PULL = 0, AA_SHIFT = 1, AA_LOCAL = 2;

// Stochastic rounding of binary16 stores (SR kernels): a value between two
// binary16 neighbours goes to the upper one with probability equal to its
// distance from the lower one in units of their spacing, so the stored value
// is unbiased and updates smaller than half a spacing are kept on average
// (round to nearest drops them).  cvt.rs.f16x2.f32 takes 13 random bits per
// half: bits 0-12 for the low half, 16-28 for the high half.  The bits are a
// fixed function of (first cell of the pair, step, population), so a run is
// reproducible and independent of the launch decomposition: a per-pair seed
// from two multiply-xorshift rounds, then, per population, the middle 32 bits
// of the 64-bit product of the seed (offset by a Weyl sequence in i) with an
// odd constant.
__device__ __forceinline__ unsigned sr_seed(unsigned cell, unsigned tmix)
{
    unsigned s = (cell * 0x9E3779B1u) ^ tmix;
    s = (s ^ (s >> 15)) * 0x2C1B3C6Du;
    return s ^ (s >> 12);
}
__device__ __forceinline__ unsigned sr_tmix(long long t) { return (unsigned)t * 0x85EBCA77u; }
__device__ __forceinline__ unsigned sr_bits(unsigned seed, int i)
{
    const unsigned long long p = (unsigned long long)(seed ^ (0x9E3779B9u * (unsigned)(i + 1))) * 0xD168AAADull;
    return (unsigned)(p >> 16);
}
// one binary16 by stochastic rounding (the low half of the pair conversion)
__device__ __forceinline__ void st_half_rs(__half *p, float g, unsigned rb)
{
    unsigned v;
    asm("cvt.rs.f16x2.f32 %0, %1, %2, %3;" : "=r"(v) : "f"(0.0f), "f"(g), "r"(rb));
    __stcs(p, __ushort_as_half((unsigned short)(v & 0xffffu)));
}

constexpr int BX = 32;
constexpr int BZ = 8;

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

// One block = one 32-wide (x chunk, y) column over all z, one cell per
// thread.  EDGE selects the general pull (walls, wraps, inlet/outlet
// rebuild); the interior variant only sees columns whose x chunk is neither
// the first nor the last and whose y has both neighbours inside the lattice.
template <typename S, bool REG, bool FORCE, bool EDGE, bool SP, bool SR = false>
__device__ __forceinline__ void step_column(const StepArgs &a, int bx, int y)
{
    const S *__restrict__ src = static_cast<const S *>(a.src);
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
                        const float drb = (fmaf(2.0f, lv, par) + ubx) / (1.0f - ubx);
                        rebuild<1>(g, drb, ubx, uby, ubz);
                    } else {
                        // zero-gradient pressure outlet: rho = 1 and the velocity of the
                        // neighbour x = nx-2 at this step, from its streamed populations
                        float gn[Q];
                        gather_general<S>(src, P, nx, ny, nx - 2, y, z, nx - 3, nx - 1, true, true, ym, yp, ym_w,
                                          yp_w, zm, zp, ((unsigned)z * ny + y) * nx + (nx - 2), gn);
                        float r = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
                        for (int i = 0; i < Q; ++i) {
                            r += gn[i];
                            jx += cx_of(i) * gn[i];
                            jy += cy_of(i) * gn[i];
                            jz += cz_of(i) * gn[i];
                        }
                        const float ir = 1.0f / (1.0f + r);
                        if (FORCE) {
                            jx += 0.5f * Fx;
                            jy += 0.5f * Fy;
                            jz += 0.5f * Fz;
                        }
                        rebuild<-1>(g, 0.0f, jx * ir, jy * ir, jz * ir);
                    }
                }
            }
            float drho, ux, uy, uz;
            collide<REG, FORCE, SP>(g, tau0, kq, Fx, Fy, Fz, drho, ux, uy, uz, SP ? __ldg(a.spf + x) : 1.0f);
#pragma unroll
            if constexpr (SR) {
                const unsigned seed = sr_seed(here, sr_tmix(t));
#pragma unroll
                for (int i = 0; i < Q; ++i) st_half_rs(static_cast<__half *>(a.dstp[i]) + here, g[i], sr_bits(seed, i));
            } else {
#pragma unroll
                for (int i = 0; i < Q; ++i) Pop<S>::st(static_cast<S *>(a.dstp[i]) + here, g[i]);
            }
            if (do_stats) {
                su0 += ux; su1 += uy; su2 += uz;
                s00 = __fmaf_rn(ux, ux, s00); s11 = __fmaf_rn(uy, uy, s11); s22 = __fmaf_rn(uz, uz, s22);
                s01 = __fmaf_rn(ux, uy, s01); s02 = __fmaf_rn(ux, uz, s02); s12 = __fmaf_rn(uy, uz, s12);
            }
            if (do_check) sdr += drho;
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
    if (do_check) mass_finish<BX * BZ>(a, sdr);
}

// Scalar interior columns: x chunks [il, ir), y = 1..ny-2 (odd nx or narrow lattices).
template <typename S, bool REG, bool FORCE, bool SP, bool SR>
__global__ void __launch_bounds__(BX *BZ, 4) lbm_step_kernel(const StepArgs a)
{
    step_column<S, REG, FORCE, false, SP, SR>(a, a.il + blockIdx.x, blockIdx.y + 1);
}

// ---------------------------------------------------------------------------
// Several cells per lane: lane l of a warp owns CPL consecutive cells starting
// at x = 32 CPL b + CPL l, so every population row is read and written as
// aligned vectors (FP32 pairs: 8 B, 256 B per warp instruction; FP16 pairs:
// 4 B, 128 B; FP16 quads: 8 B, 256 B).  A pull with c_x = +1 needs the cells shifted by one: the
// missing x-1 value is the top cell of the left lane's vector (warp shuffle;
// lane 0 reads it directly, wrapping in x when x is periodic), and c_x = -1
// mirrors this on the right.  The wide accesses keep enough bytes in flight
// per SM to saturate HBM, which 2-byte accesses cannot (and, in FP16, which
// 4-byte pairs reach only at about 0.87 of the copy bandwidth).
template <typename S, int CPL>
struct Vec;

template <>
struct Vec<float, 2> {
    using raw = float2;
    static __device__ __forceinline__ raw ld(const float *p) { return __ldg(reinterpret_cast<const float2 *>(p)); }
    static __device__ __forceinline__ float cell(raw v, int j) { return j ? v.y : v.x; }
    static __device__ __forceinline__ float2 pair(raw v, int = 0) { return v; }
    static __device__ __forceinline__ void set_pair(raw &v, int, float lo, float hi) { v = make_float2(lo, hi); }
    static __device__ __forceinline__ void put(raw &v, int j, float f)
    {
        if (j) v.y = f;
        else v.x = f;
    }
    static __device__ __forceinline__ raw pack(float lo, float hi) { return make_float2(lo, hi); }
    static __device__ __forceinline__ void st(float *p, raw v) { __stcs(reinterpret_cast<float2 *>(p), v); }
    static __device__ __forceinline__ void st1(float *p, raw v, int j) { __stcs(p + j, cell(v, j)); }
    // (x-1, x) from the left lane's (x-2, x-1) and ours (x, x+1); xl = x-1 when read directly
    static __device__ __forceinline__ raw shift_left(raw cur, const float *xl, bool side)
    {
        float l = __shfl_up_sync(0xffffffffu, cur.y, 1);
        if (side) l = __ldg(xl);
        return make_float2(l, cur.x);
    }
    // (x+1, x+2) from ours and the right lane's (x+2, x+3); xr = x+2 when read directly
    static __device__ __forceinline__ raw shift_right(raw cur, const float *xr, bool side)
    {
        float r = __shfl_down_sync(0xffffffffu, cur.x, 1);
        if (side) r = __ldg(xr);
        return make_float2(cur.y, r);
    }
};


template <>
struct Vec<__half, 2> {
    using raw = unsigned;  // two binary16: low half = first cell
    // read-only load with a 256-byte L2 fetch: a warp reads 128 B of a row and
    // the next x chunk's warp reads the following 128 B (measured +1 % of the
    // FP16 pass)
    static __device__ __forceinline__ raw ld(const __half *p)
    {
        unsigned v;
        asm volatile("ld.global.nc.L2::256B.b32 %0, [%1];" : "=r"(v) : "l"(p));
        return v;
    }
    // the halves of the pair as 16-bit registers: one conversion per value,
    // no masking or shifting (measured 0.63 -> 0.66 of the FP16 pass)
    static __device__ __forceinline__ float cell(raw v, int j)
    {
        float f;
        if (j) asm("{.reg .b16 lo, hi; mov.b32 {lo, hi}, %1; cvt.f32.f16 %0, hi;}" : "=f"(f) : "r"(v));
        else asm("{.reg .b16 lo, hi; mov.b32 {lo, hi}, %1; cvt.f32.f16 %0, lo;}" : "=f"(f) : "r"(v));
        return f;
    }
    // both halves in FP32 (.x the first cell)
    static __device__ __forceinline__ float2 pair(raw v, int = 0)
    {
        float2 f;
        asm("{.reg .b16 lo, hi; mov.b32 {lo, hi}, %2; cvt.f32.f16 %0, lo; cvt.f32.f16 %1, hi;}"
            : "=f"(f.x), "=f"(f.y) : "r"(v));
        return f;
    }
    // h_j + c and h_j - c in FP32 with the binary16 half j of the pair as an
    // operand (mixed-precision add/sub, sm_100 and later; the half converts
    // exactly, so each equals the FP32 sum of the converted value)
    static __device__ __forceinline__ float add_h(raw v, int j, float c)
    {
        float r;
        if (j) asm("{.reg .b16 lo, hi; mov.b32 {lo, hi}, %1; add.rn.f32.f16 %0, hi, %2;}" : "=f"(r) : "r"(v), "f"(c));
        else asm("{.reg .b16 lo, hi; mov.b32 {lo, hi}, %1; add.rn.f32.f16 %0, lo, %2;}" : "=f"(r) : "r"(v), "f"(c));
        return r;
    }
    static __device__ __forceinline__ float sub_h(raw v, int j, float c)
    {
        float r;
        if (j) asm("{.reg .b16 lo, hi; mov.b32 {lo, hi}, %1; sub.rn.f32.f16 %0, hi, %2;}" : "=f"(r) : "r"(v), "f"(c));
        else asm("{.reg .b16 lo, hi; mov.b32 {lo, hi}, %1; sub.rn.f32.f16 %0, lo, %2;}" : "=f"(r) : "r"(v), "f"(c));
        return r;
    }
    static __device__ __forceinline__ void put(raw &v, int j, float f)
    {
        if (j) asm("{.reg .b16 lo, hi, n; mov.b32 {lo, hi}, %0; cvt.rn.f16.f32 n, %1; mov.b32 %0, {lo, n};}" : "+r"(v) : "f"(f));
        else asm("{.reg .b16 lo, hi, n; mov.b32 {lo, hi}, %0; cvt.rn.f16.f32 n, %1; mov.b32 %0, {n, hi};}" : "+r"(v) : "f"(f));
    }
    // both cells of the pair in one conversion (round to nearest even, as
    // the one-value form): the first cell's results wait in FP32 registers,
    // which the pair's inputs free as the second cell reads them
    static __device__ __forceinline__ raw pack(float lo, float hi)
    {
        unsigned v;
        asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(v) : "f"(hi), "f"(lo));
        return v;
    }
    // the same by stochastic rounding (random bits rb: 0-12 for lo, 16-28 for hi)
    static __device__ __forceinline__ raw pack_rs(float lo, float hi, unsigned rb)
    {
        unsigned v;
        asm("cvt.rs.f16x2.f32 %0, %1, %2, %3;" : "=r"(v) : "f"(hi), "f"(lo), "r"(rb));
        return v;
    }
    static __device__ __forceinline__ void set_pair(raw &v, int, float lo, float hi) { v = pack(lo, hi); }
    static __device__ __forceinline__ void set_pair_rs(raw &v, int, float lo, float hi, unsigned rb) { v = pack_rs(lo, hi, rb); }
    static __device__ __forceinline__ void st(__half *p, raw v) { __stcs(reinterpret_cast<unsigned *>(p), v); }
    static __device__ __forceinline__ void st1(__half *p, raw v, int j)
    {
        __stcs(p + j, __ushort_as_half((unsigned short)(j ? v >> 16 : v & 0xffffu)));
    }
    // (x-1, x) and (x+1, x+2) with the missing value read as one binary16 at
    // a fixed offset from the pair's own address (row = element x): no
    // shuffle, no separate halo address; valid wherever row[-1] and row[2]
    // lie inside the allocation (the caller ensures it)
    static __device__ __forceinline__ raw halo_left(raw cur, const __half *row)
    {
        const unsigned short h = __half_as_ushort(__ldg(row - 1));
        raw v;
        asm("{.reg .b16 lo, hi; mov.b32 {lo, hi}, %1; mov.b32 %0, {%2, lo};}" : "=r"(v) : "r"(cur), "h"(h));
        return v;
    }
    static __device__ __forceinline__ raw halo_right(raw cur, const __half *row)
    {
        const unsigned short h = __half_as_ushort(__ldg(row + 2));
        raw v;
        asm("{.reg .b16 lo, hi; mov.b32 {lo, hi}, %1; mov.b32 %0, {hi, %2};}" : "=r"(v) : "r"(cur), "h"(h));
        return v;
    }
    // (x-1, x)
    static __device__ __forceinline__ raw shift_left(raw cur, const __half *xl, bool side)
    {
        unsigned l = __shfl_up_sync(0xffffffffu, cur, 1);
        if (side) l = (unsigned)__half_as_ushort(__ldg(xl)) << 16;
        return __byte_perm(l, cur, 0x5432);
    }
    // (x+1, x+2); xr = x+2 when read directly
    static __device__ __forceinline__ raw shift_right(raw cur, const __half *xr, bool side)
    {
        unsigned r = __shfl_down_sync(0xffffffffu, cur, 1);
        if (side) r = (unsigned)__half_as_ushort(__ldg(xr));
        return __byte_perm(cur, r, 0x5432);
    }
};

template <>
struct Vec<__half, 4> {
    using raw = uint2;  // x: cells 0, 1 (low half first); y: cells 2, 3
    // 8-byte read-only load with the 256-byte L2 fetch (a warp reads a 256 B row piece)
    static __device__ __forceinline__ raw ld(const __half *p)
    {
        raw v;
        asm volatile("ld.global.nc.L2::256B.v2.b32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "l"(p));
        return v;
    }
    static __device__ __forceinline__ unsigned word(raw v, int j) { return j < 2 ? v.x : v.y; }
    static __device__ __forceinline__ float cell(raw v, int j) { return Vec<__half, 2>::cell(word(v, j), j & 1); }
    // cells 2k and 2k + 1 in FP32
    static __device__ __forceinline__ float2 pair(raw v, int k) { return Vec<__half, 2>::pair(k ? v.y : v.x); }
    static __device__ __forceinline__ float add_h(raw v, int j, float c) { return Vec<__half, 2>::add_h(word(v, j), j & 1, c); }
    static __device__ __forceinline__ float sub_h(raw v, int j, float c) { return Vec<__half, 2>::sub_h(word(v, j), j & 1, c); }
    // cells 2k, 2k + 1 <- lo, hi (round to nearest, or stochastic rounding with bits rb)
    static __device__ __forceinline__ void set_pair(raw &v, int k, float lo, float hi)
    {
        (k ? v.y : v.x) = Vec<__half, 2>::pack(lo, hi);
    }
    static __device__ __forceinline__ void set_pair_rs(raw &v, int k, float lo, float hi, unsigned rb)
    {
        (k ? v.y : v.x) = Vec<__half, 2>::pack_rs(lo, hi, rb);
    }
    static __device__ __forceinline__ void st(__half *p, raw v) { __stcs(reinterpret_cast<uint2 *>(p), v); }
    // cell j at p + j
    static __device__ __forceinline__ void st1(__half *p, raw v, int j) { Vec<__half, 2>::st1(p + (j & 2), word(v, j), j & 1); }
    // cells 1 and 2 as one aligned pair at p
    static __device__ __forceinline__ void st_mid(__half *p, raw v)
    {
        __stcs(reinterpret_cast<unsigned *>(p), __byte_perm(v.x, v.y, 0x5432));
    }
    // (x-1 .. x+2) and (x+1 .. x+4) with the missing value read as one binary16
    // beside the quad (row = element x; the caller keeps row[-1] and row[4]
    // inside the allocation)
    static __device__ __forceinline__ raw halo_left(raw cur, const __half *row)
    {
        const unsigned h = __half_as_ushort(__ldg(row - 1));
        return make_uint2(__byte_perm(h, cur.x, 0x5410), __byte_perm(cur.x, cur.y, 0x5432));
    }
    static __device__ __forceinline__ raw halo_right(raw cur, const __half *row)
    {
        const unsigned h = __half_as_ushort(__ldg(row + 4));
        return make_uint2(__byte_perm(cur.x, cur.y, 0x5432), __byte_perm(cur.y, h, 0x5432));
    }
    // (x-1 .. x+2) from the left lane's cell 3 and ours; xl = x-1 when read directly
    static __device__ __forceinline__ raw shift_left(raw cur, const __half *xl, bool side)
    {
        unsigned l = __shfl_up_sync(0xffffffffu, cur.y, 1);
        if (side) l = (unsigned)__half_as_ushort(__ldg(xl)) << 16;
        return make_uint2(__byte_perm(l, cur.x, 0x5432), __byte_perm(cur.x, cur.y, 0x5432));
    }
    // (x+1 .. x+4) from ours and the right lane's cell 0; xr = x+4 when read directly
    static __device__ __forceinline__ raw shift_right(raw cur, const __half *xr, bool side)
    {
        unsigned r = __shfl_down_sync(0xffffffffu, cur.x, 1);
        if (side) r = (unsigned)__half_as_ushort(__ldg(xr));
        return make_uint2(__byte_perm(cur.x, cur.y, 0x5432), __byte_perm(cur.y, r, 0x5432));
    }
};

// One vector column (CPL 32 cells wide) at row y over the planes z = zb,
// zb + zs, ... below ze.  YEDGE rows
// (y = 0 or ny-1) take the y neighbour by half-way bounce-back (walls: the
// cell's own opposite population) or by the periodic wrap.  In inlet/outlet
// mode the inlet node x = 0 is rebuilt by the regularized Zou-He
// reconstruction (Sec. III.B) and the outlet node x = nx-1 by the regularized
// pressure outlet, whose velocity is that of the same lane's previous cell
// x = nx-2; their pulled values from outside the lattice are never read.
// STATS adds the per-cell velocity sums to the block's shared-memory slots.
// H16 (binary16, inlet/outlet in x only): the x-shifted pairs or quads take
// their missing value by a 2-byte load beside the vector instead of a warp
// shuffle.  Lane 0 of the first chunk then reads the element before its row
// and the last lane the element after it; both lie inside the 19-plane
// allocation (they are used only for c_x > 0 at x = 0, planes 1..13, and
// c_x < 0 at x = nx-1, planes 2..14) and are the unknowns that the inlet and
// outlet rebuilds replace.
// Returns the thread's sum of rho - 1.
template <typename S, int CPL, bool REG, bool FORCE, bool STATS, bool YEDGE, bool SP, bool H16, int MODE, bool SR>
__device__ __forceinline__ float vec_loop(const StepArgs &a, float (*sacc)[9][BX * CPL], int x0, int y, int zb,
                                          int ze, int zs)
{
    static_assert(CPL == 2 || (CPL == 4 && sizeof(S) == 2), "pairs, or binary16 quads");
    using V = Vec<S, CPL>;
    using raw = typename V::raw;
    // binary16, regularized collision: pair sums by mixed-precision adds
    constexpr bool MIXED = REG && sizeof(S) == 2;
    // binary16, regularized unforced collision: the lane's cells go through
    // the collision two at a time in packed FP32 (lbm_pair.cuh) wherever the
    // warp's 32 CPL cells hold no inlet or outlet node; the warps that do, the
    // other collisions and FP32 storage (whose step is bound by memory either
    // way) update cell by cell.  A warp's chunk is the same in every kernel and
    // tile, so each cell always takes the same form.
    constexpr bool PACKED = REG && !FORCE && sizeof(S) == 2;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int nxy = nx * ny;
    const int lane = threadIdx.x, wi = threadIdx.y;
    const int x = x0 + CPL * lane;
    const bool active = x < nx;
    const bool inout = a.bc_x == 0;
    // x halo read directly by lane 0 / by the last active lane
    const bool side_l = active && lane == 0;
    const bool side_r = active && (lane == 31 || x + CPL == nx);
    const int xl = x == 0 ? (inout ? 0 : nx - 1) : x - 1;        // element read for x-1
    const int xr = x + CPL == nx ? (inout ? nx - 1 : 0) : x + CPL; // element read for x+CPL
    // inlet/outlet mode: the first lane's first cell is the inlet node x = 0,
    // the last lane's last cell the outlet node x = nx-1 (nx is a multiple of
    // CPL); both are rebuilt here from the values already in registers
    const bool at_inlet = inout && x == 0;
    const bool at_outlet = inout && active && x + CPL == nx;
    const bool node_warp = inout && (x0 == 0 || x0 + BX * CPL >= nx);
    // y neighbours of this row (YEDGE rows only)
    bool ym_bb = false, yp_bb = false;
    int ym_off = nx, yp_off = -nx;  // element offset of the source row for c_y = +1 / -1 (subtracted)
    if (YEDGE) {
        const bool walls = a.bc_y == 0;
        if (y == 0) {
            if (walls) ym_bb = true;
            else ym_off = -(ny - 1) * nx;
        }
        if (y == ny - 1) {
            if (walls) yp_bb = true;
            else yp_off = (ny - 1) * nx;
        }
    }
    const float tau0 = a.tau0, kq = a.kq;
    const float Fx = a.Fx, Fy = a.Fy, Fz = a.Fz;
    const S *__restrict__ sbase = static_cast<const S *>(a.src);
    S *__restrict__ dbase = static_cast<S *>(a.dst);
    float sdr = 0.f;
    const unsigned tmix = SR ? sr_tmix(a.ctl->t[a.parity]) : 0u;
    for (int z = zb; z < ze; z += zs) {
        // Plane offsets i P are recomputed in every iteration from an opaque
        // copy of P: hoisting 19 + 19 plane pointers out of the loop would
        // cost 76 registers.  Element offsets are 32-bit (19 P < 2^32).
        unsigned Pv, nxv;
        asm volatile("mov.u32 %0, %1;" : "=r"(Pv) : "r"(a.P));
        asm volatile("mov.u32 %0, %1;" : "=r"(nxv) : "r"((unsigned)nx));
        // plane stride in bytes (opaque too): a population's address is one
        // wide multiply-add i * Pb on its row's byte pointer
        unsigned Pb;
        asm volatile("mov.u32 %0, %1;" : "=r"(Pb) : "r"(a.P * (unsigned)sizeof(S)));
        const unsigned row0 = ((unsigned)z * ny + y) * nx;
        const unsigned here = row0 + x;
        const unsigned dzm = (z == 0) ? -(nz - 1) * nxy : nxy;
        const unsigned dzp = (z == nz - 1) ? (nz - 1) * nxy : -nxy;
        raw v[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int cx = cx_of(i), cz = cz_of(i), cy = cy_of(i);
            if (MODE == AA_LOCAL) {
                // in place, odd steps: the cell's own slot i holds f_i(x)
                raw cur;
                if (active) cur = V::ld(reinterpret_cast<const S *>(reinterpret_cast<const char *>(sbase + here) + (size_t)i * Pb));
                else cur = raw{};
                v[i] = cur;
                continue;
            }
            const bool bb = YEDGE && ((cy > 0 && ym_bb) || (cy < 0 && yp_bb));
            if (bb) {
                // half-way bounce-back: f_i(x) = f*_opp(i)(x), same cell (two
                // lattices: slot opp(i); in place: the local step left it in slot i)
                raw cur;
                if (active) cur = V::ld(sbase + ((MODE == PULL ? opp_of(i) : i) * Pv + here));
                else cur = raw{};
                v[i] = cur;
                continue;
            }
            // source plane: i (two lattices) or opp(i) (in place, even steps)
            const int pl = MODE == PULL ? i : opp_of(i);
            const unsigned dz = cz > 0 ? dzm : (cz < 0 ? dzp : 0u);
            const unsigned dy = cy > 0 ? (YEDGE ? (unsigned)ym_off : nxv) : (cy < 0 ? (YEDGE ? (unsigned)yp_off : 0u - nxv) : 0u);
            const unsigned rbase = pl * Pv + row0 - dz - dy;  // plane pl, row (y - c_y, z - c_z)
            const unsigned rofs = row0 - dz - dy + x;          // element x of that row in plane 0
            const S *row = reinterpret_cast<const S *>(reinterpret_cast<const char *>(sbase + rofs) + (size_t)pl * Pb);
            raw cur;
            if (active) cur = V::ld(row);
            else cur = raw{};
            if (cx == 0) v[i] = cur;
            else if constexpr (H16) {
                if (!active) v[i] = raw{};
                else if (cx > 0) v[i] = V::halo_left(cur, row);
                else v[i] = V::halo_right(cur, row);
            }
            else if (cx > 0) v[i] = V::shift_left(cur, sbase + (rbase + xl), side_l && !(inout && x == 0));
            else v[i] = V::shift_right(cur, sbase + (rbase + xr), side_r && !(inout && x + CPL == nx));
        }
        // stochastic rounding: the bits of a pair's conversion depend on the
        // pair's first cell, so pairs and quads round a lattice alike
        auto seed_of = [&](int k) { return SR ? sr_seed(here + 2 * k, tmix) : 0u; };
        if (PACKED && !node_warp) {
            // the lane's cells two at a time (packed FP32 pairs)
#pragma unroll
            for (int k = 0; k < CPL / 2; ++k) {
                float2 nuf = make_float2(1.0f, 1.0f);
                if (SP && active) nuf = __ldg(reinterpret_cast<const float2 *>(a.spf + x + 2 * k));
                const unsigned seed = seed_of(k);
                const PairMoments m = pair_moments([&](int i) { return V::pair(v[i], k); });
                float2 drho, ux, uy, uz;
                collide_pair<SP>(m, tau0, kq, nuf, [&](int i, float2 r) {
                    if constexpr (SR) V::set_pair_rs(v[i], k, r.x, r.y, sr_bits(seed, i));
                    else V::set_pair(v[i], k, r.x, r.y);
                }, drho, ux, uy, uz);
                if (active) {
                    if (STATS) {
                        constexpr int L = BX * CPL;
#pragma unroll
                        for (int j = 0; j < 2; ++j) {
                            float *sp = &sacc[wi][0][CPL * lane + 2 * k + j];
                            const float vx = j ? ux.y : ux.x, vy = j ? uy.y : uy.x, vz = j ? uz.y : uz.x;
                            sp[0 * L] += vx; sp[1 * L] += vy; sp[2 * L] += vz;
                            sp[3 * L] = __fmaf_rn(vx, vx, sp[3 * L]); sp[4 * L] = __fmaf_rn(vy, vy, sp[4 * L]);
                            sp[5 * L] = __fmaf_rn(vz, vz, sp[5 * L]); sp[6 * L] = __fmaf_rn(vx, vy, sp[6 * L]);
                            sp[7 * L] = __fmaf_rn(vx, vz, sp[7 * L]); sp[8 * L] = __fmaf_rn(vy, vz, sp[8 * L]);
                        }
                    }
                    sdr += drho.x;
                    sdr += drho.y;
                }
            }
        } else {
        float upx = 0.f, upy = 0.f, upz = 0.f;  // velocity of the lane's previous cell
        float gp[Q];                            // results of the pair's first cell
#pragma unroll
        for (int j = 0; j < CPL; ++j) {
            float g[Q];
            // boundary nodes of this cell (inlet x = 0 at j = 0, outlet x = nx-1 at the last j)
            const bool node = (j == 0 && at_inlet) || (j == CPL - 1 && at_outlet);
            auto rebuild_node = [&](float (&gg)[Q]) {
                if (j == 0 && at_inlet) {
                    // Zou-He density, eq. (density_bc): parallel set + 2 x leaving set,
                    // rho_bc - 1 = (S_g + u_x)/(1 - u_x) in shifted variables; the
                    // unknowns (c_x > 0, their sources lie outside) are not read
                    const size_t pc = (size_t)z * ny + y, pl3 = (size_t)ny * nz;
                    const float ubx = a.ubc[pc], uby = a.ubc[pl3 + pc], ubz = a.ubc[2 * pl3 + pc];
                    float par = 0.f, lv = 0.f;
#pragma unroll
                    for (int i = 0; i < Q; ++i) {
                        if (cx_of(i) == 0) par += gg[i];
                        if (cx_of(i) < 0) lv += gg[i];
                    }
                    rebuild<1>(gg, (fmaf(2.0f, lv, par) + ubx) / (1.0f - ubx), ubx, uby, ubz);
                }
                if (j == CPL - 1 && at_outlet) {
                    // zero-gradient pressure outlet: rho = 1 and the velocity of the
                    // neighbour x = nx-2 (this lane's previous cell) at this step
                    rebuild<-1>(gg, 0.0f, upx, upy, upz);
                }
            };
            float drho, ux, uy, uz;
            const float nuf = SP && active ? __ldg(a.spf + x + j) : 1.0f;
            if constexpr (MIXED) {
                // regularized collision of binary16 pairs: only the pair sums and
                // differences enter, formed with one conversion per pair
                float s[9], d[9], drho0;
                if (node) {
#pragma unroll
                    for (int i = 0; i < Q; ++i) g[i] = V::cell(v[i], j);
                    rebuild_node(g);
#pragma unroll
                    for (int p = 0; p < 9; ++p) {
                        s[p] = g[2 * p + 1] + g[2 * p + 2];
                        d[p] = g[2 * p + 1] - g[2 * p + 2];
                    }
                    drho0 = g[0] + s[0];
                } else {
#pragma unroll
                    for (int p = 0; p < 9; ++p) {
                        const float b = V::cell(v[2 * p + 2], j);
                        s[p] = V::add_h(v[2 * p + 1], j, b);
                        d[p] = V::sub_h(v[2 * p + 1], j, b);
                    }
                    drho0 = V::add_h(v[0], j, s[0]);
                }
                collide_sd<REG, FORCE, SP>(g, s, d, drho0, tau0, kq, Fx, Fy, Fz, drho, ux, uy, uz, nuf);
            } else {
#pragma unroll
                for (int i = 0; i < Q; ++i) g[i] = V::cell(v[i], j);
                if (node) rebuild_node(g);
                collide<REG, FORCE, SP>(g, tau0, kq, Fx, Fy, Fz, drho, ux, uy, uz, nuf);
            }
            upx = ux;
            upy = uy;
            upz = uz;
            // the pair's first cell waits in FP32; the second completes the pair,
            // which replaces the pair's (already read) inputs
            const unsigned seed = (j & 1) ? seed_of(j >> 1) : 0u;
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                if ((j & 1) == 0) gp[i] = g[i];
                else if constexpr (SR) V::set_pair_rs(v[i], j >> 1, gp[i], g[i], sr_bits(seed, i));
                else V::set_pair(v[i], j >> 1, gp[i], g[i]);
            }
            const bool counted = active;
            if (STATS && counted) {
                float *sp = &sacc[wi][0][CPL * lane + j];
                constexpr int L = BX * CPL;
                // explicit fused multiply-adds: every kernel instance rounds the sums
                // alike (the compiler would otherwise fuse them or not depending on
                // how it shares the products with the collision)
                sp[0 * L] += ux; sp[1 * L] += uy; sp[2 * L] += uz;
                sp[3 * L] = __fmaf_rn(ux, ux, sp[3 * L]); sp[4 * L] = __fmaf_rn(uy, uy, sp[4 * L]);
                sp[5 * L] = __fmaf_rn(uz, uz, sp[5 * L]); sp[6 * L] = __fmaf_rn(ux, uy, sp[6 * L]);
                sp[7 * L] = __fmaf_rn(ux, uz, sp[7 * L]); sp[8 * L] = __fmaf_rn(uy, uz, sp[8 * L]);
            }
            if (counted) sdr += drho;
        }
        }
        if (active) {
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                if (MODE == PULL) {
                    V::st(reinterpret_cast<S *>(reinterpret_cast<char *>(dbase + here) + (size_t)i * Pb), v[i]);
                    continue;
                }
                // the cell's own slot opp(i): the target of every local result,
                // and of a shifted result whose target lies outside the lattice
                auto own_slot = [&](int k) {
                    return reinterpret_cast<S *>(reinterpret_cast<char *>(dbase + here) + (size_t)opp_of(k) * Pb);
                };
                if (MODE == AA_LOCAL) {
                    V::st(own_slot(i), v[i]);
                    continue;
                }
                // in place, even steps: result of population i to slot i at x + c_i
                const int cx = cx_of(i), cz = cz_of(i), cy = cy_of(i);
                const bool yout = YEDGE && ((cy > 0 && yp_bb) || (cy < 0 && ym_bb));
                if (yout) {
                    V::st(own_slot(i), v[i]);
                    continue;
                }
                // target row (y + c_y, z + c_z): the source row of population opp(i)
                const unsigned tz = cz > 0 ? 0u - dzp : (cz < 0 ? 0u - dzm : 0u);
                const unsigned ty = cy > 0 ? (YEDGE ? 0u - (unsigned)yp_off : nxv) : (cy < 0 ? (YEDGE ? 0u - (unsigned)ym_off : 0u - nxv) : 0u);
                S *trow = reinterpret_cast<S *>(reinterpret_cast<char *>(dbase + (row0 + tz + ty)) + (size_t)i * Pb);
                S *tx = trow + x;
                if (cx == 0) {
                    V::st(tx, v[i]);
                } else if (cx < 0) {
                    // cells x + 1 .. x + CPL - 1 -> x .. x + CPL - 2 (quads: cells 1, 2
                    // as one aligned pair), cell x -> x - 1; the row's first cell
                    // (lanes with x = 0 only): outside at the inlet (the own slot),
                    // wraps to x = nx - 1 when x is periodic
                    if constexpr (CPL == 4) {
                        V::st_mid(tx, v[i]);
                        V::st1(tx - 1, v[i], 3);
                    } else {
                        V::st1(tx - 1, v[i], 1);
                    }
                    if (x > 0) V::st1(tx - 1, v[i], 0);
                    else V::st1(inout ? own_slot(i) : tx + (nx - 1), v[i], 0);
                } else {
                    // cells x .. x + CPL - 2 -> x + 1 .. x + CPL - 1 (quads: cells 1, 2
                    // as one aligned pair), cell x + CPL - 1 -> x + CPL; the row's last
                    // cell (lanes with x = nx - CPL only): outside at the outlet, wraps to 0
                    V::st1(tx + 1, v[i], 0);
                    if constexpr (CPL == 4) V::st_mid(tx + 2, v[i]);
                    if (x + CPL < nx) V::st1(tx + 1, v[i], CPL - 1);
                    else V::st1(inout ? own_slot(i) : tx - (x + CPL - 1), v[i], CPL - 1);
                }
            }
        }
    }
    return sdr;
}

// Sampling-step vector kernel over all x of rows 1..ny-2 (YEDGE false) or of
// rows 0 and ny-1 (YEDGE true; that launch also advances the device step
// counter).  Block (4 consecutive 64-cell x chunks, or one 128-cell quad
// chunk, row, group of STAT_GROUP z planes); each warp walks the group's planes in order for its own chunk
// (the plain kernel's layout 1), its lanes adding the velocity moments of
// their cells to private shared-memory slots, and writes the group's FP32
// sums per (x, y) to the group's slot of a.stat_part; stats_reduce_kernel
// then adds the groups in order.  The decomposition is fixed (no tile), so
// the statistics are deterministic and independent of the launch tile.
// H16 as in vec_loop.  STATS is chosen on the host (it knows the step
// count); plain steps use lbm_vec_zc_kernel.
// warps (x chunks) per block of the layout-1 and sampling kernels: 4 with
// pairs (256 cells), one with quads (128 cells: wider quad blocks leave warps
// idle on rows that are not a multiple of their width, e.g. a quarter of them
// on 768-cell rows, and were no faster on 1536-cell rows)
constexpr int QUAD_NW = 1;
template <int CPL>
constexpr int chunk_warps() { return CPL == 4 ? QUAD_NW : 4; }
template <typename S, int CPL, bool REG, bool FORCE, bool STATS, bool YEDGE, bool SP, bool H16, int MODE, bool SR>
// (the wall rows, on the branch beside the interior launch, may take 128
// registers so that they need no stack frame; binary16 quads take 96)
__global__ void __launch_bounds__(BX *chunk_warps<CPL>(), (YEDGE ? 16 : ((REG && !FORCE) ? (CPL == 4 ? 20 : 32) : 24)) / chunk_warps<CPL>())
    lbm_vec_kernel(const StepArgs a)
{
    constexpr int STAT_NW = chunk_warps<CPL>();
    __shared__ float sacc[STATS ? STAT_NW : 1][9][BX * CPL];  // per-thread statistics slots
    const int nx = a.nx, ny = a.ny;
    const int lane = threadIdx.x, wi = threadIdx.y;
    const int x0 = BX * CPL * (STAT_NW * blockIdx.x + wi);
    const int y = YEDGE ? (blockIdx.y == 0 ? 0 : ny - 1) : blockIdx.y + 1;
    const long long t = a.ctl->t[a.parity];
    const bool do_check = a.check_every > 0 && ((t + 1) % a.check_every) == 0;
    if (STATS) {
#pragma unroll
        for (int q = 0; q < 9; ++q)
#pragma unroll
            for (int j = 0; j < CPL; ++j) sacc[wi][q][CPL * lane + j] = 0.f;
    }
    const int zb = STATS ? blockIdx.z * STAT_GROUP : 0;
    const float sdr = vec_loop<S, CPL, REG, FORCE, STATS, YEDGE, SP, H16, MODE, SR>(
        a, sacc, x0, y, zb, STATS ? min(zb + STAT_GROUP, a.nz) : a.nz, 1);
    if (STATS) {
        // each thread wrote only its own slots: no barrier
        const size_t m = (size_t)nx * ny;
        float *part = a.stat_part + (size_t)blockIdx.z * 9 * m;
#pragma unroll
        for (int j = 0; j < CPL; ++j) {
            const int xc = x0 + CPL * lane + j;
            if (xc >= nx) continue;
            const size_t xy = (size_t)y * nx + xc;
#pragma unroll
            for (int q = 0; q < 9; ++q) part[q * m + xy] = sacc[wi][q][CPL * lane + j];
        }
    }
    if (do_check) mass_finish<BX * STAT_NW>(a, sdr);
    if (YEDGE && a.bump_t && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && lane == 0 && wi == 0)
        a.ctl->t[a.parity ^ 1] = t + 1;
}

// Plain-step vector kernel, tiled in z: block (x chunk, row, z chunk of
// a.tile_zc planes, or of a.tile_wall_zc planes for the wall rows).  Many
// short blocks instead of one block per z column keep the last wave of the
// grid small.  LAYOUT 0: 8 warps on one 64-cell x chunk, warp w taking the
// planes w, w + 8, ... of the chunk; LAYOUT 1: 4 warps on 4 consecutive x
// chunks (256 cells), all walking the chunk's planes together (binary16
// quads: one warp on one 128-cell chunk).  The regularized unforced interior variants fit 64
// registers with pairs (32 warps per SM) and 96 with quads (20 warps per SM:
// with 8-byte row pieces those warps keep as many bytes in flight as FP32);
// BGK, forced and wall-row ones get 80 with pairs (24 warps per SM) and 128
// with quads.
template <int LAYOUT, bool LEAN, int CPL = 2>
struct ZcShape {
    static constexpr int NW = LAYOUT == 0 ? BZ : chunk_warps<CPL>();  // warps per block
    static constexpr int MINB = (CPL == 4 ? (LEAN ? 20 : 16) : (LEAN ? 32 : 24)) / NW;  // resident blocks per SM
};

template <typename S, int CPL, bool REG, bool FORCE, int LAYOUT, bool YEDGE, bool SP, bool H16, int MODE, bool SR>
__global__ void __launch_bounds__(BX *ZcShape<LAYOUT, REG && !FORCE && !YEDGE, CPL>::NW,
                                  ZcShape<LAYOUT, REG && !FORCE && !YEDGE, CPL>::MINB)
    lbm_vec_zc_kernel(const StepArgs a)
{
    constexpr int NW = ZcShape<LAYOUT, REG && !FORCE && !YEDGE, CPL>::NW;
    const int wi = threadIdx.y;
    const int y = YEDGE ? (blockIdx.y == 0 ? 0 : a.ny - 1) : blockIdx.y + 1;
    const int zc0 = YEDGE ? a.tile_wall_zc : a.tile_zc;
    const int zc = zc0 > 0 ? zc0 : a.nz;
    const int zb = blockIdx.z * zc, ze = min(zb + zc, a.nz);
    const long long t = a.ctl->t[a.parity];
    const bool do_check = a.check_every > 0 && ((t + 1) % a.check_every) == 0;
    float sdr;
    if (LAYOUT == 0)
        sdr = vec_loop<S, CPL, REG, FORCE, false, YEDGE, SP, H16, MODE, SR>(a, nullptr, BX * CPL * blockIdx.x, y, zb + wi, ze, NW);
    else
        sdr = vec_loop<S, CPL, REG, FORCE, false, YEDGE, SP, H16, MODE, SR>(a, nullptr, BX * CPL * (NW * blockIdx.x + wi), y, zb, ze, 1);
    if (do_check) mass_finish<BX * NW>(a, sdr);
    if (YEDGE && a.bump_t && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && threadIdx.x == 0 && wi == 0)
        a.ctl->t[a.parity ^ 1] = t + 1;
}

// Edge columns of the one-cell-per-thread split (32 wide, general pull):
// every chunk of rows 0 and ny-1, and the chunks outside [il, ir) of rows
// 1..ny-2.  Block 0 also advances the device step counter (read by the next
// step only).
template <typename S, bool REG, bool FORCE, bool SP, bool SR>
__global__ void __launch_bounds__(BX *BZ, 2) lbm_edge_kernel(const StepArgs a)
{
    const int nxc = (a.nx + BX - 1) / BX;
    const int b = blockIdx.x;
    const int nwall = (a.ny >= 2 ? 2 : 1) * nxc;
    int bx, y;
    if (b < nwall) {
        y = (b < nxc) ? 0 : a.ny - 1;
        bx = b % nxc;
    } else {
        const int emid = nxc - (a.ir - a.il);
        const int r = b - nwall;
        y = 1 + r / emid;
        const int k = r % emid;
        bx = k < a.il ? k : a.ir + (k - a.il);
    }
    const long long t = a.ctl->t[a.parity];
    step_column<S, REG, FORCE, true, SP, SR>(a, bx, y);
    if (a.bump_t && b == 0 && threadIdx.x == 0 && threadIdx.y == 0) a.ctl->t[a.parity ^ 1] = t + 1;
}

// How a pass covers the lattice.
//  vector split: vector kernel on rows 1..ny-2 and on rows {0, ny-1} (all x,
//                inlet/outlet nodes included);
//  scalar split: interior kernel (one cell per thread) on the
//                32-wide chunks [1, nxc-1) of rows 1..ny-2, edge kernel on the
//                rest.
struct Split {
    bool vec;
    int il, ir, gx, gy;        // scalar split interior
    int n_edge;
};

static Split split_of(const StepArgs &a, int cpl)
{
    Split sp{};
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int nxc = (nx + BX - 1) / BX;
    // the in-place scheme exists for the vector kernels only (the host checks
    // its lattice conditions), so it ignores the interior override
    sp.vec = (a.aa || a.interior == 0 || a.interior == 2) && nx % cpl == 0 && nx >= 2 * cpl &&
             19.0 * nx * ny * nz < 4294967296.0 && (a.bc_x != 0 || nx >= 3);
    if (sp.vec) return sp;
    if (nxc >= 3 && ny >= 3) {
        sp.il = 1;
        sp.ir = nxc - 1;
        sp.gy = ny - 2;
        sp.gx = sp.ir - sp.il;
    }
    const int nwall = (ny >= 2 ? 2 : 1) * nxc;
    sp.n_edge = nwall + (ny > 2 ? ny - 2 : 0) * (nxc - (sp.ir - sp.il));
    return sp;
}

// Vector split of one pass in streaming mode MODE.
template <typename S, int CPL, bool REG, bool FORCE, bool SP, int MODE, bool SR>
static void launch_vec(StepArgs a, bool stats, cudaStream_t s, cudaStream_t side)
{
    const dim3 block(BX, BZ);
    {
        constexpr int cpl = CPL;
        const int nx = a.nx, ny = a.ny;
        const int nxv = (nx + BX * cpl - 1) / (BX * cpl);  // vector chunks per row
        const int rows_in = ny > 2 ? ny - 2 : 0, rows_edge = ny >= 2 ? 2 : 1;
        const int nz = a.nz;
        // grids: sampling steps take fixed groups of STAT_GROUP planes (their
        // sums go to a.stat_part and are reduced after the pass); plain steps
        // take the tile's z chunks
        const int groups = (nz + STAT_GROUP - 1) / STAT_GROUP;
        constexpr int STAT_NW = chunk_warps<CPL>();
        const int nxs = (nx + BX * cpl * STAT_NW - 1) / (BX * cpl * STAT_NW);  // sampling blocks along x
        dim3 gi(nxs, rows_in, groups), ge(nxs, rows_edge, groups);
        const dim3 bs(BX, STAT_NW);
        dim3 bi = block;
        if (!stats) {
            const int zc = a.tile_zc > 0 ? a.tile_zc : nz, wzc = a.tile_wall_zc > 0 ? a.tile_wall_zc : nz;
            if (a.tile_layout == 1) {
                constexpr int W = ZcShape<1, true, CPL>::NW;
                gi = dim3((nx + BX * cpl * W - 1) / (BX * cpl * W), rows_in, (nz + zc - 1) / zc);
                bi = dim3(BX, W);
            } else {
                gi = dim3(nxv, rows_in, (nz + zc - 1) / zc);
            }
            ge = dim3(nxv, rows_edge, (nz + wzc - 1) / wzc);
        }
        const int n_in = rows_in > 0 ? (int)(gi.x * gi.y * gi.z) : 0;
        const int n_edge = (int)(ge.x * ge.y * ge.z);
        // binary16 in an inlet/outlet lattice: x halo by 2-byte loads
        // (the local in-place step reads no x neighbour)
        constexpr bool H = sizeof(S) == 2 && MODE != AA_LOCAL;
        const bool h16 = H && a.bc_x == 0;
        a.total_blocks = (unsigned)(n_in + n_edge);
        StepArgs ai = a, ae = a;
        ai.slot_base = 0;
        ae.slot_base = n_in;
        ae.bump_t = 1;
        if (n_in > 0) {
            if (stats && h16) lbm_vec_kernel<S, CPL, REG, FORCE, true, false, SP, H, MODE, SR><<<gi, bs, 0, s>>>(ai);
            else if (stats) lbm_vec_kernel<S, CPL, REG, FORCE, true, false, SP, false, MODE, SR><<<gi, bs, 0, s>>>(ai);
            else if (h16 && a.tile_layout == 1) lbm_vec_zc_kernel<S, CPL, REG, FORCE, 1, false, SP, H, MODE, SR><<<gi, bi, 0, s>>>(ai);
            else if (h16) lbm_vec_zc_kernel<S, CPL, REG, FORCE, 0, false, SP, H, MODE, SR><<<gi, bi, 0, s>>>(ai);
            else if (a.tile_layout == 1) lbm_vec_zc_kernel<S, CPL, REG, FORCE, 1, false, SP, false, MODE, SR><<<gi, bi, 0, s>>>(ai);
            else lbm_vec_zc_kernel<S, CPL, REG, FORCE, 0, false, SP, false, MODE, SR><<<gi, bi, 0, s>>>(ai);
        }
        if (stats && h16) lbm_vec_kernel<S, CPL, REG, FORCE, true, true, SP, H, MODE, SR><<<ge, bs, 0, side>>>(ae);
        else if (stats) lbm_vec_kernel<S, CPL, REG, FORCE, true, true, SP, false, MODE, SR><<<ge, bs, 0, side>>>(ae);
        else if (h16) lbm_vec_zc_kernel<S, CPL, REG, FORCE, 0, true, SP, H, MODE, SR><<<ge, block, 0, side>>>(ae);
        else lbm_vec_zc_kernel<S, CPL, REG, FORCE, 0, true, SP, false, MODE, SR><<<ge, block, 0, side>>>(ae);
    }
}

// Returns true when the pass left z-group statistics in a.stat_part.
template <typename S, bool REG, bool FORCE, bool SP, bool SR>
static bool launch_forced(StepArgs a, const Split &sp, bool stats, cudaStream_t s,
                          cudaStream_t side)
{
    const dim3 block(BX, BZ);
    if (sp.vec) {
        // binary16, regularized unforced, rows of whole quads: four cells per lane
        constexpr bool QUAD = sizeof(S) == 2 && REG && !FORCE;
        // in place: steps with even index shift, steps with odd index stay local
        const int mode = !a.aa ? PULL : (a.parity == 0 ? AA_SHIFT : AA_LOCAL);
        if (QUAD && quads_fit(a.nx)) {
            if constexpr (QUAD) {
                if (mode == PULL) launch_vec<S, 4, REG, FORCE, SP, PULL, SR>(a, stats, s, side);
                else if (mode == AA_SHIFT) launch_vec<S, 4, REG, FORCE, SP, AA_SHIFT, SR>(a, stats, s, side);
                else launch_vec<S, 4, REG, FORCE, SP, AA_LOCAL, SR>(a, stats, s, side);
            }
        } else {
            if (mode == PULL) launch_vec<S, 2, REG, FORCE, SP, PULL, SR>(a, stats, s, side);
            else if (mode == AA_SHIFT) launch_vec<S, 2, REG, FORCE, SP, AA_SHIFT, SR>(a, stats, s, side);
            else launch_vec<S, 2, REG, FORCE, SP, AA_LOCAL, SR>(a, stats, s, side);
        }
        return stats;
    }
    const int n_in = sp.gy > 0 ? sp.gx * sp.gy : 0;
    a.il = sp.il;
    a.ir = sp.ir;
    a.total_blocks = (unsigned)(n_in + sp.n_edge);
    StepArgs ai = a, ae = a;
    ai.slot_base = 0;
    ae.slot_base = n_in;
    ae.bump_t = 1;
    lbm_edge_kernel<S, REG, FORCE, SP, SR><<<sp.n_edge, block, 0, side>>>(ae);
    if (n_in > 0) {
        lbm_step_kernel<S, REG, FORCE, SP, SR><<<dim3(sp.gx, sp.gy), block, 0, s>>>(ai);
    }
    return false;
}

// SR: binary16 stores by stochastic rounding (S = __half only)
template <typename S, bool REG, bool SR = false>
bool launch_typed(const StepArgs &a0, bool stats, cudaStream_t s, cudaStream_t side)
{
    const Split sp = split_of(a0, 2);
    StepArgs a = a0;
    a.bump_t = 0;
    // the sponge is only compiled for unforced lattices (the host refuses a sponge with a force)
    if (a.spf) return launch_forced<S, REG, false, true, SR>(a, sp, stats, s, side);
    if (a.has_force) return launch_forced<S, REG, true, false, SR>(a, sp, stats, s, side);
    return launch_forced<S, REG, false, false, SR>(a, sp, stats, s, side);
}

}  // namespace stg
