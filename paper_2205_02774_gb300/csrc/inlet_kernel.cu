// Synthetic turbulence generator on the inlet plane (Algorithm 1 steps 5-8)
// and the FP64 setup kernel for the per-node inlet tables (steps 3-4).
//
// Per inlet node (j, k) and step t:
//   v'  = sqrt(6) sum_n sqrt(q^n(j)) sigma^n cos(k^n d^n . x' + phi^n)     eq. (aux_vec)
//   with k^n d^n . x' = -2 pi d^n_x U_b t / max l_e + k^n (d^n_y y_j + d^n_z z_k)  eq. (psu), x = 0
//   u'  = a(j) v'                                                           eqs. (v_fluc), (cholesky)
//   u_f = a u_f + (1 - a) u'   (first-order temporal filter; u_f = u' at the first step)
//   u_bc = u_int(j) e_x + u_f                                               eqs. (u_phys), (u_transfer)
// The phase is split into three parts each already reduced to [0, 2 pi):
// the y part and the z part (tables built in FP64 on the host) and the time
// part phi^n + omega^n t, kept as Q0.64 fractions of a turn and advanced by
// wrapping 64-bit integer arithmetic (a phase accumulator: exact modulo a
// turn for any step count, no floating point); their FP32 sum is below 6 pi
// and is reduced to [-pi, pi] before the cosine.
//
// Work split: a block covers 32 consecutive j (one per lane) by 8 span nodes
// k; its 8 warps are 4 pairs of span nodes times 2 halves of the mode sum
// (modes of even and odd index within a chunk).  Everything a mode term
// needs is staged in shared memory per chunk of INLET_CHUNK modes by
// coalesced loads of the whole block (any mode count fits the fixed
// footprint): the time phase and sigma^n, the block's 8 z parts, and its 32
// y parts and amplitudes sqrt(6 q^n(j)).  A thread reads the y part and the
// amplitude of a mode once and uses them for its two span nodes, so a mode
// term costs a few shared-memory reads, the phase sum and its reduction, one
// cosine and four multiply-adds; the two halves of the mode sum are added in
// a fixed order at the end.
// The plane of step t + 1 is computed during step t (ahead = 1), beside the
// step pass that reads the plane of step t; the first plane after a reset is
// computed with ahead = 0.
#include "internal.h"

namespace stg {

constexpr int INLET_J = 32;      // wall-normal nodes per block (one per lane)
constexpr int INLET_KPT = 2;     // span nodes per thread
constexpr int INLET_KG = 4;      // span-node pairs per block
constexpr int INLET_H = 2;       // halves of the mode sum
constexpr int INLET_WARPS = INLET_KG * INLET_H;
constexpr int INLET_K = INLET_KPT * INLET_KG;  // span nodes per block
constexpr int INLET_CHUNK = 128; // modes staged per pass through shared memory

// At least 4 blocks per SM caps the kernel at 64 registers, which it fits without
// spilling; left to itself ptxas aims at the 5 blocks the shared memory allows and
// spills to a stack frame, and with local memory the kernel no longer ran beside
// the interior pass (0.75 ms more per step on 1536x256x384 in FP32).
__global__ void __launch_bounds__(INLET_J * INLET_WARPS, 4) stg_inlet_kernel(const InletArgs a)
{
    __shared__ float4 ts[INLET_CHUNK];           // (time phase, sigma_x, sigma_y, sigma_z) per mode
    __shared__ float2 bz[INLET_CHUNK][INLET_KG]; // z parts of the block's span nodes per mode
    __shared__ float ay_s[INLET_CHUNK][INLET_J]; // y parts of the block's wall-normal nodes per mode
    __shared__ float sq_s[INLET_CHUNK][INLET_J]; // amplitudes sqrt(6 q^n(j)) per mode
    __shared__ float part[INLET_KG][INLET_KPT][3][INLET_J];  // second half of the mode sum
    const int lane = threadIdx.x, w = threadIdx.y;
    const int g = w % INLET_KG, h = w / INLET_KG;
    const int tid = w * INLET_J + lane;
    const int ny = a.ny, nz = a.nz, N = a.N;
    const int j0 = blockIdx.x * INLET_J;
    const int j = j0 + lane;
    const int k0 = blockIdx.y * INLET_K;
    const bool jl = j < ny;
    const long long t = a.ctl->t[a.parity] + a.ahead;
    const bool first = (t == a.ctl->t0_filter);
    float v[INLET_KPT][3];
#pragma unroll
    for (int q = 0; q < INLET_KPT; ++q) v[q][0] = v[q][1] = v[q][2] = 0.f;
    for (int n0 = 0; n0 < N; n0 += INLET_CHUNK) {
        const int cn = min(INLET_CHUNK, N - n0);
        __syncthreads();  // the previous chunk is consumed
        for (int m = tid; m < cn; m += INLET_J * INLET_WARPS) {
            const int n = n0 + m;
            // time part of the phase in turns: phi^n + omega^n t modulo one turn
            const unsigned long long q = a.phq[n] + a.omq[n] * (unsigned long long)t;
            const float th = (float)(unsigned)(q >> 32) * 1.4629180792671596e-09f;  // 2 pi / 2^32
            ts[m] = make_float4(th, a.sig[3 * n + 0], a.sig[3 * n + 1], a.sig[3 * n + 2]);
        }
        for (int e = tid; e < cn * INLET_K; e += INLET_J * INLET_WARPS) {
            const int m = e / INLET_K, kk = e % INLET_K;
            const int k = min(k0 + kk, nz - 1);  // span nodes past nz are computed and not stored
            reinterpret_cast<float *>(&bz[m][0])[kk] = a.B[(size_t)(n0 + m) * nz + k];
        }
        for (int e = tid; e < cn * INLET_J; e += INLET_J * INLET_WARPS) {
            const int m = e / INLET_J, jj = min(j0 + e % INLET_J, ny - 1);  // rows past ny are not stored
            ay_s[m][e % INLET_J] = a.A[(size_t)(n0 + m) * ny + jj];
            sq_s[m][e % INLET_J] = a.SQ[(size_t)(n0 + m) * ny + jj];
        }
        __syncthreads();
#pragma unroll 4
        for (int m = h; m < cn; m += INLET_H) {
            const float4 tm = ts[m];
            const float ay = ay_s[m][lane] + tm.x;  // in [0, 4 pi)
            const float sq = sq_s[m][lane];
            const float2 b2 = bz[m][g];
            const float bq[INLET_KPT] = {b2.x, b2.y};
#pragma unroll
            for (int q = 0; q < INLET_KPT; ++q) {
                float arg = ay + bq[q];                           // in [0, 6 pi)
                arg -= 6.2831853f * rintf(arg * 0.15915494f);     // to [-pi, pi]
                const float amp = sq * __cosf(arg);
                v[q][0] = fmaf(amp, tm.y, v[q][0]);
                v[q][1] = fmaf(amp, tm.z, v[q][1]);
                v[q][2] = fmaf(amp, tm.w, v[q][2]);
            }
        }
    }
    if (h == 1) {
#pragma unroll
        for (int q = 0; q < INLET_KPT; ++q)
#pragma unroll
            for (int c = 0; c < 3; ++c) part[g][q][c][lane] = v[q][c];
    }
    __syncthreads();
    if (h == 1 || !jl) return;
    const float *L = a.a6 + 6 * j;
    const float l11 = L[0], l21 = L[1], l22 = L[2], l31 = L[3], l32 = L[4], l33 = L[5];
    const float af = a.a_filter, bf = 1.0f - a.a_filter, ui = a.u_int[j];
    const size_t plane = (size_t)ny * nz;
#pragma unroll
    for (int q = 0; q < INLET_KPT; ++q) {
        const int k = k0 + g * INLET_KPT + q;
        if (k >= nz) break;
        const float v0 = v[q][0] + part[g][q][0][lane];
        const float v1 = v[q][1] + part[g][q][1][lane];
        const float v2 = v[q][2] + part[g][q][2][lane];
        const size_t node = (size_t)k * ny + j;
        const float u0 = l11 * v0;
        const float u1 = l21 * v0 + l22 * v1;
        const float u2 = l31 * v0 + l32 * v1 + l33 * v2;
        float f0 = u0, f1 = u1, f2 = u2;
        if (!first) {
            f0 = af * a.uf[node] + bf * u0;
            f1 = af * a.uf[plane + node] + bf * u1;
            f2 = af * a.uf[2 * plane + node] + bf * u2;
        }
        a.uf[node] = f0;
        a.uf[plane + node] = f1;
        a.uf[2 * plane + node] = f2;
        a.ubc[node] = ui + f0;
        a.ubc[plane + node] = f1;
        a.ubc[2 * plane + node] = f2;
    }
}

cudaError_t launch_inlet(const InletArgs &a, cudaStream_t s)
{
    const dim3 grid((a.ny + INLET_J - 1) / INLET_J, (a.nz + INLET_K - 1) / INLET_K);
    if (grid.y > 65535u) return cudaErrorInvalidConfiguration;  // nz > 524 280
    stg_inlet_kernel<<<grid, dim3(INLET_J, INLET_WARPS), 0, s>>>(a);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// FP64 setup per inlet node j: Cholesky factor of the lattice-unit Reynolds
// stress (eq. cholesky; a negative radicand counts as zero, a zero pivot
// zeroes the column).  The mode amplitudes are built on the host.
__global__ void setup_nodes_kernel(int ny, const double *R6, float *a6)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= ny) return;
    const double *R = R6 + 6 * j;  // 11 22 33 12 13 23
    const double l11 = sqrt(fmax(R[0], 0.0));
    const double l21 = l11 > 0.0 ? R[3] / l11 : 0.0;
    const double l31 = l11 > 0.0 ? R[4] / l11 : 0.0;
    const double l22 = sqrt(fmax(R[1] - l21 * l21, 0.0));
    const double l32 = l22 > 0.0 ? (R[5] - l21 * l31) / l22 : 0.0;
    const double l33 = sqrt(fmax(R[2] - l31 * l31 - l32 * l32, 0.0));
    float *o = a6 + 6 * j;
    o[0] = (float)l11; o[1] = (float)l21; o[2] = (float)l22;
    o[3] = (float)l31; o[4] = (float)l32; o[5] = (float)l33;
}

cudaError_t launch_setup_nodes(int ny, const double *R6, float *a6, cudaStream_t s)
{
    setup_nodes_kernel<<<(ny + 127) / 128, 128, 0, s>>>(ny, R6, a6);
    return cudaGetLastError();
}

}  // namespace stg
