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
// part phi^n + omega^n t (evaluated in FP64 per block); their FP32 sum is
// below 6 pi whatever the step count and is reduced to [-pi, pi] before the
// cosine.  Each block serves 32 nodes; its 8 warps split the mode sum.
// The plane of step t + 1 is computed during step t (ahead = 1), beside the
// step pass that reads the plane of step t; the first plane after a reset is
// computed with ahead = 0.
#include "internal.h"

namespace stg {

constexpr int INLET_NODES = 32;  // nodes per block (one per lane)
constexpr int INLET_WARPS = 8;   // the mode sum of each node is split over 8 warps
constexpr double TWO_PI = 6.283185307179586476925286766559;

__global__ void __launch_bounds__(INLET_NODES *INLET_WARPS) stg_inlet_kernel(const InletArgs a)
{
    extern __shared__ float sm[];  // theta[N], sigma[3N]
    __shared__ float part[INLET_WARPS][3][INLET_NODES];
    float *theta = sm;
    float *sig = sm + a.N;
    const int tid = threadIdx.y * INLET_NODES + threadIdx.x;
    const long long t = a.ctl->t[a.parity] + a.ahead;
    const bool first = (t == a.ctl->t0_filter);
    // time part of the phase, phi^n + omega^n t, reduced to [0, 2 pi) in FP64
    for (int n = tid; n < a.N; n += INLET_NODES * INLET_WARPS) {
        double th = a.phi[n] + a.omg[n] * (double)t;
        th -= TWO_PI * floor(th / TWO_PI);
        theta[n] = (float)th;
        sig[3 * n + 0] = a.sig[3 * n + 0];
        sig[3 * n + 1] = a.sig[3 * n + 1];
        sig[3 * n + 2] = a.sig[3 * n + 2];
    }
    __syncthreads();
    const int ny = a.ny, nz = a.nz;
    const int node = blockIdx.x * INLET_NODES + threadIdx.x;
    const bool live = node < ny * nz;
    const int j = live ? node % ny : 0, k = live ? node / ny : 0;
    float v0 = 0.f, v1 = 0.f, v2 = 0.f;
    if (live) {
        for (int n = threadIdx.y; n < a.N; n += INLET_WARPS) {
            float arg = a.A[(size_t)n * ny + j] + a.B[(size_t)n * nz + k] + theta[n];  // in [0, 6 pi)
            arg -= 6.2831853f * rintf(arg * 0.15915494f);                             // to [-pi, pi]
            const float amp = a.SQ[(size_t)n * ny + j] * __cosf(arg);
            v0 = fmaf(amp, sig[3 * n + 0], v0);
            v1 = fmaf(amp, sig[3 * n + 1], v1);
            v2 = fmaf(amp, sig[3 * n + 2], v2);
        }
    }
    part[threadIdx.y][0][threadIdx.x] = v0;
    part[threadIdx.y][1][threadIdx.x] = v1;
    part[threadIdx.y][2][threadIdx.x] = v2;
    __syncthreads();
    if (threadIdx.y != 0 || !live) return;
    v0 = v1 = v2 = 0.f;
#pragma unroll
    for (int w = 0; w < INLET_WARPS; ++w) {
        v0 += part[w][0][threadIdx.x];
        v1 += part[w][1][threadIdx.x];
        v2 += part[w][2][threadIdx.x];
    }
    const float *L = a.a6 + 6 * j;
    const float u0 = L[0] * v0;
    const float u1 = L[1] * v0 + L[2] * v1;
    const float u2 = L[3] * v0 + L[4] * v1 + L[5] * v2;
    const size_t plane = (size_t)ny * nz;
    float f0 = u0, f1 = u1, f2 = u2;
    if (!first) {
        const float af = a.a_filter, bf = 1.0f - a.a_filter;
        f0 = af * a.uf[node] + bf * u0;
        f1 = af * a.uf[plane + node] + bf * u1;
        f2 = af * a.uf[2 * plane + node] + bf * u2;
    }
    a.uf[node] = f0;
    a.uf[plane + node] = f1;
    a.uf[2 * plane + node] = f2;
    a.ubc[node] = a.u_int[j] + f0;
    a.ubc[plane + node] = f1;
    a.ubc[2 * plane + node] = f2;
}

cudaError_t launch_inlet(const InletArgs &a, cudaStream_t s)
{
    const int nodes = a.ny * a.nz;
    const int blocks = (nodes + INLET_NODES - 1) / INLET_NODES;
    const size_t smem = sizeof(float) * 4 * (size_t)(a.N > 0 ? a.N : 1);
    stg_inlet_kernel<<<blocks, dim3(INLET_NODES, INLET_WARPS), smem, s>>>(a);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// FP64 setup per inlet node j: Cholesky factor of the lattice-unit Reynolds
// stress (eq. cholesky; a negative radicand counts as zero, a zero pivot
// zeroes the column) and the mode weights sqrt(6 q^n) from the modified von
// Karman spectrum (eq. qn; Shur et al.'s form, cited by the paper):
//   E(k) = (k/k_e)^4 [1 + 2.4 (k/k_e)^2]^(-17/6) exp(-(12 k/k_eta)^2)
//          exp(-(4 max(k - 0.9 k_cut, 0)/k_cut)^3).
__device__ double vk_spectrum(double k, double le, double leta, double lcut)
{
    if (le <= 0.0) return 0.0;
    const double r = k * le / TWO_PI;  // k / k_e
    const double r2 = r * r;
    double e = r2 * r2 * pow(1.0 + 2.4 * r2, -17.0 / 6.0);
    if (leta > 0.0) {
        const double g = 12.0 * k * leta / TWO_PI;  // 12 k / k_eta
        e *= exp(-g * g);
    }
    if (lcut > 0.0) {
        const double kc = TWO_PI / lcut;
        const double h = 4.0 * fmax(k - 0.9 * kc, 0.0) / kc;
        e *= exp(-h * h * h);
    }
    return e;
}

// One block per inlet node j; its threads share the mode sum (FP64, fixed
// reduction order).
constexpr int SETUP_THREADS = 128;

__global__ void __launch_bounds__(SETUP_THREADS) setup_nodes_kernel(int ny, int N, const double *R6, const double *le,
                                                                     const double *leta, const double *lcut,
                                                                     const double *kn, const double *dk, float *a6,
                                                                     float *SQ)
{
    __shared__ double red[SETUP_THREADS];
    const int j = blockIdx.x;
    if (threadIdx.x == 0) {
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
    const double lej = le[j], letaj = leta[j], lcutj = lcut[j];
    double acc = 0.0;
    for (int n = threadIdx.x; n < N; n += SETUP_THREADS) acc += vk_spectrum(kn[n], lej, letaj, lcutj) * dk[n];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int off = SETUP_THREADS / 2; off > 0; off >>= 1) {
        if (threadIdx.x < off) red[threadIdx.x] += red[threadIdx.x + off];
        __syncthreads();
    }
    const double total = red[0];
    for (int n = threadIdx.x; n < N; n += SETUP_THREADS) {
        const double q = total > 0.0 ? vk_spectrum(kn[n], lej, letaj, lcutj) * dk[n] / total : 0.0;
        SQ[(size_t)n * ny + j] = (float)sqrt(6.0 * q);
    }
}

cudaError_t launch_setup_nodes(int ny, int N, const double *R6, const double *le, const double *leta,
                               const double *lcut, const double *kn, const double *dk, float *a6, float *SQ,
                               cudaStream_t s)
{
    setup_nodes_kernel<<<ny, SETUP_THREADS, 0, s>>>(ny, N, R6, le, leta, lcut, kn, dk, a6, SQ);
    return cudaGetLastError();
}

}  // namespace stg
