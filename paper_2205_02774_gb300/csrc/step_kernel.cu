// Host-side launch of one fused step pass (the kernels: step_kernel.cuh and
// its six instantiation units), the initial-state kernel, the statistics
// reduction of sampling steps and the FP64 mass reduction.
#include <cuda_fp16.h>

#include "d3q19.cuh"
#include "internal.h"
#include "lbm_cell.cuh"
#include "reduce.cuh"

namespace stg {

constexpr int BX = 32;

// instantiation units (step_f32_*.cu, step_f16_*.cu, step_f16sr_*.cu; reg / bgk collision)
bool launch_f32_reg(const StepArgs &a, bool stats, cudaStream_t s, cudaStream_t side);
bool launch_f32_bgk(const StepArgs &a, bool stats, cudaStream_t s, cudaStream_t side);
bool launch_f16_reg(const StepArgs &a, bool stats, cudaStream_t s, cudaStream_t side);
bool launch_f16_bgk(const StepArgs &a, bool stats, cudaStream_t s, cudaStream_t side);
bool launch_f16sr_reg(const StepArgs &a, bool stats, cudaStream_t s, cudaStream_t side);
bool launch_f16sr_bgk(const StepArgs &a, bool stats, cudaStream_t s, cudaStream_t side);

int step_grid_blocks(int nx, int ny, int nz)
{
    const long long vec = (long long)((nx + 2 * BX - 1) / (2 * BX)) * ny * ((nz + MIN_ZC - 1) / MIN_ZC);
    const long long col = (long long)((nx + BX - 1) / BX) * ny;
    return (int)((vec > col ? vec : col) + 2LL * ny + 64);
}

// Adds the z-group sums of a sampling step to the FP64 statistics, group by
// group in index order (one thread per (x, y) and moment).
__global__ void stats_reduce_kernel(const float *part, int groups, size_t m, double *stat_mean, double *stat_rey)
{
    const size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x;  // q * m + xy
    if (k >= 9 * m) return;
    // the groups in index order as a compensated FP32 sum (the two-sum error
    // of every addition is kept: hi + lo holds the sum to about 2^-44 of its
    // size), then one FP64 addition into the running sum; GB300's FP64 rate
    // is a small fraction of its FP32 rate, and an FP64 conversion and add per
    // group made this kernel FP64-bound
    float hi = 0.f, lo = 0.f;
#pragma unroll 4
    for (int g = 0; g < groups; ++g) {
        const float x = __ldcs(part + (size_t)g * 9 * m + k);
        const float s = hi + x;
        const float z = s - hi;
        lo += (hi - (s - z)) + (x - z);
        hi = s;
    }
    const double sum = (double)hi + (double)lo;
    if (k < 3 * m) stat_mean[k] += sum;
    else stat_rey[k - 3 * m] += sum;
}

// One fused step pass.  With a side stream and two events the wall rows (or
// the edge kernel on the scalar path) run on a forked branch concurrently
// with the interior (they read and write disjoint slots: the previous and the
// next lattice, or, in place, the slots of their own cells); `s` waits for
// both.  `inlet`
// (may be NULL) computes the next step's inlet plane on the branch.
cudaError_t launch_step(const StepArgs &a, int storage, int collision, bool stats,
                        cudaStream_t s, cudaStream_t side, cudaEvent_t fork, cudaEvent_t join, const InletArgs *inlet)
{
    cudaError_t e = cudaSuccess;
    const bool forked = side != nullptr && fork != nullptr && join != nullptr;
    if (forked) {
        if ((e = cudaEventRecord(fork, s)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(side, fork, 0)) != cudaSuccess) return e;
    }
    cudaStream_t es = forked ? side : s;
    // the inlet kernel writes the plane of the next step, which nothing in
    // this pass reads, so it runs on the branch beside the interior; beside a
    // quad interior (96-register warps filling the SMs' registers) its
    // 256-thread blocks waited for room and the step ran slower than with the
    // inlet ahead of the pass (FP16-SR 1.813 against 1.771 ms on 1536x256x384),
    // so there it goes first on the main stream
    const bool quad = storage != 0 && collision == 0 && !a.has_force && quads_fit(a.nx);
    if (inlet && (e = launch_inlet(*inlet, quad ? s : es)) != cudaSuccess) return e;
    bool reduce = false;
    if (storage == 0) {
        if (collision == 0) reduce = launch_f32_reg(a, stats, s, es);
        else reduce = launch_f32_bgk(a, stats, s, es);
    } else if (storage == 1) {
        if (collision == 0) reduce = launch_f16_reg(a, stats, s, es);
        else reduce = launch_f16_bgk(a, stats, s, es);
    } else {
        if (collision == 0) reduce = launch_f16sr_reg(a, stats, s, es);
        else reduce = launch_f16sr_bgk(a, stats, s, es);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (forked) {
        if ((e = cudaEventRecord(join, side)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(s, join, 0)) != cudaSuccess) return e;
    }
    if (reduce) {
        const size_t m = (size_t)a.nx * a.ny;
        const int groups = (a.nz + STAT_GROUP - 1) / STAT_GROUP;
        const unsigned blocks = (unsigned)((9 * m + 255) / 256);
        stats_reduce_kernel<<<blocks, 256, 0, s>>>(a.stat_part, groups, m, a.stat_mean, a.stat_rey);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// ---------------------------------------------------------------------------
// Initial state f^eq(1, (u_int(y), 0, 0)) (u_int == nullptr: rest state),
// stored shifted; `swap` stores population i in slot opp(i) (the in-place
// layout before a step with even index).
template <typename S>
__global__ void init_eq_kernel(S *dst, int nx, int ny, int nz, const float *u_int, int swap)
{
    const size_t P = (size_t)nx * ny * nz;
    for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < P; c += (size_t)gridDim.x * blockDim.x) {
        const int y = (int)((c / nx) % ny);
        const float ux = u_int ? u_int[y] : 0.0f;
#pragma unroll
        for (int i = 0; i < Q; ++i)
            Pop<S>::st(dst + (size_t)(swap ? opp_of(i) : i) * P + c, geq(w_of(i), 0.0f, 1.0f, cx_of(i) * ux, ux * ux));
    }
}

cudaError_t launch_init_equilibrium(void *dst, int storage, int nx, int ny, int nz, const float *u_int, int swap,
                                    cudaStream_t s)
{
    const int blocks = 152 * 8;
    if (storage == 0) init_eq_kernel<float><<<blocks, 256, 0, s>>>(static_cast<float *>(dst), nx, ny, nz, u_int, swap);
    else init_eq_kernel<__half><<<blocks, 256, 0, s>>>(static_cast<__half *>(dst), nx, ny, nz, u_int, swap);
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
    __shared__ double ws[MASS_THREADS / 32];
    __shared__ int s_last;
    double acc = 0.0;
    for (size_t c = blockIdx.x * (size_t)MASS_THREADS + threadIdx.x; c < a.P; c += (size_t)gridDim.x * MASS_THREADS) {
        float r = 0.f;
#pragma unroll
        for (int i = 0; i < Q; ++i) r += Pop<S>::ld(src + (size_t)i * a.P + c);
        acc += (double)r;
    }
    const int tid = threadIdx.x;
    const double bs = block_sum<MASS_THREADS>(acc, ws);
    if (tid == 0) {
        a.partial[blockIdx.x] = bs;
        __threadfence();
        s_last = (atomicAdd(a.counter, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (s_last) {
        double v = 0.0;
        for (unsigned k = tid; k < gridDim.x; k += MASS_THREADS) v += __ldcg(a.partial + k);
        const double tot = block_sum<MASS_THREADS>(v, ws);
        if (tid == 0) {
            a.out[0] = tot + (double)a.P;
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
