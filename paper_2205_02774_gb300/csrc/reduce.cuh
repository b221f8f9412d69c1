// Block-level reductions shared by the step kernels.
#pragma once

#include "internal.h"

namespace stg {

// Sum of one double per thread over a block of NT threads (a multiple of 32,
// at most 1024) in a fixed order: a butterfly of warp shuffles inside each
// warp, then warp 0 adds the warp sums by the same butterfly.  Every thread of
// the block must call it (it holds a barrier); the result is meant for thread
// 0 (each lane's butterfly associates the terms its own way, lane 0's always
// the same).  ws: shared scratch of NT / 32 doubles.
template <int NT>
__device__ __forceinline__ double block_sum(double v, double *ws)
{
    static_assert(NT % 32 == 0 && NT <= 1024, "whole warps");
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((tid & 31) == 0) ws[tid >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (tid < 32) {
        s = tid < NT / 32 ? ws[tid] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    }
    return s;
}

// Deterministic FP64 mass of a step pass: each block leaves the sum of its
// threads' (rho - 1) in its own slot, a.slot_base + its linear block index
// (x fastest, then y, then z); the last of all total_blocks blocks of the pass
// (all kernels) adds the slots in index order (each thread a strided subset,
// then the block sum) and writes nx ny nz + sum.  NT = threads per block.
template <int NT>
__device__ __forceinline__ void mass_finish(const StepArgs &a, float sdr)
{
    __shared__ double ws[NT / 32];
    __shared__ int s_last;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const double bs = block_sum<NT>((double)sdr, ws);
    if (tid == 0) {
        a.mass_partial[a.slot_base + (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = bs;
        __threadfence();
        const unsigned prev = atomicAdd(a.mass_counter, 1u);
        s_last = (prev == a.total_blocks - 1);
    }
    __syncthreads();
    if (s_last) {
        __threadfence();
        double acc = 0.0;
        for (unsigned k = tid; k < a.total_blocks; k += NT) acc += __ldcg(a.mass_partial + k);
        const double tot = block_sum<NT>(acc, ws);
        if (tid == 0) {
            a.mass_out[0] = tot + (double)a.P;
            *a.mass_counter = 0u;
        }
    }
}

}  // namespace stg
