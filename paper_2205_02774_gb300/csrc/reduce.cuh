// Block-level reductions shared by the step kernels.
#pragma once

#include "internal.h"

namespace stg {

// Deterministic FP64 mass of a step pass: each block leaves the sum of its
// threads' (rho - 1) in its own slot, a.slot_base + its linear block index
// (x fastest, then y, then z);
// the last of all total_blocks blocks of the pass (all kernels) adds the
// slots in index order and writes nx ny nz + sum.  NT = threads per block (a
// power of two, at most 256).
template <int NT>
__device__ __forceinline__ void mass_finish(const StepArgs &a, float sdr)
{
    __shared__ double rd[NT];
    __shared__ int s_last;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    rd[tid] = (double)sdr;
    __syncthreads();
    for (int off = NT / 2; off > 0; off >>= 1) {
        if (tid < off) rd[tid] += rd[tid + off];
        __syncthreads();
    }
    if (tid == 0) {
        a.mass_partial[a.slot_base + (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = rd[0];
        __threadfence();
        const unsigned prev = atomicAdd(a.mass_counter, 1u);
        s_last = (prev == a.total_blocks - 1);
    }
    __syncthreads();
    if (s_last) {
        __threadfence();
        double acc = 0.0;
        for (unsigned k = tid; k < a.total_blocks; k += NT) acc += __ldcg(a.mass_partial + k);
        rd[tid] = acc;
        __syncthreads();
        for (int off = NT / 2; off > 0; off >>= 1) {
            if (tid < off) rd[tid] += rd[tid + off];
            __syncthreads();
        }
        if (tid == 0) {
            a.mass_out[0] = rd[0] + (double)a.P;
            *a.mass_counter = 0u;
        }
    }
}

}  // namespace stg
