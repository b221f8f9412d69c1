// Velocity probes: the velocity of chosen cells, read from a stored lattice
// (post-collision populations g_i = f_i - w_i), for time series such as the
// auto-correlation B_uu of Sec. V.  u = (sum_i c_i g_i - F/2) / (1 + sum_i g_i).
#include <cuda_fp16.h>

#include "d3q19.cuh"
#include "internal.h"

namespace stg {

template <typename S>
__device__ __forceinline__ float ldg_pop(const S *p);
template <>
__device__ __forceinline__ float ldg_pop<float>(const float *p) { return __ldg(p); }
template <>
__device__ __forceinline__ float ldg_pop<__half>(const __half *p) { return __half2float(__ldg(p)); }

template <typename S>
__global__ void probe_kernel(const S *src, size_t P, int nx, int ny, int n, const int *xyz, float Fx, float Fy,
                             float Fz, float *out)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const size_t c = ((size_t)xyz[3 * k + 2] * ny + xyz[3 * k + 1]) * nx + xyz[3 * k + 0];
    float r = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const float g = ldg_pop<S>(src + (size_t)i * P + c);
        r += g;
        jx += cx_of(i) * g;
        jy += cy_of(i) * g;
        jz += cz_of(i) * g;
    }
    const float ir = 1.0f / (1.0f + r);
    out[3 * k + 0] = (jx - 0.5f * Fx) * ir;
    out[3 * k + 1] = (jy - 0.5f * Fy) * ir;
    out[3 * k + 2] = (jz - 0.5f * Fz) * ir;
}

cudaError_t launch_probe(const void *src, int storage, size_t P, int nx, int ny, int n, const int *xyz, float Fx,
                         float Fy, float Fz, float *out, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    const int T = 128, B = (n + T - 1) / T;
    if (storage == 0)
        probe_kernel<float><<<B, T, 0, s>>>(static_cast<const float *>(src), P, nx, ny, n, xyz, Fx, Fy, Fz, out);
    else
        probe_kernel<__half><<<B, T, 0, s>>>(static_cast<const __half *>(src), P, nx, ny, n, xyz, Fx, Fy, Fz, out);
    return cudaGetLastError();
}

}  // namespace stg
