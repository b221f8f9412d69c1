// Reads of a stored lattice: velocity probes (the velocity of chosen cells,
// from the post-collision populations g_i = f_i - w_i, for time series such as
// the auto-correlation B_uu of Sec. V; u = (sum_i c_i g_i - F/2) / (1 + sum_i
// g_i)) and the canonical sub-block gather of an in-place lattice.
#include <cuda_fp16.h>

#include "aa_layout.cuh"
#include "d3q19.cuh"
#include "internal.h"

namespace stg {

template <typename S>
__device__ __forceinline__ float ldg_pop(const S *p);
template <>
__device__ __forceinline__ float ldg_pop<float>(const float *p) { return __ldg(p); }
template <>
__device__ __forceinline__ float ldg_pop<__half>(const __half *p) { return __half2float(__ldg(p)); }

// element of canonical population i of cell (x, y, z): slot i of the cell in
// a two-lattice state, the in-place arrangement of LatticeView::t otherwise
__device__ __forceinline__ size_t pop_index(const LatticeView &v, int i, int x, int y, int z)
{
    if (!v.aa) return (size_t)i * v.P + ((size_t)z * v.ny + y) * v.nx + x;
    return aa_slot(i, x, y, z, v.t, v.nx, v.ny, v.nz, v.bc_x, v.bc_y);
}

template <typename S>
__global__ void probe_kernel(const S *src, LatticeView lv, int n, const int *xyz, float Fx, float Fy, float Fz,
                             float *out)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int x = xyz[3 * k + 0], y = xyz[3 * k + 1], z = xyz[3 * k + 2];
    float r = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const float g = ldg_pop<S>(src + pop_index(lv, i, x, y, z));
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

cudaError_t launch_probe(const void *src, int storage, const LatticeView &lv, int n, const int *xyz, float Fx,
                         float Fy, float Fz, float *out, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    const int T = 128, B = (n + T - 1) / T;
    if (storage == 0)
        probe_kernel<float><<<B, T, 0, s>>>(static_cast<const float *>(src), lv, n, xyz, Fx, Fy, Fz, out);
    else
        probe_kernel<__half><<<B, T, 0, s>>>(static_cast<const __half *>(src), lv, n, xyz, Fx, Fy, Fz, out);
    return cudaGetLastError();
}

// Canonical sub-block [19][bz][by][bx] of a stored lattice, bit for bit
// (E: the 4- or 2-byte element).
template <typename E>
__global__ void gather_block_kernel(const E *src, LatticeView lv, int x0, int y0, int z0, int bx, int by, int bz,
                                    E *out)
{
    const size_t n = (size_t)19 * bx * by * bz;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        size_t r = e;
        const int x = (int)(r % bx);
        r /= bx;
        const int y = (int)(r % by);
        r /= by;
        const int z = (int)(r % bz);
        const int i = (int)(r / bz);
        out[e] = src[pop_index(lv, i, x0 + x, y0 + y, z0 + z)];
    }
}

cudaError_t launch_gather_block(const void *src, int storage, const LatticeView &lv, int x0, int y0, int z0, int bx,
                                int by, int bz, void *out, cudaStream_t s)
{
    const size_t n = (size_t)19 * bx * by * bz;
    const int T = 256;
    const int B = (int)((n + T - 1) / T < 152 * 16 ? (n + T - 1) / T : 152 * 16);
    if (storage == 0)
        gather_block_kernel<uint32_t><<<B, T, 0, s>>>(static_cast<const uint32_t *>(src), lv, x0, y0, z0, bx, by, bz,
                                                     static_cast<uint32_t *>(out));
    else
        gather_block_kernel<uint16_t><<<B, T, 0, s>>>(static_cast<const uint16_t *>(src), lv, x0, y0, z0, bx, by, bz,
                                                     static_cast<uint16_t *>(out));
    return cudaGetLastError();
}

}  // namespace stg
