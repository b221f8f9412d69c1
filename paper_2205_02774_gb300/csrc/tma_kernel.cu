// Interior columns of the fused step with the pull staged by the TMA engine.
//
// A block is TW warps on one 64-wide x chunk (from x = 32 il) at one y.  The z-planes are taken
// in groups of TW (warp w owns plane z = TW g + w of group g).  For each group
// and each population i one tiled tensor copy (a box of 80 x-values, 1 row,
// TW planes of plane i, starting at (x0 - 8, y - c_iy, TW g - c_iz)) lands in
// a shared-memory stage; D stages form a ring completed by mbarriers.  Warp w
// then finds the source row of every population of its plane at row w of
// that population's box, so the x +-1 shifts of the pull are plain
// shared-memory offsets.  The warp that finishes reading a stage last (a
// shared-memory counter) issues the stage's refill, so no warp ever waits for
// another.  Source rows that wrap periodically in z (planes 0 and nz-1) fall
// outside the box and are read from global memory instead.  Lane l collides
// cells (x0 + 2l, x0 + 2l + 1) (lbm_cell.cuh) and stores them as one aligned
// pair.  Every mbarrier wait is bounded: on expiry the warp records an error
// bit in StepCtl::err, waits (bounded) for the copies it may still need to
// see complete, and stops.
#include <cstdint>

#include <cuda.h>
#include <cuda_fp16.h>

#include "d3q19.cuh"
#include "internal.h"
#include "lbm_cell.cuh"
#include "reduce.cuh"

namespace stg {

constexpr int TW = 4;    // warps per block
constexpr int ROW = 80;  // staged elements per row: x0-8 .. x0+72

template <typename S>
struct TmaDepth {
    static constexpr int D = 3;
};
template <>
struct TmaDepth<float> {
    static constexpr int D = 2;
};

template <typename S>
constexpr uint32_t stage_bytes() { return (uint32_t)(Q * TW * ROW * sizeof(S)); }

template <typename S, bool STATS>
constexpr size_t tma_smem_bytes()
{
    return (size_t)TmaDepth<S>::D * stage_bytes<S>() + 128 + (STATS ? (size_t)TW * 9 * 64 * sizeof(float) : 0);
}

// ---- PTX wrappers (mbarrier, bulk async copy, proxy fences) ----
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_inval(uint32_t bar)
{
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait: false after about 2^24 polls (far beyond any legitimate copy)
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity)
{
    for (int it = 0; it < (1 << 24); ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// ---- reading cell pairs from a staged row (b = 8 + 2 lane) ----
template <typename S>
struct Staged;

template <>
struct Staged<float> {
    using raw = float2;
    static __device__ __forceinline__ raw at(const float *row, int b, int cx)
    {
        if (cx == 0) return *reinterpret_cast<const float2 *>(row + b);
        if (cx > 0) return make_float2(row[b - 1], row[b]);
        return make_float2(row[b + 1], row[b + 2]);
    }
    static __device__ __forceinline__ float lo(raw v) { return v.x; }
    static __device__ __forceinline__ float hi(raw v) { return v.y; }
    static __device__ __forceinline__ raw put_lo(raw v, float a) { return make_float2(a, v.y); }
    static __device__ __forceinline__ void st(float *p, raw v, float b)
    {
        __stcs(reinterpret_cast<float2 *>(p), make_float2(v.x, b));
    }
};

template <>
struct Staged<__half> {
    using raw = unsigned;  // low half: first cell
    static __device__ __forceinline__ raw at(const __half *row, int b, int cx)
    {
        const unsigned *r = reinterpret_cast<const unsigned *>(row);
        const int q = b >> 1;  // pair index of cell b
        if (cx == 0) return r[q];
        if (cx > 0) return __byte_perm(r[q - 1], r[q], 0x5432);  // (b-1, b)
        return __byte_perm(r[q], r[q + 1], 0x5432);              // (b+1, b+2)
    }
    static __device__ __forceinline__ float lo(raw v) { return __half2float(__ushort_as_half((unsigned short)(v & 0xffffu))); }
    static __device__ __forceinline__ float hi(raw v) { return __half2float(__ushort_as_half((unsigned short)(v >> 16))); }
    static __device__ __forceinline__ raw put_lo(raw v, float a)
    {
        return (v & 0xffff0000u) | (unsigned)__half_as_ushort(__float2half_rn(a));
    }
    static __device__ __forceinline__ void st(__half *p, raw v, float b)
    {
        const unsigned out = (v & 0xffffu) | ((unsigned)__half_as_ushort(__float2half_rn(b)) << 16);
        __stcs(reinterpret_cast<unsigned *>(p), out);
    }
};

__device__ __forceinline__ void tensor_g2s_4d(uint32_t dst, const CUtensorMap *map, int c0, int c1, int c2, int c3,
                                              uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
        : "memory");
}

// a pair of cells read straight from global memory (periodic z-wrap rows)
template <typename S>
__device__ __forceinline__ typename Staged<S>::raw global_pair(const S *row, int x, int cx);
template <>
__device__ __forceinline__ float2 global_pair<float>(const float *row, int x, int cx)
{
    return make_float2(__ldg(row + x - cx), __ldg(row + x + 1 - cx));
}
template <>
__device__ __forceinline__ unsigned global_pair<__half>(const __half *row, int x, int cx)
{
    return (unsigned)__half_as_ushort(__ldg(row + x - cx)) | ((unsigned)__half_as_ushort(__ldg(row + x + 1 - cx)) << 16);
}

template <typename S, bool REG, bool FORCE, bool STATS>
__global__ void __launch_bounds__(32 * TW, 6) lbm_tma_kernel(const StepArgs a, const __grid_constant__ CUtensorMap tmap)
{
    constexpr int D = TmaDepth<S>::D;
    constexpr uint32_t BOX = TW * ROW;  // elements of one population's box
    constexpr uint32_t SB = stage_bytes<S>();
    using ST = Staged<S>;
    using raw = typename ST::raw;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + (size_t)D * SB);
    unsigned *cnt = reinterpret_cast<unsigned *>(full + D);
    float *sacc = reinterpret_cast<float *>(smem + (size_t)D * SB + 128);  // [TW][9][64]

    const int w = threadIdx.y, lane = threadIdx.x;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int y = blockIdx.y + 1;
    const int x0 = 32 * a.il + 64 * blockIdx.x;  // interior chunk pairs from x = 32 il
    const int ngroups = (nz + TW - 1) / TW;
    const long long t = a.ctl->t[a.parity];
    const bool do_check = a.check_every > 0 && ((t + 1) % a.check_every) == 0;
    const float tau0 = a.tau0, kq = a.kq;
    const float Fx = a.Fx, Fy = a.Fy, Fz = a.Fz;
    const S *sbase = static_cast<const S *>(a.src);
    S *dbase = static_cast<S *>(a.dst);

    if (w == 0 && lane == 0) {
        for (int s = 0; s < D; ++s) {
            mbar_init(smem_u32(full + s), 1);
            cnt[s] = 0u;
        }
        fence_mbar_init();
    }
    if (STATS) {
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            sacc[(w * 9 + q) * 64 + 2 * lane] = 0.f;
            sacc[(w * 9 + q) * 64 + 2 * lane + 1] = 0.f;
        }
    }
    __syncthreads();

    // one box per population for group g into stage s (one thread)
    auto issue = [&](int g, int s) {
        const uint32_t bar = smem_u32(full + s);
        const uint32_t dst = smem_u32(smem + (size_t)s * SB);
        mbar_arrive_expect_tx(bar, SB);
#pragma unroll
        for (int i = 0; i < Q; ++i)
            tensor_g2s_4d(dst + (uint32_t)(i * BOX * sizeof(S)), &tmap, x0 - 8, y - cy_of(i), TW * g - cz_of(i), i, bar);
    };
    if (w == 0 && lane == 0)
        for (int g = 0; g < D && g < ngroups; ++g) issue(g, g);

    float sdr = 0.f;
    int g = 0;
    bool failed = false;
    for (; g < ngroups; ++g) {
        const int s = g % D;
        if (!mbar_wait_bounded(smem_u32(full + s), (uint32_t)((g / D) & 1))) {
            failed = true;
            break;
        }
        const int z = TW * g + w;
        const bool live = z < nz;
        const S *stg = reinterpret_cast<const S *>(smem + (size_t)s * SB);
        const int b = 8 + 2 * lane;
        const int x = x0 + 2 * lane;
        raw v[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int cz = cz_of(i);
            const int zs = z - cz;
            if (cz != 0 && live && (zs < 0 || zs >= nz)) {
                const int zw = zs < 0 ? zs + nz : zs - nz;
                const S *row = sbase + (size_t)i * a.P + ((size_t)zw * ny + (y - cy_of(i))) * nx;
                v[i] = global_pair<S>(row, x, cx_of(i));
            } else {
                v[i] = ST::at(stg + i * BOX + w * ROW, b, cx_of(i));
            }
        }
        // release the stage: the last warp to finish reading refills it
        __syncwarp();
        if (lane == 0) {
            __threadfence_block();
            const unsigned prev = atomicAdd(cnt + s, 1u);
            if (prev == TW - 1) {
                cnt[s] = 0u;
                __threadfence_block();
                fence_proxy_async();  // all reads of stage s precede the copies that overwrite it
                if (g + D < ngroups) issue(g + D, s);
            }
        }
        if (live) {
            unsigned Pv;  // opaque copy: keeps the 19 store-plane offsets out of registers
            asm volatile("mov.u32 %0, %1;" : "=r"(Pv) : "r"(a.P));
            const unsigned here = ((unsigned)z * ny + y) * nx + x;
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                float gg[Q];
#pragma unroll
                for (int i = 0; i < Q; ++i) gg[i] = half ? ST::hi(v[i]) : ST::lo(v[i]);
                float drho, ux, uy, uz;
                collide<REG, FORCE>(gg, tau0, kq, Fx, Fy, Fz, drho, ux, uy, uz);
                if (half == 0) {
#pragma unroll
                    for (int i = 0; i < Q; ++i) v[i] = ST::put_lo(v[i], gg[i]);
                } else {
#pragma unroll
                    for (int i = 0; i < Q; ++i) ST::st(dbase + (i * Pv + here), v[i], gg[i]);
                }
                if (STATS) {
                    float *sp = sacc + (w * 9) * 64 + 2 * lane + half;
                    sp[0 * 64] += ux; sp[1 * 64] += uy; sp[2 * 64] += uz;
                    sp[3 * 64] += ux * ux; sp[4 * 64] += uy * uy; sp[5 * 64] += uz * uz;
                    sp[6 * 64] += ux * uy; sp[7 * 64] += ux * uz; sp[8 * 64] += uy * uz;
                }
                sdr += drho;
            }
        }
    }
    if (failed) {
        if (lane == 0) atomicOr(&a.ctl->err, 1ull);
        // wait (bounded) for the copies of the stages still ahead of this warp
        for (int j = g; j < ngroups && j < g + D; ++j) mbar_wait_bounded(smem_u32(full + (j % D)), (uint32_t)((j / D) & 1));
    }
    __syncthreads();
    if (w == 0 && lane == 0)
        for (int s = 0; s < D; ++s) mbar_inval(smem_u32(full + s));

    if (STATS) {
        if (w == 0) {
            const size_t m = (size_t)nx * ny;
#pragma unroll
            for (int k2 = 0; k2 < 2; ++k2) {
                const int col = 2 * lane + k2;
                const size_t xy = (size_t)y * nx + x0 + col;
#pragma unroll
                for (int q = 0; q < 9; ++q) {
                    double sum = 0.0;
                    for (int ww = 0; ww < TW; ++ww) sum += (double)sacc[(ww * 9 + q) * 64 + col];
                    if (q < 3) a.stat_mean[q * m + xy] += sum;
                    else a.stat_rey[(q - 3) * m + xy] += sum;
                }
            }
        }
    }
    if (do_check) {
        mass_finish<32 * TW>(a, sdr);
    }
}

template <typename S, bool REG, bool FORCE, bool STATS>
static cudaError_t set_smem_attr()
{
    return cudaFuncSetAttribute(lbm_tma_kernel<S, REG, FORCE, STATS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)tma_smem_bytes<S, STATS>());
}

template <typename S, bool REG, bool FORCE>
static cudaError_t prepare3()
{
    cudaError_t e = set_smem_attr<S, REG, FORCE, false>();
    if (e == cudaSuccess) e = set_smem_attr<S, REG, FORCE, true>();
    return e;
}

cudaError_t tma_prepare()
{
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = prepare3<float, true, false>();
    if (e == cudaSuccess) e = prepare3<float, true, true>();
    if (e == cudaSuccess) e = prepare3<float, false, false>();
    if (e == cudaSuccess) e = prepare3<float, false, true>();
    if (e == cudaSuccess) e = prepare3<__half, true, false>();
    if (e == cudaSuccess) e = prepare3<__half, true, true>();
    if (e == cudaSuccess) e = prepare3<__half, false, false>();
    if (e == cudaSuccess) e = prepare3<__half, false, true>();
    return e;
}

bool tma_usable(int nx, int storage)
{
    const int esize = storage == 0 ? 4 : 2;
    return (nx * esize) % 16 == 0;
}

template <typename S, bool REG, bool FORCE>
static void launch3(const StepArgs &a, const CUtensorMap &map, dim3 grid, bool stats, cudaStream_t s)
{
    const dim3 block(32, TW);
    if (stats) lbm_tma_kernel<S, REG, FORCE, true><<<grid, block, tma_smem_bytes<S, true>(), s>>>(a, map);
    else lbm_tma_kernel<S, REG, FORCE, false><<<grid, block, tma_smem_bytes<S, false>(), s>>>(a, map);
}

cudaError_t launch_tma(const StepArgs &a, const void *tensor_map, int gx, int gy, int storage, int collision,
                       bool stats, cudaStream_t s)
{
    const dim3 grid(gx, gy);
    const bool force = a.has_force != 0;
    const CUtensorMap &m = *static_cast<const CUtensorMap *>(tensor_map);
    if (storage == 0) {
        if (collision == 0) force ? launch3<float, true, true>(a, m, grid, stats, s) : launch3<float, true, false>(a, m, grid, stats, s);
        else force ? launch3<float, false, true>(a, m, grid, stats, s) : launch3<float, false, false>(a, m, grid, stats, s);
    } else {
        if (collision == 0) force ? launch3<__half, true, true>(a, m, grid, stats, s) : launch3<__half, true, false>(a, m, grid, stats, s);
        else force ? launch3<__half, false, true>(a, m, grid, stats, s) : launch3<__half, false, false>(a, m, grid, stats, s);
    }
    return cudaGetLastError();
}

// Tensor map of one stored lattice: dims (nx, ny, nz, 19), box (ROW, 1, TW, 1).
int tma_encode(void *map_out, const void *lattice, int storage, int nx, int ny, int nz)
{
    using Encode = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    static Encode encode = nullptr;
    if (!encode) {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn)
            return 1;
        encode = reinterpret_cast<Encode>(fn);
    }
    const size_t es = storage == 0 ? 4 : 2;
    const cuuint64_t dims[4] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz, 19};
    const cuuint64_t strides[3] = {(cuuint64_t)nx * es, (cuuint64_t)nx * ny * es, (cuuint64_t)nx * ny * nz * es};
    const cuuint32_t box[4] = {(cuuint32_t)ROW, 1, (cuuint32_t)TW, 1};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    const CUresult r = encode(static_cast<CUtensorMap *>(map_out),
                              storage == 0 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 4,
                              const_cast<void *>(lattice), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? 0 : 2;
}

}  // namespace stg
