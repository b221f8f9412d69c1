// Interior columns of the fused step with the pull staged by the TMA engine.
//
// A block is TW warps on one 64-wide x chunk at one y; warp w walks the
// z-planes w, w + TW, ...  For each plane it needs, per population i, the row
// (y - c_iy, z - c_iz) of plane i over x in [x0 - 1, x0 + 64].  Lane 0 of the
// warp copies those 19 rows (x0 - 8 .. x0 + 72, 16-byte aligned) into a
// shared-memory stage with cp.async.bulk, completing on an mbarrier; the warp
// keeps D stages in flight, so the memory system always holds the next planes'
// bytes while the current plane is collided.  Lane l then takes cells
// (x0 + 2l, x0 + 2l + 1) from shared memory (the x +-1 shifts are plain
// shared-memory offsets), collides both (lbm_cell.cuh) and stores them as one
// aligned pair.  Every mbarrier wait is bounded: on expiry the warp records an
// error bit in StepCtl::err, drains its own copies (also bounded) and stops.
#include <cstdint>

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
constexpr uint32_t stage_bytes() { return (uint32_t)(Q * ROW * sizeof(S)); }

template <typename S, bool STATS>
constexpr size_t tma_smem_bytes()
{
    return (size_t)TW * TmaDepth<S>::D * stage_bytes<S>() + (size_t)TW * TmaDepth<S>::D * 8 +
           (STATS ? (size_t)TW * 9 * 64 * sizeof(float) : 0);
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
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
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

template <typename S, bool REG, bool FORCE, bool STATS>
__global__ void __launch_bounds__(32 * TW, 6) lbm_tma_kernel(const StepArgs a)
{
    constexpr int D = TmaDepth<S>::D;
    constexpr uint32_t SB = stage_bytes<S>();
    using ST = Staged<S>;
    using raw = typename ST::raw;
    extern __shared__ __align__(128) unsigned char smem[];
    const int w = threadIdx.y, lane = threadIdx.x;
    unsigned char *wbase = smem + (size_t)w * D * SB;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + (size_t)TW * D * SB) + w * D;
    float *sacc = reinterpret_cast<float *>(smem + (size_t)TW * D * SB + (size_t)TW * D * 8);  // [TW][9][64]

    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int c = a.il / 2 + blockIdx.x;
    const int y = blockIdx.y + 1;
    const int x0 = 64 * c;
    const int count = (nz - w + TW - 1) / TW;  // planes z = w + k TW
    const long long t = a.ctl->t[a.parity];
    const bool do_check = a.check_every > 0 && ((t + 1) % a.check_every) == 0;
    const float tau0 = a.tau0, kq = a.kq;
    const float Fx = a.Fx, Fy = a.Fy, Fz = a.Fz;
    const S *sbase = static_cast<const S *>(a.src);
    S *dbase = static_cast<S *>(a.dst);

    if (lane == 0) {
        for (int s = 0; s < D; ++s) mbar_init(smem_u32(bars + s), 1);
        fence_mbar_init();
    }
    if (STATS) {
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            sacc[(w * 9 + q) * 64 + 2 * lane] = 0.f;
            sacc[(w * 9 + q) * 64 + 2 * lane + 1] = 0.f;
        }
    }
    __syncwarp();

    // lane 0: copy the 19 source rows of plane k into stage s
    auto issue = [&](int k, int s) {
        const int z = w + k * TW;
        const uint32_t bar = smem_u32(bars + s);
        const uint32_t dst = smem_u32(wbase + (size_t)s * SB);
        mbar_arrive_expect_tx(bar, SB);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            int zs = z - cz_of(i);
            zs = zs < 0 ? zs + nz : (zs >= nz ? zs - nz : zs);
            const size_t off = (size_t)i * a.P + ((size_t)zs * ny + (y - cy_of(i))) * nx + (x0 - 8);
            bulk_g2s(dst + (uint32_t)(i * ROW * sizeof(S)), sbase + off, ROW * (uint32_t)sizeof(S), bar);
        }
    };
    if (lane == 0)
        for (int k = 0; k < D && k < count; ++k) issue(k, k);

    float sdr = 0.f;
    int k = 0;
    bool failed = false;
    for (; k < count; ++k) {
        const int s = k % D;
        if (!mbar_wait_bounded(smem_u32(bars + s), (uint32_t)((k / D) & 1))) {
            failed = true;
            break;
        }
        const S *stg = reinterpret_cast<const S *>(wbase + (size_t)s * SB);
        const int b = 8 + 2 * lane;
        raw v[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) v[i] = ST::at(stg + i * ROW, b, cx_of(i));
        __syncwarp();
        if (lane == 0 && k + D < count) {
            fence_proxy_async();  // our reads of stage s precede the copy that overwrites it
            issue(k + D, s);
        }
        const int z = w + k * TW;
        unsigned Pv;  // opaque copy: keeps the 19 store-plane offsets out of registers
        asm volatile("mov.u32 %0, %1;" : "=r"(Pv) : "r"(a.P));
        const unsigned here = ((unsigned)z * ny + y) * nx + x0 + 2 * lane;
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            float g[Q];
#pragma unroll
            for (int i = 0; i < Q; ++i) g[i] = half ? ST::hi(v[i]) : ST::lo(v[i]);
            float rho, ux, uy, uz;
            collide<REG, FORCE>(g, tau0, kq, Fx, Fy, Fz, rho, ux, uy, uz);
            if (half == 0) {
#pragma unroll
                for (int i = 0; i < Q; ++i) v[i] = ST::put_lo(v[i], g[i]);
            } else {
#pragma unroll
                for (int i = 0; i < Q; ++i) ST::st(dbase + (i * Pv + here), v[i], g[i]);
            }
            if (STATS) {
                float *sp = sacc + (w * 9) * 64 + 2 * lane + half;
                sp[0 * 64] += ux; sp[1 * 64] += uy; sp[2 * 64] += uz;
                sp[3 * 64] += ux * ux; sp[4 * 64] += uy * uy; sp[5 * 64] += uz * uz;
                sp[6 * 64] += ux * uy; sp[7 * 64] += ux * uz; sp[8 * 64] += uy * uz;
            }
            sdr += rho - 1.0f;
        }
    }
    if (failed) {
        if (lane == 0) atomicOr(&a.ctl->err, 1ull);
        // drain the copies this warp still has in flight (bounded as well)
        for (int j = k; j < count && j < k + D; ++j) mbar_wait_bounded(smem_u32(bars + (j % D)), (uint32_t)((j / D) & 1));
    }
    __syncwarp();
    if (lane == 0)
        for (int s = 0; s < D; ++s) mbar_inval(smem_u32(bars + s));

    if (STATS) {
        __syncthreads();
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
        const int nxc = (nx + 31) / 32;
        mass_finish<32 * TW>(a, sdr, y * nxc + 2 * c, y * nxc + 2 * c + 1);
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
static void launch3(const StepArgs &a, dim3 grid, bool stats, cudaStream_t s)
{
    const dim3 block(32, TW);
    if (stats) lbm_tma_kernel<S, REG, FORCE, true><<<grid, block, tma_smem_bytes<S, true>(), s>>>(a);
    else lbm_tma_kernel<S, REG, FORCE, false><<<grid, block, tma_smem_bytes<S, false>(), s>>>(a);
}

cudaError_t launch_tma(const StepArgs &a, int gx, int gy, int storage, int collision, bool stats, cudaStream_t s)
{
    const dim3 grid(gx, gy);
    const bool force = a.has_force != 0;
    if (storage == 0) {
        if (collision == 0) force ? launch3<float, true, true>(a, grid, stats, s) : launch3<float, true, false>(a, grid, stats, s);
        else force ? launch3<float, false, true>(a, grid, stats, s) : launch3<float, false, false>(a, grid, stats, s);
    } else {
        if (collision == 0) force ? launch3<__half, true, true>(a, grid, stats, s) : launch3<__half, true, false>(a, grid, stats, s);
        else force ? launch3<__half, false, true>(a, grid, stats, s) : launch3<__half, false, false>(a, grid, stats, s);
    }
    return cudaGetLastError();
}

}  // namespace stg
