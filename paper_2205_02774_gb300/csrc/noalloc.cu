// stg_lattice_mass_noalloc: the FP64 mass of a stored population field,
// computed by the library's mass-reduction kernel with its scratch (block
// partials and a completion counter) in a file-scope device array instead of
// memory the library allocates.  For callers that must not allocate.
#include <mutex>
#include <string>

#include "internal.h"
#include "stg_lbm.h"

namespace {

constexpr int kMaxPartials = 1024;  // block partials the scratch holds
constexpr int kMaxDevices = 64;

struct __align__(256) NoAllocScratch {
    double partial[kMaxPartials];
    unsigned counter;
};

// Every GPU that loads the library holds one copy (8 KB) until the process
// exits.  All calls on a device share it: overlapping calls race.
static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

std::mutex g_mu;
NoAllocScratch *g_scratch_ptr[kMaxDevices] = {};

}  // namespace

namespace stg {
void record_error(const std::string &msg);
}

extern "C" int stg_lattice_mass_noalloc(const void *pops, int32_t storage, int32_t nx, int32_t ny, int32_t nz,
                                        double *mass_out, void *stream)
{
    if (!pops || !mass_out) {
        stg::record_error("stg_lattice_mass_noalloc: NULL pointer");
        return STG_ERR_INVALID;
    }
    if (storage != STG_FP32 && storage != STG_FP16_SHIFTED && storage != STG_FP16_SHIFTED_SR) {
        stg::record_error("stg_lattice_mass_noalloc: bad storage");
        return STG_ERR_INVALID;
    }
    if (nx < 1 || ny < 1 || nz < 1 || (double)nx * ny * nz > 2147483647.0) {
        stg::record_error("stg_lattice_mass_noalloc: lattice sizes must be >= 1 with at most 2^31-1 cells");
        return STG_ERR_INVALID;
    }
    if (stg::mass_grid_blocks() > kMaxPartials) {
        stg::record_error("stg_lattice_mass_noalloc: reduction grid exceeds the static scratch");
        return STG_ERR_INVALID;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        stg::record_error(std::string("stg_lattice_mass_noalloc: ") + cudaGetErrorString(e));
        return STG_ERR_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        stg::record_error("stg_lattice_mass_noalloc: device index beyond the supported 64");
        return STG_ERR_INVALID;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(s, &cap);
    if (e != cudaSuccess) {
        stg::record_error(std::string("stg_lattice_mass_noalloc: ") + cudaGetErrorString(e));
        return STG_ERR_CUDA;
    }
    NoAllocScratch *scratch = nullptr;
    {
        // set-up per device (with that device current): the device address of
        // the scratch array (host code may not use its name directly).  Looked
        // up on the first call and again on every call outside stream capture,
        // so that an address invalidated by a device reset is replaced.
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_scratch_ptr[dev] || cap == cudaStreamCaptureStatusNone) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess) {
                stg::record_error(std::string("stg_lattice_mass_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
                return STG_ERR_CUDA;
            }
            g_scratch_ptr[dev] = static_cast<NoAllocScratch *>(p);
        }
        scratch = g_scratch_ptr[dev];
    }
    // the completion counter must start at zero (the kernel leaves it at zero)
    e = cudaMemsetAsync(&scratch->counter, 0, sizeof(unsigned), s);
    if (e == cudaSuccess) {
        stg::MassArgs m{};
        m.src = pops;
        m.P = (unsigned)((size_t)nx * ny * nz);
        m.storage = storage;
        m.partial = scratch->partial;
        m.counter = &scratch->counter;
        m.out = mass_out;
        e = stg::launch_mass(m, s);
    }
    if (e != cudaSuccess) {
        stg::record_error(std::string("stg_lattice_mass_noalloc: ") + cudaGetErrorString(e));
        return STG_ERR_CUDA;
    }
    return STG_OK;
}
