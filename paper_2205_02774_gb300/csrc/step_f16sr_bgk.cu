// Step kernels of shifted binary16 storage written by stochastic rounding,
// with the plain BGK collision (one of the instantiation units of
// step_kernel.cuh, compiled in parallel).
#include "step_kernel.cuh"

namespace stg {

bool launch_f16sr_bgk(const StepArgs &a, bool stats, cudaStream_t s, cudaStream_t side)
{
    return launch_typed<__half, false, true>(a, stats, s, side);
}

}  // namespace stg
