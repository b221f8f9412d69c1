// Step kernels of FP32 storage with the plain BGK collision (one of four
// instantiation units of step_kernel.cuh, compiled in parallel).
#include "step_kernel.cuh"

namespace stg {

bool launch_f32_bgk(const StepArgs &a, bool stats, cudaStream_t s, cudaStream_t side)
{
    return launch_typed<float, false>(a, stats, s, side);
}

}  // namespace stg
