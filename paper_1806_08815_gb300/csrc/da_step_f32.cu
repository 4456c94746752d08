// da_step_f32.cu -- the step kernel for real couplings (fp32 W and fields).
#include "da_step.cuh"

namespace da {
cudaError_t launch_step_f32(const StepShape& s, const StepParams& p, bool trace, cudaStream_t st)
{
    return step_detail::launch_typed<float>(s, p, trace, st);
}
}  // namespace da
