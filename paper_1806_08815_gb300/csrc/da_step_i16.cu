// da_step_i16.cu -- the step kernel for 16-bit integer couplings (int16 W, int32 fields).
#include "da_step.cuh"

namespace da {
cudaError_t launch_step_i16(const StepShape& s, const StepParams& p, bool trace, cudaStream_t st)
{
    return step_detail::launch_typed<int16_t>(s, p, trace, st);
}
}  // namespace da
