// da_step_i8.cu -- the step kernel for integer couplings (int8 W, int32 fields).
#include "da_step.cuh"

namespace da {
cudaError_t launch_step_i8(const StepShape& s, const StepParams& p, bool trace, cudaStream_t st)
{
    return step_detail::launch_typed<int8_t>(s, p, trace, st);
}
}  // namespace da
