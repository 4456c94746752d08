// da_step_i8f.cu -- the step kernel for DA_INT8 contexts: the int8 couplings
// held as exact fp32 (f32e in da_step_common.cuh), int64 energies.
#include "da_step.cuh"

namespace da {
cudaError_t launch_step_i8f(const StepShape& s, const StepParams& p, bool trace, cudaStream_t st)
{
    return step_detail::launch_typed<step_detail::f32e>(s, p, trace, st);
}
}  // namespace da
