// da_step.cu -- launch-shape checks and dispatch of the step kernel
// (da_step.cuh; instantiated per coupling type in da_step_i8.cu and
// da_step_f32.cu so that the two compile in parallel).
#include "da_internal.h"

namespace da {

cudaError_t launch_step_i8(const StepShape& s, const StepParams& p, bool trace, cudaStream_t st);
cudaError_t launch_step_f32(const StepShape& s, const StepParams& p, bool trace, cudaStream_t st);
cudaError_t launch_step_i16(const StepShape& s, const StepParams& p, bool trace, cudaStream_t st);
cudaError_t launch_step_i8f(const StepShape& s, const StepParams& p, bool trace, cudaStream_t st);

bool step_shape_supported(const StepShape& s)
{
    bool vg = false;
    switch (s.G) {
    case 1: vg = s.V == 4 || s.V == 8 || s.V == 16 || s.V == 32; break;
    case 2: vg = s.V == 4 || s.V == 8 || s.V == 16 || s.V == 32; break;
    case 4: vg = s.V == 4 || s.V == 8 || s.V == 16 || s.V == 32; break;
    case 8: vg = s.V == 8 || s.V == 16 || s.V == 32; break;
    default: vg = false;
    }
    const int max_rpb = s.G == 1 ? 4 : s.G == 2 ? 2 : 1;
    return vg && s.rpb >= 1 && s.rpb <= max_rpb;
}

cudaError_t launch_step(int wtype, const StepShape& s, const StepParams& p, bool trace, cudaStream_t st)
{
    if (!step_shape_supported(s)) return cudaErrorInvalidConfiguration;
    switch (wtype) {
    case kWInt8: return launch_step_i8(s, p, trace, st);
    case kWFp32: return launch_step_f32(s, p, trace, st);
    case kWInt16: return launch_step_i16(s, p, trace, st);
    case kWInt8AsF32: return launch_step_i8f(s, p, trace, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t prepare_step(int wtype)
{
    StepParams p;
    p.R = 0;   // no blocks: the launch only sets the kernel's attributes
    for (int G = 1; G <= 8; G *= 2)
        for (int V = 4; V <= 32; V *= 2)
            for (int rpb = 1; rpb <= 4; rpb *= 2) {
                StepShape s;
                s.V = V;
                s.G = G;
                s.rpb = rpb;
                if (!step_shape_supported(s)) continue;
                for (int full = 0; full < 2; ++full) {
                    p.N = 32 * V * G - (full ? 0 : 1);
                    const cudaError_t e = launch_step(wtype, s, p, false, nullptr);
                    if (e != cudaSuccess) return e;
                }
            }
    return cudaSuccess;
}

}  // namespace da
