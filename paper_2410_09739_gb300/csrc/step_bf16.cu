// step_bf16.cu -- step-kernel instantiations for __nv_bfloat16 storage, float arithmetic: the
// even parity here, the odd parity in step_bf16_odd.cu (two translation units
// compile in parallel).
#include "step_kernel.cuh"

namespace fpc {

cudaError_t launch_step_bf16_odd(int bc, int force, int mode, const StepArgs<float>& a, const StepLaunch& cfg,
                             cudaStream_t st);

cudaError_t launch_step_bf16(int odd, int bc, int force, int mode, const StepArgs<float>& a, const StepLaunch& cfg,
                          cudaStream_t st)
{
    if (odd) return launch_step_bf16_odd(bc, force, mode, a, cfg, st);
    return step_by_bc<__nv_bfloat16, float, false>(bc, force, mode, a, cfg, st);
}

}  // namespace fpc
