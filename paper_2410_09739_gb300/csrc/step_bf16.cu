// step_bf16.cu -- step-kernel instantiations for __nv_bfloat16 storage, float arithmetic.
#include "step_kernel.cuh"

namespace fpc {

cudaError_t launch_step_bf16(int odd, int bc, int force, int mode, const StepArgs<float>& a, const StepLaunch& cfg,
                          cudaStream_t st)
{
    return step_dispatch<__nv_bfloat16, float>(odd, bc, force, mode, a, cfg, st);
}

}  // namespace fpc
