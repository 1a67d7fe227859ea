// step_fp16.cu -- step-kernel instantiations for __half storage, float arithmetic.
#include "step_kernel.cuh"

namespace fpc {

cudaError_t launch_step_fp16(int odd, int bc, int force, int mode, const StepArgs<float>& a, const StepLaunch& cfg,
                          cudaStream_t st)
{
    return step_dispatch<__half, float>(odd, bc, force, mode, a, cfg, st);
}

}  // namespace fpc
