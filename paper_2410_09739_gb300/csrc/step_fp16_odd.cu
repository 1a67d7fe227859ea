// step_fp16_odd.cu -- odd-parity step-kernel instantiations for __half storage, float
// arithmetic (the even parity and the dispatch are in step_fp16.cu).
#include "step_kernel.cuh"

namespace fpc {

cudaError_t launch_step_fp16_odd(int bc, int force, int mode, const StepArgs<float>& a, const StepLaunch& cfg,
                             cudaStream_t st)
{
    return step_by_bc<__half, float, true>(bc, force, mode, a, cfg, st);
}

}  // namespace fpc
