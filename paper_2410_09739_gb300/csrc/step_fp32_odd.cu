// step_fp32_odd.cu -- odd-parity step-kernel instantiations for float storage, float
// arithmetic (the even parity and the dispatch are in step_fp32.cu).
#include "step_kernel.cuh"

namespace fpc {

cudaError_t launch_step_fp32_odd(int bc, int force, int mode, const StepArgs<float>& a, const StepLaunch& cfg,
                             cudaStream_t st)
{
    return step_by_bc<float, float, true>(bc, force, mode, a, cfg, st);
}

}  // namespace fpc
