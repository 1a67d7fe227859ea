// step_bf16_odd.cu -- odd-parity step-kernel instantiations for __nv_bfloat16 storage, float
// arithmetic (the even parity and the dispatch are in step_bf16.cu).
#include "step_kernel.cuh"

namespace fpc {

cudaError_t launch_step_bf16_odd(int bc, int force, int mode, const StepArgs<float>& a, const StepLaunch& cfg,
                             cudaStream_t st)
{
    return step_by_bc<__nv_bfloat16, float, true>(bc, force, mode, a, cfg, st);
}

}  // namespace fpc
