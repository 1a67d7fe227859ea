// step_fp64.cu -- step-kernel instantiations for double storage, double arithmetic.
#include "step_kernel.cuh"

namespace fpc {

cudaError_t launch_step_fp64(int odd, int bc, int force, int mode, const StepArgs<double>& a, const StepLaunch& cfg,
                          cudaStream_t st)
{
    return step_dispatch<double, double>(odd, bc, force, mode, a, cfg, st);
}

}  // namespace fpc
