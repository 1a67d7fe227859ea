// step_kernels.cu -- precision dispatch of the single-box step kernel (the
// instantiations live in step_fp64.cu, step_fp32.cu, step_fp16.cu, step_bf16.cu).
#include "internal.h"

namespace fpc {

cudaError_t launch_step_fp64(int, int, int, int, const StepArgs<double>&, const StepLaunch&, cudaStream_t);
cudaError_t launch_step_fp32(int, int, int, int, const StepArgs<float>&, const StepLaunch&, cudaStream_t);
cudaError_t launch_step_fp16(int, int, int, int, const StepArgs<float>&, const StepLaunch&, cudaStream_t);
cudaError_t launch_step_bf16(int, int, int, int, const StepArgs<float>&, const StepLaunch&, cudaStream_t);

cudaError_t launch_step(int precision, int odd, int bc, int force, int mode, const StepArgs<double>& a64,
                        const StepArgs<float>& a32, const StepLaunch& cfg, cudaStream_t st)
{
    switch (precision) {
        case P_FP64: return launch_step_fp64(odd, bc, force, mode, a64, cfg, st);
        case P_FP32: return launch_step_fp32(odd, bc, force, mode, a32, cfg, st);
        case P_FP16: return launch_step_fp16(odd, bc, force, mode, a32, cfg, st);
        case P_BF16: return launch_step_bf16(odd, bc, force, mode, a32, cfg, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace fpc
