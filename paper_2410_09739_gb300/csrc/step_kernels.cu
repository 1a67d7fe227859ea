// step_kernels.cu -- fused collide-and-stream kernel of one box (AA pattern,
// see cell.cuh): one thread per cell, one launch per time step.
#include "cell.cuh"
#include "internal.h"

namespace fpc {

template <typename S, typename R, bool ODD, bool WALLS, bool FORCE, int MODE>
__global__ void __launch_bounds__(256) k_step(const StepArgs<R> a)
{
    const unsigned cell = blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= a.ncells) return;
    CellGeom G;
    G.stride = a.stride;
    G.nx = a.nx;
    G.ny = a.ny;
    G.nz = a.nz;
    G.div_nx = a.div_nx;
    G.div_nxny = a.div_nxny;
    const Rates<R>& rt = a.rates;
    update_cell<S, R, ODD, WALLS, FORCE, MODE>(static_cast<S*>(a.buf), G, cell, rt, a.Fx, a.Fy, a.Fz, rt.om[4],
                                               rt.om[5], rt.om[6], rt.om[8], rt.om[9], a.closure, a.flag);
}

template <typename S, typename R, bool ODD, bool WALLS, bool FORCE, int MODE>
static cudaError_t go(const StepArgs<R>& a, const StepLaunch& cfg, cudaStream_t st)
{
    const int block = cfg.block > 0 ? cfg.block : 256;
    const unsigned grid = (a.ncells + block - 1) / block;
    k_step<S, R, ODD, WALLS, FORCE, MODE><<<grid, block, 0, st>>>(a);
    return cudaGetLastError();
}

template <typename S, typename R, bool ODD, bool WALLS, bool FORCE>
static cudaError_t by_mode(int mode, const StepArgs<R>& a, const StepLaunch& cfg, cudaStream_t st)
{
    switch (mode) {
        case MODE_FP: return go<S, R, ODD, WALLS, FORCE, MODE_FP>(a, cfg, st);
        case MODE_EQ: return go<S, R, ODD, WALLS, FORCE, MODE_EQ>(a, cfg, st);
        case MODE_LEARNED: return go<S, R, ODD, WALLS, FORCE, MODE_LEARNED>(a, cfg, st);
    }
    return cudaErrorInvalidValue;
}

template <typename S, typename R, bool ODD, bool WALLS>
static cudaError_t by_force(int force, int mode, const StepArgs<R>& a, const StepLaunch& cfg, cudaStream_t st)
{
    return force ? by_mode<S, R, ODD, WALLS, true>(mode, a, cfg, st)
                 : by_mode<S, R, ODD, WALLS, false>(mode, a, cfg, st);
}

template <typename S, typename R>
static cudaError_t by_geom(int odd, int walls, int force, int mode, const StepArgs<R>& a, const StepLaunch& cfg,
                           cudaStream_t st)
{
    if (odd)
        return walls ? by_force<S, R, true, true>(force, mode, a, cfg, st)
                     : by_force<S, R, true, false>(force, mode, a, cfg, st);
    return walls ? by_force<S, R, false, true>(force, mode, a, cfg, st)
                 : by_force<S, R, false, false>(force, mode, a, cfg, st);
}

cudaError_t launch_step(int precision, int odd, int walls, int force, int mode, const StepArgs<double>& a64,
                        const StepArgs<float>& a32, const StepLaunch& cfg, cudaStream_t st)
{
    switch (precision) {
        case P_FP64: return by_geom<double, double>(odd, walls, force, mode, a64, cfg, st);
        case P_FP32: return by_geom<float, float>(odd, walls, force, mode, a32, cfg, st);
        case P_FP16: return by_geom<__half, float>(odd, walls, force, mode, a32, cfg, st);
        case P_BF16: return by_geom<__nv_bfloat16, float>(odd, walls, force, mode, a32, cfg, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace fpc
