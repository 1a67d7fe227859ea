// step_kernel.cuh -- fused collide-and-stream kernel of one box (AA pattern,
// see cell.cuh): one thread per cell, one launch per time step.  MINB is the
// minimum resident blocks per SM handed to __launch_bounds__, i.e. the
// register cap (2: ~120, 3: ~80, 4: 64 registers); the autotuner times the
// variants and keeps the fastest.  BC is one of the BC_* boundary kinds.
#pragma once
#include "cell.cuh"
#include "internal.h"
#include "stage.cuh"

namespace fpc {

template <typename S, typename R, bool ODD, int BC, bool FORCE, int MODE, int MINB>
__global__ void __launch_bounds__(256, MINB) k_step(const StepArgs<R> a)
{
    unsigned cell = blockIdx.x * blockDim.x + threadIdx.x;
    bool active = true;
    if (cell >= a.ncells) {
        // the learned closure is warp-collective: tail lanes stay, on a valid cell, without writing
        if (!learned_mode(MODE)) return;
        active = false;
        cell = a.ncells - 1;
    }
    CellGeom G;
    G.stride = a.stride;
    G.nx = a.nx;
    G.ny = a.ny;
    G.nz = a.nz;
    G.div_nx = a.div_nx;
    G.div_nxny = a.div_nxny;
    const Rates<R>& rt = a.rates;
    update_cell<S, R, ODD, BC, FORCE, MODE>(static_cast<S*>(a.buf), G, cell, rt, a.Fx, a.Fy, a.Fz, rt.om[4],
                                            rt.om[5], rt.om[6], rt.om[8], rt.om[9], a.closure, a.flag, active,
                                            a.lid6x, a.lid6z, a.smag);
}

// ---------------------------------------------------------------------------
// Software-pipelined variant: a persistent grid walks tiles of blockDim cells;
// while a thread collides its cell of tile t, the 27 loads of its cell of the
// next tile are already in flight as cp.async copies into the thread's own
// column of a two-stage shared-memory buffer [2][27][blockDim].  Bytes in
// flight no longer cost registers, so the load and compute phases of a warp
// overlap.  Each thread reads back only what it copied itself, so a per-thread
// cp.async.wait_group is the only synchronisation.  Storage of 4 or 8 bytes.
// ---------------------------------------------------------------------------

template <int BYTES>
__device__ __forceinline__ void cp_async(void* smem, const void* gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(s), "l"(gmem), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

template <typename S, typename R, bool ODD, int BC, bool FORCE, int MODE, int MINB>
__global__ void __launch_bounds__(128, MINB) k_step_pipe(const StepArgs<R> a, unsigned ntiles)
{
    static_assert(sizeof(S) == 4 || sizeof(S) == 8, "cp.async moves 4, 8 or 16 bytes");
    static_assert(BC == BC_PERIODIC || BC == BC_WALLS_Y, "periodic or channel boxes only");
    static_assert(plain_mode(MODE), "FP and MCM modes only");
    extern __shared__ __align__(16) unsigned char fpc_smem[];
    S* sm = reinterpret_cast<S*>(fpc_smem);
    const unsigned T = blockDim.x, tid = threadIdx.x;
    CellGeom G;
    G.stride = a.stride;
    G.nx = a.nx;
    G.ny = a.ny;
    G.nz = a.nz;
    G.div_nx = a.div_nx;
    G.div_nxny = a.div_nxny;
    S* __restrict__ buf = static_cast<S*>(a.buf);
    const unsigned stride = a.stride;
    const Rates<R>& rt = a.rates;

    auto issue = [&](unsigned tile, int stage) {
        const unsigned cell = tile * T + tid;
        if (tile < ntiles && cell < a.ncells) {
            Nbr n;
            if (ODD) n = make_nbr<BC>(G, cell);
            S* dst = sm + (size_t)stage * 27 * T + tid;
#pragma unroll
            for (int s = 0; s < 27; ++s)
                cp_async<sizeof(S)>(dst + s * T, load_ptr<S, ODD, BC>(buf, s, n, stride, cell));
        }
        cp_async_commit();
    };

    int stage = 0;
    unsigned t = blockIdx.x;
    issue(t, 0);
    for (; t < ntiles; t += gridDim.x) {
        issue(t + gridDim.x, stage ^ 1);
        cp_async_wait<1>();
        const unsigned cell = t * T + tid;
        if (cell < a.ncells) {
            R g[27];
            const S* src = sm + (size_t)stage * 27 * T + tid;
#pragma unroll
            for (int s = 0; s < 27; ++s) g[s] = Store<S>::ld(src + s * T);
            const bool ok = collide_cell<R, FORCE, MODE>(g, rt, a.Fx, a.Fy, a.Fz, rt.om[4], rt.om[5], rt.om[6],
                                                         rt.om[8], rt.om[9], a.closure);
            if (!ok) atomicOr(a.flag, 1);
            Nbr n;
            if (ODD) n = make_nbr<BC>(G, cell);
#pragma unroll
            for (int s = 0; s < 27; ++s) Store<S>::st(store_ptr<S, ODD, BC>(buf, s, n, stride, cell), g[s]);
        }
        stage ^= 1;
    }
    cp_async_wait<0>();
}

template <typename S, typename R, bool ODD, int BC, bool FORCE, int MODE, int MINB>
cudaError_t step_go_pipe(const StepArgs<R>& a, cudaStream_t st)
{
    constexpr int T = 128;
    const size_t smem = 2ull * 27 * T * sizeof(S);
    auto kern = k_step_pipe<S, R, ODD, BC, FORCE, MODE, 2 * MINB>;
    static int per_sm = 0, sms = 0;  // benign race: every thread computes the same values
    if (per_sm == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int n = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, T, smem) != cudaSuccess || n < 1) n = 1;
        per_sm = n;
    }
    const unsigned ntiles = (a.ncells + T - 1) / T;
    unsigned grid = (unsigned)(per_sm * sms);
    if (grid > ntiles) grid = ntiles;
    kern<<<grid, T, smem, st>>>(a, ntiles);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Paired variant: each thread updates two cells with the packed fp32
// arithmetic of pair.cuh (one instruction per operation for both cells).  The
// odd step pairs cells c and c + half, with per-cell loads and stores as
// coalesced as in k_step; the even step pairs neighbouring cells 2c, 2c + 1,
// whose values of a slot are adjacent, with one vector access per slot.  Each
// cell still reads and writes only its own AA addresses.
// ---------------------------------------------------------------------------

template <typename S, bool ODD, int BC, bool FORCE, int MODE, int MINB, bool ADJ>
__global__ void __launch_bounds__(128, MINB) k_step_pair(const StepArgs<f2> a, unsigned half)
{
    unsigned c1 = blockIdx.x * blockDim.x + threadIdx.x;
    bool active = true;
    if (c1 >= half) {
        // the learned closure is warp-collective: tail lanes stay, on a valid pair, without writing
        if (!learned_mode(MODE)) return;
        active = false;
        c1 = half - 1;
    }
    CellGeom G;
    G.stride = a.stride;
    G.nx = a.nx;
    G.ny = a.ny;
    G.nz = a.nz;
    G.div_nx = a.div_nx;
    G.div_nxny = a.div_nxny;
    const Rates<f2>& rt = a.rates;
    if constexpr (ODD && ADJ)  // neighbouring cells 2 c1, 2 c1 + 1 with a shared neighbour table
        update_pair_odd_adj<S, BC, FORCE, MODE>(static_cast<S*>(a.buf), G, c1, rt, a.Fx, a.Fy, a.Fz, rt.om[4],
                                                rt.om[5], rt.om[6], rt.om[8], rt.om[9], a.flag, a.lid6x, a.lid6z,
                                                a.closure, active);
    else if constexpr (ODD)  // cells c1 and c1 + half
        update_pair<S, ODD, BC, FORCE, MODE>(static_cast<S*>(a.buf), G, c1, half, a.ncells, rt, a.Fx, a.Fy, a.Fz,
                                             rt.om[4], rt.om[5], rt.om[6], rt.om[8], rt.om[9], a.flag, a.lid6x,
                                             a.lid6z, a.closure, active);
    else  // neighbouring cells 2 c1 and 2 c1 + 1, vector loads and stores
        update_pair_even<S, BC, FORCE, MODE>(static_cast<S*>(a.buf), G, c1, a.ncells, rt, a.Fx, a.Fy, a.Fz,
                                             rt.om[4], rt.om[5], rt.om[6], rt.om[8], rt.om[9], a.flag, a.lid6x,
                                             a.lid6z, a.closure, active);
}

// The launch arguments with every scalar duplicated into both lanes.
inline StepArgs<f2> pair_args(const StepArgs<float>& a)
{
    StepArgs<f2> p;
    p.buf = a.buf;
    p.stride = a.stride;
    p.ncells = a.ncells;
    p.nx = a.nx;
    p.ny = a.ny;
    p.nz = a.nz;
    p.div_nx = a.div_nx;
    p.div_nxny = a.div_nxny;
    p.Fx = f2(a.Fx, a.Fx);
    p.Fy = f2(a.Fy, a.Fy);
    p.Fz = f2(a.Fz, a.Fz);
    p.lid6x = f2(a.lid6x, a.lid6x);
    p.lid6z = f2(a.lid6z, a.lid6z);
    for (int j = 0; j < 27; ++j) {
        p.rates.om[j] = f2(a.rates.om[j], a.rates.om[j]);
        p.rates.keep[j] = f2(a.rates.keep[j], a.rates.keep[j]);
        p.rates.src[j] = f2(a.rates.src[j], a.rates.src[j]);
    }
    p.flag = a.flag;
    p.closure = a.closure;
    p.smag = nullptr;
    return p;
}

template <typename S, bool ODD, int BC, bool FORCE, int MODE, int MINB>
cudaError_t step_go_pair(const StepArgs<float>& a, cudaStream_t st)
{
    const unsigned half = (a.ncells + 1) / 2;
    // the even step without force or moving wall (vector accesses, no neighbour table, no source
    // terms) fits in 96 registers without spilling: one block more per SM.  The learned modes run
    // four blocks (128 registers, about 90 bytes of spills: 2.5 % faster than three blocks at 168)
    constexpr bool LID = BC == BC_WALLS_Y_LID || BC == BC_BOX_LID;
    constexpr int BLOCKS = learned_mode(MODE) ? 4 : (ODD || FORCE || LID) ? 2 * MINB : 2 * MINB + 1;
    const unsigned grid = (half + 127) / 128;
    // neighbouring cells on the odd step: nx even (rows hold whole pairs), no symmetry plane; the
    // closed box only with fp32 storage (its per-cell x-wall tests spill with 16-bit unpacking)
    constexpr bool ADJ_OK = ODD && BC != BC_HALF_CHANNEL && (BC != BC_BOX_LID || sizeof(S) == 4);
    if (ADJ_OK && (a.nx & 1) == 0)
        k_step_pair<S, ODD, BC, FORCE, MODE, BLOCKS, ADJ_OK><<<grid, 128, 0, st>>>(pair_args(a), half);
    else
        k_step_pair<S, ODD, BC, FORCE, MODE, BLOCKS, false><<<grid, 128, 0, st>>>(pair_args(a), half);
    return cudaGetLastError();
}

template <typename S, typename R, bool ODD, int BC, bool FORCE, int MODE, int MINB>
cudaError_t step_go(const StepArgs<R>& a, const StepLaunch& cfg, cudaStream_t st)
{
    // paired variant: fp32 arithmetic, FP and MCM modes, every boundary kind, one register cap
    // (4 blocks of 128 threads: 128 registers hold two cells without spilling)
    // the learned modes too, on periodic boxes and channels with resting walls (the paired MLP
    // calls are warp-collective like the one-cell ones)
    constexpr bool pair_learned = learned_mode(MODE) && (BC == BC_PERIODIC || BC == BC_WALLS_Y);
    if constexpr (sizeof(R) == 4 && pair_learned && MINB == 2) {
        if (cfg.pipe == 2) return step_go_pair<S, ODD, BC, FORCE, MODE, MINB>(a, st);
    }
    if constexpr (sizeof(R) == 4 && plain_mode(MODE) && MINB == 2) {
        if (cfg.pipe == 2) return step_go_pair<S, ODD, BC, FORCE, MODE, MINB>(a, st);
        // row-staged variant (stage.cuh): periodic boxes and channels
        if constexpr (BC == BC_PERIODIC || BC == BC_WALLS_Y) {
            if (cfg.pipe == 3) return step_go_stage<S, ODD, BC, FORCE, MODE>(a, cfg.stages, st);
        }
    }
    // the pipelined variant retires tail lanes early, so it never runs the warp-collective
    // learned mode; it exists for the FP and MCM modes of periodic and channel boxes
    if constexpr (sizeof(S) >= 4 && plain_mode(MODE) && BC <= BC_WALLS_Y) {
        if (cfg.pipe == 1) return step_go_pipe<S, R, ODD, BC, FORCE, MODE, MINB>(a, st);
    }
    const int block = cfg.block > 0 ? cfg.block : 256;
    const unsigned grid = (a.ncells + block - 1) / block;
    k_step<S, R, ODD, BC, FORCE, MODE, MINB><<<grid, block, 0, st>>>(a);
    return cudaGetLastError();
}

// Register-cap variants exist for fp32 arithmetic: 2, 3, 4 for the FP and EQ
// modes (every boundary kind); 1 (no cap) and 2 (128 registers) for the
// learned mode on boxes with resting walls, whose tensor-core MLP keeps the
// cell's state live.  fp64 and the Smagorinsky mode have one variant each.
template <typename S, typename R, bool ODD, int BC, bool FORCE, int MODE>
cudaError_t step_by_minb(const StepArgs<R>& a, const StepLaunch& cfg, cudaStream_t st)
{
    constexpr bool fp32_capped = sizeof(R) == 4 && plain_mode(MODE);
    constexpr bool fp32_learned = sizeof(R) == 4 && learned_mode(MODE) && bc_fixed(BC);
    if constexpr (fp32_capped) {
        if (cfg.minb == 3) return step_go<S, R, ODD, BC, FORCE, MODE, 3>(a, cfg, st);
        if (cfg.minb == 4) return step_go<S, R, ODD, BC, FORCE, MODE, 4>(a, cfg, st);
        return step_go<S, R, ODD, BC, FORCE, MODE, 2>(a, cfg, st);
    } else if constexpr (fp32_learned) {
        if (cfg.minb == 2) return step_go<S, R, ODD, BC, FORCE, MODE, 2>(a, cfg, st);
        return step_go<S, R, ODD, BC, FORCE, MODE, 1>(a, cfg, st);
    } else {
        return step_go<S, R, ODD, BC, FORCE, MODE, 1>(a, cfg, st);
    }
}

template <typename S, typename R, bool ODD, int BC, bool FORCE>
cudaError_t step_by_mode(int mode, const StepArgs<R>& a, const StepLaunch& cfg, cudaStream_t st)
{
    switch (mode) {
        case MODE_FP: return step_by_minb<S, R, ODD, BC, FORCE, MODE_FP>(a, cfg, st);
        case MODE_EQ: return step_by_minb<S, R, ODD, BC, FORCE, MODE_EQ>(a, cfg, st);
        case MODE_FP_R1: return step_by_minb<S, R, ODD, BC, FORCE, MODE_FP_R1>(a, cfg, st);  // unit rates, orders >= 3
        case MODE_EQ_R1: return step_by_minb<S, R, ODD, BC, FORCE, MODE_EQ_R1>(a, cfg, st);
        case MODE_LEARNED:  // periodic and channel boxes (the closure's training data come from them)
            if constexpr (BC == BC_PERIODIC || BC == BC_WALLS_Y)
                return step_by_minb<S, R, ODD, BC, FORCE, MODE_LEARNED>(a, cfg, st);
            break;
        case MODE_LEARNED_R1:  // the same with unit rates of orders 3-6
            if constexpr (BC == BC_PERIODIC || BC == BC_WALLS_Y)
                return step_by_minb<S, R, ODD, BC, FORCE, MODE_LEARNED_R1>(a, cfg, st);
            break;
        case MODE_SMAG:  // resting walls
            if constexpr (bc_fixed(BC)) return step_by_minb<S, R, ODD, BC, FORCE, MODE_SMAG>(a, cfg, st);
            break;
    }
    return cudaErrorInvalidValue;
}

template <typename S, typename R, bool ODD, int BC>
cudaError_t step_by_force(int force, int mode, const StepArgs<R>& a, const StepLaunch& cfg, cudaStream_t st)
{
    return force ? step_by_mode<S, R, ODD, BC, true>(mode, a, cfg, st)
                 : step_by_mode<S, R, ODD, BC, false>(mode, a, cfg, st);
}

template <typename S, typename R, bool ODD>
cudaError_t step_by_bc(int bc, int force, int mode, const StepArgs<R>& a, const StepLaunch& cfg, cudaStream_t st)
{
    switch (bc) {
        case BC_PERIODIC: return step_by_force<S, R, ODD, BC_PERIODIC>(force, mode, a, cfg, st);
        case BC_WALLS_Y: return step_by_force<S, R, ODD, BC_WALLS_Y>(force, mode, a, cfg, st);
        case BC_WALLS_Y_LID: return step_by_force<S, R, ODD, BC_WALLS_Y_LID>(force, mode, a, cfg, st);
        case BC_BOX_LID: return step_by_force<S, R, ODD, BC_BOX_LID>(force, mode, a, cfg, st);
        case BC_HALF_CHANNEL: return step_by_force<S, R, ODD, BC_HALF_CHANNEL>(force, mode, a, cfg, st);
    }
    return cudaErrorInvalidValue;
}

template <typename S, typename R>
cudaError_t step_dispatch(int odd, int bc, int force, int mode, const StepArgs<R>& a, const StepLaunch& cfg,
                          cudaStream_t st)
{
    return odd ? step_by_bc<S, R, true>(bc, force, mode, a, cfg, st)
               : step_by_bc<S, R, false>(bc, force, mode, a, cfg, st);
}

}  // namespace fpc
