// closure.cuh -- per-cell inference of the learned shear-rate correction.
//
// MLP 9 -> 64 -> 64 -> 1 with tanh hidden layers, evaluated for the 32 cells of
// a warp at once on the tensor cores: both hidden layers are
// mma.sync.m16n8k16 bf16 x bf16 -> fp32 products (rows = cells, the 9 inputs
// padded to K = 16), the output layer and biases in fp32.  The fp32
// accumulator fragments of layer 1 are exactly the A-operand fragments of
// layer 2 (row g / g+8, columns 2t, 2t+1 per n-tile), so the hidden
// activations never leave registers.  tanh uses the MUFU approximation
// (relative error ~2^-11, below the bf16 rounding of the activations).
//
// The weights are the bf16 values installed by fpclbm_set_closure, re-packed
// on the host into per-lane fragment order (ClosurePack below).  The function
// is warp-collective: every lane of the warp must call it (inactive lanes pass
// any finite inputs and ignore the result).
#pragma once
#include <stdint.h>

#include "common.cuh"
#include "pair.cuh"

namespace fpc {

enum { CL_W1 = 0, CL_B1 = 576, CL_W2 = 640, CL_B2 = 4736, CL_W3 = 4800, CL_B3 = 4864, CL_N = 4865 };

// Device layout of the packed closure (32-bit words):
//   [0, 512)      layer-1 B fragments: (nt * 32 + lane) * 2 + {0, 1}, nt = 0..7
//   [512, 2560)   layer-2 B fragments: ((nt * 4 + kt) * 32 + lane) * 2 + {0, 1}
//   [2560, 2624)  b1 (fp32), [2624, 2688) b2, [2688, 2752) W3, [2752] b3
enum { CP_F1 = 0, CP_F2 = 512, CP_B1 = 2560, CP_B2 = 2624, CP_W3 = 2688, CP_B3 = 2752, CP_WORDS = 2756 };

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);  // .x (low 16 bits) = lo
    return *reinterpret_cast<const uint32_t*>(&v);
}

__device__ __forceinline__ float tanh_mufu(float x)
{
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                               uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// delta omega of this lane's cell from its 9 inputs (warp-collective).
template <typename R>
__device__ R closure_delta_omega(const uint32_t* __restrict__ P, const R in[9])
{
    __syncwarp();  // the .aligned mma below needs the whole warp converged
    const unsigned lane = threadIdx.x & 31u, g = lane >> 2, t = lane & 3u;
    const float* Pf = reinterpret_cast<const float*>(P);
    // this lane's inputs as bf16 pairs (x0,x1) (x2,x3) (x4,x5) (x6,x7) (x8,0)
    uint32_t q[5];
    q[0] = pack_bf16x2((float)in[0], (float)in[1]);
    q[1] = pack_bf16x2((float)in[2], (float)in[3]);
    q[2] = pack_bf16x2((float)in[4], (float)in[5]);
    q[3] = pack_bf16x2((float)in[6], (float)in[7]);
    q[4] = pack_bf16x2((float)in[8], 0.f);
    float mine = 0.f;
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
        // layer-1 A fragments: rows g and g+8 of this 16-cell tile, K columns 2t, 2t+1 (and +8)
        const unsigned rlo = 16u * mt + g, rhi = rlo + 8u;
        uint32_t plo[5], phi[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            plo[k] = __shfl_sync(0xffffffffu, q[k], rlo);
            phi[k] = __shfl_sync(0xffffffffu, q[k], rhi);
        }
        const uint32_t a0 = t == 0 ? plo[0] : t == 1 ? plo[1] : t == 2 ? plo[2] : plo[3];
        const uint32_t a1 = t == 0 ? phi[0] : t == 1 ? phi[1] : t == 2 ? phi[2] : phi[3];
        const uint32_t a2 = t == 0 ? plo[4] : 0u;
        const uint32_t a3 = t == 0 ? phi[4] : 0u;
        // layer 1 + tanh, re-packed as the layer-2 A fragments
        uint32_t A2[4][4];
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            float c[4] = {0.f, 0.f, 0.f, 0.f};
            mma_bf16_16816(c, a0, a1, a2, a3, __ldg(P + CP_F1 + (nt * 32 + lane) * 2),
                           __ldg(P + CP_F1 + (nt * 32 + lane) * 2 + 1));
            const float bb0 = __ldg(Pf + CP_B1 + 8 * nt + 2 * t), bb1 = __ldg(Pf + CP_B1 + 8 * nt + 2 * t + 1);
            const uint32_t lo = pack_bf16x2(tanh_mufu(c[0] + bb0), tanh_mufu(c[1] + bb1));  // row g
            const uint32_t hi = pack_bf16x2(tanh_mufu(c[2] + bb0), tanh_mufu(c[3] + bb1));  // row g+8
            const int kt = nt >> 1;
            if ((nt & 1) == 0) {
                A2[kt][0] = lo;
                A2[kt][1] = hi;
            } else {
                A2[kt][2] = lo;
                A2[kt][3] = hi;
            }
        }
        // layer 2 + tanh + output layer partial sums over this lane's columns
        float ylo = 0.f, yhi = 0.f;
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int kt = 0; kt < 4; ++kt)
                mma_bf16_16816(c, A2[kt][0], A2[kt][1], A2[kt][2], A2[kt][3],
                               __ldg(P + CP_F2 + ((nt * 4 + kt) * 32 + lane) * 2),
                               __ldg(P + CP_F2 + ((nt * 4 + kt) * 32 + lane) * 2 + 1));
            const int n0 = 8 * nt + 2 * t;
            const float bb0 = __ldg(Pf + CP_B2 + n0), bb1 = __ldg(Pf + CP_B2 + n0 + 1);
            const float w0 = __ldg(Pf + CP_W3 + n0), w1 = __ldg(Pf + CP_W3 + n0 + 1);
            ylo = fmaf(w0, tanh_mufu(c[0] + bb0), fmaf(w1, tanh_mufu(c[1] + bb1), ylo));
            yhi = fmaf(w0, tanh_mufu(c[2] + bb0), fmaf(w1, tanh_mufu(c[3] + bb1), yhi));
        }
        // sum over the quad (the 4 lanes sharing rows g, g+8), then hand row r to lane 16 mt + r
        ylo += __shfl_xor_sync(0xffffffffu, ylo, 1);
        ylo += __shfl_xor_sync(0xffffffffu, ylo, 2);
        yhi += __shfl_xor_sync(0xffffffffu, yhi, 1);
        yhi += __shfl_xor_sync(0xffffffffu, yhi, 2);
        const unsigned r = lane & 15u;
        const float vlo = __shfl_sync(0xffffffffu, ylo, 4u * (r & 7u));
        const float vhi = __shfl_sync(0xffffffffu, yhi, 4u * (r & 7u));
        if ((lane >> 4) == (unsigned)mt) mine = r < 8 ? vlo : vhi;
    }
    return (R)(mine + __ldg(Pf + CP_B3));
}

// Two cells per thread (pair.cuh): the network runs once for the cells in the x lanes of the
// warp and once for those in the y lanes (warp-collective, like the scalar version).
template <>
__device__ __forceinline__ f2 closure_delta_omega<f2>(const uint32_t* __restrict__ P, const f2 in[9])
{
    float ix[9], iy[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        ix[k] = in[k].v.x;
        iy[k] = in[k].v.y;
    }
    const float dx = closure_delta_omega<float>(P, ix);
    const float dy = closure_delta_omega<float>(P, iy);
    return f2(dx, dy);
}

}  // namespace fpc
