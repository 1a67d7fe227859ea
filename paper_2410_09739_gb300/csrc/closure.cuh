// closure.cuh -- per-cell inference of the learned shear-rate correction.
//
// MLP 9 -> 64 -> 64 -> 1 with tanh hidden layers.  Weights are the bf16
// values installed by fpclbm_set_closure, widened to fp32 once on the host;
// accumulation is fp32.  Layout (row-major, out x in):
//   W1[64][9] at 0, b1[64] at 576, W2[64][64] at 640, b2[64] at 4736,
//   W3[64] at 4800, b3 at 4864 (4865 values).
// Inputs are raw (normalisation is folded into W1, b1 by the trainer).
#pragma once
#include "collide.cuh"

namespace fpc {

enum { CL_W1 = 0, CL_B1 = 576, CL_W2 = 640, CL_B2 = 4736, CL_W3 = 4800, CL_B3 = 4864, CL_N = 4865 };

template <typename R>
__device__ R closure_delta_omega(const float* __restrict__ W, const R in[9])
{
    float x[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) x[i] = (float)in[i];
    float h1[64];
#pragma unroll
    for (int j = 0; j < 64; ++j) {
        float acc = __ldg(W + CL_B1 + j);
#pragma unroll
        for (int i = 0; i < 9; ++i) acc = fmaf(__ldg(W + CL_W1 + 9 * j + i), x[i], acc);
        h1[j] = tanhf(acc);
    }
    float out = __ldg(W + CL_B3);
#pragma unroll 4
    for (int j = 0; j < 64; ++j) {
        const float4* row = reinterpret_cast<const float4*>(W + CL_W2 + 64 * j);
        float acc = __ldg(W + CL_B2 + j);
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const float4 w = __ldg(row + k);
            acc = fmaf(w.x, h1[4 * k + 0], acc);
            acc = fmaf(w.y, h1[4 * k + 1], acc);
            acc = fmaf(w.z, h1[4 * k + 2], acc);
            acc = fmaf(w.w, h1[4 * k + 3], acc);
        }
        out = fmaf(__ldg(W + CL_W3 + j), tanhf(acc), out);
    }
    return (R)out;
}

}  // namespace fpc
