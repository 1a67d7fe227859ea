// closure.cuh -- per-cell inference of the learned shear-rate correction.
//
// MLP 9 -> 64 -> 64 -> 1 with tanh hidden layers, evaluated for the 32 cells of
// a warp at once on the tensor cores: both hidden layers are
// mma.sync.m16n8k16 bf16 x bf16 -> fp32 products (rows = cells, the 9 inputs and
// a constant 1 for the bias padded to K = 16), the output layer in fp32.  The fp32
// accumulator fragments of layer 1 are exactly the A-operand fragments of
// layer 2 (row g / g+8, columns 2t, 2t+1 per n-tile), so the hidden
// activations never leave registers.  tanh uses the MUFU approximation
// (relative error ~2^-11, below the bf16 rounding of the activations).
//
// The weights are the bf16 values installed by fpclbm_set_closure, re-packed
// on the host into per-lane fragment order (the layout below).  The function
// is warp-collective: every lane of the warp must call it (inactive lanes pass
// any finite inputs and ignore the result).
#pragma once
#include <stdint.h>

#include "common.cuh"
#include "pair.cuh"

namespace fpc {

enum { CL_W1 = 0, CL_B1 = 576, CL_W2 = 640, CL_B2 = 4736, CL_W3 = 4800, CL_B3 = 4864, CL_N = 4865 };

// Device layout of the packed closure (32-bit words):
//   [0, 512)      layer-1 B fragments: (nt * 32 + lane) * 2 + {0, 1}, nt = 0..7; K column 9
//                 holds b1 (the A operand's input 9 is the constant 1)
//   [512, 2560)   layer-2 B fragments: ((nt * 4 + kt) * 32 + lane) * 2 + {0, 1}
//   [2560, 2624)  b1 (fp32), [2624, 2688) b2, [2688, 2752) W3, [2752] b3
//   [2756, 3012)  layer-2 bias fragments: nt * 32 + lane, the first word of the B fragment of a
//                 K tile whose only non-zero row holds b2 (the second word is zero)
// The weights, biases included, are bf16 values, so b1 and b2 enter the products exactly.
enum { CP_F1 = 0, CP_F2 = 512, CP_B1 = 2560, CP_B2 = 2624, CP_W3 = 2688, CP_B3 = 2752, CP_F2B = 2756,
       CP_WORDS = 3012 };

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

// D += A B (bf16 x bf16 -> fp32, accumulator in place)
__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                               uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// D = A B + C with the accumulator input C given separately (a bias row), so no register copy of
// it is needed before the product.
__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], const uint32_t (&a)[4], uint2 b, float c0, float c1,
                                               float c2, float c3)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%10,%11,%12,%13};\n"
        : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b.x), "r"(b.y), "f"(c0), "f"(c1), "f"(c2), "f"(c3));
}

// Two consecutive words of the packed closure (every pair read here starts at an even word of a
// cudaMalloc'd array, so one 8-byte load).
__device__ __forceinline__ uint2 ldg_pair(const uint32_t* p) { return __ldg(reinterpret_cast<const uint2*>(p)); }
__device__ __forceinline__ float2 ldg_pair(const float* p) { return __ldg(reinterpret_cast<const float2*>(p)); }

// delta omega of this lane's cell from its 9 inputs (warp-collective).  The warp's 32 cells form
// two 16-row tiles; every weight fragment is loaded once and used by both tiles.  The biases enter
// the products as weights of a constant input 1: b1 in the spare K column 9 of layer 1, b2 in a
// fifth K tile of layer 2 whose A fragment is the constant 1 in column 64.
template <typename R>
__device__ R closure_delta_omega(const uint32_t* __restrict__ P, const R in[9])
{
    __syncwarp();  // the .aligned mma below needs the whole warp converged
    const unsigned lane = threadIdx.x & 31u, g = lane >> 2, t = lane & 3u;
    const float* Pf = reinterpret_cast<const float*>(P);
    // this lane's inputs as bf16 pairs (x0,x1) (x2,x3) (x4,x5) (x6,x7) (x8,1)
    uint32_t q[5];
    q[0] = pack_bf16x2((float)in[0], (float)in[1]);
    q[1] = pack_bf16x2((float)in[2], (float)in[3]);
    q[2] = pack_bf16x2((float)in[4], (float)in[5]);
    q[3] = pack_bf16x2((float)in[6], (float)in[7]);
    q[4] = pack_bf16x2((float)in[8], 1.f);  // input 9: the constant 1 that carries b1
    // layer-1 A fragments of tile mt: rows g and g+8 (cells 16 mt + g, 16 mt + g + 8), K columns
    // 2t, 2t+1 (and + 8: only input 8 and zeros)
    uint32_t a1[2][4];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
        const unsigned rlo = 16u * mt + g, rhi = rlo + 8u;
        uint32_t plo[5], phi[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            plo[k] = __shfl_sync(0xffffffffu, q[k], rlo);
            phi[k] = __shfl_sync(0xffffffffu, q[k], rhi);
        }
        a1[mt][0] = t == 0 ? plo[0] : t == 1 ? plo[1] : t == 2 ? plo[2] : plo[3];
        a1[mt][1] = t == 0 ? phi[0] : t == 1 ? phi[1] : t == 2 ? phi[2] : phi[3];
        a1[mt][2] = t == 0 ? plo[4] : 0u;
        a1[mt][3] = t == 0 ? phi[4] : 0u;
    }
    // layer 1 (+ b1 through input 9) + tanh, re-packed in registers as the layer-2 A fragments
    // A2[mt][kt]
    uint32_t A2[2][4][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        const uint2 b = ldg_pair(P + CP_F1 + (nt * 32 + lane) * 2);
        const int kt = nt >> 1, h = (nt & 1) * 2;
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
            float c[4];
            mma_bf16_16816(c, a1[mt], b, 0.f, 0.f, 0.f, 0.f);
            A2[mt][kt][h] = pack_bf16x2(tanh_mufu(c[0]), tanh_mufu(c[1]));      // row g
            A2[mt][kt][h + 1] = pack_bf16x2(tanh_mufu(c[2]), tanh_mufu(c[3]));  // row g+8
        }
    }
    // layer 2 (b2 first, through the constant-1 K tile) + tanh + output-layer partial sums over
    // this lane's columns 2t, 2t+1 of each n-tile
    const uint32_t one = t == 0 ? pack_bf16x2(1.f, 0.f) : 0u;  // A fragment: 1 in K column 64
    const uint32_t aone[4] = {one, one, 0u, 0u};
    float ylo[2] = {0.f, 0.f}, yhi[2] = {0.f, 0.f};
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        const int n0 = 8 * nt + 2 * t;
        const uint2 bias = make_uint2(__ldg(P + CP_F2B + nt * 32 + lane), 0u);
        float c[2][4];
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) mma_bf16_16816(c[mt], aone, bias, 0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int kt = 0; kt < 4; ++kt) {
            const uint2 b = ldg_pair(P + CP_F2 + ((nt * 4 + kt) * 32 + lane) * 2);
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
                mma_bf16_16816(c[mt], A2[mt][kt], b, c[mt][0], c[mt][1], c[mt][2], c[mt][3]);
        }
        const float2 w = ldg_pair(Pf + CP_W3 + n0);
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
            ylo[mt] = fmaf(w.x, tanh_mufu(c[mt][0]), fmaf(w.y, tanh_mufu(c[mt][1]), ylo[mt]));
            yhi[mt] = fmaf(w.x, tanh_mufu(c[mt][2]), fmaf(w.y, tanh_mufu(c[mt][3]), yhi[mt]));
        }
    }
    // sum over the quad (the 4 lanes sharing rows g, g+8), then hand row r of tile mt to lane 16 mt + r
    float mine = 0.f;
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
        float lo = ylo[mt], hi = yhi[mt];
        lo += __shfl_xor_sync(0xffffffffu, lo, 1);
        lo += __shfl_xor_sync(0xffffffffu, lo, 2);
        hi += __shfl_xor_sync(0xffffffffu, hi, 1);
        hi += __shfl_xor_sync(0xffffffffu, hi, 2);
        const unsigned r = lane & 15u;
        const float vlo = __shfl_sync(0xffffffffu, lo, 4u * (r & 7u));
        const float vhi = __shfl_sync(0xffffffffu, hi, 4u * (r & 7u));
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
