// closure_train.cu -- training data and training kernels of the learned closure.
//
// The learned closure (no counterpart in the paper, whose channel flow uses a
// Smagorinsky LES) is a per-cell MLP 9 -> 64 -> 64 -> 1 that corrects the shear
// relaxation rate of a coarse-grid FPC-LBM (inference: closure.cuh).
//
// fpclbm_closure_sample: box filter of a fine run onto r^3 blocks, features
//   and labels per block (definitions in include/fpclbm.h).
// fpclbm_closure_train:  Adam on the mean squared error, mini-batches, bf16
//   weights in the forward and backward kernels, fp32 accumulation and
//   gradients, fp64 loss accumulation, fp32 master weights.
// fpclbm_closure_grad:   one loss/gradient evaluation, for checking.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "rtalloc.h"
#include "aux.cuh"
#include "closure.cuh"
#include "handle.h"

namespace fpc {
namespace {

constexpr double kCs2 = 1.0 / 3.0;

// ---------------------------------------------------------------------------
// Training data: filter, strain rate, eddy viscosity, labels
// ---------------------------------------------------------------------------

struct FilterArgs {
    BoxGeom b;
    int parity, r;
    int cx, cy, cz;  // coarse dimensions
    double Fx, Fy, Fz;
    double* acc;     // [10][Nc]: rho, ux, uy, uz, uxx, uyy, uzz, uxy, uxz, uyz
};

template <typename S>
__global__ void k_cl_filter(FilterArgs a)
{
    const unsigned nc = (unsigned)a.cx * a.cy * a.cz;
    const unsigned c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nc) return;
    const unsigned X = c % a.cx, Y = (c / a.cx) % a.cy, Z = c / (a.cx * a.cy);
    double s[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int k = 0; k < a.r; ++k)
        for (int j = 0; j < a.r; ++j)
            for (int i = 0; i < a.r; ++i) {
                const unsigned x = X * a.r + i, y = Y * a.r + j, z = Z * a.r + k;
                const unsigned cell = x + (unsigned)a.b.nx * (y + (unsigned)a.b.ny * z);
                double g[27], rho, u, v, w;
                load_cell<S>(a.b, a.parity, cell, g);
                fields_of(g, a.Fx, a.Fy, a.Fz, rho, u, v, w);
                s[0] += rho;
                s[1] += u;
                s[2] += v;
                s[3] += w;
                s[4] += u * u;
                s[5] += v * v;
                s[6] += w * w;
                s[7] += u * v;
                s[8] += u * w;
                s[9] += v * w;
            }
    const double inv = 1.0 / ((double)a.r * a.r * a.r);
    for (int q = 0; q < 10; ++q) a.acc[(size_t)q * nc + c] = s[q] * inv;
}

// Strain rate of the filtered velocity (central differences in coarse cells,
// periodic in x and z, periodic in y or, at y walls, through the no-slip wall
// value), eddy viscosity from the sub-filter stress, label and features.
__global__ void k_cl_label(const double* __restrict__ acc, int cx, int cy, int cz, int walls, double tau_c,
                           float* X, float* T)
{
    const unsigned nc = (unsigned)cx * cy * cz;
    const unsigned c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nc) return;
    const int x = c % cx, y = (c / cx) % cy, z = c / (cx * cy);
    auto at = [&](int q, int xx, int yy, int zz) {
        return acc[(size_t)q * nc + (unsigned)(xx + cx * (yy + cy * zz))];
    };
    // d u_i / d x_j, i = 0..2 (u, v, w), j = 0..2 (x, y, z)
    double gr[3][3];
    for (int i = 0; i < 3; ++i) {
        const int q = 1 + i;
        gr[i][0] = 0.5 * (at(q, (x + 1) % cx, y, z) - at(q, (x - 1 + cx) % cx, y, z));
        gr[i][2] = 0.5 * (at(q, x, y, (z + 1) % cz) - at(q, x, y, (z - 1 + cz) % cz));
        // next to a no-slip wall (y = -1/2 or cy - 1/2) the derivative of the quadratic through the
        // wall value 0 and the two nearest rows
        if (!walls)
            gr[i][1] = 0.5 * (at(q, x, (y + 1) % cy, z) - at(q, x, (y - 1 + cy) % cy, z));
        else if (y == 0)
            gr[i][1] = at(q, x, 0, z) + at(q, x, 1, z) / 3.0;
        else if (y == cy - 1)
            gr[i][1] = -(at(q, x, cy - 1, z) + at(q, x, cy - 2, z) / 3.0);
        else
            gr[i][1] = 0.5 * (at(q, x, y + 1, z) - at(q, x, y - 1, z));
    }
    double S[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) S[i][j] = 0.5 * (gr[i][j] + gr[j][i]);
    const double u[3] = {at(1, x, y, z), at(2, x, y, z), at(3, x, y, z)};
    const double rho = at(0, x, y, z);
    // <u_i u_j>: q = 4 uu, 5 vv, 6 ww, 7 uv, 8 uw, 9 vw
    const int uq[3][3] = {{4, 7, 8}, {7, 5, 9}, {8, 9, 6}};
    double tau[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) tau[i][j] = at(uq[i][j], x, y, z) - u[i] * u[j];
    const double tr = (tau[0][0] + tau[1][1] + tau[2][2]) / 3.0;
    double num = 0, den = 0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            const double td = tau[i][j] - (i == j ? tr : 0.0);
            num += td * S[i][j];
            den += S[i][j] * S[i][j];
        }
    double nut = den > 0 ? -num / (2.0 * den) : 0.0;
    if (!(nut > 0)) nut = 0.0;
    const double nu = kCs2 * (tau_c - 0.5);
    const double label = 1.0 / ((nu + nut) / kCs2 + 0.5) - 1.0 / (nu / kCs2 + 0.5);
    const double f = -2.0 * rho * kCs2 * tau_c;
    float* xo = X + (size_t)9 * c;
    xo[0] = (float)(f * S[0][0]);
    xo[1] = (float)(f * S[1][1]);
    xo[2] = (float)(f * S[2][2]);
    xo[3] = (float)(f * S[0][1]);
    xo[4] = (float)(f * S[0][2]);
    xo[5] = (float)(f * S[1][2]);
    xo[6] = (float)u[0];
    xo[7] = (float)u[1];
    xo[8] = (float)u[2];
    T[c] = (float)label;
}

// ---------------------------------------------------------------------------
// Network forward/backward on mini-batches
// ---------------------------------------------------------------------------

// Mini-batch forward and backward on the tensor cores.  A block takes kMB = 128
// samples, 32 per warp (two 16-row tiles).  Every contraction is an
// mma.sync.m16n8k16 bf16 x bf16 -> fp32 product:
//   forward   Z1 = [x, 1] [W1 | b1]^T (K = 16: 9 inputs, the bias input 1, zeros),
//             Z2 = H1 W2^T (K = 64), H = tanh(Z) in fp32, y = w3 . H2 + b3 in fp32;
//   backward  G2 = gy w3 (1 - H2^2), G1 = (G2 W2) (1 - H1^2)  (K = 64);
//   weights   dW2 = G2^T [H1, 1] and dW1 = G1^T [x, 1] over the block's samples
//             (K = 128); the column of ones gives the bias gradients db2, db1;
//             dw3 = sum gy H2 and db3 = sum gy in fp32.
// The operands x, H1, G2, G1 are rounded to bf16 (the weights are bf16 already);
// products accumulate in fp32.  The fp32 accumulator fragments of one product
// are the A-operand fragments of the next (row g / g+8, columns 2t, 2t+1), so
// H1 and G2 stay in registers; for the weight gradients, whose K runs over the
// samples, H1, G2, G1 and x are also written feature-major to shared memory.
// Each block writes its gradient (4865 fp32) and its loss (fp64) to its own
// slot of a scratch array; k_cl_reduce_adam / k_cl_reduce_grad sum the blocks
// in a fixed order, so training is deterministic.

constexpr int kMB = 128;        // samples per block (4 warps x 32)
constexpr int kTP = kMB + 8;    // row pitch of the feature-major tables (bank offset between rows)

struct NetArgs {
    const float* X;             // [n][9]
    const float* T;             // [n]
    unsigned long long n;       // samples in the data set
    unsigned long long first;   // first position of this batch in the epoch order
    unsigned long long count;   // samples in this batch
    unsigned long long perm_a, perm_c;  // epoch order: sample(i) = (a i + c) mod n
    float mu[10], inv_sd[10];   // standardisation of the 9 inputs and the target
    float scale;                // dL/dy factor 2 / batch
    const __nv_bfloat16* W;     // bf16 weights (closure layout)
    float* part;                // per-block gradients [blocks][4865]
    double* part_loss;          // per-block sums of squared errors [blocks]
};

struct TrainSmem {
    __nv_bfloat16 W1p[64][16];  // [j][i]: W1, then b1 in column 9, zeros
    __nv_bfloat16 W2s[64][64];  // W2[j][k]
    __nv_bfloat16 W2T[64][64];  // W2[j][k] at [k][j]
    __nv_bfloat16 XS[kMB][16];  // [m][i] inputs of the block's samples, 1 in column 9
    __nv_bfloat16 XT[16][kTP];  // [i][m]
    __nv_bfloat16 H1T[72][kTP]; // [k][m], row 64 = 1, rows 65..71 = 0
    __nv_bfloat16 G2T[64][kTP]; // [j][m]
    __nv_bfloat16 G1T[64][kTP]; // [j][m]
    float b2[64], w3[64], tgt[kMB], vld[kMB], dw3[4][64];
    float b3, db3[4];
    double loss[4];
};

__device__ __forceinline__ uint32_t lds32(const __nv_bfloat16* p) { return *reinterpret_cast<const uint32_t*>(p); }
__device__ __forceinline__ __nv_bfloat16 bf_lo(uint32_t v) { return __ushort_as_bfloat16((unsigned short)(v & 0xffffu)); }
__device__ __forceinline__ __nv_bfloat16 bf_hi(uint32_t v) { return __ushort_as_bfloat16((unsigned short)(v >> 16)); }

__global__ void __launch_bounds__(kMB) k_cl_mma(NetArgs a)
{
    extern __shared__ __align__(16) unsigned char cl_smem[];
    TrainSmem& S = *reinterpret_cast<TrainSmem*>(cl_smem);
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5, g = lane >> 2, t = lane & 3;
    const __nv_bfloat16 zero = __float2bfloat16_rn(0.f), one = __float2bfloat16_rn(1.f);

    for (int i = tid; i < 64 * 16; i += kMB) {
        const int j = i >> 4, c = i & 15;
        S.W1p[j][c] = c < 9 ? a.W[CL_W1 + 9 * j + c] : (c == 9 ? a.W[CL_B1 + j] : zero);
    }
    for (int i = tid; i < 4096; i += kMB) {
        const __nv_bfloat16 v = a.W[CL_W2 + i];
        S.W2s[i >> 6][i & 63] = v;
        S.W2T[i & 63][i >> 6] = v;
    }
    for (int j = tid; j < 64; j += kMB) {
        S.b2[j] = __bfloat162float(a.W[CL_B2 + j]);
        S.w3[j] = __bfloat162float(a.W[CL_W3 + j]);
    }
    if (tid == 0) S.b3 = __bfloat162float(a.W[CL_B3]);
    for (int i = tid; i < 8 * kTP; i += kMB) S.H1T[64 + i / kTP][i % kTP] = i < kTP ? one : zero;
    // this thread's sample: standardised inputs (bf16), bias input 1, target
    {
        const unsigned long long pos = a.first + (unsigned long long)blockIdx.x * kMB + tid;
        const bool valid = pos < a.first + a.count;
        float x[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) x[i] = 0.f;
        x[9] = 1.f;
        float tt = 0.f;
        if (valid) {
            const unsigned long long idx = (a.perm_a * pos + a.perm_c) % a.n;
#pragma unroll
            for (int i = 0; i < 9; ++i) x[i] = (a.X[idx * 9 + i] - a.mu[i]) * a.inv_sd[i];
            tt = (a.T[idx] - a.mu[9]) * a.inv_sd[9];
        }
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const __nv_bfloat16 b = __float2bfloat16_rn(x[i]);
            S.XS[tid][i] = b;
            S.XT[i][tid] = b;
        }
        S.tgt[tid] = tt;
        S.vld[tid] = valid ? 1.f : 0.f;  // padding rows of a short batch: no error, no gradient
    }
    __syncthreads();

    float dw3a[8][2];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) dw3a[nt][0] = dw3a[nt][1] = 0.f;
    float db3a = 0.f;
    double lossa = 0.0;
#pragma unroll 1
    for (int mt = 0; mt < 2; ++mt) {
        const int r0 = 32 * w + 16 * mt + g, r1 = r0 + 8;
        // ---- layer 1: Z1 = [x, 1] [W1 | b1]^T, H1 = tanh(Z1)
        const uint32_t xa0 = lds32(&S.XS[r0][2 * t]), xa1 = lds32(&S.XS[r1][2 * t]);
        const uint32_t xa2 = lds32(&S.XS[r0][2 * t + 8]), xa3 = lds32(&S.XS[r1][2 * t + 8]);
        float h1[8][4];
        uint32_t A2[4][4];
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            float c[4] = {0.f, 0.f, 0.f, 0.f};
            mma_bf16_16816(c, xa0, xa1, xa2, xa3, lds32(&S.W1p[8 * nt + g][2 * t]), lds32(&S.W1p[8 * nt + g][2 * t + 8]));
#pragma unroll
            for (int q = 0; q < 4; ++q) h1[nt][q] = tanhf(c[q]);
            const uint32_t lo = pack_bf16x2(h1[nt][0], h1[nt][1]), hi = pack_bf16x2(h1[nt][2], h1[nt][3]);
            A2[nt >> 1][(nt & 1) * 2] = lo;
            A2[nt >> 1][(nt & 1) * 2 + 1] = hi;
            const int c0 = 8 * nt + 2 * t;
            S.H1T[c0][r0] = bf_lo(lo);
            S.H1T[c0 + 1][r0] = bf_hi(lo);
            S.H1T[c0][r1] = bf_lo(hi);
            S.H1T[c0 + 1][r1] = bf_hi(hi);
            // the backward pass needs 1 - H1^2 of the bf16 operand's source value
            h1[nt][0] = 1.f - h1[nt][0] * h1[nt][0];
            h1[nt][1] = 1.f - h1[nt][1] * h1[nt][1];
            h1[nt][2] = 1.f - h1[nt][2] * h1[nt][2];
            h1[nt][3] = 1.f - h1[nt][3] * h1[nt][3];
        }
        // ---- layer 2 and output: Z2 = H1 W2^T + b2, H2 = tanh(Z2), y = w3 . H2 + b3
        float h2[8][4];
        float y0 = 0.f, y1 = 0.f;
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int kt = 0; kt < 4; ++kt)
                mma_bf16_16816(c, A2[kt][0], A2[kt][1], A2[kt][2], A2[kt][3], lds32(&S.W2s[8 * nt + g][16 * kt + 2 * t]),
                               lds32(&S.W2s[8 * nt + g][16 * kt + 2 * t + 8]));
            const int c0 = 8 * nt + 2 * t;
            h2[nt][0] = tanhf(c[0] + S.b2[c0]);
            h2[nt][1] = tanhf(c[1] + S.b2[c0 + 1]);
            h2[nt][2] = tanhf(c[2] + S.b2[c0]);
            h2[nt][3] = tanhf(c[3] + S.b2[c0 + 1]);
            y0 = fmaf(S.w3[c0], h2[nt][0], fmaf(S.w3[c0 + 1], h2[nt][1], y0));
            y1 = fmaf(S.w3[c0], h2[nt][2], fmaf(S.w3[c0 + 1], h2[nt][3], y1));
        }
        y0 += __shfl_xor_sync(0xffffffffu, y0, 1);
        y0 += __shfl_xor_sync(0xffffffffu, y0, 2);
        y1 += __shfl_xor_sync(0xffffffffu, y1, 1);
        y1 += __shfl_xor_sync(0xffffffffu, y1, 2);
        const float e0 = S.vld[r0] * (y0 + S.b3 - S.tgt[r0]), e1 = S.vld[r1] * (y1 + S.b3 - S.tgt[r1]);
        const float gy0 = a.scale * e0, gy1 = a.scale * e1;
        if (t == 0) {
            lossa += (double)e0 * e0 + (double)e1 * e1;
            db3a += gy0 + gy1;
        }
        // ---- G2 = gy w3 (1 - H2^2): A operand of G2 W2 and feature-major copy for dW2
        uint32_t AG[4][4];
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const int c0 = 8 * nt + 2 * t;
            dw3a[nt][0] = fmaf(gy0, h2[nt][0], fmaf(gy1, h2[nt][2], dw3a[nt][0]));
            dw3a[nt][1] = fmaf(gy0, h2[nt][1], fmaf(gy1, h2[nt][3], dw3a[nt][1]));
            const float wa = S.w3[c0], wb = S.w3[c0 + 1];
            const uint32_t lo = pack_bf16x2(gy0 * wa * (1.f - h2[nt][0] * h2[nt][0]), gy0 * wb * (1.f - h2[nt][1] * h2[nt][1]));
            const uint32_t hi = pack_bf16x2(gy1 * wa * (1.f - h2[nt][2] * h2[nt][2]), gy1 * wb * (1.f - h2[nt][3] * h2[nt][3]));
            AG[nt >> 1][(nt & 1) * 2] = lo;
            AG[nt >> 1][(nt & 1) * 2 + 1] = hi;
            S.G2T[c0][r0] = bf_lo(lo);
            S.G2T[c0 + 1][r0] = bf_hi(lo);
            S.G2T[c0][r1] = bf_lo(hi);
            S.G2T[c0 + 1][r1] = bf_hi(hi);
        }
        // ---- G1 = (G2 W2) (1 - H1^2), feature-major copy for dW1
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int kt = 0; kt < 4; ++kt)
                mma_bf16_16816(c, AG[kt][0], AG[kt][1], AG[kt][2], AG[kt][3], lds32(&S.W2T[8 * nt + g][16 * kt + 2 * t]),
                               lds32(&S.W2T[8 * nt + g][16 * kt + 2 * t + 8]));
            const int c0 = 8 * nt + 2 * t;
            const uint32_t lo = pack_bf16x2(c[0] * h1[nt][0], c[1] * h1[nt][1]);
            const uint32_t hi = pack_bf16x2(c[2] * h1[nt][2], c[3] * h1[nt][3]);
            S.G1T[c0][r0] = bf_lo(lo);
            S.G1T[c0 + 1][r0] = bf_hi(lo);
            S.G1T[c0][r1] = bf_lo(hi);
            S.G1T[c0 + 1][r1] = bf_hi(hi);
        }
    }
    // warp sums of dw3 (over the rows, lane bits 2..4), db3 and the loss
#pragma unroll
    for (int nt = 0; nt < 8; ++nt)
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            float v = dw3a[nt][q];
            v += __shfl_xor_sync(0xffffffffu, v, 4);
            v += __shfl_xor_sync(0xffffffffu, v, 8);
            v += __shfl_xor_sync(0xffffffffu, v, 16);
            if (g == 0) S.dw3[w][8 * nt + 2 * t + q] = v;
        }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        db3a += __shfl_xor_sync(0xffffffffu, db3a, o);
        lossa += __shfl_xor_sync(0xffffffffu, lossa, o);
    }
    if (lane == 0) {
        S.db3[w] = db3a;
        S.loss[w] = lossa;
    }
    __syncthreads();

    // ---- weight gradients over the block's samples: warp w owns rows j = 16 w .. 16 w + 15
    float* part = a.part + (size_t)blockIdx.x * CL_N;
    const int j0 = 16 * w + g, j1 = j0 + 8;
#pragma unroll 1
    for (int nt = 0; nt < 9; ++nt) {  // dW2 (k = 0..63) and db2 (k = 64)
        float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int kt = 0; kt < kMB / 16; ++kt) {
            const int m0 = 16 * kt + 2 * t;
            mma_bf16_16816(c, lds32(&S.G2T[j0][m0]), lds32(&S.G2T[j1][m0]), lds32(&S.G2T[j0][m0 + 8]),
                           lds32(&S.G2T[j1][m0 + 8]), lds32(&S.H1T[8 * nt + g][m0]), lds32(&S.H1T[8 * nt + g][m0 + 8]));
        }
        const int k0 = 8 * nt + 2 * t;
        if (nt < 8) {
            part[CL_W2 + 64 * j0 + k0] = c[0];
            part[CL_W2 + 64 * j0 + k0 + 1] = c[1];
            part[CL_W2 + 64 * j1 + k0] = c[2];
            part[CL_W2 + 64 * j1 + k0 + 1] = c[3];
        } else if (t == 0) {
            part[CL_B2 + j0] = c[0];
            part[CL_B2 + j1] = c[2];
        }
    }
#pragma unroll 1
    for (int nt = 0; nt < 2; ++nt) {  // dW1 (i = 0..8) and db1 (i = 9)
        float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int kt = 0; kt < kMB / 16; ++kt) {
            const int m0 = 16 * kt + 2 * t;
            mma_bf16_16816(c, lds32(&S.G1T[j0][m0]), lds32(&S.G1T[j1][m0]), lds32(&S.G1T[j0][m0 + 8]),
                           lds32(&S.G1T[j1][m0 + 8]), lds32(&S.XT[8 * nt + g][m0]), lds32(&S.XT[8 * nt + g][m0 + 8]));
        }
        const int i0 = 8 * nt + 2 * t;
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int i = i0 + q;
            if (i < 9) {
                part[CL_W1 + 9 * j0 + i] = c[q];
                part[CL_W1 + 9 * j1 + i] = c[2 + q];
            } else if (i == 9) {
                part[CL_B1 + j0] = c[q];
                part[CL_B1 + j1] = c[2 + q];
            }
        }
    }
    if (tid < 64) part[CL_W3 + tid] = (S.dw3[0][tid] + S.dw3[1][tid]) + (S.dw3[2][tid] + S.dw3[3][tid]);
    if (tid == 64) part[CL_B3] = (S.db3[0] + S.db3[1]) + (S.db3[2] + S.db3[3]);
    if (tid == 65) a.part_loss[blockIdx.x] = (S.loss[0] + S.loss[1]) + (S.loss[2] + S.loss[3]);
}

// Second stage: sum of the block gradients in block order; the loss (fp64) is added to *loss.
__device__ __forceinline__ float sum_blocks(const float* part, int blocks, int p)
{
    float s = 0.f;
    for (int b = 0; b < blocks; ++b) s += part[(size_t)b * CL_N + p];
    return s;
}

__global__ void k_cl_reduce_grad(const float* part, const double* part_loss, int blocks, float* grad, double* loss)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < CL_N) grad[p] = sum_blocks(part, blocks, p);
    if (p == 0) {
        double l = 0.0;
        for (int b = 0; b < blocks; ++b) l += part_loss[b];
        *loss += l;
    }
}

// Adam (Kingma & Ba 2015) on fp32 master weights; the gradient is the sum of the block partials.
__global__ void k_cl_reduce_adam(float* w, float* m, float* v, const float* part, const double* part_loss, int blocks,
                                 double* loss, __nv_bfloat16* wb, float lr, float b1, float b2, float c1, float c2,
                                 float eps)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p == 0) {
        double l = 0.0;
        for (int b = 0; b < blocks; ++b) l += part_loss[b];
        *loss += l;
    }
    if (p >= CL_N) return;
    const float g = sum_blocks(part, blocks, p);
    const float mm = b1 * m[p] + (1.f - b1) * g;
    const float vv = b2 * v[p] + (1.f - b2) * g * g;
    m[p] = mm;
    v[p] = vv;
    const float wn = w[p] - lr * (mm * c1) / (sqrtf(vv * c2) + eps);
    w[p] = wn;
    wb[p] = __float2bfloat16_rn(wn);
}

// Column sums and sums of squares of the inputs and the target (column 9): per-block partials in
// out[block][20], each block's in a fixed tree order, summed over blocks by the host in block order.
constexpr int kStatBlocks = 256, kStatThreads = 256;

__global__ void __launch_bounds__(kStatThreads) k_cl_stats(const float* X, const float* T, unsigned long long n,
                                                            double* out)
{
    __shared__ double sh[20][kStatThreads];
    double s[20];
    for (int k = 0; k < 20; ++k) s[k] = 0.0;
    for (unsigned long long i = (unsigned long long)blockIdx.x * kStatThreads + threadIdx.x; i < n;
         i += (unsigned long long)kStatBlocks * kStatThreads) {
        for (int k = 0; k < 10; ++k) {
            const double v = k < 9 ? X[i * 9 + k] : T[i];
            s[k] += v;
            s[10 + k] += v * v;
        }
    }
    for (int k = 0; k < 20; ++k) sh[k][threadIdx.x] = s[k];
    __syncthreads();
    for (int w = kStatThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < (unsigned)w)
            for (int k = 0; k < 20; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < 20) out[blockIdx.x * 20 + threadIdx.x] = sh[threadIdx.x][0];
}

// splitmix64 (Steele, Lea & Flood 2014) for the initial weights and epoch orders
uint64_t splitmix(uint64_t& s)
{
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

uint64_t gcd64(uint64_t a, uint64_t b)
{
    while (b) {
        const uint64_t t = a % b;
        a = b;
        b = t;
    }
    return a;
}

unsigned short bf16_bits(float v)
{
    const __nv_bfloat16 b = __float2bfloat16_rn(v);
    unsigned short u;
    std::memcpy(&u, &b, sizeof u);
    return u;
}

int err(int code, const std::string& m)
{
    g_create_error = m;
    return code;
}

}  // namespace
}  // namespace fpc

using namespace fpc;

#define FPC_CL_CK(call, what)                                                                   \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess)                                                                  \
            return err(e_ == cudaErrorMemoryAllocation ? FPCLBM_ERR_ALLOC : FPCLBM_ERR_CUDA,      \
                       std::string(what) + ": " + cudaGetErrorString(e_));                        \
    } while (0)

extern "C" int fpclbm_closure_sample(fpclbm_t h, int r, double tau_coarse, float* X, float* T, int on_device)
{
    if (!h) return FPCLBM_ERR_ARG;
    h->err.clear();
    if (h->ensemble) return fail(h, FPCLBM_ERR_ARG, "closure_sample needs a single box");
    if (!h->initialized) return fail(h, FPCLBM_ERR_STATE, "populations not initialised");
    const Box& B = h->boxes[0];
    if (r < 1 || B.nx % r || B.ny % r || B.nz % r) return fail(h, FPCLBM_ERR_ARG, "nx, ny, nz must be multiples of r");
    if (!X || !T) return fail(h, FPCLBM_ERR_ARG, "null output");
    if (!(tau_coarse > 0.5) || !std::isfinite(tau_coarse)) return fail(h, FPCLBM_ERR_ARG, "tau_coarse must be > 1/2");
    const int cx = B.nx / r, cy = B.ny / r, cz = B.nz / r;
    if (h->bc != FPCLBM_BC_PERIODIC && h->bc != FPCLBM_BC_WALLS_Y)
        return fail(h, FPCLBM_ERR_ARG, "closure sampling needs a periodic or channel box");
    const bool walls = h->bc == FPCLBM_BC_WALLS_Y;
    if (walls && cy < 2) return fail(h, FPCLBM_ERR_ARG, "walls need ny / r >= 2");
    const size_t nc = (size_t)cx * cy * cz;
    double* acc = nullptr;
    float *dX = X, *dT = T;
    cudaError_t e = rt_malloc(&acc, sizeof(double) * 10 * nc);
    if (e == cudaSuccess && !on_device) {
        e = rt_malloc(&dX, sizeof(float) * 9 * nc);
        if (e == cudaSuccess) e = rt_malloc(&dT, sizeof(float) * nc);
    }
    if (e != cudaSuccess) {
        rt_free(acc);
        if (!on_device) {
            rt_free(dX != X ? dX : nullptr);
        }
        return fail(h, FPCLBM_ERR_ALLOC, "closure_sample scratch");
    }
    BoxGeom g;
    g.buf = static_cast<char*>(h->d_pop) + B.off * elem_size(h->precision);
    g.stride = B.stride;
    g.ncells = B.ncells;
    g.nx = B.nx;
    g.ny = B.ny;
    g.nz = B.nz;
    g.walls = walls;
    g.div_nx = make_fastdiv((unsigned)B.nx);
    g.div_nxny = make_fastdiv((unsigned)(B.nx * B.ny));
    FilterArgs fa{g, (int)(h->steps & 1), r, cx, cy, cz, h->F[0], h->F[1], h->F[2], acc};
    const unsigned blocks = (unsigned)((nc + 127) / 128);
    switch (h->precision) {
        case FPCLBM_FP64: k_cl_filter<double><<<blocks, 128, 0, h->stream>>>(fa); break;
        case FPCLBM_FP32: k_cl_filter<float><<<blocks, 128, 0, h->stream>>>(fa); break;
        case FPCLBM_FP32_STORE_FP16: k_cl_filter<__half><<<blocks, 128, 0, h->stream>>>(fa); break;
        default: k_cl_filter<__nv_bfloat16><<<blocks, 128, 0, h->stream>>>(fa); break;
    }
    k_cl_label<<<blocks, 128, 0, h->stream>>>(acc, cx, cy, cz, walls, tau_coarse, dX, dT);
    e = cudaGetLastError();
    if (e == cudaSuccess && !on_device) {
        e = cudaMemcpyAsync(X, dX, sizeof(float) * 9 * nc, cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(T, dT, sizeof(float) * nc, cudaMemcpyDeviceToHost, h->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    rt_free(acc);
    if (!on_device) {
        rt_free(dX);
        rt_free(dT);
    }
    if (e != cudaSuccess) return fail(h, FPCLBM_ERR_CUDA, std::string("closure_sample: ") + cudaGetErrorString(e));
    return FPCLBM_OK;
}

namespace {

// Run the forward/backward kernel over `count` samples starting at epoch position `first`: one
// block per kMB samples, each writing its gradient and loss to a.part / a.part_loss.
int batch_blocks(unsigned long long count) { return (int)((count + kMB - 1) / kMB); }

cudaError_t run_batch(const NetArgs& a, cudaStream_t st)
{
    const size_t smem = sizeof(TrainSmem);
    static bool attr = false;
    if (!attr) {
        const cudaError_t e = cudaFuncSetAttribute(k_cl_mma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    k_cl_mma<<<batch_blocks(a.count), kMB, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace

extern "C" int fpclbm_closure_grad(const float* X, const float* T, int n, const unsigned short* w, float* grad,
                                   double* loss, void* cuda_stream)
{
    g_create_error.clear();
    if (!X || !T || !w || !grad || !loss || n < 1) return err(FPCLBM_ERR_ARG, "closure_grad: bad arguments");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const int blocks = batch_blocks((unsigned long long)n);
    __nv_bfloat16* dW = nullptr;
    float *dG = nullptr, *dP = nullptr;
    double *dL = nullptr, *dPL = nullptr;
    cudaError_t e = rt_malloc(&dW, sizeof(__nv_bfloat16) * CL_N);
    if (e == cudaSuccess) e = rt_malloc(&dG, sizeof(float) * CL_N);
    if (e == cudaSuccess) e = rt_malloc(&dL, sizeof(double));
    if (e == cudaSuccess) e = rt_malloc(&dP, sizeof(float) * CL_N * (size_t)blocks);
    if (e == cudaSuccess) e = rt_malloc(&dPL, sizeof(double) * (size_t)blocks);
    auto cleanup = [&]() {
        rt_free(dW);
        rt_free(dG);
        rt_free(dL);
        rt_free(dP);
        rt_free(dPL);
    };
    if (e != cudaSuccess) {
        cleanup();
        return err(FPCLBM_ERR_ALLOC, "closure_grad buffers");
    }
    NetArgs a;
    std::memset(&a, 0, sizeof a);
    a.X = X;
    a.T = T;
    a.n = (unsigned long long)n;
    a.first = 0;
    a.count = (unsigned long long)n;
    a.perm_a = 1;
    a.perm_c = 0;
    for (int k = 0; k < 10; ++k) {
        a.mu[k] = 0.f;
        a.inv_sd[k] = 1.f;
    }
    a.scale = 2.0f / (float)n;
    a.W = dW;
    a.part = dP;
    a.part_loss = dPL;
    e = cudaMemcpyAsync(dW, w, sizeof(unsigned short) * CL_N, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(dL, 0, sizeof(double), st);
    if (e == cudaSuccess) e = run_batch(a, st);
    if (e == cudaSuccess) {
        k_cl_reduce_grad<<<(CL_N + 255) / 256, 256, 0, st>>>(dP, dPL, blocks, dG, dL);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(grad, dG, sizeof(float) * CL_N, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(loss, dL, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cleanup();
    if (e != cudaSuccess) return err(FPCLBM_ERR_CUDA, std::string("closure_grad: ") + cudaGetErrorString(e));
    *loss /= n;
    return FPCLBM_OK;
}

extern "C" int fpclbm_closure_train(const float* X, const float* T, long long n, int epochs, int batch, double lr,
                                    unsigned long long seed, unsigned short* out_w, double* loss_per_epoch,
                                    void* cuda_stream)
{
    g_create_error.clear();
    if (!X || !T || !out_w || n < 2 || epochs < 1 || batch < 1 || !(lr > 0) || !std::isfinite(lr))
        return err(FPCLBM_ERR_ARG, "closure_train: bad arguments");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    // standardisation of inputs and target
    double* dS = nullptr;
    FPC_CL_CK(rt_malloc(&dS, sizeof(double) * 20 * kStatBlocks), "closure_train stats");
    k_cl_stats<<<kStatBlocks, kStatThreads, 0, st>>>(X, T, (unsigned long long)n, dS);
    std::vector<double> parts(20 * kStatBlocks);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(parts.data(), dS, sizeof(double) * parts.size(), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    rt_free(dS);
    double sums[20] = {0};
    for (int b = 0; b < kStatBlocks; ++b)
        for (int k = 0; k < 20; ++k) sums[k] += parts[20 * b + k];
    if (e != cudaSuccess) return err(FPCLBM_ERR_CUDA, std::string("closure_train stats: ") + cudaGetErrorString(e));
    double mu[10], sd[10];
    for (int k = 0; k < 10; ++k) {
        mu[k] = sums[k] / n;
        const double var = sums[10 + k] / n - mu[k] * mu[k];
        sd[k] = var > 0 ? std::sqrt(var) : 1.0;
        if (!(sd[k] > 1e-30)) sd[k] = 1.0;
    }
    // initial weights (standardised space): uniform(+-1/sqrt(fan_in)), zero biases
    std::vector<float> w0(CL_N, 0.f);
    uint64_t rs = seed;
    auto unif = [&](double lim) { return (float)(lim * (2.0 * ((splitmix(rs) >> 11) * 0x1.0p-53) - 1.0)); };
    for (int i = 0; i < 576; ++i) w0[CL_W1 + i] = unif(1.0 / 3.0);
    for (int i = 0; i < 4096; ++i) w0[CL_W2 + i] = unif(1.0 / 8.0);
    for (int i = 0; i < 64; ++i) w0[CL_W3 + i] = unif(1.0 / 8.0);
    std::vector<unsigned short> wb0(CL_N);
    for (int i = 0; i < CL_N; ++i) wb0[i] = bf16_bits(w0[i]);
    const int max_blocks = batch_blocks((unsigned long long)std::min<long long>(batch, n));
    float *dw = nullptr, *dm = nullptr, *dv = nullptr, *dP = nullptr;
    __nv_bfloat16* dwb = nullptr;
    double *dL = nullptr, *dPL = nullptr;
    e = rt_malloc(&dw, sizeof(float) * CL_N);
    if (e == cudaSuccess) e = rt_malloc(&dm, sizeof(float) * CL_N);
    if (e == cudaSuccess) e = rt_malloc(&dv, sizeof(float) * CL_N);
    if (e == cudaSuccess) e = rt_malloc(&dP, sizeof(float) * CL_N * (size_t)max_blocks);
    if (e == cudaSuccess) e = rt_malloc(&dPL, sizeof(double) * (size_t)max_blocks);
    if (e == cudaSuccess) e = rt_malloc(&dwb, sizeof(__nv_bfloat16) * CL_N);
    if (e == cudaSuccess) e = rt_malloc(&dL, sizeof(double));
    auto cleanup = [&]() {
        rt_free(dw);
        rt_free(dm);
        rt_free(dv);
        rt_free(dP);
        rt_free(dPL);
        rt_free(dwb);
        rt_free(dL);
    };
    if (e != cudaSuccess) {
        cleanup();
        return err(FPCLBM_ERR_ALLOC, "closure_train buffers");
    }
    e = cudaMemcpyAsync(dw, w0.data(), sizeof(float) * CL_N, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dwb, wb0.data(), sizeof(unsigned short) * CL_N, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(dm, 0, sizeof(float) * CL_N, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(dv, 0, sizeof(float) * CL_N, st);
    NetArgs a;
    std::memset(&a, 0, sizeof a);
    a.X = X;
    a.T = T;
    a.n = (unsigned long long)n;
    for (int k = 0; k < 10; ++k) {
        a.mu[k] = (float)mu[k];
        a.inv_sd[k] = (float)(1.0 / sd[k]);
    }
    a.W = dwb;
    a.part = dP;
    a.part_loss = dPL;
    const float b1 = 0.9f, b2 = 0.999f;
    long long step = 0;
    for (int ep = 0; ep < epochs && e == cudaSuccess; ++ep) {
        // epoch order: i -> (perm_a i + perm_c) mod n with gcd(perm_a, n) = 1
        uint64_t pa = splitmix(rs) % (uint64_t)n;
        while (pa == 0 || gcd64(pa, (uint64_t)n) != 1) pa = (pa + 1) % (uint64_t)n;
        a.perm_a = pa;
        a.perm_c = splitmix(rs) % (uint64_t)n;
        e = cudaMemsetAsync(dL, 0, sizeof(double), st);
        for (long long first = 0; first < n && e == cudaSuccess; first += batch) {
            const long long cnt = (n - first < batch) ? n - first : batch;
            a.first = (unsigned long long)first;
            a.count = (unsigned long long)cnt;
            a.scale = 2.0f / (float)cnt;
            e = run_batch(a, st);
            ++step;
            const float c1 = (float)(1.0 / (1.0 - std::pow((double)b1, (double)step)));
            const float c2 = (float)(1.0 / (1.0 - std::pow((double)b2, (double)step)));
            if (e == cudaSuccess) {
                k_cl_reduce_adam<<<(CL_N + 255) / 256, 256, 0, st>>>(dw, dm, dv, dP, dPL, batch_blocks(a.count), dL, dwb,
                                                                     (float)lr, b1, b2, c1, c2, 1e-8f);
                e = cudaGetLastError();
            }
        }
        if (loss_per_epoch && e == cudaSuccess) {
            double l = 0;
            e = cudaMemcpyAsync(&l, dL, sizeof(double), cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            loss_per_epoch[ep] = l / n;
        }
    }
    std::vector<float> w(CL_N);
    if (e == cudaSuccess) e = cudaMemcpyAsync(w.data(), dw, sizeof(float) * CL_N, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cleanup();
    if (e != cudaSuccess) return err(FPCLBM_ERR_CUDA, std::string("closure_train: ") + cudaGetErrorString(e));
    // fold the standardisation into the first and last layers (raw inputs, raw output)
    std::vector<double> out(CL_N);
    for (int j = 0; j < 64; ++j) {
        double b = w[CL_B1 + j];
        for (int i = 0; i < 9; ++i) {
            const double wij = (double)w[CL_W1 + 9 * j + i] / sd[i];
            out[CL_W1 + 9 * j + i] = wij;
            b -= wij * mu[i];
        }
        out[CL_B1 + j] = b;
    }
    for (int i = 0; i < 4096; ++i) out[CL_W2 + i] = w[CL_W2 + i];
    for (int j = 0; j < 64; ++j) out[CL_B2 + j] = w[CL_B2 + j];
    for (int j = 0; j < 64; ++j) out[CL_W3 + j] = (double)w[CL_W3 + j] * sd[9];
    out[CL_B3] = (double)w[CL_B3] * sd[9] + mu[9];
    for (int i = 0; i < CL_N; ++i) out_w[i] = bf16_bits((float)out[i]);
    return FPCLBM_OK;
}
