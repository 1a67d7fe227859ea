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
#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

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
// periodic in x and z, periodic or one-sided at y walls), eddy viscosity from
// the sub-filter stress, label and features.
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
        if (!walls)
            gr[i][1] = 0.5 * (at(q, x, (y + 1) % cy, z) - at(q, x, (y - 1 + cy) % cy, z));
        else if (y == 0)
            gr[i][1] = at(q, x, 1, z) - at(q, x, 0, z);
        else if (y == cy - 1)
            gr[i][1] = at(q, x, cy - 1, z) - at(q, x, cy - 2, z);
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

constexpr int kB = 64;          // samples per block
constexpr int kPad = kB + 1;    // padded row length of the per-sample tables

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
    float* grad;                // fp32 gradient accumulator [4865]
    double* loss;               // fp64 sum of squared errors
};

// dynamic shared memory: weights (4868 floats) then per-sample tables
constexpr int kSmemFloats = 4868 + kPad * (9 + 64 * 4 + 1);

__global__ void __launch_bounds__(kB) k_cl_fwd_bwd(NetArgs a)
{
    extern __shared__ __align__(16) float sm[];
    float* sW = sm;                     // closure layout
    float* sX = sm + 4868;              // [9][kPad]
    float* sH1 = sX + 9 * kPad;         // [64][kPad]
    float* sH2 = sH1 + 64 * kPad;       // [64][kPad]
    float* sG2 = sH2 + 64 * kPad;       // [64][kPad]  dL/da2
    float* sG1 = sG2 + 64 * kPad;       // [64][kPad]  dL/da1
    float* sGY = sG1 + 64 * kPad;       // [kPad]      dL/dy
    __shared__ double sLoss[kB];

    for (int i = threadIdx.x; i < CL_N; i += kB) sW[i] = __bfloat162float(a.W[i]);
    __syncthreads();

    const int tid = threadIdx.x;
    const unsigned long long pos = a.first + (unsigned long long)blockIdx.x * kB + tid;
    const bool valid = pos < a.first + a.count;
    float x[9], t = 0.f;
    if (valid) {
        const unsigned long long idx = (a.perm_a * pos + a.perm_c) % a.n;
        for (int i = 0; i < 9; ++i) x[i] = (a.X[idx * 9 + i] - a.mu[i]) * a.inv_sd[i];
        t = (a.T[idx] - a.mu[9]) * a.inv_sd[9];
    } else {
        for (int i = 0; i < 9; ++i) x[i] = 0.f;
    }
    // layer 1 (h1 kept in registers with compile-time indices, and in shared memory)
    float h1[64];
#pragma unroll
    for (int j = 0; j < 64; ++j) {
        float s = sW[CL_B1 + j];
#pragma unroll
        for (int i = 0; i < 9; ++i) s = fmaf(sW[CL_W1 + 9 * j + i], x[i], s);
        h1[j] = tanhf(s);
        sH1[j * kPad + tid] = h1[j];
    }
    for (int i = 0; i < 9; ++i) sX[i * kPad + tid] = x[i];
    // layer 2 and output
    float y = sW[CL_B3];
    for (int j = 0; j < 64; ++j) {
        float s = sW[CL_B2 + j];
#pragma unroll
        for (int k = 0; k < 64; ++k) s = fmaf(sW[CL_W2 + 64 * j + k], h1[k], s);
        const float h = tanhf(s);
        sH2[j * kPad + tid] = h;
        y = fmaf(sW[CL_W3 + j], h, y);
    }
    const float err = valid ? (y - t) : 0.f;
    const float gy = a.scale * err;
    sLoss[tid] = (double)err * (double)err;
    sGY[tid] = gy;
    for (int j = 0; j < 64; ++j) {
        const float h = sH2[j * kPad + tid];
        sG2[j * kPad + tid] = gy * sW[CL_W3 + j] * (1.f - h * h);
    }
    // dL/dh1 = W2^T dL/da2, then through tanh
    for (int k = 0; k < 64; ++k) {
        float s = 0.f;
#pragma unroll 8
        for (int j = 0; j < 64; ++j) s = fmaf(sW[CL_W2 + 64 * j + k], sG2[j * kPad + tid], s);
        const float h = sH1[k * kPad + tid];
        sG1[k * kPad + tid] = s * (1.f - h * h);
    }
    __syncthreads();

    // parameter gradients summed over the block's samples
    for (int p = tid; p < CL_N; p += kB) {
        float s = 0.f;
        if (p < CL_B1) {  // W1[j][i]
            const int j = p / 9, i = p % 9;
            for (int m = 0; m < kB; ++m) s = fmaf(sG1[j * kPad + m], sX[i * kPad + m], s);
        } else if (p < CL_W2) {  // b1[j]
            const int j = p - CL_B1;
            for (int m = 0; m < kB; ++m) s += sG1[j * kPad + m];
        } else if (p < CL_B2) {  // W2[j][k]
            const int j = (p - CL_W2) / 64, k = (p - CL_W2) % 64;
            for (int m = 0; m < kB; ++m) s = fmaf(sG2[j * kPad + m], sH1[k * kPad + m], s);
        } else if (p < CL_W3) {  // b2[j]
            const int j = p - CL_B2;
            for (int m = 0; m < kB; ++m) s += sG2[j * kPad + m];
        } else if (p < CL_B3) {  // W3[j]
            const int j = p - CL_W3;
            for (int m = 0; m < kB; ++m) s = fmaf(sGY[m], sH2[j * kPad + m], s);
        } else {  // b3
            for (int m = 0; m < kB; ++m) s += sGY[m];
        }
        atomicAdd(a.grad + p, s);
    }
    if (tid == 0) {
        double l = 0;
        for (int m = 0; m < kB; ++m) l += sLoss[m];
        atomicAdd(a.loss, l);
    }
}

__global__ void k_cl_adam(float* w, float* m, float* v, float* grad, __nv_bfloat16* wb, float lr, float b1, float b2,
                          float c1, float c2, float eps)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= CL_N) return;
    const float g = grad[p];
    const float mm = b1 * m[p] + (1.f - b1) * g;
    const float vv = b2 * v[p] + (1.f - b2) * g * g;
    m[p] = mm;
    v[p] = vv;
    const float wn = w[p] - lr * (mm * c1) / (sqrtf(vv * c2) + eps);
    w[p] = wn;
    wb[p] = __float2bfloat16_rn(wn);
    grad[p] = 0.f;
}

__global__ void k_cl_stats(const float* X, const float* T, unsigned long long n, double* sums)
{
    // sums[0..9] = sum of column, sums[10..19] = sum of squares (column 9 = target)
    double s[10] = {0}, q[10] = {0};
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        for (int k = 0; k < 9; ++k) {
            const double v = X[i * 9 + k];
            s[k] += v;
            q[k] += v * v;
        }
        const double v = T[i];
        s[9] += v;
        q[9] += v * v;
    }
    for (int k = 0; k < 10; ++k) {
        atomicAdd(sums + k, s[k]);
        atomicAdd(sums + 10 + k, q[k]);
    }
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
        if (e_ != cudaSuccess) return err(FPCLBM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e_)); \
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
    cudaError_t e = cudaMalloc(&acc, sizeof(double) * 10 * nc);
    if (e == cudaSuccess && !on_device) {
        e = cudaMalloc(&dX, sizeof(float) * 9 * nc);
        if (e == cudaSuccess) e = cudaMalloc(&dT, sizeof(float) * nc);
    }
    if (e != cudaSuccess) {
        cudaFree(acc);
        if (!on_device) {
            cudaFree(dX != X ? dX : nullptr);
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
    cudaFree(acc);
    if (!on_device) {
        cudaFree(dX);
        cudaFree(dT);
    }
    if (e != cudaSuccess) return fail(h, FPCLBM_ERR_CUDA, std::string("closure_sample: ") + cudaGetErrorString(e));
    return FPCLBM_OK;
}

namespace {

// Run fwd/bwd over `count` samples starting at epoch position `first`.
cudaError_t run_batch(NetArgs a, cudaStream_t st)
{
    const size_t smem = sizeof(float) * kSmemFloats;
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_cl_fwd_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr = true;
    }
    const unsigned blocks = (unsigned)((a.count + kB - 1) / kB);
    k_cl_fwd_bwd<<<blocks, kB, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace

extern "C" int fpclbm_closure_grad(const float* X, const float* T, int n, const unsigned short* w, float* grad,
                                   double* loss, void* cuda_stream)
{
    g_create_error.clear();
    if (!X || !T || !w || !grad || !loss || n < 1) return err(FPCLBM_ERR_ARG, "closure_grad: bad arguments");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    __nv_bfloat16* dW = nullptr;
    float* dG = nullptr;
    double* dL = nullptr;
    cudaError_t e = cudaMalloc(&dW, sizeof(__nv_bfloat16) * CL_N);
    if (e == cudaSuccess) e = cudaMalloc(&dG, sizeof(float) * CL_N);
    if (e == cudaSuccess) e = cudaMalloc(&dL, sizeof(double));
    if (e != cudaSuccess) {
        cudaFree(dW);
        cudaFree(dG);
        cudaFree(dL);
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
    a.grad = dG;
    a.loss = dL;
    e = cudaMemcpyAsync(dW, w, sizeof(unsigned short) * CL_N, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(dG, 0, sizeof(float) * CL_N, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(dL, 0, sizeof(double), st);
    if (e == cudaSuccess) e = run_batch(a, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(grad, dG, sizeof(float) * CL_N, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(loss, dL, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(dW);
    cudaFree(dG);
    cudaFree(dL);
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
    FPC_CL_CK(cudaMalloc(&dS, sizeof(double) * 20), "closure_train stats");
    cudaMemsetAsync(dS, 0, sizeof(double) * 20, st);
    k_cl_stats<<<256, 256, 0, st>>>(X, T, (unsigned long long)n, dS);
    double sums[20];
    cudaError_t e = cudaMemcpyAsync(sums, dS, sizeof sums, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(dS);
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
    float *dw = nullptr, *dm = nullptr, *dv = nullptr, *dg = nullptr;
    __nv_bfloat16* dwb = nullptr;
    double* dL = nullptr;
    e = cudaMalloc(&dw, sizeof(float) * CL_N);
    if (e == cudaSuccess) e = cudaMalloc(&dm, sizeof(float) * CL_N);
    if (e == cudaSuccess) e = cudaMalloc(&dv, sizeof(float) * CL_N);
    if (e == cudaSuccess) e = cudaMalloc(&dg, sizeof(float) * CL_N);
    if (e == cudaSuccess) e = cudaMalloc(&dwb, sizeof(__nv_bfloat16) * CL_N);
    if (e == cudaSuccess) e = cudaMalloc(&dL, sizeof(double));
    auto cleanup = [&]() {
        cudaFree(dw);
        cudaFree(dm);
        cudaFree(dv);
        cudaFree(dg);
        cudaFree(dwb);
        cudaFree(dL);
    };
    if (e != cudaSuccess) {
        cleanup();
        return err(FPCLBM_ERR_ALLOC, "closure_train buffers");
    }
    e = cudaMemcpyAsync(dw, w0.data(), sizeof(float) * CL_N, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dwb, wb0.data(), sizeof(unsigned short) * CL_N, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(dm, 0, sizeof(float) * CL_N, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(dv, 0, sizeof(float) * CL_N, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(dg, 0, sizeof(float) * CL_N, st);
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
    a.grad = dg;
    a.loss = dL;
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
                k_cl_adam<<<(CL_N + 255) / 256, 256, 0, st>>>(dw, dm, dv, dg, dwb, (float)lr, b1, b2, c1, c2, 1e-8f);
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
