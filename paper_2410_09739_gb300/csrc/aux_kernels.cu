// aux_kernels.cu -- initialisation, field export, population I/O and fp64
// diagnostics of one box.  None of these is on the time-step hot path.  Fields
// and populations cross the boundary in fp64; the arithmetic is fp64 except
// where k_init_eq and k_moments state otherwise for fp32 and 16-bit storage.
#include "aux.cuh"
#include "internal.h"

namespace fpc {

// Velocity list of the paper (Sec. 3, D3Q27), alpha = 0..26, and the tensor
// slot (ex+1) + 3 (ey+1) + 9 (ez+1) of each alpha.
static const int kEx[27] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1};
static const int kEy[27] = {0, 0, 0, 1, -1, 0, 0, 1, 1, -1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, 1, -1, -1, 1, 1, -1, -1};
static const int kEz[27] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, 1, -1, -1, 1, 1, -1, -1, 1, 1, 1, 1, -1, -1, -1, -1};

#define FPC_SLOT(a) ((kEx[a] + 1) + 3 * (kEy[a] + 1) + 9 * (kEz[a] + 1))
const int kSlotOfAlpha[27] = {FPC_SLOT(0),  FPC_SLOT(1),  FPC_SLOT(2),  FPC_SLOT(3),  FPC_SLOT(4),  FPC_SLOT(5),
                              FPC_SLOT(6),  FPC_SLOT(7),  FPC_SLOT(8),  FPC_SLOT(9),  FPC_SLOT(10), FPC_SLOT(11),
                              FPC_SLOT(12), FPC_SLOT(13), FPC_SLOT(14), FPC_SLOT(15), FPC_SLOT(16), FPC_SLOT(17),
                              FPC_SLOT(18), FPC_SLOT(19), FPC_SLOT(20), FPC_SLOT(21), FPC_SLOT(22), FPC_SLOT(23),
                              FPC_SLOT(24), FPC_SLOT(25), FPC_SLOT(26)};
#undef FPC_SLOT

struct AlphaMap {
    int slot[27];   // tensor slot of each alpha
    int alpha[27];  // alpha of each tensor slot
};

static AlphaMap alpha_map()
{
    AlphaMap m;
    for (int a = 0; a < 27; ++a) {
        m.slot[a] = kSlotOfAlpha[a];
        m.alpha[kSlotOfAlpha[a]] = a;
    }
    return m;
}

// Equilibrium deviation f^eq(rho, u) - w in product form: per axis
// phi(0) = 2/3 - u^2, phi(+-1) = 1/6 + (u^2 +- u)/2, i.e. w1 + dphi; the
// product (w1x + ax)(w1y + ay)(w1z + az) - w1x w1y w1z is expanded so that
// only small terms are summed.  (Equal to C(u)^-1 kappa^eq with kappa^eq the
// Maxwellian central moments (1, 0, cs^2) per axis.)
//
// The arithmetic follows the storage type.  This GPU's fp64 pipe is a small
// fraction of its fp32 one, and the fp64 form below took ~220 fp64
// instructions per cell, which made the kernel fp64-bound (5.7 ms for 256^3)
// rather than bound by reading the fields.  FP64 storage keeps it.  FP32
// storage forms the three per-axis factors w1 + dphi in fp64 and then
// g = rho X Y Z - w with one fma per slot: the cancellation against w costs at
// most ~8 of fp64's 53 bits, far below the 24 bits stored.  16-bit storage
// evaluates the expanded form in fp32 (a few fp32 ulps of error against at
// most 11 stored bits).
template <typename S>
__global__ void k_init_eq(BoxGeom b, const double* rho, const double* ux, const double* uy, const double* uz,
                          unsigned c0, unsigned n)
{
    const unsigned i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const unsigned cell = c0 + i;
    if constexpr (std::is_same<S, float>::value) {
        const double r = rho[i], u[3] = {ux[i], uy[i], uz[i]};
        double X[3][3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const double v = u[d], v2 = v * v;
            X[d][0] = w1(0) + 0.5 * (v2 - v);
            X[d][1] = w1(1) - v2;
            X[d][2] = w1(2) + 0.5 * (v2 + v);
        }
        float* buf = static_cast<float*>(b.buf);
#pragma unroll
        for (int iz = 0; iz < 3; ++iz)
#pragma unroll
            for (int iy = 0; iy < 3; ++iy) {
                const double yz = X[1][iy] * X[2][iz];
#pragma unroll
                for (int ix = 0; ix < 3; ++ix) {
                    const int s = ix + 3 * iy + 9 * iz;
                    buf[(size_t)s * b.stride + cell] = (float)(r * (X[0][ix] * yz) - wslot(s));
                }
            }
        return;
    } else if constexpr (!std::is_same<S, double>::value) {
        const float dr = (float)(rho[i] - 1.0), u[3] = {(float)ux[i], (float)uy[i], (float)uz[i]};
        float dphi[3][3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const float v = u[d], v2 = v * v;
            dphi[d][0] = 0.5f * (v2 - v);
            dphi[d][1] = -v2;
            dphi[d][2] = 0.5f * (v2 + v);
        }
        S* buf = static_cast<S*>(b.buf);
#pragma unroll
        for (int s = 0; s < 27; ++s) {
            const int ix = s % 3, iy = (s / 3) % 3, iz = s / 9;
            const float A = (float)w1(ix), B = (float)w1(iy), C = (float)w1(iz);
            const float a = dphi[0][ix], bb = dphi[1][iy], c = dphi[2][iz];
            const float dprod = a * (B + bb) * (C + c) + A * (bb * (C + c) + B * c);
            Store<S>::st(buf + (size_t)s * b.stride + cell, dr * ((A + a) * (B + bb) * (C + c)) + dprod);
        }
        return;
    }
    const double r = rho[i], u[3] = {ux[i], uy[i], uz[i]};
    double dphi[3][3];
    for (int d = 0; d < 3; ++d) {
        const double v = u[d], v2 = v * v;
        dphi[d][0] = 0.5 * (v2 - v);
        dphi[d][1] = -v2;
        dphi[d][2] = 0.5 * (v2 + v);
    }
    S* buf = static_cast<S*>(b.buf);
    for (int s = 0; s < 27; ++s) {
        const int ix = s % 3, iy = (s / 3) % 3, iz = s / 9;
        const double A = w1(ix), B = w1(iy), C = w1(iz);
        const double a = dphi[0][ix], bb = dphi[1][iy], c = dphi[2][iz];
        // (A+a)(B+bb)(C+c) - ABC
        const double dprod = a * (B + bb) * (C + c) + A * (bb * (C + c) + B * c);
        const double feq_dev = (r - 1.0) * ((A + a) * (B + bb) * (C + c)) + dprod;
        buf[(size_t)s * b.stride + cell] = Store<S>::fromd(feq_dev);
    }
}

// Density and half-force velocity (Step 7) of every cell, in fp64.  For fp32
// and 16-bit storage the 27 deviations are summed in fp32 with compensation
// (sum2_add), which gives the fp64 sums in all but the last bits at fp32 cost,
// and the three divisions by rho become one reciprocal: the fp64 form below
// made the kernel fp64-bound on this GPU.  FP64 storage keeps the fp64 form.
template <typename S>
__global__ void k_moments(BoxGeom b, int parity, double Fx, double Fy, double Fz, double* rho, double* ux,
                          double* uy, double* uz, unsigned c0, unsigned n)
{
    const unsigned i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if constexpr (!std::is_same<S, double>::value) {
        float g[27];
        load_cell<S>(b, parity, c0 + i, g);
        float ds = 0.f, dc = 0.f, xs = 0.f, xc = 0.f, ys = 0.f, yc = 0.f, zs = 0.f, zc = 0.f;
#pragma unroll
        for (int s = 0; s < 27; ++s) {
            const int ex = s % 3 - 1, ey = (s / 3) % 3 - 1, ez = s / 9 - 1;
            sum2_add(ds, dc, g[s]);
            if (ex != 0) sum2_add(xs, xc, ex > 0 ? g[s] : -g[s]);
            if (ey != 0) sum2_add(ys, yc, ey > 0 ? g[s] : -g[s]);
            if (ez != 0) sum2_add(zs, zc, ez > 0 ? g[s] : -g[s]);
        }
        const double r = 1.0 + ((double)ds + (double)dc), inv = 1.0 / r;
        if (rho) rho[i] = r;
        if (ux) ux[i] = ((double)xs + (double)xc + 0.5 * Fx) * inv;
        if (uy) uy[i] = ((double)ys + (double)yc + 0.5 * Fy) * inv;
        if (uz) uz[i] = ((double)zs + (double)zc + 0.5 * Fz) * inv;
        return;
    }
    double g[27];
    load_cell<S>(b, parity, c0 + i, g);
    double dr = 0, jx = 0, jy = 0, jz = 0;
#pragma unroll
    for (int s = 0; s < 27; ++s) {
        dr += g[s];
        jx += (s % 3 - 1) * g[s];
        jy += ((s / 3) % 3 - 1) * g[s];
        jz += (s / 9 - 1) * g[s];
    }
    const double r = 1.0 + dr;
    if (rho) rho[i] = r;
    if (ux) ux[i] = (jx + 0.5 * Fx) / r;
    if (uy) uy[i] = (jy + 0.5 * Fy) / r;
    if (uz) uz[i] = (jz + 0.5 * Fz) / r;
}

template <typename S>
__global__ void k_get_pops(BoxGeom b, AlphaMap am, int parity, double* out, unsigned ld, unsigned c0, unsigned n)
{
    const unsigned i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double g[27];
    load_cell<S>(b, parity, c0 + i, g);
#pragma unroll
    for (int s = 0; s < 27; ++s) out[(size_t)am.alpha[s] * ld + i] = wslot(s) + g[s];
}

template <typename S>
__global__ void k_get_pops_at(BoxGeom b, AlphaMap am, int parity, const unsigned* cells, unsigned n, double* out)
{
    const unsigned i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const unsigned cell = cells[i];
    if (cell >= b.ncells) return;
    double g[27];
    load_cell<S>(b, parity, cell, g);
#pragma unroll
    for (int s = 0; s < 27; ++s) out[(size_t)am.alpha[s] * n + i] = wslot(s) + g[s];
}

template <typename S>
__global__ void k_set_pops(BoxGeom b, AlphaMap am, const double* in, unsigned ld, unsigned c0, unsigned n)
{
    const unsigned i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    S* buf = static_cast<S*>(b.buf);
    for (int a = 0; a < 27; ++a) {
        const int s = am.slot[a];
        buf[(size_t)s * b.stride + c0 + i] = Store<S>::fromd(in[(size_t)a * ld + i] - wslot(s));
    }
}

// Diagnostics: per-block sums of (rho, rho u, rho |u|^2 / 2) in fp64 with a
// fixed tree order, then one block sums the partials in index order.
constexpr int kDiagThreads = 256;

int diag_blocks(unsigned ncells)
{
    const unsigned per = kDiagThreads * 8u;
    unsigned nb = (ncells + per - 1) / per;
    return (int)(nb < 1 ? 1 : nb);
}

template <typename S>
__global__ void __launch_bounds__(kDiagThreads) k_diag_partial(BoxGeom b, int parity, double Fx, double Fy,
                                                               double Fz, double* part)
{
    __shared__ double sh[5][kDiagThreads];
    double acc[5] = {0, 0, 0, 0, 0};
    const unsigned base = blockIdx.x * kDiagThreads * 8u;
    for (int k = 0; k < 8; ++k) {
        const unsigned cell = base + k * kDiagThreads + threadIdx.x;
        if (cell >= b.ncells) break;
        double g[27];
        load_cell<S>(b, parity, cell, g);
        double dr = 0, jx = 0, jy = 0, jz = 0;
#pragma unroll
        for (int s = 0; s < 27; ++s) {
            dr += g[s];
            jx += (s % 3 - 1) * g[s];
            jy += ((s / 3) % 3 - 1) * g[s];
            jz += (s / 9 - 1) * g[s];
        }
        const double r = 1.0 + dr;
        const double mx = jx + 0.5 * Fx, my = jy + 0.5 * Fy, mz = jz + 0.5 * Fz;  // rho u
        acc[0] += r;
        acc[1] += mx;
        acc[2] += my;
        acc[3] += mz;
        acc[4] += 0.5 * (mx * mx + my * my + mz * mz) / r;
    }
    for (int q = 0; q < 5; ++q) sh[q][threadIdx.x] = acc[q];
    __syncthreads();
    for (int w = kDiagThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < (unsigned)w)
            for (int q = 0; q < 5; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int q = 0; q < 5; ++q) part[(size_t)5 * blockIdx.x + q] = sh[q][0];
}

__global__ void __launch_bounds__(kDiagThreads) k_diag_final(const double* part, int nblocks, double* out)
{
    __shared__ double sh[5][kDiagThreads];
    double acc[5] = {0, 0, 0, 0, 0};
    for (int i = threadIdx.x; i < nblocks; i += kDiagThreads)
        for (int q = 0; q < 5; ++q) acc[q] += part[(size_t)5 * i + q];
    for (int q = 0; q < 5; ++q) sh[q][threadIdx.x] = acc[q];
    __syncthreads();
    for (int w = kDiagThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < (unsigned)w)
            for (int q = 0; q < 5; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int q = 0; q < 5; ++q) out[q] = sh[q][0];
}

// ---------------------------------------------------------------------------
// dispatch
// ---------------------------------------------------------------------------

#define FPC_DISPATCH(prec, KCALL)                                   \
    switch (prec) {                                                 \
        case P_FP64: { using S = double; KCALL; break; }            \
        case P_FP32: { using S = float; KCALL; break; }             \
        case P_FP16: { using S = __half; KCALL; break; }            \
        case P_BF16: { using S = __nv_bfloat16; KCALL; break; }     \
        default: return cudaErrorInvalidValue;                      \
    }

static inline unsigned blocks_for(unsigned n, int t) { return (n + t - 1) / t; }

cudaError_t launch_init_eq(int precision, const BoxGeom& b, const double* rho, const double* ux, const double* uy,
                           const double* uz, unsigned c0, unsigned n, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    FPC_DISPATCH(precision, (k_init_eq<S><<<blocks_for(n, 256), 256, 0, st>>>(b, rho, ux, uy, uz, c0, n)));
    return cudaGetLastError();
}

cudaError_t launch_moments(int precision, const BoxGeom& b, int parity, double Fx, double Fy, double Fz, double* rho,
                           double* ux, double* uy, double* uz, unsigned c0, unsigned n, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    FPC_DISPATCH(precision,
                 (k_moments<S><<<blocks_for(n, 256), 256, 0, st>>>(b, parity, Fx, Fy, Fz, rho, ux, uy, uz, c0, n)));
    return cudaGetLastError();
}

cudaError_t launch_get_pops(int precision, const BoxGeom& b, int parity, double* out, unsigned ld, unsigned c0,
                            unsigned n, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    const AlphaMap am = alpha_map();
    FPC_DISPATCH(precision, (k_get_pops<S><<<blocks_for(n, 128), 128, 0, st>>>(b, am, parity, out, ld, c0, n)));
    return cudaGetLastError();
}

cudaError_t launch_get_pops_at(int precision, const BoxGeom& b, int parity, const unsigned* cells, unsigned n,
                               double* out, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    const AlphaMap am = alpha_map();
    FPC_DISPATCH(precision, (k_get_pops_at<S><<<blocks_for(n, 128), 128, 0, st>>>(b, am, parity, cells, n, out)));
    return cudaGetLastError();
}

cudaError_t launch_set_pops(int precision, const BoxGeom& b, const double* in, unsigned ld, unsigned c0, unsigned n,
                            cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    const AlphaMap am = alpha_map();
    FPC_DISPATCH(precision, (k_set_pops<S><<<blocks_for(n, 128), 128, 0, st>>>(b, am, in, ld, c0, n)));
    return cudaGetLastError();
}

cudaError_t launch_diag_partial(int precision, const BoxGeom& b, int parity, double Fx, double Fy, double Fz,
                                double* part, cudaStream_t st)
{
    const int nb = diag_blocks(b.ncells);
    FPC_DISPATCH(precision, (k_diag_partial<S><<<nb, kDiagThreads, 0, st>>>(b, parity, Fx, Fy, Fz, part)));
    return cudaGetLastError();
}

cudaError_t launch_diag_final(const double* part, int nparts, double* out, cudaStream_t st)
{
    k_diag_final<<<1, kDiagThreads, 0, st>>>(part, nparts, out);
    return cudaGetLastError();
}

}  // namespace fpc
