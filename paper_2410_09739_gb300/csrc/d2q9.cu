// d2q9.cu -- the 2D FPC-LBM on the D2Q9 lattice (Sec. 2 and the appendix on
// the 2D algorithm): kernels and the fpclbm2d_* entry points.
//
// Layout and update scheme as in 3D (see common.cuh, cell.cuh): one buffer
// buf[s * stride + cell], tensor slot s = (ex+1) + 3 (ey+1), cell = x + nx y,
// deviations g = f - w from the rest weights w = w1(ex) w1(ey) (4/9, 1/9,
// 1/36), AA pattern in place (even step: own slots -> opposite slot 8 - s;
// odd step: neighbour gather / scatter), periodic in x and y or a closed
// square box (half-way bounce-back on all four sides, the wall y = ny - 1/2
// moving along x: the 2D lid-driven cavity of Sec. 4, handled as in 3D, see
// cell.cuh).  One thread per cell: 9 loads, the collision in registers, 9
// stores.
//
// Collision (Step 3 of the 2D appendix) in deviation form: the central
// moments come from two 3-point passes (y lines, then x lines; see fwd3 in
// collide.cuh), the groups 2s = 20 + 02 (rate omega_3, bulk), 2d = 20 - 02
// (omega_4) and 11 (omega_5) relax toward c_s^2 rho delta, 21 and 12
// (omega_6, omega_7) toward 0 with the sources of Eq. (sourceCM2D), and 22
// (omega_8) toward (k~20 k~02 + 2 k~11^2) / rho built from the relaxed second
// moments (FP mode) or toward c_s^4 rho (MCM mode).  First-order moments
// enter sources as 0; the force enters kappa_10, kappa_01 directly (as in 3D).
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "rtalloc.h"
#include "collide.cuh"
#include "fpclbm.h"
#include "hostmem.h"
#include "internal.h"

namespace fpc {
namespace {

template <typename R>
struct Rates2 {
    R om[9], keep[9], src[9];
};

template <typename R>
struct Args2 {
    void* buf;
    unsigned stride, ncells;
    int nx, ny;
    FastDiv div_nx;
    R Fx, Fy;
    R lid6;  // 6 x the velocity of the wall y = ny - 1/2 (closed box)
    Rates2<R> rt;
    int* flag;
};

// 1D rest weights and rest central moments per axis index i = e + 1.
__host__ __device__ constexpr double w1d(int i) { return i == 1 ? 2.0 / 3.0 : 1.0 / 6.0; }
__host__ __device__ constexpr double r1d(int k) { return k == 0 ? 1.0 : (k == 1 ? 0.0 : 1.0 / 3.0); }

template <typename R, bool FORCE, int MODE>
__device__ __forceinline__ bool collide2(R (&g)[9], const Rates2<R>& rt, R Fx, R Fy)
{
    // y lines at fixed ix: sums give rho and j
    R S[3], Dy[3], Py[3];
#pragma unroll
    for (int ix = 0; ix < 3; ++ix) {
        Py[ix] = g[ix] + g[ix + 6];
        Dy[ix] = g[ix + 6] - g[ix];
        S[ix] = Py[ix] + g[ix + 3];
    }
    const R drho = (S[0] + S[1]) + S[2];
    const R jx = S[2] - S[0];
    const R jy = (Dy[0] + Dy[1]) + Dy[2];
    const R rho = R(1) + drho;
    const R inv_rho = R(1) / rho;
    const bool ok = (rho > R(0)) && (rho < R(1e30));
    const R ux = (FORCE ? fmaR(R(0.5), Fx, jx) : jx) * inv_rho;
    const R uy = (FORCE ? fmaR(R(0.5), Fy, jy) : jy) * inv_rho;
    const R ux2 = ux * ux, uy2 = uy * uy, tux = R(2) * ux, tuy = R(2) * uy;
#pragma unroll
    for (int ix = 0; ix < 3; ++ix) {
        const R U = R(w1d(ix)) + S[ix];
        g[ix] = S[ix];
        g[ix + 3] = fmaR(-uy, U, Dy[ix]);
        g[ix + 6] = fmaR(uy2, U, fmaR(-tuy, Dy[ix], Py[ix]));
    }
    // x lines at fixed n
    fwd3<R, false>(g[0], g[1], g[2], ux, ux2, tux, R(1));
    fwd3<R, true>(g[3], g[4], g[5], ux, ux2, tux, R(0));
    fwd3<R, false>(g[6], g[7], g[8], ux, ux2, tux, R(1.0 / 3.0));
    // now g[m + 3n] = kappa_mn - r_m r_n

    const R third = R(1.0 / 3.0), ninth = R(1.0 / 9.0);
    R fx = R(0), fy = R(0), s21 = R(0), s12 = R(0), s22 = R(0);
    if (FORCE) {
        fx = Fx * inv_rho;
        fy = Fy * inv_rho;
        const R k20 = third + g[2], k02 = third + g[6], k11 = g[4];
        s21 = fmaR(R(2) * fx, k11, fy * k20);
        s12 = fmaR(fx, k02, R(2) * fy * k11);
        s22 = R(2) * fmaR(fx, g[7], fy * g[5]);  // 2 (Fx/rho k12 + Fy/rho k21); k12 at g[7], k21 at g[5]
        g[1] += Fx;
        g[3] += Fy;
    }
    // order 2: 2s (attractor deviation 2/3 drho), 2d and 11 (attractor 0)
    {
        const R y2s = g[2] + g[6], y2d = g[2] - g[6];
        const R t2s = fmaR(rt.om[3], R(2.0 / 3.0) * drho, rt.keep[3] * y2s);
        const R t2d = rt.keep[4] * y2d;
        g[4] = rt.keep[5] * g[4];
        g[2] = R(0.5) * (t2s + t2d);
        g[6] = R(0.5) * (t2s - t2d);
    }
    // order 3 (attractors 0): 21 at g[5], 12 at g[7]
    g[5] = rt.keep[6] * g[5];
    g[7] = rt.keep[7] * g[7];
    if (FORCE) {
        g[5] = fmaR(rt.src[6], s21, g[5]);
        g[7] = fmaR(rt.src[7], s12, g[7]);
    }
    // order 4
    {
        R A22;
        if constexpr (MODE == MODE_EQ) {
            A22 = ninth * drho;  // cs^4 rho - 1/9
        } else {
            const R pa = g[2], pb = g[6], o = g[4];
            A22 = (fmaR(third, pa + pb, fmaR(pa, pb, R(2) * o * o)) - ninth * drho) * inv_rho;
        }
        R t = fmaR(rt.om[8], A22, rt.keep[8] * g[8]);
        if (FORCE) t = fmaR(rt.src[8], s22, t);
        g[8] = t;
    }
    // back: x lines, then y lines
    inv3<R, false>(g[0], g[1], g[2], ux, ux2, tux, R(1));
    inv3<R, true>(g[3], g[4], g[5], ux, ux2, tux, R(0));
    inv3<R, false>(g[6], g[7], g[8], ux, ux2, tux, R(1.0 / 3.0));
#pragma unroll
    for (int ix = 0; ix < 3; ++ix) inv3<R, false>(g[ix], g[ix + 3], g[ix + 6], uy, uy2, tuy, R(w1d(ix)));
    return ok;
}

template <typename S, typename R, bool ODD, bool FORCE, int MODE, bool BOX>
__global__ void __launch_bounds__(256) k_step2d(const Args2<R> a)
{
    const unsigned cell = blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= a.ncells) return;
    S* __restrict__ buf = static_cast<S*>(a.buf);
    const unsigned stride = a.stride, nx = a.nx, ny = a.ny;
    unsigned xs[3], ys[3];  // column / row offset of x - e for e = -1, 0, +1
    bool xin[3] = {true, true, true}, yin[3] = {true, true, true};  // x - e inside the box
    unsigned y = 0;
    if (ODD || BOX) y = fdiv(cell, a.div_nx);
    if (ODD) {
        const unsigned x = cell - y * nx;
        xs[0] = (x + 1 == nx) ? 0u : x + 1;
        xs[1] = x;
        xs[2] = (x == 0) ? nx - 1 : x - 1;
        ys[0] = ((y + 1 == ny) ? 0u : y + 1) * nx;
        ys[1] = y * nx;
        ys[2] = ((y == 0) ? ny - 1 : y - 1) * nx;
        if (BOX) {
            xin[0] = x + 1 < nx;
            xin[2] = x > 0;
            yin[0] = y + 1 < ny;
            yin[2] = y > 0;
        }
    }
    R g[9];
#pragma unroll
    for (int s = 0; s < 9; ++s) {
        const int ix = s % 3, iy = s / 3;
        const S* p;
        if (!ODD || (BOX && !(xin[ix] && yin[iy])))  // even step, or bounce-back
            p = buf + (size_t)s * stride + cell;
        else
            p = buf + (size_t)(8 - s) * stride + (xs[ix] + ys[iy]);
        g[s] = Store<S>::ld(p);
    }
    const bool ok = collide2<R, FORCE, MODE>(g, a.rt, a.Fx, a.Fy);
    if (!ok) atomicOr(a.flag, 1);
    if (BOX && y + 1 == ny) {  // moving wall: -2 w_s rho e_sx u_w / cs^2 on the three e_y = +1 slots
        R rho = R(1);
#pragma unroll
        for (int s = 0; s < 9; ++s) rho += g[s];
        g[6] -= R(w1d(0) * w1d(2)) * rho * (-a.lid6);
        g[8] -= R(w1d(2) * w1d(2)) * rho * a.lid6;
    }
#pragma unroll
    for (int s = 0; s < 9; ++s) {
        const int ix = s % 3, iy = s / 3;
        S* p;
        if (!ODD || (BOX && !(xin[2 - ix] && yin[2 - iy])))  // even step, or bounce-back
            p = buf + (size_t)(8 - s) * stride + cell;
        else
            p = buf + (size_t)s * stride + (xs[2 - ix] + ys[2 - iy]);
        Store<S>::st(p, g[s]);
    }
}

// Deviations at the current time whatever the AA parity (as aux.cuh in 3D).
template <typename S>
__device__ void load2(const void* bufv, unsigned stride, int nx, int ny, int box, int parity, unsigned cell,
                      double g[9])
{
    const S* buf = static_cast<const S*>(bufv);
    if (parity == 0) {
        for (int s = 0; s < 9; ++s) g[s] = Store<S>::ldd(buf + (size_t)s * stride + cell);
        return;
    }
    const int y = (int)(cell / (unsigned)nx), x = (int)(cell - (unsigned)y * nx);
    for (int s = 0; s < 9; ++s) {
        const int ex = s % 3 - 1, ey = s / 3 - 1;
        if (box && (x - ex < 0 || x - ex >= nx || y - ey < 0 || y - ey >= ny)) {  // bounce-back
            g[s] = Store<S>::ldd(buf + (size_t)s * stride + cell);
            continue;
        }
        const int sx = (x - ex + nx) % nx, sy = (y - ey + ny) % ny;
        g[s] = Store<S>::ldd(buf + (size_t)(8 - s) * stride + (size_t)sx + (size_t)nx * sy);
    }
}

// Product-form equilibrium deviation (equal to C(u)^-1 kappa^eq with the
// Maxwellian central moments (1, 0, cs^2) per axis, times rho).
template <typename S>
__global__ void k_init2d(void* bufv, unsigned stride, unsigned n, const double* rho, const double* ux,
                         const double* uy)
{
    const unsigned c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    const double r = rho[c], u[2] = {ux[c], uy[c]};
    double dphi[2][3];
    for (int d = 0; d < 2; ++d) {
        const double v = u[d], v2 = v * v;
        dphi[d][0] = 0.5 * (v2 - v);
        dphi[d][1] = -v2;
        dphi[d][2] = 0.5 * (v2 + v);
    }
    S* buf = static_cast<S*>(bufv);
    for (int s = 0; s < 9; ++s) {
        const int ix = s % 3, iy = s / 3;
        const double A = w1d(ix), B = w1d(iy), a = dphi[0][ix], b = dphi[1][iy];
        const double dprod = a * (B + b) + A * b;  // (A+a)(B+b) - AB
        buf[(size_t)s * stride + c] = Store<S>::fromd((r - 1.0) * ((A + a) * (B + b)) + dprod);
    }
}

template <typename S>
__global__ void k_moments2d(const void* buf, unsigned stride, int nx, int ny, int box, unsigned n, int parity,
                            double Fx, double Fy, double* rho, double* ux, double* uy)
{
    const unsigned c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    double g[9];
    load2<S>(buf, stride, nx, ny, box, parity, c, g);
    double dr = 0, jx = 0, jy = 0;
    for (int s = 0; s < 9; ++s) {
        dr += g[s];
        jx += (s % 3 - 1) * g[s];
        jy += (s / 3 - 1) * g[s];
    }
    const double r = 1.0 + dr;
    if (rho) rho[c] = r;
    if (ux) ux[c] = (jx + 0.5 * Fx) / r;
    if (uy) uy[c] = (jy + 0.5 * Fy) / r;
}

// alpha order of Sec. 2 -> tensor slot
__constant__ int c_slot2[9];
const int kEx2[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
const int kEy2[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};

template <typename S>
__global__ void k_get_pops2d(const void* buf, unsigned stride, int nx, int ny, int box, unsigned n, int parity,
                             double* out)
{
    const unsigned c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    double g[9];
    load2<S>(buf, stride, nx, ny, box, parity, c, g);
    for (int a = 0; a < 9; ++a) {
        const int s = c_slot2[a];
        out[(size_t)a * n + c] = w1d(s % 3) * w1d(s / 3) + g[s];
    }
}

template <typename S>
__global__ void k_set_pops2d(void* bufv, unsigned stride, unsigned n, const double* in)
{
    const unsigned c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    S* buf = static_cast<S*>(bufv);
    for (int a = 0; a < 9; ++a) {
        const int s = c_slot2[a];
        buf[(size_t)s * stride + c] = Store<S>::fromd(in[(size_t)a * n + c] - w1d(s % 3) * w1d(s / 3));
    }
}

template <typename S, typename R, bool BOX>
cudaError_t step2d_go(int odd, int force, int mode, const Args2<R>& a, cudaStream_t st)
{
    const unsigned grid = (a.ncells + 255) / 256;
#define FPC2_K(O, FO, M) k_step2d<S, R, O, FO, M, BOX><<<grid, 256, 0, st>>>(a)
    if (odd) {
        if (force) { if (mode == MODE_EQ) FPC2_K(true, true, MODE_EQ); else FPC2_K(true, true, MODE_FP); }
        else { if (mode == MODE_EQ) FPC2_K(true, false, MODE_EQ); else FPC2_K(true, false, MODE_FP); }
    } else {
        if (force) { if (mode == MODE_EQ) FPC2_K(false, true, MODE_EQ); else FPC2_K(false, true, MODE_FP); }
        else { if (mode == MODE_EQ) FPC2_K(false, false, MODE_EQ); else FPC2_K(false, false, MODE_FP); }
    }
#undef FPC2_K
    return cudaGetLastError();
}

constexpr int kGraph2 = 32;

}  // namespace
}  // namespace fpc

using namespace fpc;

struct fpclbm2d {
    int nx = 0, ny = 0, precision = 0;
    unsigned ncells = 0, stride = 0;
    cudaStream_t stream = nullptr, cap = nullptr;
    void* d_pop = nullptr;
    int* d_flag = nullptr;
    int* h_flag = nullptr;
    double omega[9];
    double F[2] = {0, 0};
    int diffusion = FPCLBM_DIFF_FP;
    int bc = FPCLBM_BC_PERIODIC;
    double lid = 0;
    long long steps = 0;
    bool initialized = false;
    cudaGraphExec_t graph = nullptr;
    bool graph_valid = false;
    std::string err;
};

namespace {

thread_local std::string g_err2;

int fail2(fpclbm2d* h, int code, const std::string& m)
{
    h->err = m;
    return code;
}

#define FPC2_CK(h, call, what)                                                                     \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) return fail2(h, FPCLBM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e_)); \
    } while (0)

size_t esize2(int p) { return p == FPCLBM_FP64 ? 8 : p == FPCLBM_FP32 ? 4 : 2; }

template <typename R>
Args2<R> args_of(const fpclbm2d* h)
{
    Args2<R> a;
    a.buf = h->d_pop;
    a.stride = h->stride;
    a.ncells = h->ncells;
    a.nx = h->nx;
    a.ny = h->ny;
    a.div_nx = make_fastdiv((unsigned)h->nx);
    a.Fx = (R)h->F[0];
    a.Fy = (R)h->F[1];
    a.lid6 = (R)(6.0 * h->lid);
    for (int j = 0; j < 9; ++j) {
        a.rt.om[j] = (R)h->omega[j];
        a.rt.keep[j] = (R)(1.0 - h->omega[j]);
        a.rt.src[j] = (R)(1.0 - 0.5 * h->omega[j]);
    }
    a.flag = h->d_flag;
    return a;
}

cudaError_t one_step2(fpclbm2d* h, long long t, cudaStream_t st)
{
    const int odd = (int)(t & 1), force = h->F[0] != 0.0 || h->F[1] != 0.0;
    const int mode = h->diffusion == FPCLBM_DIFF_EQUILIBRIUM ? MODE_EQ : MODE_FP;
    const bool box = h->bc == FPCLBM_BC_BOX;
#define FPC2_GO(S, R) (box ? step2d_go<S, R, true>(odd, force, mode, args_of<R>(h), st) \
                           : step2d_go<S, R, false>(odd, force, mode, args_of<R>(h), st))
    switch (h->precision) {
        case FPCLBM_FP64: return FPC2_GO(double, double);
        case FPCLBM_FP32: return FPC2_GO(float, float);
        case FPCLBM_FP32_STORE_FP16: return FPC2_GO(__half, float);
        case FPCLBM_FP32_STORE_BF16: return FPC2_GO(__nv_bfloat16, float);
    }
#undef FPC2_GO
    return cudaErrorInvalidValue;
}

bool rates2_valid(const double om[9], std::string& why)
{
    for (int j = 3; j < 9; ++j)
        if (!(om[j] > 0.0 && om[j] < 2.0)) {
            why = "relaxation rate omega_" + std::to_string(j) + " outside (0, 2)";
            return false;
        }
    for (int j = 0; j < 3; ++j)
        if (!std::isfinite(om[j])) {
            why = "omega_0..2 must be finite";
            return false;
        }
    return true;
}

void drop_graph2(fpclbm2d* h)
{
    if (h->graph) cudaGraphExecDestroy(h->graph);
    h->graph = nullptr;
    h->graph_valid = false;
}

}  // namespace

extern "C" {

int fpclbm2d_create(fpclbm2d_t* out, int nx, int ny, int precision, void* cuda_stream)
{
    g_err2.clear();
    if (!out) return FPCLBM_ERR_ARG;
    *out = nullptr;
    if (nx < 1 || ny < 1 || (unsigned long long)nx * ny >= (1ull << 31)) {
        g_err2 = "need 1 <= nx, ny and nx * ny < 2^31";
        return FPCLBM_ERR_ARG;
    }
    if (precision < FPCLBM_FP64 || precision > FPCLBM_FP32_STORE_BF16) {
        g_err2 = "unknown precision";
        return FPCLBM_ERR_ARG;
    }
    fpclbm2d* h = new (std::nothrow) fpclbm2d();
    if (!h) return FPCLBM_ERR_ALLOC;
    h->nx = nx;
    h->ny = ny;
    h->ncells = (unsigned)nx * (unsigned)ny;
    h->stride = (h->ncells + 63) / 64 * 64;
    h->precision = precision;
    h->stream = static_cast<cudaStream_t>(cuda_stream);
    for (int j = 0; j < 9; ++j) h->omega[j] = 1.0;
    cudaError_t e = rt_malloc(&h->d_pop, 9ull * h->stride * esize2(precision));
    if (e == cudaSuccess) e = rt_malloc(&h->d_flag, sizeof(int));
    if (e == cudaSuccess) e = rt_malloc_host(&h->h_flag, sizeof(int));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMemset(h->d_flag, 0, sizeof(int));
    if (e != cudaSuccess) {
        g_err2 = std::string("allocation: ") + cudaGetErrorString(e);
        fpclbm2d_destroy(h);
        return FPCLBM_ERR_ALLOC;
    }
    *out = h;
    return FPCLBM_OK;
}

int fpclbm2d_destroy(fpclbm2d_t h)
{
    if (!h) return FPCLBM_OK;
    if (h->stream) cudaStreamSynchronize(h->stream);
    drop_graph2(h);
    if (h->d_pop) rt_free(h->d_pop);
    if (h->d_flag) rt_free(h->d_flag);
    if (h->h_flag) rt_free_host(h->h_flag);
    if (h->cap) cudaStreamDestroy(h->cap);
    delete h;
    return FPCLBM_OK;
}

const char* fpclbm2d_last_error(fpclbm2d_t h) { return h ? h->err.c_str() : g_err2.c_str(); }

int fpclbm2d_init_fields(fpclbm2d_t h, const double* rho, const double* ux, const double* uy, int on_device)
{
    if (!h) return FPCLBM_ERR_ARG;
    h->err.clear();
    if (!rho || !ux || !uy) return fail2(h, FPCLBM_ERR_ARG, "null field");
    const size_t n = h->ncells;
    double* d = nullptr;
    const double *pr = rho, *px = ux, *py = uy;
    if (!on_device) {  // page-locked host fields are read in place by the init kernel
        const double *mr = mapped_host(rho), *mx = mapped_host(ux), *my = mapped_host(uy);
        if (mr && mx && my) {
            pr = mr;
            px = mx;
            py = my;
            on_device = 1;
        }
    }
    if (!on_device) {
        FPC2_CK(h, rt_malloc(&d, 3 * n * sizeof(double)), "staging");
        cudaError_t ec = cudaMemcpyAsync(d, rho, n * sizeof(double), cudaMemcpyHostToDevice, h->stream);
        if (ec == cudaSuccess) ec = cudaMemcpyAsync(d + n, ux, n * sizeof(double), cudaMemcpyHostToDevice, h->stream);
        if (ec == cudaSuccess)
            ec = cudaMemcpyAsync(d + 2 * n, uy, n * sizeof(double), cudaMemcpyHostToDevice, h->stream);
        if (ec != cudaSuccess) {
            cudaStreamSynchronize(h->stream);
            rt_free(d);
            FPC2_CK(h, ec, "copy fields");
        }
        pr = d;
        px = d + n;
        py = d + 2 * n;
    }
    const unsigned blocks = (h->ncells + 255) / 256;
    cudaError_t e = cudaSuccess;
    switch (h->precision) {
        case FPCLBM_FP64: k_init2d<double><<<blocks, 256, 0, h->stream>>>(h->d_pop, h->stride, h->ncells, pr, px, py); break;
        case FPCLBM_FP32: k_init2d<float><<<blocks, 256, 0, h->stream>>>(h->d_pop, h->stride, h->ncells, pr, px, py); break;
        case FPCLBM_FP32_STORE_FP16: k_init2d<__half><<<blocks, 256, 0, h->stream>>>(h->d_pop, h->stride, h->ncells, pr, px, py); break;
        default: k_init2d<__nv_bfloat16><<<blocks, 256, 0, h->stream>>>(h->d_pop, h->stride, h->ncells, pr, px, py); break;
    }
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (d) rt_free(d);
    FPC2_CK(h, e, "init");
    h->steps = 0;
    h->initialized = true;
    return FPCLBM_OK;
}

int fpclbm2d_set_params(fpclbm2d_t h, double tau, double bulk_rate, double drift, int diffusion)
{
    if (!h) return FPCLBM_ERR_ARG;
    h->err.clear();
    if (diffusion != FPCLBM_DIFF_FP && diffusion != FPCLBM_DIFF_EQUILIBRIUM)
        return fail2(h, FPCLBM_ERR_ARG, "2D diffusion mode must be FP or EQUILIBRIUM");
    if (!std::isfinite(tau) || !std::isfinite(bulk_rate) || !std::isfinite(drift) || drift < 0 || bulk_rate < 0)
        return fail2(h, FPCLBM_ERR_ARG, "tau, bulk_rate, drift must be finite; bulk_rate, drift >= 0");
    double om[9];
    for (int j = 0; j < 9; ++j) om[j] = 1.0;
    om[3] = bulk_rate > 0 ? bulk_rate : 1.0;
    om[4] = om[5] = 1.0 / tau;
    om[6] = om[7] = drift > 0 ? 3.0 * drift : 1.0;
    om[8] = drift > 0 ? 4.0 * drift : 1.0;
    std::string why;
    if (!rates2_valid(om, why)) return fail2(h, FPCLBM_ERR_PARAM, why);
    std::memcpy(h->omega, om, sizeof om);
    h->diffusion = diffusion;
    h->graph_valid = false;
    return FPCLBM_OK;
}

int fpclbm2d_set_rates(fpclbm2d_t h, const double omega[9])
{
    if (!h) return FPCLBM_ERR_ARG;
    h->err.clear();
    if (!omega) return fail2(h, FPCLBM_ERR_ARG, "omega is NULL");
    std::string why;
    if (!rates2_valid(omega, why)) return fail2(h, FPCLBM_ERR_PARAM, why);
    std::memcpy(h->omega, omega, sizeof(double) * 9);
    h->graph_valid = false;
    return FPCLBM_OK;
}

int fpclbm2d_set_force(fpclbm2d_t h, double Fx, double Fy)
{
    if (!h) return FPCLBM_ERR_ARG;
    h->err.clear();
    if (!std::isfinite(Fx) || !std::isfinite(Fy)) return fail2(h, FPCLBM_ERR_ARG, "force must be finite");
    h->F[0] = Fx;
    h->F[1] = Fy;
    h->graph_valid = false;
    return FPCLBM_OK;
}

int fpclbm2d_set_boundary(fpclbm2d_t h, int bc, double lid_ux)
{
    if (!h) return FPCLBM_ERR_ARG;
    h->err.clear();
    if (bc != FPCLBM_BC_PERIODIC && bc != FPCLBM_BC_BOX) return fail2(h, FPCLBM_ERR_ARG, "2D boundary must be PERIODIC or BOX");
    if (!std::isfinite(lid_ux) || (bc == FPCLBM_BC_PERIODIC && lid_ux != 0.0))
        return fail2(h, FPCLBM_ERR_ARG, "lid velocity must be finite and needs the closed box");
    if (bc != h->bc && h->initialized && (h->steps & 1))
        return fail2(h, FPCLBM_ERR_STATE, "change the boundary at an even step count");
    h->bc = bc;
    h->lid = lid_ux;
    h->graph_valid = false;
    return FPCLBM_OK;
}

int fpclbm2d_step(fpclbm2d_t h, long long n)
{
    if (!h) return FPCLBM_ERR_ARG;
    h->err.clear();
    if (n < 0) return fail2(h, FPCLBM_ERR_ARG, "negative step count");
    if (!h->initialized) return fail2(h, FPCLBM_ERR_STATE, "populations not initialised");
    if (n == 0) return FPCLBM_OK;
    FPC2_CK(h, cudaMemsetAsync(h->d_flag, 0, sizeof(int), h->stream), "flag reset");
    long long done = 0;
    while (done < n && ((h->steps + done) & 1)) {
        FPC2_CK(h, one_step2(h, h->steps + done, h->stream), "step launch");
        ++done;
    }
    if (n - done >= kGraph2) {
        if (!h->graph_valid) {
            drop_graph2(h);
            cudaGraph_t g = nullptr;
            FPC2_CK(h, cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal), "capture begin");
            cudaError_t e = cudaSuccess;
            for (int k = 0; k < kGraph2 && e == cudaSuccess; ++k) e = one_step2(h, k, h->cap);
            cudaError_t e2 = cudaStreamEndCapture(h->cap, &g);
            if (e != cudaSuccess) {
                if (g) cudaGraphDestroy(g);
                FPC2_CK(h, e, "step launch during capture");
            }
            FPC2_CK(h, e2, "capture end");
            e = cudaGraphInstantiate(&h->graph, g, 0);
            cudaGraphDestroy(g);
            FPC2_CK(h, e, "graph instantiate");
            h->graph_valid = true;
        }
        while (n - done >= kGraph2) {
            FPC2_CK(h, cudaGraphLaunch(h->graph, h->stream), "graph launch");
            done += kGraph2;
        }
    }
    while (done < n) {
        FPC2_CK(h, one_step2(h, h->steps + done, h->stream), "step launch");
        ++done;
    }
    h->steps += n;
    FPC2_CK(h, cudaMemcpyAsync(h->h_flag, h->d_flag, sizeof(int), cudaMemcpyDeviceToHost, h->stream), "flag read");
    FPC2_CK(h, cudaStreamSynchronize(h->stream), "step sync");
    if (*h->h_flag) return fail2(h, FPCLBM_ERR_DIVERGED, "a cell reached rho <= 0 or a non-finite value");
    return FPCLBM_OK;
}

int fpclbm2d_moments(fpclbm2d_t h, double* rho, double* ux, double* uy, int on_device)
{
    if (!h) return FPCLBM_ERR_ARG;
    h->err.clear();
    if (!h->initialized) return fail2(h, FPCLBM_ERR_STATE, "populations not initialised");
    const size_t n = h->ncells;
    double* d = nullptr;
    double* o[3] = {rho, ux, uy};
    if (!on_device) {  // page-locked host outputs are written in place by the moments kernel
        double* m[3] = {mapped_host(rho), mapped_host(ux), mapped_host(uy)};
        if ((!rho || m[0]) && (!ux || m[1]) && (!uy || m[2])) {
            for (int k = 0; k < 3; ++k) o[k] = m[k];
            on_device = 1;
        }
    }
    if (!on_device) {
        FPC2_CK(h, rt_malloc(&d, 3 * n * sizeof(double)), "staging");
        for (int k = 0; k < 3; ++k) o[k] = o[k] ? d + k * n : nullptr;
    }
    const unsigned blocks = (h->ncells + 255) / 256;
    const int parity = (int)(h->steps & 1);
    switch (h->precision) {
        case FPCLBM_FP64: k_moments2d<double><<<blocks, 256, 0, h->stream>>>(h->d_pop, h->stride, h->nx, h->ny, h->bc == FPCLBM_BC_BOX, h->ncells, parity, h->F[0], h->F[1], o[0], o[1], o[2]); break;
        case FPCLBM_FP32: k_moments2d<float><<<blocks, 256, 0, h->stream>>>(h->d_pop, h->stride, h->nx, h->ny, h->bc == FPCLBM_BC_BOX, h->ncells, parity, h->F[0], h->F[1], o[0], o[1], o[2]); break;
        case FPCLBM_FP32_STORE_FP16: k_moments2d<__half><<<blocks, 256, 0, h->stream>>>(h->d_pop, h->stride, h->nx, h->ny, h->bc == FPCLBM_BC_BOX, h->ncells, parity, h->F[0], h->F[1], o[0], o[1], o[2]); break;
        default: k_moments2d<__nv_bfloat16><<<blocks, 256, 0, h->stream>>>(h->d_pop, h->stride, h->nx, h->ny, h->bc == FPCLBM_BC_BOX, h->ncells, parity, h->F[0], h->F[1], o[0], o[1], o[2]); break;
    }
    cudaError_t e = cudaGetLastError();
    double* host[3] = {rho, ux, uy};
    if (!on_device && e == cudaSuccess)
        for (int k = 0; k < 3 && e == cudaSuccess; ++k)
            if (host[k]) e = cudaMemcpyAsync(host[k], o[k], n * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (d) rt_free(d);
    FPC2_CK(h, e, "moments");
    return FPCLBM_OK;
}

int fpclbm2d_get_populations(fpclbm2d_t h, double* f)
{
    if (!h) return FPCLBM_ERR_ARG;
    h->err.clear();
    if (!f) return fail2(h, FPCLBM_ERR_ARG, "null output");
    if (!h->initialized) return fail2(h, FPCLBM_ERR_STATE, "populations not initialised");
    int slots[9];
    for (int a = 0; a < 9; ++a) slots[a] = (kEx2[a] + 1) + 3 * (kEy2[a] + 1);
    FPC2_CK(h, cudaMemcpyToSymbolAsync(c_slot2, slots, sizeof slots, 0, cudaMemcpyHostToDevice, h->stream), "slot table");
    const size_t n = h->ncells;
    double* d = nullptr;
    FPC2_CK(h, rt_malloc(&d, 9 * n * sizeof(double)), "staging");
    const unsigned blocks = (h->ncells + 255) / 256;
    const int parity = (int)(h->steps & 1);
    switch (h->precision) {
        case FPCLBM_FP64: k_get_pops2d<double><<<blocks, 256, 0, h->stream>>>(h->d_pop, h->stride, h->nx, h->ny, h->bc == FPCLBM_BC_BOX, h->ncells, parity, d); break;
        case FPCLBM_FP32: k_get_pops2d<float><<<blocks, 256, 0, h->stream>>>(h->d_pop, h->stride, h->nx, h->ny, h->bc == FPCLBM_BC_BOX, h->ncells, parity, d); break;
        case FPCLBM_FP32_STORE_FP16: k_get_pops2d<__half><<<blocks, 256, 0, h->stream>>>(h->d_pop, h->stride, h->nx, h->ny, h->bc == FPCLBM_BC_BOX, h->ncells, parity, d); break;
        default: k_get_pops2d<__nv_bfloat16><<<blocks, 256, 0, h->stream>>>(h->d_pop, h->stride, h->nx, h->ny, h->bc == FPCLBM_BC_BOX, h->ncells, parity, d); break;
    }
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(f, d, 9 * n * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    rt_free(d);
    FPC2_CK(h, e, "get populations");
    return FPCLBM_OK;
}

int fpclbm2d_set_populations(fpclbm2d_t h, const double* f)
{
    if (!h) return FPCLBM_ERR_ARG;
    h->err.clear();
    if (!f) return fail2(h, FPCLBM_ERR_ARG, "null input");
    int slots[9];
    for (int a = 0; a < 9; ++a) slots[a] = (kEx2[a] + 1) + 3 * (kEy2[a] + 1);
    FPC2_CK(h, cudaMemcpyToSymbolAsync(c_slot2, slots, sizeof slots, 0, cudaMemcpyHostToDevice, h->stream), "slot table");
    const size_t n = h->ncells;
    double* d = nullptr;
    FPC2_CK(h, rt_malloc(&d, 9 * n * sizeof(double)), "staging");
    cudaError_t e = cudaMemcpyAsync(d, f, 9 * n * sizeof(double), cudaMemcpyHostToDevice, h->stream);
    const unsigned blocks = (h->ncells + 255) / 256;
    if (e == cudaSuccess) {
        switch (h->precision) {
            case FPCLBM_FP64: k_set_pops2d<double><<<blocks, 256, 0, h->stream>>>(h->d_pop, h->stride, h->ncells, d); break;
            case FPCLBM_FP32: k_set_pops2d<float><<<blocks, 256, 0, h->stream>>>(h->d_pop, h->stride, h->ncells, d); break;
            case FPCLBM_FP32_STORE_FP16: k_set_pops2d<__half><<<blocks, 256, 0, h->stream>>>(h->d_pop, h->stride, h->ncells, d); break;
            default: k_set_pops2d<__nv_bfloat16><<<blocks, 256, 0, h->stream>>>(h->d_pop, h->stride, h->ncells, d); break;
        }
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    rt_free(d);
    FPC2_CK(h, e, "set populations");
    h->steps = 0;  // written in the even-parity layout
    h->initialized = true;
    return FPCLBM_OK;
}

}  // extern "C"
