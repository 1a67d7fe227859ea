// noalloc.cu -- fpclbm_diagnostics_noalloc: the fp64 diagnostics reduction for
// callers that cannot allocate device memory.
//
// Who needs it: code that runs inside a host application which owns all
// device memory through its own pool or arena (a plugin, a solver coupled to
// another code), or a loop whose latency budget forbids the implicit
// synchronisation of cudaMalloc/cudaFree.  Such callers hold device pointers
// to their inputs and outputs but must not create new allocations.
//
// The regular fpclbm_diagnostics keeps its block partials in a buffer the
// handle allocated.  This variant keeps them in a fixed file-scope device
// array instead, so it allocates nothing:
//   * the array holds kMaxBlocks partial sums (5 doubles each, 40 KB) and
//     lives on every device that loads the library until the process exits;
//   * host code must not use the array's name as a device address: at the
//     first call on a device (with that device current) the library asks the
//     runtime for the array's device address with cudaGetSymbolAddress and
//     caches it, so that first call should come before any stream capture;
//   * every call shares the array and overwrites only the partials it then
//     reads (nothing has to start at zero), so two calls that overlap on the
//     GPU race: order them on one stream or synchronise between them.
#include <cmath>
#include <cstdio>
#include <mutex>
#include <string>

#include "handle.h"

namespace fpc {
namespace {

constexpr int kThreads = 256;
constexpr int kMaxBlocks = 1024;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_partials[5 * kMaxBlocks];

std::mutex g_mu;
double* g_partials_addr[kMaxDevices] = {};

// Block partials of (rho, rho u, rho |u|^2 / 2) over cells c = blockIdx.x + k
// gridDim.x blocks of the grid-stride loop; f is alpha-major, full f.
__global__ void __launch_bounds__(kThreads) k_noalloc_partial(const double* __restrict__ f, unsigned long long n,
                                                              double Fx, double Fy, double Fz, double* part)
{
    // velocity components of the paper's alpha order (Sec. 3, D3Q27 list)
    const signed char ex[27] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1};
    const signed char ey[27] = {0, 0, 0, 1, -1, 0, 0, 1, 1, -1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, 1, -1, -1, 1, 1, -1, -1};
    const signed char ez[27] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, 1, -1, -1, 1, 1, -1, -1, 1, 1, 1, 1, -1, -1, -1, -1};
    __shared__ double sh[5][kThreads];
    double acc[5] = {0, 0, 0, 0, 0};
    for (unsigned long long c = (unsigned long long)blockIdx.x * kThreads + threadIdx.x; c < n;
         c += (unsigned long long)gridDim.x * kThreads) {
        double r = 0, jx = 0, jy = 0, jz = 0;
        for (int a = 0; a < 27; ++a) {
            const double v = f[(size_t)a * n + c];
            r += v;
            jx += ex[a] * v;
            jy += ey[a] * v;
            jz += ez[a] * v;
        }
        const double mx = jx + 0.5 * Fx, my = jy + 0.5 * Fy, mz = jz + 0.5 * Fz;
        acc[0] += r;
        acc[1] += mx;
        acc[2] += my;
        acc[3] += mz;
        acc[4] += 0.5 * (mx * mx + my * my + mz * mz) / r;
    }
    for (int q = 0; q < 5; ++q) sh[q][threadIdx.x] = acc[q];
    __syncthreads();
    for (int w = kThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < (unsigned)w)
            for (int q = 0; q < 5; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int q = 0; q < 5; ++q) part[5 * blockIdx.x + q] = sh[q][0];
}

__global__ void __launch_bounds__(kThreads) k_noalloc_final(const double* __restrict__ part, int nblocks, double* out)
{
    __shared__ double sh[5][kThreads];
    double acc[5] = {0, 0, 0, 0, 0};
    for (int i = threadIdx.x; i < nblocks; i += kThreads)
        for (int q = 0; q < 5; ++q) acc[q] += part[5 * i + q];
    for (int q = 0; q < 5; ++q) sh[q][threadIdx.x] = acc[q];
    __syncthreads();
    for (int w = kThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < (unsigned)w)
            for (int q = 0; q < 5; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int q = 0; q < 5; ++q) out[q] = sh[q][0];
}

// Device address of the partials array on the current device (set up once).
cudaError_t partials_address(double** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_partials_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_partials);
        if (e != cudaSuccess) return e;
        g_partials_addr[dev] = static_cast<double*>(p);
    }
    *out = g_partials_addr[dev];
    return cudaSuccess;
}

}  // namespace
}  // namespace fpc

using namespace fpc;

extern "C" int fpclbm_diagnostics_noalloc(const double* f, long long ncells, double Fx, double Fy, double Fz,
                                          double* out, void* cuda_stream)
{
    g_create_error.clear();
    if (!f || !out) {
        g_create_error = "diagnostics_noalloc: f and out must be device pointers";
        return FPCLBM_ERR_ARG;
    }
    if (ncells < 1 || ncells > FPCLBM_NOALLOC_MAX_CELLS) {
        g_create_error = "diagnostics_noalloc: ncells must be in [1, FPCLBM_NOALLOC_MAX_CELLS = 2^31 - 1]";
        return FPCLBM_ERR_ARG;
    }
    if (!std::isfinite(Fx) || !std::isfinite(Fy) || !std::isfinite(Fz)) {
        g_create_error = "diagnostics_noalloc: force must be finite";
        return FPCLBM_ERR_ARG;
    }
    double* part = nullptr;
    cudaError_t e = partials_address(&part);
    if (e != cudaSuccess) {
        g_create_error = std::string("diagnostics_noalloc: scratch address: ") + cudaGetErrorString(e);
        return FPCLBM_ERR_CUDA;
    }
    const unsigned long long n = (unsigned long long)ncells;
    unsigned long long nb = (n + kThreads - 1) / kThreads;
    const int blocks = (int)(nb < (unsigned long long)kMaxBlocks ? nb : kMaxBlocks);
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    k_noalloc_partial<<<blocks, kThreads, 0, st>>>(f, n, Fx, Fy, Fz, part);
    k_noalloc_final<<<1, kThreads, 0, st>>>(part, blocks, out);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        g_create_error = std::string("diagnostics_noalloc: launch: ") + cudaGetErrorString(e);
        return FPCLBM_ERR_CUDA;
    }
    return FPCLBM_OK;
}
