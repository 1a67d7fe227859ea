// fpclbm.cu -- host runtime and C ABI of libfpclbm.so (see include/fpclbm.h).
//
// A handle owns one population buffer (AA pattern, one copy), a divergence
// flag, staging buffers for host transfers, and a cached CUDA graph of the
// step loop.  Relaxation rates (Appendix D Step 3 numbering) and the body
// force live in the handle and are passed to every launch by value.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/fpclbm.h"
#include "internal.h"

using namespace fpc;

namespace {

thread_local std::string g_create_error;

constexpr int kGraphSteps = 32;           // steps per captured graph (even)
constexpr unsigned kChunk = 1u << 20;     // cells per host-transfer chunk

}  // namespace

struct fpclbm {
    // geometry
    int nx = 0, ny = 0, nz = 0;
    unsigned ncells = 0, stride = 0;
    int precision = 0, bc = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;
    int device = 0;
    // state
    void* d_pop = nullptr;
    int* d_flag = nullptr;
    int* h_flag = nullptr;  // pinned
    double* d_stage = nullptr;
    size_t stage_bytes = 0;
    double* d_part = nullptr;
    double* d_diag = nullptr;
    double* h_diag = nullptr;  // pinned
    float* d_closure = nullptr;
    bool have_closure = false;
    bool initialized = false;
    long long steps = 0;
    // parameters
    double omega[27];
    double F[3] = {0, 0, 0};
    int diffusion = FPCLBM_DIFF_FP;
    // launch config and graph cache
    StepLaunch launch{256};
    cudaGraphExec_t graph = nullptr;
    bool graph_valid = false;
    std::string err;
};

namespace {

int fail(fpclbm* h, int code, const std::string& msg)
{
    if (h) h->err = msg;
    return code;
}

int cuda_fail(fpclbm* h, cudaError_t e, const char* what)
{
    return fail(h, FPCLBM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define FPC_CK(h, call, what)                          \
    do {                                               \
        cudaError_t e_ = (call);                       \
        if (e_ != cudaSuccess) return cuda_fail(h, e_, what); \
    } while (0)

// Rates from (tau, drift): shear 1/tau on 4,5,6,8,9; bulk 1 on 7; 1 on 0..3;
// orders >= 3: k * drift, or 1 when drift == 0.
void rates_from_params(double tau, double drift, double om[27])
{
    static const int order[27] = {0, 1, 1, 1, 2, 2, 2, 2, 2, 2, 3, 3, 3, 3, 3, 3, 3, 4, 4, 4, 4, 4, 4, 5, 5, 5, 6};
    for (int j = 0; j < 27; ++j) {
        const int k = order[j];
        if (k <= 1) om[j] = 1.0;
        else if (k == 2) om[j] = 1.0 / tau;
        else om[j] = drift > 0 ? k * drift : 1.0;
    }
    om[7] = 1.0;
}

bool rates_valid(const double om[27], std::string& why)
{
    for (int j = 0; j < 27; ++j) {
        if (!std::isfinite(om[j])) {
            why = "omega_" + std::to_string(j) + " is not finite";
            return false;
        }
        if (j >= 4 && !(om[j] > 0.0 && om[j] < 2.0)) {
            char buf[96];
            std::snprintf(buf, sizeof buf, "omega_%d = %.17g outside (0, 2)", j, om[j]);
            why = buf;
            return false;
        }
    }
    return true;
}

template <typename R>
StepArgs<R> make_args(const fpclbm* h)
{
    StepArgs<R> a;
    a.buf = h->d_pop;
    a.stride = h->stride;
    a.ncells = h->ncells;
    a.nx = h->nx;
    a.ny = h->ny;
    a.nz = h->nz;
    a.div_nx = make_fastdiv((unsigned)h->nx);
    a.div_nxny = make_fastdiv((unsigned)(h->nx * h->ny));
    a.Fx = (R)h->F[0];
    a.Fy = (R)h->F[1];
    a.Fz = (R)h->F[2];
    for (int j = 0; j < 27; ++j) {
        a.rates.om[j] = (R)h->omega[j];
        a.rates.keep[j] = (R)(1.0 - h->omega[j]);
        a.rates.src[j] = (R)(1.0 - 0.5 * h->omega[j]);
    }
    a.flag = h->d_flag;
    a.closure = h->d_closure;
    return a;
}

BoxGeom geom_of(const fpclbm* h)
{
    BoxGeom b;
    b.buf = h->d_pop;
    b.stride = h->stride;
    b.ncells = h->ncells;
    b.nx = h->nx;
    b.ny = h->ny;
    b.nz = h->nz;
    b.walls = h->bc == FPCLBM_BC_WALLS_Y;
    b.div_nx = make_fastdiv((unsigned)h->nx);
    b.div_nxny = make_fastdiv((unsigned)(h->nx * h->ny));
    return b;
}

int mode_of(const fpclbm* h)
{
    if (h->diffusion == FPCLBM_DIFF_EQUILIBRIUM) return MODE_EQ;
    if (h->diffusion == FPCLBM_DIFF_FP_LEARNED) return MODE_LEARNED;
    return MODE_FP;
}

bool has_force(const fpclbm* h) { return h->F[0] != 0.0 || h->F[1] != 0.0 || h->F[2] != 0.0; }

cudaError_t one_step(fpclbm* h, long long t, cudaStream_t st)
{
    const StepArgs<double> a64 = make_args<double>(h);
    const StepArgs<float> a32 = make_args<float>(h);
    return launch_step(h->precision, (int)(t & 1), h->bc == FPCLBM_BC_WALLS_Y, has_force(h), mode_of(h), a64, a32,
                       h->launch, st);
}

void drop_graph(fpclbm* h)
{
    if (h->graph) cudaGraphExecDestroy(h->graph);
    h->graph = nullptr;
    h->graph_valid = false;
}

int build_graph(fpclbm* h)
{
    drop_graph(h);
    cudaGraph_t g = nullptr;
    FPC_CK(h, cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal), "graph capture begin");
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < kGraphSteps && e == cudaSuccess; ++k) e = one_step(h, k, h->cap_stream);
    cudaError_t e2 = cudaStreamEndCapture(h->cap_stream, &g);
    if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_fail(h, e, "step launch during capture");
    }
    FPC_CK(h, e2, "graph capture end");
    e = cudaGraphInstantiate(&h->graph, g, 0);
    cudaGraphDestroy(g);
    FPC_CK(h, e, "graph instantiate");
    h->graph_valid = true;
    return FPCLBM_OK;
}

int ensure_stage(fpclbm* h, size_t bytes)
{
    if (h->stage_bytes >= bytes) return FPCLBM_OK;
    if (h->d_stage) cudaFree(h->d_stage);
    h->d_stage = nullptr;
    h->stage_bytes = 0;
    cudaError_t e = cudaMalloc(&h->d_stage, bytes);
    if (e != cudaSuccess) return fail(h, FPCLBM_ERR_ALLOC, std::string("staging buffer: ") + cudaGetErrorString(e));
    h->stage_bytes = bytes;
    return FPCLBM_OK;
}

size_t elem_size(int precision)
{
    switch (precision) {
        case FPCLBM_FP64: return 8;
        case FPCLBM_FP32: return 4;
        default: return 2;
    }
}

}  // namespace

extern "C" {

int fpclbm_create(fpclbm_t* out, int nx, int ny, int nz, int precision, int bc, void* cuda_stream)
{
    g_create_error.clear();
    if (!out) {
        g_create_error = "out is NULL";
        return FPCLBM_ERR_ARG;
    }
    *out = nullptr;
    if (nx < 1 || ny < 1 || nz < 1) {
        g_create_error = "dimensions must be >= 1";
        return FPCLBM_ERR_ARG;
    }
    const unsigned long long n = (unsigned long long)nx * ny * nz;
    const unsigned long long stride = (n + 63) / 64 * 64;
    if (n >= (1ull << 31) || 27ull * stride >= (1ull << 32)) {
        g_create_error = "too many cells: need 27 * ceil64(nx*ny*nz) < 2^32";
        return FPCLBM_ERR_ARG;
    }
    if (precision < FPCLBM_FP64 || precision > FPCLBM_FP32_STORE_BF16) {
        g_create_error = "unknown precision";
        return FPCLBM_ERR_ARG;
    }
    if (bc != FPCLBM_BC_PERIODIC && bc != FPCLBM_BC_WALLS_Y) {
        g_create_error = "unknown boundary condition";
        return FPCLBM_ERR_ARG;
    }
    if (bc == FPCLBM_BC_WALLS_Y && ny < 1) {
        g_create_error = "walls need ny >= 1";
        return FPCLBM_ERR_ARG;
    }
    fpclbm* h = new (std::nothrow) fpclbm();
    if (!h) {
        g_create_error = "host allocation failed";
        return FPCLBM_ERR_ALLOC;
    }
    h->nx = nx;
    h->ny = ny;
    h->nz = nz;
    h->ncells = (unsigned)n;
    h->stride = (unsigned)stride;
    h->precision = precision;
    h->bc = bc;
    h->stream = static_cast<cudaStream_t>(cuda_stream);
    rates_from_params(1.0, 0.0, h->omega);
    cudaError_t e = cudaGetDevice(&h->device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&h->d_pop, 27ull * stride * elem_size(precision));
    if (e == cudaSuccess) e = cudaMalloc(&h->d_flag, sizeof(int));
    if (e == cudaSuccess) e = cudaMallocHost(&h->h_flag, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&h->d_part, sizeof(double) * 5 * (size_t)diag_blocks(h->ncells));
    if (e == cudaSuccess) e = cudaMalloc(&h->d_diag, sizeof(double) * 5);
    if (e == cudaSuccess) e = cudaMallocHost(&h->h_diag, sizeof(double) * 5);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->d_flag, 0, sizeof(int), h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
        g_create_error = std::string("CUDA: ") + cudaGetErrorString(e);
        const int code = (e == cudaErrorMemoryAllocation) ? FPCLBM_ERR_ALLOC : FPCLBM_ERR_CUDA;
        fpclbm_destroy(h);
        return code;
    }
    *out = h;
    return FPCLBM_OK;
}

int fpclbm_create_ensemble(fpclbm_t* out, int n_boxes, const int* dims, const double* tau, int precision,
                           void* cuda_stream);  // ensemble.cu

int fpclbm_destroy(fpclbm_t h)
{
    if (!h) return FPCLBM_OK;
    drop_graph(h);
    if (h->d_pop) cudaFree(h->d_pop);
    if (h->d_flag) cudaFree(h->d_flag);
    if (h->h_flag) cudaFreeHost(h->h_flag);
    if (h->d_stage) cudaFree(h->d_stage);
    if (h->d_part) cudaFree(h->d_part);
    if (h->d_diag) cudaFree(h->d_diag);
    if (h->h_diag) cudaFreeHost(h->h_diag);
    if (h->d_closure) cudaFree(h->d_closure);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    delete h;
    return FPCLBM_OK;
}

const char* fpclbm_last_error(fpclbm_t h)
{
    if (!h) return g_create_error.c_str();
    return h->err.c_str();
}

int fpclbm_init_fields(fpclbm_t h, const double* rho, const double* ux, const double* uy, const double* uz,
                       int on_device)
{
    if (!h) return FPCLBM_ERR_ARG;
    h->err.clear();
    if (!rho || !ux || !uy || !uz) return fail(h, FPCLBM_ERR_ARG, "null field pointer");
    const BoxGeom b = geom_of(h);
    if (on_device) {
        FPC_CK(h, launch_init_eq(h->precision, b, rho, ux, uy, uz, 0, h->ncells, h->stream), "init kernel");
    } else {
        const unsigned chunk = h->ncells < kChunk ? h->ncells : kChunk;
        int rc = ensure_stage(h, sizeof(double) * 4 * (size_t)chunk);
        if (rc) return rc;
        double* d = h->d_stage;
        for (unsigned c0 = 0; c0 < h->ncells; c0 += chunk) {
            const unsigned n = (h->ncells - c0 < chunk) ? h->ncells - c0 : chunk;
            const size_t bytes = sizeof(double) * n;
            FPC_CK(h, cudaMemcpyAsync(d, rho + c0, bytes, cudaMemcpyHostToDevice, h->stream), "copy rho");
            FPC_CK(h, cudaMemcpyAsync(d + chunk, ux + c0, bytes, cudaMemcpyHostToDevice, h->stream), "copy ux");
            FPC_CK(h, cudaMemcpyAsync(d + 2 * (size_t)chunk, uy + c0, bytes, cudaMemcpyHostToDevice, h->stream),
                   "copy uy");
            FPC_CK(h, cudaMemcpyAsync(d + 3 * (size_t)chunk, uz + c0, bytes, cudaMemcpyHostToDevice, h->stream),
                   "copy uz");
            FPC_CK(h,
                   launch_init_eq(h->precision, b, d, d + chunk, d + 2 * (size_t)chunk, d + 3 * (size_t)chunk, c0, n,
                                  h->stream),
                   "init kernel");
        }
    }
    FPC_CK(h, cudaStreamSynchronize(h->stream), "init sync");
    h->initialized = true;
    h->steps = 0;
    return FPCLBM_OK;
}

int fpclbm_set_params(fpclbm_t h, double tau, double drift, int diffusion)
{
    if (!h) return FPCLBM_ERR_ARG;
    h->err.clear();
    if (diffusion < FPCLBM_DIFF_FP || diffusion > FPCLBM_DIFF_FP_LEARNED)
        return fail(h, FPCLBM_ERR_ARG, "unknown diffusion mode");
    if (!std::isfinite(tau) || !std::isfinite(drift) || drift < 0)
        return fail(h, FPCLBM_ERR_ARG, "tau and drift must be finite, drift >= 0");
    if (diffusion == FPCLBM_DIFF_FP_LEARNED && !h->have_closure)
        return fail(h, FPCLBM_ERR_STATE, "learned diffusion mode needs fpclbm_set_closure first");
    double om[27];
    rates_from_params(tau, drift, om);
    std::string why;
    if (!rates_valid(om, why)) return fail(h, FPCLBM_ERR_PARAM, why);
    std::memcpy(h->omega, om, sizeof om);
    h->diffusion = diffusion;
    h->graph_valid = false;
    return FPCLBM_OK;
}

int fpclbm_set_rates(fpclbm_t h, const double omega[27])
{
    if (!h) return FPCLBM_ERR_ARG;
    h->err.clear();
    if (!omega) return fail(h, FPCLBM_ERR_ARG, "omega is NULL");
    std::string why;
    if (!rates_valid(omega, why)) return fail(h, FPCLBM_ERR_PARAM, why);
    std::memcpy(h->omega, omega, sizeof(double) * 27);
    h->graph_valid = false;
    return FPCLBM_OK;
}

int fpclbm_set_force(fpclbm_t h, double Fx, double Fy, double Fz)
{
    if (!h) return FPCLBM_ERR_ARG;
    h->err.clear();
    if (!std::isfinite(Fx) || !std::isfinite(Fy) || !std::isfinite(Fz))
        return fail(h, FPCLBM_ERR_ARG, "force must be finite");
    h->F[0] = Fx;
    h->F[1] = Fy;
    h->F[2] = Fz;
    h->graph_valid = false;
    return FPCLBM_OK;
}

int fpclbm_step(fpclbm_t h, long long n)
{
    if (!h) return FPCLBM_ERR_ARG;
    h->err.clear();
    if (n < 0) return fail(h, FPCLBM_ERR_ARG, "negative step count");
    if (!h->initialized) return fail(h, FPCLBM_ERR_STATE, "populations not initialised");
    if (n == 0) return FPCLBM_OK;
    FPC_CK(h, cudaMemsetAsync(h->d_flag, 0, sizeof(int), h->stream), "flag reset");
    long long done = 0;
    // bring the AA parity to even with single launches
    while (done < n && ((h->steps + done) & 1)) {
        FPC_CK(h, one_step(h, h->steps + done, h->stream), "step launch");
        ++done;
    }
    if (n - done >= kGraphSteps) {
        if (!h->graph_valid) {
            int rc = build_graph(h);
            if (rc) return rc;
        }
        while (n - done >= kGraphSteps) {
            FPC_CK(h, cudaGraphLaunch(h->graph, h->stream), "graph launch");
            done += kGraphSteps;
        }
    }
    while (done < n) {
        FPC_CK(h, one_step(h, h->steps + done, h->stream), "step launch");
        ++done;
    }
    h->steps += n;
    FPC_CK(h, cudaMemcpyAsync(h->h_flag, h->d_flag, sizeof(int), cudaMemcpyDeviceToHost, h->stream), "flag read");
    FPC_CK(h, cudaStreamSynchronize(h->stream), "step sync");
    if (*h->h_flag) return fail(h, FPCLBM_ERR_DIVERGED, "a cell reached rho <= 0 or a non-finite value");
    return FPCLBM_OK;
}

int fpclbm_get_step_count(fpclbm_t h, long long* steps)
{
    if (!h || !steps) return FPCLBM_ERR_ARG;
    *steps = h->steps;
    return FPCLBM_OK;
}

int fpclbm_moments(fpclbm_t h, double* rho, double* ux, double* uy, double* uz, int on_device)
{
    if (!h) return FPCLBM_ERR_ARG;
    h->err.clear();
    if (!h->initialized) return fail(h, FPCLBM_ERR_STATE, "populations not initialised");
    const BoxGeom b = geom_of(h);
    const int parity = (int)(h->steps & 1);
    if (on_device) {
        FPC_CK(h,
               launch_moments(h->precision, b, parity, h->F[0], h->F[1], h->F[2], rho, ux, uy, uz, 0, h->ncells,
                              h->stream),
               "moments kernel");
    } else {
        const unsigned chunk = h->ncells < kChunk ? h->ncells : kChunk;
        int rc = ensure_stage(h, sizeof(double) * 4 * (size_t)chunk);
        if (rc) return rc;
        double* d = h->d_stage;
        double* outs[4] = {rho, ux, uy, uz};
        for (unsigned c0 = 0; c0 < h->ncells; c0 += chunk) {
            const unsigned n = (h->ncells - c0 < chunk) ? h->ncells - c0 : chunk;
            double* dd[4];
            for (int q = 0; q < 4; ++q) dd[q] = outs[q] ? d + (size_t)q * chunk : nullptr;
            FPC_CK(h,
                   launch_moments(h->precision, b, parity, h->F[0], h->F[1], h->F[2], dd[0], dd[1], dd[2], dd[3], c0,
                                  n, h->stream),
                   "moments kernel");
            for (int q = 0; q < 4; ++q)
                if (outs[q])
                    FPC_CK(h,
                           cudaMemcpyAsync(outs[q] + c0, dd[q], sizeof(double) * n, cudaMemcpyDeviceToHost, h->stream),
                           "copy moments");
        }
    }
    FPC_CK(h, cudaStreamSynchronize(h->stream), "moments sync");
    return FPCLBM_OK;
}

int fpclbm_diagnostics(fpclbm_t h, double out[5])
{
    if (!h) return FPCLBM_ERR_ARG;
    h->err.clear();
    if (!out) return fail(h, FPCLBM_ERR_ARG, "out is NULL");
    if (!h->initialized) return fail(h, FPCLBM_ERR_STATE, "populations not initialised");
    FPC_CK(h,
           launch_diagnostics(h->precision, geom_of(h), (int)(h->steps & 1), h->F[0], h->F[1], h->F[2], h->d_part,
                              h->d_diag, h->stream),
           "diagnostics kernels");
    FPC_CK(h, cudaMemcpyAsync(h->h_diag, h->d_diag, sizeof(double) * 5, cudaMemcpyDeviceToHost, h->stream),
           "copy diagnostics");
    FPC_CK(h, cudaStreamSynchronize(h->stream), "diagnostics sync");
    std::memcpy(out, h->h_diag, sizeof(double) * 5);
    return FPCLBM_OK;
}

int fpclbm_get_populations(fpclbm_t h, double* f)
{
    if (!h) return FPCLBM_ERR_ARG;
    h->err.clear();
    if (!f) return fail(h, FPCLBM_ERR_ARG, "f is NULL");
    if (!h->initialized) return fail(h, FPCLBM_ERR_STATE, "populations not initialised");
    const unsigned chunk = h->ncells < kChunk ? h->ncells : kChunk;
    int rc = ensure_stage(h, sizeof(double) * 27 * (size_t)chunk);
    if (rc) return rc;
    const BoxGeom b = geom_of(h);
    const int parity = (int)(h->steps & 1);
    for (unsigned c0 = 0; c0 < h->ncells; c0 += chunk) {
        const unsigned n = (h->ncells - c0 < chunk) ? h->ncells - c0 : chunk;
        FPC_CK(h, launch_get_pops(h->precision, b, parity, h->d_stage, chunk, c0, n, h->stream), "populations kernel");
        FPC_CK(h,
               cudaMemcpy2DAsync(f + c0, sizeof(double) * h->ncells, h->d_stage, sizeof(double) * chunk,
                                 sizeof(double) * n, 27, cudaMemcpyDeviceToHost, h->stream),
               "copy populations");
    }
    FPC_CK(h, cudaStreamSynchronize(h->stream), "populations sync");
    return FPCLBM_OK;
}

int fpclbm_get_populations_at(fpclbm_t h, const long long* cells, int n, double* f)
{
    if (!h) return FPCLBM_ERR_ARG;
    h->err.clear();
    if (n < 0 || (n > 0 && (!cells || !f))) return fail(h, FPCLBM_ERR_ARG, "bad cell list");
    if (!h->initialized) return fail(h, FPCLBM_ERR_STATE, "populations not initialised");
    if (n == 0) return FPCLBM_OK;
    if (n > (int)kChunk) return fail(h, FPCLBM_ERR_ARG, "at most 2^20 cells per call");
    std::vector<unsigned> idx(n);
    for (int i = 0; i < n; ++i) {
        if (cells[i] < 0 || cells[i] >= (long long)h->ncells) return fail(h, FPCLBM_ERR_ARG, "cell index out of range");
        idx[i] = (unsigned)cells[i];
    }
    const size_t out_bytes = sizeof(double) * 27 * (size_t)n;
    const size_t idx_bytes = (sizeof(unsigned) * (size_t)n + 255) / 256 * 256;
    int rc = ensure_stage(h, out_bytes + idx_bytes);
    if (rc) return rc;
    double* d_out = h->d_stage;
    unsigned* d_idx = reinterpret_cast<unsigned*>(reinterpret_cast<char*>(h->d_stage) + out_bytes);
    FPC_CK(h, cudaMemcpyAsync(d_idx, idx.data(), sizeof(unsigned) * n, cudaMemcpyHostToDevice, h->stream), "copy cells");
    FPC_CK(h, launch_get_pops_at(h->precision, geom_of(h), (int)(h->steps & 1), d_idx, (unsigned)n, d_out, h->stream),
           "populations kernel");
    FPC_CK(h, cudaMemcpyAsync(f, d_out, out_bytes, cudaMemcpyDeviceToHost, h->stream), "copy populations");
    FPC_CK(h, cudaStreamSynchronize(h->stream), "populations sync");
    return FPCLBM_OK;
}

int fpclbm_set_populations(fpclbm_t h, const double* f)
{
    if (!h) return FPCLBM_ERR_ARG;
    h->err.clear();
    if (!f) return fail(h, FPCLBM_ERR_ARG, "f is NULL");
    const unsigned chunk = h->ncells < kChunk ? h->ncells : kChunk;
    int rc = ensure_stage(h, sizeof(double) * 27 * (size_t)chunk);
    if (rc) return rc;
    const BoxGeom b = geom_of(h);
    for (unsigned c0 = 0; c0 < h->ncells; c0 += chunk) {
        const unsigned n = (h->ncells - c0 < chunk) ? h->ncells - c0 : chunk;
        FPC_CK(h,
               cudaMemcpy2DAsync(h->d_stage, sizeof(double) * chunk, f + c0, sizeof(double) * h->ncells,
                                 sizeof(double) * n, 27, cudaMemcpyHostToDevice, h->stream),
               "copy populations");
        FPC_CK(h, launch_set_pops(h->precision, b, h->d_stage, chunk, c0, n, h->stream), "populations kernel");
    }
    FPC_CK(h, cudaStreamSynchronize(h->stream), "populations sync");
    h->initialized = true;
    h->steps = 0;
    return FPCLBM_OK;
}

int fpclbm_set_closure(fpclbm_t h, const unsigned short* w, int n_params)
{
    if (!h) return FPCLBM_ERR_ARG;
    h->err.clear();
    if (!w) return fail(h, FPCLBM_ERR_ARG, "weights are NULL");
    if (n_params != 4865) return fail(h, FPCLBM_ERR_ARG, "closure needs exactly 4865 parameters");
    std::vector<float> wf(n_params);
    for (int i = 0; i < n_params; ++i) {
        const unsigned bits = (unsigned)w[i] << 16;  // bf16 -> fp32 is exact
        float v;
        std::memcpy(&v, &bits, sizeof v);
        if (!std::isfinite(v)) return fail(h, FPCLBM_ERR_ARG, "non-finite closure weight");
        wf[i] = v;
    }
    if (!h->d_closure) {
        cudaError_t e = cudaMalloc(&h->d_closure, sizeof(float) * 4868);  // 16-byte padded
        if (e != cudaSuccess) return fail(h, FPCLBM_ERR_ALLOC, "closure weights");
    }
    FPC_CK(h, cudaMemcpyAsync(h->d_closure, wf.data(), sizeof(float) * n_params, cudaMemcpyHostToDevice, h->stream),
           "copy closure");
    FPC_CK(h, cudaStreamSynchronize(h->stream), "closure sync");
    h->have_closure = true;
    h->graph_valid = false;
    return FPCLBM_OK;
}

}  // extern "C"
