// fpclbm.cu -- host runtime and C ABI of libfpclbm.so (see include/fpclbm.h).
//
// A handle owns one population buffer (AA pattern, one copy per box), a
// divergence flag, staging buffers for host transfers, and a cached CUDA
// graph of the step loop.  Relaxation rates (Appendix D Step 3 numbering) and
// the body force live in the handle and are passed to every launch by value.
// On the first fpclbm_step of a large enough handle the launch configuration
// is autotuned on a saved copy of the state (the state is restored bit for
// bit afterwards), and the choice is cached per device and configuration.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "rtalloc.h"
#include <nvtx3/nvToolsExt.h>

#include "closure.cuh"
#include "handle.h"
#include "hostmem.h"

using namespace fpc;

namespace fpc {

thread_local std::string g_create_error;

int fail(fpclbm* h, int code, const std::string& msg)
{
    if (h) h->err = msg;
    return code;
}

int cuda_fail(fpclbm* h, cudaError_t e, const char* what)
{
    return fail(h, FPCLBM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// Rates from (tau, drift): shear 1/tau on 4,5,6,8,9 (Eq. transportcoeff3DFPCLBM);
// bulk 1 on 7 and 1 on 0..3; orders >= 3: k * drift (omega_mnp = (m+n+p) omega_FP),
// or 1 when drift == 0 (unit higher-order rates, Sec. 4).
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

// Allocation wrappers (rtalloc.h): live-allocation count and the test hook's failure countdown
// (-1: disarmed; k >= 0: the allocation after k more successful ones fails).
std::atomic<long long> g_live_allocs{0};
std::atomic<long long> g_fail_countdown{-1};

cudaError_t rt_malloc_raw(void** p, size_t bytes, bool host)
{
    *p = nullptr;
    long long c = g_fail_countdown.load();
    while (c >= 0 && !g_fail_countdown.compare_exchange_weak(c, c - 1)) {
    }
    if (c == 0) return cudaErrorMemoryAllocation;  // injected failure, as if the device were full
    const cudaError_t e = host ? cudaMallocHost(p, bytes) : cudaMalloc(p, bytes);
    if (e == cudaSuccess) {
        ++g_live_allocs;
    } else {
        *p = nullptr;
    }
    return e;
}

void rt_free_raw(void* p, bool host)
{
    if (!p) return;
    if (host) cudaFreeHost(p);
    else cudaFree(p);
    --g_live_allocs;
}

size_t elem_size(int precision)
{
    switch (precision) {
        case FPCLBM_FP64: return 8;
        case FPCLBM_FP32: return 4;
        default: return 2;
    }
}

int alloc_common(fpclbm* h)
{
    cudaError_t e = cudaGetDevice(&h->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, h->device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = rt_malloc(&h->d_flag, sizeof(int));
    if (e == cudaSuccess) e = rt_malloc_host(&h->h_flag, sizeof(int));
    unsigned parts = 0;
    for (auto& b : h->boxes) {
        b.diag0 = parts;
        parts += (unsigned)diag_blocks(b.ncells);
    }
    h->diag_parts = parts;
    if (e == cudaSuccess) e = rt_malloc(&h->d_part, sizeof(double) * 5 * (size_t)parts);
    if (e == cudaSuccess) e = rt_malloc(&h->d_diag, sizeof(double) * 5);
    if (e == cudaSuccess) e = rt_malloc_host(&h->h_diag, sizeof(double) * 5);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->d_flag, 0, sizeof(int), h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
        g_create_error = std::string("CUDA: ") + cudaGetErrorString(e);
        return e == cudaErrorMemoryAllocation ? FPCLBM_ERR_ALLOC : FPCLBM_ERR_CUDA;
    }
    return FPCLBM_OK;
}

}  // namespace fpc

namespace {

constexpr int kGraphSteps = 32;        // steps per captured graph (even)
constexpr unsigned kChunk = 1u << 20;  // cells per host-transfer chunk

#define FPC_CK(h, call, what)                                 \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return cuda_fail(h, e_, what); \
    } while (0)

void* box_ptr(const fpclbm* h, const Box& b)
{
    return static_cast<char*>(h->d_pop) + b.off * elem_size(h->precision);
}

template <typename R>
StepArgs<R> make_args(const fpclbm* h)
{
    const Box& b = h->boxes[0];
    StepArgs<R> a;
    a.buf = box_ptr(h, b);
    a.stride = b.stride;
    a.ncells = b.ncells;
    a.nx = b.nx;
    a.ny = b.ny;
    a.nz = b.nz;
    a.div_nx = make_fastdiv((unsigned)b.nx);
    a.div_nxny = make_fastdiv((unsigned)(b.nx * b.ny));
    a.Fx = (R)h->F[0];
    a.Fy = (R)h->F[1];
    a.Fz = (R)h->F[2];
    a.lid6x = (R)(6.0 * h->lid[0]);
    a.lid6z = (R)(6.0 * h->lid[1]);
    for (int j = 0; j < 27; ++j) {
        a.rates.om[j] = (R)h->omega[j];
        a.rates.keep[j] = (R)(1.0 - h->omega[j]);
        a.rates.src[j] = (R)(1.0 - 0.5 * h->omega[j]);
    }
    a.flag = h->d_flag;
    a.closure = h->d_closure;
    a.smag = h->diffusion == FPCLBM_DIFF_FP_SMAGORINSKY ? static_cast<const R*>(h->d_smag) : nullptr;
    return a;
}

EnsArgs make_ens_args(const fpclbm* h)
{
    EnsArgs a;
    a.buf = h->d_pop;
    a.boxes = h->d_ens_boxes;
    a.tile_box = h->d_tile_box;
    a.ntiles = h->ntiles;
    a.tile_cells = (unsigned)h->tile_cells;
    for (int j = 0; j < 27; ++j) {
        a.rates.om[j] = (float)h->omega[j];
        a.rates.keep[j] = (float)(1.0 - h->omega[j]);
        a.rates.src[j] = (float)(1.0 - 0.5 * h->omega[j]);
    }
    a.Fx = (float)h->F[0];
    a.Fy = (float)h->F[1];
    a.Fz = (float)h->F[2];
    for (int j = 0; j < 27; ++j) {
        a.rates2.om[j] = f2(a.rates.om[j], a.rates.om[j]);
        a.rates2.keep[j] = f2(a.rates.keep[j], a.rates.keep[j]);
        a.rates2.src[j] = f2(a.rates.src[j], a.rates.src[j]);
    }
    a.Fx2 = f2(a.Fx, a.Fx);
    a.Fy2 = f2(a.Fy, a.Fy);
    a.Fz2 = f2(a.Fz, a.Fz);
    a.flag = h->d_flag;
    return a;
}

BoxGeom geom_of(const fpclbm* h, const Box& b)
{
    BoxGeom g;
    g.buf = box_ptr(h, b);
    g.stride = b.stride;
    g.ncells = b.ncells;
    g.nx = b.nx;
    g.ny = b.ny;
    g.nz = b.nz;
    g.walls = h->bc == FPCLBM_BC_WALLS_Y ? 1 : h->bc == FPCLBM_BC_BOX ? 2 : h->bc == FPCLBM_BC_HALF_CHANNEL ? 3 : 0;
    g.div_nx = make_fastdiv((unsigned)b.nx);
    g.div_nxny = make_fastdiv((unsigned)(b.nx * b.ny));
    return g;
}

bool has_force(const fpclbm* h) { return h->F[0] != 0.0 || h->F[1] != 0.0 || h->F[2] != 0.0; }

// Collision mode of the step kernel.  A box or ensemble in the FP or MCM mode whose rates of
// orders 3-6 (Step 3 indices 10..26) are all exactly 1 takes the unit-rate variant, which sets
// those moments to their attractors plus half their sources (and, without force, never forms
// their pre-collision values).
int mode_of(const fpclbm* h)
{
    if (h->diffusion == FPCLBM_DIFF_FP_SMAGORINSKY) return MODE_SMAG;
    const int m = h->diffusion == FPCLBM_DIFF_FP_LEARNED ? MODE_LEARNED
                  : h->diffusion == FPCLBM_DIFF_EQUILIBRIUM ? MODE_EQ : MODE_FP;
    for (int j = 10; j < 27; ++j)
        if (h->omega[j] != 1.0) return m;
    return m == MODE_EQ ? MODE_EQ_R1 : m == MODE_LEARNED ? MODE_LEARNED_R1 : MODE_FP_R1;
}

// Boundary kind of the step kernel: a channel whose upper wall moves takes the
// moving-wall variant; a closed box always does (its lid may rest).
int kernel_bc(const fpclbm* h)
{
    if (h->bc == FPCLBM_BC_BOX) return BC_BOX_LID;
    if (h->bc == FPCLBM_BC_HALF_CHANNEL) return BC_HALF_CHANNEL;
    if (h->bc == FPCLBM_BC_WALLS_Y) return (h->lid[0] != 0.0 || h->lid[1] != 0.0) ? BC_WALLS_Y_LID : BC_WALLS_Y;
    return BC_PERIODIC;
}

// (C_s Delta D(y))^2 per row y (Delta = 1): van Driest damping D = 1 - exp(-y+ / A+),
// y+ = y_w u* / nu, y_w the distance of the row centre to the nearest wall (none in a
// periodic box; u* <= 0 or A+ <= 0 switch the damping off).  nu from the shear rate omega_4.
int upload_smag(fpclbm* h)
{
    const Box& b = h->boxes[0];
    const int ny = b.ny;
    if (!h->d_smag) {
        cudaError_t e = rt_malloc(&h->d_smag, sizeof(double) * (size_t)ny);
        if (e != cudaSuccess) return fail(h, FPCLBM_ERR_ALLOC, std::string("Smagorinsky table: ") + cudaGetErrorString(e));
    }
    const double nu = (1.0 / h->omega[4] - 0.5) / 3.0;
    std::vector<double> c2(ny);
    std::vector<float> c2f(ny);
    for (int y = 0; y < ny; ++y) {
        double yw = -1.0;
        if (h->bc == FPCLBM_BC_WALLS_Y) yw = std::min(y + 0.5, ny - 0.5 - y);
        if (h->bc == FPCLBM_BC_HALF_CHANNEL) yw = y + 0.5;
        double D = 1.0;
        if (yw >= 0 && h->smag[1] > 0 && h->smag[2] > 0) D = 1.0 - std::exp(-(yw * h->smag[1] / nu) / h->smag[2]);
        c2[y] = (h->smag[0] * D) * (h->smag[0] * D);
        c2f[y] = (float)c2[y];
    }
    const bool f64 = h->precision == FPCLBM_FP64;
    FPC_CK(h, cudaMemcpyAsync(h->d_smag, f64 ? (const void*)c2.data() : (const void*)c2f.data(),
                              (f64 ? sizeof(double) : sizeof(float)) * (size_t)ny, cudaMemcpyHostToDevice, h->stream),
           "Smagorinsky table upload");
    FPC_CK(h, cudaStreamSynchronize(h->stream), "Smagorinsky table upload");
    h->smag_dirty = false;
    return FPCLBM_OK;
}

cudaError_t one_step(fpclbm* h, long long t, cudaStream_t st, int block, int minb, int grid, int pipe)
{
    if (h->ensemble)
        return launch_ens_step((int)(t & 1), has_force(h), mode_of(h), make_ens_args(h), block, minb, grid, pipe, st);
    const StepArgs<double> a64 = make_args<double>(h);
    const StepArgs<float> a32 = make_args<float>(h);
    StepLaunch cfg{block, minb, pipe, pipe == 3 ? grid : 2};  // variant 3 keeps its stage count in grid
    return launch_step(h->precision, (int)(t & 1), kernel_bc(h), has_force(h), mode_of(h), a64, a32, cfg, st);
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
    for (int k = 0; k < kGraphSteps && e == cudaSuccess; ++k) e = one_step(h, k, h->cap_stream, h->block, h->minb, h->grid, h->pipe);
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
    if (h->d_stage) rt_free(h->d_stage);
    h->d_stage = nullptr;
    h->stage_bytes = 0;
    cudaError_t e = rt_malloc(&h->d_stage, bytes);
    if (e != cudaSuccess) return fail(h, FPCLBM_ERR_ALLOC, std::string("staging buffer: ") + cudaGetErrorString(e));
    h->stage_bytes = bytes;
    return FPCLBM_OK;
}

unsigned chunk_of(const Box& b) { return b.ncells < kChunk ? b.ncells : kChunk; }


// ---------------------------------------------------------------------------
// Autotuning of the launch configuration (block size; persistent grid for
// ensembles).  Runs on the handle's own buffer after saving it to a device
// copy, times every candidate from the same state, restores the state, and
// caches the winner per device/precision/boundary/force/mode/shape class.
// ---------------------------------------------------------------------------

struct TuneChoice {
    int block, minb, grid, pipe;
};

std::mutex g_tune_mu;
std::map<std::string, TuneChoice> g_tune_cache;

bool verbose()
{
    const char* v = std::getenv("FPCLBM_VERBOSE");
    return v && v[0] && v[0] != '0';
}

// Optional persistent cache of tuning results (FPCLBM_TUNE_CACHE = path): one
// line "key block minb grid pipe" per configuration.  A run can reuse the
// choice of an earlier run, e.g. a profiler run that must time the same
// kernel variant as the plain run it profiles.
void load_tune_file()
{
    static bool loaded = false;
    if (loaded) return;
    loaded = true;
    const char* path = std::getenv("FPCLBM_TUNE_CACHE");
    if (!path || !path[0]) return;
    FILE* fp = std::fopen(path, "r");
    if (!fp) return;
    char key[200];
    TuneChoice c;
    while (std::fscanf(fp, "%199s %d %d %d %d", key, &c.block, &c.minb, &c.grid, &c.pipe) == 5)
        g_tune_cache[key] = c;
    std::fclose(fp);
}

void save_tune_file()
{
    const char* path = std::getenv("FPCLBM_TUNE_CACHE");
    if (!path || !path[0]) return;
    FILE* fp = std::fopen(path, "w");
    if (!fp) return;
    for (const auto& kv : g_tune_cache)
        std::fprintf(fp, "%s %d %d %d %d\n", kv.first.c_str(), kv.second.block, kv.second.minb, kv.second.grid,
                     kv.second.pipe);
    std::fclose(fp);
}

// FPCLBM_LAUNCH = "block:minb:variant[:stages]" forces a single-box launch configuration
// (variant 0: one cell per thread, 1: cp.async-pipelined, 2: two cells per thread, 3: two cells
// per thread through row-staged shared memory with `stages` input stages, 2..6, default 2).
bool forced_launch(TuneChoice& c)
{
    const char* v = std::getenv("FPCLBM_LAUNCH");
    if (!v || !v[0]) return false;
    int b = 0, m = 0, p = 0, ns = 2;
    const int got = std::sscanf(v, "%d:%d:%d:%d", &b, &m, &p, &ns);
    if (got < 3 || b < 32 || b > 256 || b % 32 || m < 1 || m > 4 || p < 0 || p > 3 || ns < 2 || ns > 6)
        return false;
    c = {b, m, p == 3 ? ns : 0, p};
    return true;
}

// Whether the row-staged variant (stage.cuh) can run this handle: a single periodic box or
// channel, fp32 arithmetic in the FP or MCM mode, 16- or 32-bit storage, rows of a multiple of
// 16 bytes and at most 512 cells (tiles of 256 or 512 cells).
bool stage_ok(const fpclbm* h)
{
    if (h->ensemble || h->precision == FPCLBM_FP64) return false;
    const int kb = kernel_bc(h);
    if (!(kb == BC_PERIODIC || kb == BC_WALLS_Y) || !plain_mode(mode_of(h))) return false;
    const Box& b = h->boxes[0];
    const size_t es = elem_size(h->precision);
    return (b.nx * es) % 16 == 0 && b.nx <= 512;
}

// Threads of a row-staged block: 4, 6 or 8 consumer warps and one producer warp.
int stage_threads(const fpclbm* h)
{
    const int nx = h->boxes[0].nx;
    return nx <= 256 ? 160 : nx <= 384 ? 224 : 288;
}

std::string tune_key(const fpclbm* h)
{
    char buf[160];
    std::snprintf(buf, sizeof buf, "dev%d/p%d/bc%d/f%d/m%d/%s/%llu", h->device, h->precision, kernel_bc(h), (int)has_force(h),
                  mode_of(h), h->ensemble ? "ens" : "box", (unsigned long long)(h->total_cells >> 20));
    return buf;
}

int autotune(fpclbm* h)
{
    h->tuned = true;
    std::vector<TuneChoice> cands;
    // register-cap variants: fp32 arithmetic, FP/EQ modes, any boundary; pipelined variant: the
    // same on periodic and channel boxes with 4- or 8-byte storage (cp.async moves >= 4 bytes)
    const int kb = kernel_bc(h), md = mode_of(h);
    const bool fixed_walls = bc_fixed(kb);
    const bool fp32_math = h->precision != FPCLBM_FP64 && plain_mode(md);
    const bool pipe_ok = elem_size(h->precision) >= 4 && plain_mode(md) &&
                         (kb == BC_PERIODIC || kb == BC_WALLS_Y);
    // paired variant (two cells per thread, packed fp32): fp32 arithmetic, every boundary kind
    const bool pair_ok = fp32_math;
    if (h->ensemble) {
        for (int minb : {2, 3})
            for (int block : {128, 256}) {
                const int per_sm = ens_max_blocks_per_sm(block, minb, mode_of(h), 0);
                for (int mult : {1, 2}) cands.push_back({block, minb, h->sm_count * per_sm * mult, 0});
            }
        for (int minb : {3, 4}) {  // paired variant: 3 or 4 blocks of 128 threads per SM
            const int per_sm = ens_max_blocks_per_sm(128, minb, mode_of(h), 2);
            // oversubscribed grids let the block scheduler even out boxes of different cost, up to
            // one tile per block
            for (int mult : {1, 2, 4, 8, 16}) cands.push_back({128, minb, h->sm_count * per_sm * mult, 2});
            cands.push_back({128, minb, (int)h->ntiles, 2});
        }
    } else if (fp32_math) {
        for (int minb : {2, 3, 4})
            for (int block : {128, 256}) cands.push_back({block, minb, 0, 0});
        if (pipe_ok)
            for (int minb : {2, 3, 4}) cands.push_back({128, minb, 0, 1});
        if (pair_ok) cands.push_back({128, 2, 0, 2});  // 4 blocks of 128 threads, 128 registers
        if (stage_ok(h))  // row-staged paired variant with 2 or 3 input stages
            for (int ns : {2, 3}) cands.push_back({stage_threads(h), 2, ns, 3});
    } else if (learned_mode(mode_of(h)) && h->precision != FPCLBM_FP64 && fixed_walls) {
        // two cells per thread first (the collision on the packed fp32 pipe, the MLP once per
        // lane), then one cell per thread capped at 128 registers or uncapped
        cands.push_back({128, 2, 0, 2});
        for (int minb : {2, 1})
            for (int block : {128, 256}) cands.push_back({block, minb, 0, 0});
    } else {
        for (int block : {128, 256}) cands.push_back({block, 1, 0, 0});
        if (pipe_ok) cands.push_back({128, 1, 0, 1});
    }
    TuneChoice forced;
    if (h->ensemble && forced_launch(forced)) {
        // ensembles: variant 0 (one cell per thread, minb 2 or 3) or 2 (paired, blocks of 128,
        // minb 3 or 4); persistent grid from the occupancy of the chosen kernel
        if (forced.pipe == 2) {
            forced.block = 128;
            if (forced.minb != 3) forced.minb = 4;
        } else {
            forced.pipe = 0;
            if (forced.minb != 3) forced.minb = 2;
            if (h->tile_cells % forced.block) forced.block = h->tile_cells;
        }
        h->block = forced.block;
        h->minb = forced.minb;
        h->pipe = forced.pipe;
        h->grid = h->sm_count * ens_max_blocks_per_sm(forced.block, forced.minb, mode_of(h), forced.pipe);
        return FPCLBM_OK;
    }
    if (!h->ensemble && forced_launch(forced)) {
        if (forced.pipe == 3 && !stage_ok(h)) forced.pipe = pair_ok ? 2 : 0;
        const bool pair_learned = learned_mode(mode_of(h)) && h->precision != FPCLBM_FP64 &&
                                  (kb == BC_PERIODIC || kb == BC_WALLS_Y);
        if ((forced.pipe == 1 && !pipe_ok) || (forced.pipe == 2 && !pair_ok && !pair_learned)) forced.pipe = 0;
        if (forced.pipe == 2 || forced.pipe == 3) forced.minb = 2;
        if (forced.pipe == 3) forced.block = stage_threads(h);
        if (forced.pipe != 3) forced.grid = 0;
        if (!fp32_math && !learned_mode(mode_of(h))) forced.minb = 1;  // learned: 1 or 2 (else 1)
        h->block = forced.block;
        h->minb = forced.minb;
        h->grid = forced.grid;
        h->pipe = forced.pipe;
        return FPCLBM_OK;
    }
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        load_tune_file();
        auto it = g_tune_cache.find(tune_key(h));
        if (it != g_tune_cache.end()) {
            h->block = it->second.block;
            h->minb = it->second.minb;
            h->grid = it->second.grid;
            h->pipe = it->second.pipe;
            return FPCLBM_OK;
        }
    }
    h->block = cands[0].block;
    h->minb = cands[0].minb;
    h->grid = cands[0].grid;
    h->pipe = cands[0].pipe;
    // small problems: keep the first candidate, tuning noise would dominate
    if (h->total_cells < (1ull << 20)) return FPCLBM_OK;
    size_t bytes = 0;
    for (const Box& b : h->boxes) bytes += 27ull * b.stride * elem_size(h->precision);
    void* backup = nullptr;
    if (rt_malloc(&backup, bytes) != cudaSuccess) {
        cudaGetLastError();
        return FPCLBM_OK;  // no room to tune safely: keep the default
    }
    FPC_CK(h, cudaMemcpyAsync(backup, h->d_pop, bytes, cudaMemcpyDeviceToDevice, h->stream), "tune save");
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    TuneChoice win = cands[0];
    for (const TuneChoice& c : cands) {
        cudaError_t e = cudaSuccess;
        for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = one_step(h, h->steps + k, h->stream, c.block, c.minb, c.grid, c.pipe);
        cudaEventRecord(e0, h->stream);
        for (int k = 0; k < 8 && e == cudaSuccess; ++k) e = one_step(h, h->steps + k, h->stream, c.block, c.minb, c.grid, c.pipe);
        cudaEventRecord(e1, h->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0;
        if (e == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
        if (verbose())
            std::fprintf(stderr, "fpclbm tune %s: block %d minb %d grid %d pipe %d: %.4f ms/step%s\n",
                         tune_key(h).c_str(), c.block, c.minb, c.grid, c.pipe, ms / 8,
                         e == cudaSuccess ? "" : " (launch failed)");
        if (e == cudaSuccess && ms < best) {
            best = ms;
            win = c;
        }
        if (e != cudaSuccess) cudaGetLastError();
        cudaMemcpyAsync(h->d_pop, backup, bytes, cudaMemcpyDeviceToDevice, h->stream);
    }
    cudaMemsetAsync(h->d_flag, 0, sizeof(int), h->stream);
    cudaError_t e = cudaStreamSynchronize(h->stream);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    rt_free(backup);
    FPC_CK(h, e, "tune restore");
    h->block = win.block;
    h->minb = win.minb;
    h->grid = win.grid;
    h->pipe = win.pipe;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[tune_key(h)] = win;
    save_tune_file();
    if (verbose())
        std::fprintf(stderr, "fpclbm tune %s: chose block %d minb %d grid %d pipe %d\n", tune_key(h).c_str(),
                     win.block, win.minb, win.grid, win.pipe);
    return FPCLBM_OK;
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
    if (bc != FPCLBM_BC_PERIODIC && bc != FPCLBM_BC_WALLS_Y && bc != FPCLBM_BC_BOX && bc != FPCLBM_BC_HALF_CHANNEL) {
        g_create_error = "unknown boundary condition";
        return FPCLBM_ERR_ARG;
    }
    fpclbm* h = new (std::nothrow) fpclbm();
    if (!h) {
        g_create_error = "host allocation failed";
        return FPCLBM_ERR_ALLOC;
    }
    Box b;
    b.nx = nx;
    b.ny = ny;
    b.nz = nz;
    b.ncells = (unsigned)n;
    b.stride = (unsigned)stride;
    h->boxes.push_back(b);
    h->total_cells = n;
    h->precision = precision;
    h->bc = bc;
    h->stream = static_cast<cudaStream_t>(cuda_stream);
    rates_from_params(1.0, 0.0, h->omega);
    int rc = alloc_common(h);
    if (rc == FPCLBM_OK) {
        cudaError_t e = rt_malloc(&h->d_pop, 27ull * stride * elem_size(precision));
        if (e != cudaSuccess) {
            g_create_error = std::string("populations: ") + cudaGetErrorString(e);
            rc = FPCLBM_ERR_ALLOC;
        }
    }
    if (rc != FPCLBM_OK) {
        fpclbm_destroy(h);
        return rc;
    }
    *out = h;
    return FPCLBM_OK;
}

int fpclbm_destroy(fpclbm_t h)
{
    if (!h) return FPCLBM_OK;
    drop_graph(h);
    if (h->d_pop) rt_free(h->d_pop);
    if (h->d_flag) rt_free(h->d_flag);
    if (h->h_flag) rt_free_host(h->h_flag);
    if (h->d_stage) rt_free(h->d_stage);
    if (h->d_part) rt_free(h->d_part);
    if (h->d_diag) rt_free(h->d_diag);
    if (h->h_diag) rt_free_host(h->h_diag);
    if (h->d_closure) rt_free(h->d_closure);
    if (h->d_smag) rt_free(h->d_smag);
    if (h->d_ens_boxes) rt_free(h->d_ens_boxes);
    if (h->d_tile_box) rt_free(h->d_tile_box);
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
    if (!on_device) {  // page-locked host fields: the init kernel reads them in place
        const double* m[4] = {mapped_host(rho), mapped_host(ux), mapped_host(uy), mapped_host(uz)};
        if (m[0] && m[1] && m[2] && m[3]) {
            rho = m[0];
            ux = m[1];
            uy = m[2];
            uz = m[3];
            on_device = 1;
        }
    }
    for (const Box& b : h->boxes) {
        const BoxGeom g = geom_of(h, b);
        if (on_device) {
            FPC_CK(h,
                   launch_init_eq(h->precision, g, rho + b.cell0, ux + b.cell0, uy + b.cell0, uz + b.cell0, 0,
                                  b.ncells, h->stream),
                   "init kernel");
            continue;
        }
        const unsigned chunk = chunk_of(b);
        int rc = ensure_stage(h, sizeof(double) * 4 * (size_t)chunk);
        if (rc) return rc;
        double* d = h->d_stage;
        for (unsigned c0 = 0; c0 < b.ncells; c0 += chunk) {
            const unsigned n = (b.ncells - c0 < chunk) ? b.ncells - c0 : chunk;
            const size_t bytes = sizeof(double) * n;
            const size_t at = (size_t)b.cell0 + c0;
            FPC_CK(h, cudaMemcpyAsync(d, rho + at, bytes, cudaMemcpyHostToDevice, h->stream), "copy rho");
            FPC_CK(h, cudaMemcpyAsync(d + chunk, ux + at, bytes, cudaMemcpyHostToDevice, h->stream), "copy ux");
            FPC_CK(h, cudaMemcpyAsync(d + 2 * (size_t)chunk, uy + at, bytes, cudaMemcpyHostToDevice, h->stream),
                   "copy uy");
            FPC_CK(h, cudaMemcpyAsync(d + 3 * (size_t)chunk, uz + at, bytes, cudaMemcpyHostToDevice, h->stream),
                   "copy uz");
            FPC_CK(h,
                   launch_init_eq(h->precision, g, d, d + chunk, d + 2 * (size_t)chunk, d + 3 * (size_t)chunk, c0, n,
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
    if (diffusion < FPCLBM_DIFF_FP || diffusion > FPCLBM_DIFF_FP_SMAGORINSKY)
        return fail(h, FPCLBM_ERR_ARG, "unknown diffusion mode");
    if (diffusion == FPCLBM_DIFF_FP_SMAGORINSKY && h->ensemble)
        return fail(h, FPCLBM_ERR_ARG, "Smagorinsky mode is for single boxes");
    if (!std::isfinite(tau) || !std::isfinite(drift) || drift < 0)
        return fail(h, FPCLBM_ERR_ARG, "tau and drift must be finite, drift >= 0");
    if (diffusion == FPCLBM_DIFF_FP_LEARNED && !h->have_closure)
        return fail(h, FPCLBM_ERR_STATE, "learned diffusion mode needs fpclbm_set_closure first");
    if (diffusion == FPCLBM_DIFF_FP_LEARNED && h->ensemble)
        return fail(h, FPCLBM_ERR_ARG, "learned diffusion mode is for single boxes");
    double om[27];
    rates_from_params(h->ensemble ? 1.0 : tau, drift, om);
    std::string why;
    if (!rates_valid(om, why)) return fail(h, FPCLBM_ERR_PARAM, why);
    std::memcpy(h->omega, om, sizeof om);
    h->diffusion = diffusion;
    h->graph_valid = false;
    h->tuned = false;
    h->smag_dirty = true;
    return FPCLBM_OK;
}

int fpclbm_set_rates(fpclbm_t h, const double omega[27])
{
    if (!h) return FPCLBM_ERR_ARG;
    h->err.clear();
    if (!omega) return fail(h, FPCLBM_ERR_ARG, "omega is NULL");
    if (h->ensemble) return fail(h, FPCLBM_ERR_ARG, "set_rates is for single boxes");
    std::string why;
    if (!rates_valid(omega, why)) return fail(h, FPCLBM_ERR_PARAM, why);
    const int md = mode_of(h);
    std::memcpy(h->omega, omega, sizeof(double) * 27);
    if (mode_of(h) != md) h->tuned = false;  // another kernel family: tune it
    h->graph_valid = false;
    h->smag_dirty = true;
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
    h->tuned = false;
    return FPCLBM_OK;
}

int fpclbm_set_smagorinsky(fpclbm_t h, double cs, double u_star, double a_plus)
{
    if (!h) return FPCLBM_ERR_ARG;
    h->err.clear();
    if (h->ensemble) return fail(h, FPCLBM_ERR_ARG, "Smagorinsky model is for single boxes");
    if (!std::isfinite(cs) || !std::isfinite(u_star) || !std::isfinite(a_plus) || cs < 0)
        return fail(h, FPCLBM_ERR_ARG, "C_s must be finite and >= 0, u* and A+ finite");
    h->smag[0] = cs;
    h->smag[1] = u_star;
    h->smag[2] = a_plus;
    h->smag_dirty = true;
    return FPCLBM_OK;
}

int fpclbm_set_wall_velocity(fpclbm_t h, double ux, double uz)
{
    if (!h) return FPCLBM_ERR_ARG;
    h->err.clear();
    if (h->ensemble || (h->bc != FPCLBM_BC_WALLS_Y && h->bc != FPCLBM_BC_BOX))
        return fail(h, FPCLBM_ERR_ARG, "wall velocity needs a box with walls (FPCLBM_BC_WALLS_Y or FPCLBM_BC_BOX)");
    if (!std::isfinite(ux) || !std::isfinite(uz)) return fail(h, FPCLBM_ERR_ARG, "wall velocity must be finite");
    h->lid[0] = ux;
    h->lid[1] = uz;
    h->graph_valid = false;
    h->tuned = false;
    return FPCLBM_OK;
}

int fpclbm_step(fpclbm_t h, long long n)
{
    if (!h) return FPCLBM_ERR_ARG;
    h->err.clear();
    if (n < 0) return fail(h, FPCLBM_ERR_ARG, "negative step count");
    if (!h->initialized) return fail(h, FPCLBM_ERR_STATE, "populations not initialised");
    if (n == 0) return FPCLBM_OK;
    {
        const int kb = kernel_bc(h), md = mode_of(h);
        if (learned_mode(md) && !(kb == BC_PERIODIC || kb == BC_WALLS_Y))
            return fail(h, FPCLBM_ERR_ARG, "learned mode needs a periodic box or a channel with resting walls");
        if (md == MODE_SMAG && !bc_fixed(kb))
            return fail(h, FPCLBM_ERR_ARG, "Smagorinsky mode needs resting walls (no closed box, no moving wall)");
        if (md == MODE_SMAG && h->smag_dirty) {
            int rc = upload_smag(h);
            if (rc) return rc;
        }
    }
    if (!h->tuned) {
        int rc = autotune(h);
        if (rc) return rc;
        h->graph_valid = false;
    }
    FPC_CK(h, cudaMemsetAsync(h->d_flag, 0, sizeof(int), h->stream), "flag reset");
    // profiler ranges (NVTX, header-only: free unless a tool is attached) around the host-side
    // issue of the step launches and graph replays
    struct Range {
        Range(const char* name) { nvtxRangePushA(name); }
        ~Range() { nvtxRangePop(); }
    } range("fpclbm_step");
    long long done = 0;
    // bring the AA parity to even with single launches
    while (done < n && ((h->steps + done) & 1)) {
        FPC_CK(h, one_step(h, h->steps + done, h->stream, h->block, h->minb, h->grid, h->pipe), "step launch");
        ++done;
    }
    if (n - done >= kGraphSteps) {
        if (!h->graph_valid) {
            int rc = build_graph(h);
            if (rc) return rc;
        }
        Range replays("fpclbm_step graph replays");
        while (n - done >= kGraphSteps) {
            FPC_CK(h, cudaGraphLaunch(h->graph, h->stream), "graph launch");
            done += kGraphSteps;
        }
    }
    while (done < n) {
        FPC_CK(h, one_step(h, h->steps + done, h->stream, h->block, h->minb, h->grid, h->pipe), "step launch");
        ++done;
    }
    h->steps += n;
    FPC_CK(h, cudaMemcpyAsync(h->h_flag, h->d_flag, sizeof(int), cudaMemcpyDeviceToHost, h->stream), "flag read");
    FPC_CK(h, cudaStreamSynchronize(h->stream), "step sync");
    if (*h->h_flag & 2)
        return fail(h, FPCLBM_ERR_TIMEOUT, "a step kernel's bounded wait for its staged data ran out");
    if (*h->h_flag) return fail(h, FPCLBM_ERR_DIVERGED, "a cell reached rho <= 0 or a non-finite value");
    return FPCLBM_OK;
}

int fpclbm_get_step_count(fpclbm_t h, long long* steps)
{
    if (!h || !steps) return FPCLBM_ERR_ARG;
    *steps = h->steps;
    return FPCLBM_OK;
}

int fpclbm_get_launch(fpclbm_t h, int out[4])
{
    if (!h || !out) return FPCLBM_ERR_ARG;
    h->err.clear();
    if (!h->tuned) return fail(h, FPCLBM_ERR_STATE, "no launch chosen yet: the autotuner runs at the first step");
    out[0] = h->block;
    out[1] = h->pipe == 3 ? h->grid : h->minb;  // variant 3: its shared-memory stages
    out[2] = h->pipe;
    out[3] = mode_of(h);
    return FPCLBM_OK;
}

int fpclbm_moments(fpclbm_t h, double* rho, double* ux, double* uy, double* uz, int on_device)
{
    if (!h) return FPCLBM_ERR_ARG;
    h->err.clear();
    if (!h->initialized) return fail(h, FPCLBM_ERR_STATE, "populations not initialised");
    const int parity = (int)(h->steps & 1);
    double* outs[4] = {rho, ux, uy, uz};
    if (!on_device) {  // page-locked host outputs: the moments kernel writes them in place
        bool all = true;
        double* m[4];
        for (int q = 0; q < 4; ++q) {
            m[q] = mapped_host(outs[q]);
            if (outs[q] && !m[q]) all = false;
        }
        if (all) {
            for (int q = 0; q < 4; ++q) outs[q] = m[q];
            on_device = 1;
        }
    }
    for (const Box& b : h->boxes) {
        const BoxGeom g = geom_of(h, b);
        if (on_device) {
            double* o[4];
            for (int q = 0; q < 4; ++q) o[q] = outs[q] ? outs[q] + b.cell0 : nullptr;
            FPC_CK(h,
                   launch_moments(h->precision, g, parity, h->F[0], h->F[1], h->F[2], o[0], o[1], o[2], o[3], 0,
                                  b.ncells, h->stream),
                   "moments kernel");
            continue;
        }
        const unsigned chunk = chunk_of(b);
        int rc = ensure_stage(h, sizeof(double) * 4 * (size_t)chunk);
        if (rc) return rc;
        double* d = h->d_stage;
        for (unsigned c0 = 0; c0 < b.ncells; c0 += chunk) {
            const unsigned n = (b.ncells - c0 < chunk) ? b.ncells - c0 : chunk;
            double* dd[4];
            for (int q = 0; q < 4; ++q) dd[q] = outs[q] ? d + (size_t)q * chunk : nullptr;
            FPC_CK(h,
                   launch_moments(h->precision, g, parity, h->F[0], h->F[1], h->F[2], dd[0], dd[1], dd[2], dd[3], c0,
                                  n, h->stream),
                   "moments kernel");
            for (int q = 0; q < 4; ++q)
                if (outs[q])
                    FPC_CK(h,
                           cudaMemcpyAsync(outs[q] + b.cell0 + c0, dd[q], sizeof(double) * n, cudaMemcpyDeviceToHost,
                                           h->stream),
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
    const int parity = (int)(h->steps & 1);
    for (const Box& b : h->boxes)
        FPC_CK(h,
               launch_diag_partial(h->precision, geom_of(h, b), parity, h->F[0], h->F[1], h->F[2],
                                   h->d_part + 5 * (size_t)b.diag0, h->stream),
               "diagnostics kernel");
    FPC_CK(h, launch_diag_final(h->d_part, (int)h->diag_parts, h->d_diag, h->stream), "diagnostics kernel");
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
    const int parity = (int)(h->steps & 1);
    const size_t pitch = sizeof(double) * h->total_cells;
    for (const Box& b : h->boxes) {
        const unsigned chunk = chunk_of(b);
        int rc = ensure_stage(h, sizeof(double) * 27 * (size_t)chunk);
        if (rc) return rc;
        const BoxGeom g = geom_of(h, b);
        for (unsigned c0 = 0; c0 < b.ncells; c0 += chunk) {
            const unsigned n = (b.ncells - c0 < chunk) ? b.ncells - c0 : chunk;
            FPC_CK(h, launch_get_pops(h->precision, g, parity, h->d_stage, chunk, c0, n, h->stream),
                   "populations kernel");
            FPC_CK(h,
                   cudaMemcpy2DAsync(f + b.cell0 + c0, pitch, h->d_stage, sizeof(double) * chunk, sizeof(double) * n,
                                     27, cudaMemcpyDeviceToHost, h->stream),
                   "copy populations");
        }
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
    for (int i = 0; i < n; ++i)
        if (cells[i] < 0 || (unsigned long long)cells[i] >= h->total_cells)
            return fail(h, FPCLBM_ERR_ARG, "cell index out of range");
    const size_t out_bytes = sizeof(double) * 27 * (size_t)n;
    const size_t idx_bytes = (sizeof(unsigned) * (size_t)n + 255) / 256 * 256;
    int rc = ensure_stage(h, 2 * out_bytes + idx_bytes);
    if (rc) return rc;
    double* d_out = h->d_stage;
    unsigned* d_idx = reinterpret_cast<unsigned*>(reinterpret_cast<char*>(h->d_stage) + 2 * out_bytes);
    std::vector<double> host(27 * (size_t)n);
    std::vector<unsigned> idx;
    std::vector<int> which;
    const int parity = (int)(h->steps & 1);
    for (const Box& b : h->boxes) {
        idx.clear();
        which.clear();
        for (int i = 0; i < n; ++i)
            if ((unsigned long long)cells[i] >= b.cell0 && (unsigned long long)cells[i] < (unsigned long long)b.cell0 + b.ncells) {
                idx.push_back((unsigned)(cells[i] - b.cell0));
                which.push_back(i);
            }
        if (idx.empty()) continue;
        const unsigned m = (unsigned)idx.size();
        FPC_CK(h, cudaMemcpyAsync(d_idx, idx.data(), sizeof(unsigned) * m, cudaMemcpyHostToDevice, h->stream),
               "copy cells");
        FPC_CK(h, launch_get_pops_at(h->precision, geom_of(h, b), parity, d_idx, m, d_out, h->stream),
               "populations kernel");
        std::vector<double> part(27 * (size_t)m);
        FPC_CK(h, cudaMemcpyAsync(part.data(), d_out, sizeof(double) * 27 * m, cudaMemcpyDeviceToHost, h->stream),
               "copy populations");
        FPC_CK(h, cudaStreamSynchronize(h->stream), "populations sync");
        for (unsigned k = 0; k < m; ++k)
            for (int a = 0; a < 27; ++a) host[(size_t)a * n + which[k]] = part[(size_t)a * m + k];
    }
    std::memcpy(f, host.data(), sizeof(double) * 27 * (size_t)n);
    return FPCLBM_OK;
}

int fpclbm_set_populations(fpclbm_t h, const double* f)
{
    if (!h) return FPCLBM_ERR_ARG;
    h->err.clear();
    if (!f) return fail(h, FPCLBM_ERR_ARG, "f is NULL");
    const size_t pitch = sizeof(double) * h->total_cells;
    for (const Box& b : h->boxes) {
        const unsigned chunk = chunk_of(b);
        int rc = ensure_stage(h, sizeof(double) * 27 * (size_t)chunk);
        if (rc) return rc;
        const BoxGeom g = geom_of(h, b);
        for (unsigned c0 = 0; c0 < b.ncells; c0 += chunk) {
            const unsigned n = (b.ncells - c0 < chunk) ? b.ncells - c0 : chunk;
            FPC_CK(h,
                   cudaMemcpy2DAsync(h->d_stage, sizeof(double) * chunk, f + b.cell0 + c0, pitch, sizeof(double) * n,
                                     27, cudaMemcpyHostToDevice, h->stream),
                   "copy populations");
            FPC_CK(h, launch_set_pops(h->precision, g, h->d_stage, chunk, c0, n, h->stream), "populations kernel");
        }
    }
    FPC_CK(h, cudaStreamSynchronize(h->stream), "populations sync");
    h->initialized = true;
    h->steps = 0;
    return FPCLBM_OK;
}

// The learned closure's weights (4865 bf16 bit patterns) in the device layout of closure.cuh
// (CP_WORDS 32-bit words, zero-initialised by the caller): per-lane mma fragments of both layers,
// the fp32 biases and output layer, and layer 2's bias fragments.
static void pack_closure(const unsigned short* w, uint32_t* pk)
{
    // re-pack into the per-lane mma fragment order of closure.cuh: for lane (g = lane/4,
    // t = lane%4) and n-tile nt, output n = 8 nt + g; a 32-bit word holds two bf16 of
    // consecutive k (lower k in the low half): k = 2t, 2t+1 and k = 2t+8, 2t+9
    auto wb = [&](int idx) -> uint32_t { return w[idx]; };
    // layer 1: K column 9 carries b1 (the kernel's input 9 is the constant 1)
    auto w1 = [&](int n, int k) -> uint32_t { return k < 9 ? wb(CL_W1 + 9 * n + k) : k == 9 ? wb(CL_B1 + n) : 0u; };
    auto w2 = [&](int n, int k) -> uint32_t { return wb(CL_W2 + 64 * n + k); };
    for (int lane = 0; lane < 32; ++lane) {
        const int g = lane / 4, t = lane % 4;
        for (int nt = 0; nt < 8; ++nt) {
            const int n = 8 * nt + g;
            pk[CP_F1 + (nt * 32 + lane) * 2] = w1(n, 2 * t) | (w1(n, 2 * t + 1) << 16);
            pk[CP_F1 + (nt * 32 + lane) * 2 + 1] = w1(n, 2 * t + 8) | (w1(n, 2 * t + 9) << 16);
            for (int kt = 0; kt < 4; ++kt) {
                const int k = 16 * kt + 2 * t;
                pk[CP_F2 + ((nt * 4 + kt) * 32 + lane) * 2] = w2(n, k) | (w2(n, k + 1) << 16);
                pk[CP_F2 + ((nt * 4 + kt) * 32 + lane) * 2 + 1] = w2(n, k + 8) | (w2(n, k + 9) << 16);
            }
            // layer 2's bias as a fifth K tile whose only non-zero row (k = 64, input 1) holds b2
            pk[CP_F2B + nt * 32 + lane] = t == 0 ? wb(CL_B2 + n) : 0u;
        }
    }
    for (int j = 0; j < 64; ++j) {
        pk[CP_B1 + j] = wb(CL_B1 + j) << 16;  // fp32 bit patterns of the bf16 values
        pk[CP_B2 + j] = wb(CL_B2 + j) << 16;
        pk[CP_W3 + j] = wb(CL_W3 + j) << 16;
    }
    pk[CP_B3] = wb(CL_B3) << 16;
}

int fpclbm_closure_pack(const unsigned short* w, int n_params, unsigned int* out, int out_words)
{
    if (!w || !out || n_params != CL_N || out_words != CP_WORDS) return FPCLBM_ERR_ARG;
    std::vector<uint32_t> pk(CP_WORDS, 0u);
    pack_closure(w, pk.data());
    std::memcpy(out, pk.data(), sizeof(uint32_t) * CP_WORDS);
    return FPCLBM_OK;
}

int fpclbm_set_closure(fpclbm_t h, const unsigned short* w, int n_params)
{
    if (!h) return FPCLBM_ERR_ARG;
    h->err.clear();
    if (!w) return fail(h, FPCLBM_ERR_ARG, "weights are NULL");
    if (n_params != 4865) return fail(h, FPCLBM_ERR_ARG, "closure needs exactly 4865 parameters");
    for (int i = 0; i < n_params; ++i) {
        const unsigned bits = (unsigned)w[i] << 16;  // bf16 -> fp32 is exact
        float v;
        std::memcpy(&v, &bits, sizeof v);
        if (!std::isfinite(v)) return fail(h, FPCLBM_ERR_ARG, "non-finite closure weight");
    }
    std::vector<uint32_t> pk(CP_WORDS, 0u);
    pack_closure(w, pk.data());
    if (!h->d_closure) {
        cudaError_t e = rt_malloc(&h->d_closure, sizeof(uint32_t) * CP_WORDS);
        if (e != cudaSuccess) return fail(h, FPCLBM_ERR_ALLOC, "closure weights");
    }
    FPC_CK(h, cudaMemcpyAsync(h->d_closure, pk.data(), sizeof(uint32_t) * CP_WORDS, cudaMemcpyHostToDevice, h->stream),
           "copy closure");
    FPC_CK(h, cudaStreamSynchronize(h->stream), "closure sync");
    h->have_closure = true;
    h->graph_valid = false;
    return FPCLBM_OK;
}

int fpclbm_state_bytes(fpclbm_t h, unsigned long long* bytes)
{
    if (!h) return FPCLBM_ERR_ARG;
    h->err.clear();
    if (!bytes) return fail(h, FPCLBM_ERR_ARG, "bytes is NULL");
    unsigned long long n = 0;
    for (const Box& b : h->boxes) n += 27ull * b.stride * elem_size(h->precision);
    *bytes = n;
    return FPCLBM_OK;
}

int fpclbm_get_state(fpclbm_t h, void* raw, unsigned long long bytes, long long* steps)
{
    if (!h) return FPCLBM_ERR_ARG;
    h->err.clear();
    unsigned long long need = 0;
    fpclbm_state_bytes(h, &need);
    if (!raw || !steps) return fail(h, FPCLBM_ERR_ARG, "raw and steps must not be NULL");
    if (bytes != need) return fail(h, FPCLBM_ERR_ARG, "raw state has " + std::to_string(need) + " bytes");
    if (!h->initialized) return fail(h, FPCLBM_ERR_STATE, "populations not initialised");
    FPC_CK(h, cudaMemcpyAsync(raw, h->d_pop, need, cudaMemcpyDeviceToHost, h->stream), "copy state");
    FPC_CK(h, cudaStreamSynchronize(h->stream), "state sync");
    *steps = h->steps;
    return FPCLBM_OK;
}

int fpclbm_set_state(fpclbm_t h, const void* raw, unsigned long long bytes, long long steps)
{
    if (!h) return FPCLBM_ERR_ARG;
    h->err.clear();
    unsigned long long need = 0;
    fpclbm_state_bytes(h, &need);
    if (!raw) return fail(h, FPCLBM_ERR_ARG, "raw is NULL");
    if (bytes != need) return fail(h, FPCLBM_ERR_ARG, "raw state has " + std::to_string(need) + " bytes");
    if (steps < 0) return fail(h, FPCLBM_ERR_ARG, "negative step count");
    FPC_CK(h, cudaMemcpyAsync(h->d_pop, raw, need, cudaMemcpyHostToDevice, h->stream), "copy state");
    FPC_CK(h, cudaStreamSynchronize(h->stream), "state sync");
    h->steps = steps;
    h->initialized = true;
    return FPCLBM_OK;
}

int fpclbm_test_alloc_hook(int fail_after, long long* live)
{
    if (fail_after >= -1) g_fail_countdown.store(fail_after);
    if (live) *live = g_live_allocs.load();
    return FPCLBM_OK;
}

}  // extern "C"
