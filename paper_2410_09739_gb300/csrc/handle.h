// handle.h -- the fpclbm handle shared by the host translation units.
//
// A handle owns one device allocation holding the populations of all its
// boxes (a single box, or an ensemble of independent periodic boxes).  Box b
// occupies 27 * stride_b elements starting at element offset off_b; its cells
// are numbered cell0_b .. cell0_b + ncells_b - 1 in the concatenated field and
// population arrays of the C ABI.
#pragma once
#include <string>
#include <vector>

#include "fpclbm.h"  // include/ is on the include path
#include "internal.h"
#include "pair.cuh"

namespace fpc {

struct Box {
    int nx = 0, ny = 0, nz = 0;
    unsigned ncells = 0, stride = 0;
    unsigned long long off = 0;  // element offset of slot row 0
    unsigned cell0 = 0;          // first global cell index
    double tau = 1.0;            // ensemble: per-box shear relaxation time
    unsigned tile0 = 0, ntiles = 0;
    unsigned diag0 = 0;          // first diagnostics partial of this box
};

// Device table entry of an ensemble box.
struct EnsBox {
    unsigned long long off;
    unsigned stride, ncells;
    int nx, ny, nz;
    FastDiv div_nx, div_nxny;
    float om_shear;
    unsigned tile0;
};

struct EnsArgs {
    void* buf;
    const EnsBox* boxes;
    const unsigned* tile_box;
    unsigned ntiles;
    unsigned tile_cells;  // cells per tile (a multiple of the block size; of twice it when paired)
    Rates<float> rates;
    float Fx, Fy, Fz;
    Rates<f2> rates2;     // the same, duplicated into both lanes (paired variant)
    f2 Fx2, Fy2, Fz2;
    int* flag;
};

// Ensemble step launch (ensemble.cu).  grid = persistent blocks; variant 2 =
// two cells per thread (blocks of 128 threads, tiles of 256 cells).
cudaError_t launch_ens_step(int odd, int force, int mode, const EnsArgs& a, int block, int minb, int grid,
                            int variant, cudaStream_t st);
int ens_max_blocks_per_sm(int block, int minb, int mode, int variant);

}  // namespace fpc

struct fpclbm {
    std::vector<fpc::Box> boxes;
    bool ensemble = false;
    unsigned long long total_cells = 0;
    int precision = 0, bc = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;
    int device = 0, sm_count = 0;
    // device state
    void* d_pop = nullptr;
    int* d_flag = nullptr;
    int* h_flag = nullptr;  // pinned
    double* d_stage = nullptr;
    size_t stage_bytes = 0;
    double* d_part = nullptr;
    unsigned diag_parts = 0;
    double* d_diag = nullptr;
    double* h_diag = nullptr;  // pinned
    float* d_closure = nullptr;
    bool have_closure = false;
    fpc::EnsBox* d_ens_boxes = nullptr;
    unsigned* d_tile_box = nullptr;
    unsigned ntiles = 0;
    int tile_cells = 256;
    bool initialized = false;
    long long steps = 0;
    // parameters (Appendix D Step 3 numbering)
    double omega[27];
    double F[3] = {0, 0, 0};
    double lid[2] = {0, 0};  // x and z velocity of the wall y = ny - 1/2
    double smag[3] = {0, 0, 0};  // Smagorinsky C_s, u*, A+
    void* d_smag = nullptr;      // (C_s D(y))^2 per row, storage of the arithmetic type
    bool smag_dirty = true;
    int diffusion = FPCLBM_DIFF_FP;
    // launch configuration (autotuned) and graph cache
    int block = 256;
    int minb = 2;  // register-cap variant (see step_kernel.cuh)
    int pipe = 0;  // 1: cp.async-pipelined persistent variant (see step_kernel.cuh)
    int grid = 0;  // ensemble: persistent blocks
    bool tuned = false;
    cudaGraphExec_t graph = nullptr;
    bool graph_valid = false;
    std::string err;
};

namespace fpc {
// Shared host helpers (fpclbm.cu).
int fail(fpclbm* h, int code, const std::string& msg);
int cuda_fail(fpclbm* h, cudaError_t e, const char* what);
void rates_from_params(double tau, double drift, double om[27]);
bool rates_valid(const double om[27], std::string& why);
size_t elem_size(int precision);
int alloc_common(fpclbm* h);  // flag, diagnostics, capture stream
extern thread_local std::string g_create_error;
}  // namespace fpc
