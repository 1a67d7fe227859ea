// internal.h -- host-side interfaces between the libfpclbm translation units.
#pragma once
#include <cuda_runtime.h>
#include "common.cuh"

namespace fpc {

// Storage precisions (values of the FPCLBM_* precision enum).
enum { P_FP64 = 0, P_FP32 = 1, P_FP16 = 2, P_BF16 = 3 };

// Launch configuration of the single-box step kernel (autotuned).
struct StepLaunch {
    int block;     // threads per block (<= 256)
    int minb = 2;  // register-cap variant: minimum resident blocks of 256 threads per SM (2, 3 or 4)
    int pipe = 0;  // 1: software-pipelined persistent variant (cp.async prefetch), 4/8-byte storage only;
                   // 2: paired variant (two cells per thread on the packed fp32 pipe);
                   // 3: row-staged paired variant (bulk copies of whole slot rows through shared memory)
    int stages = 2;  // variant 3: shared-memory input stages per block (2..6)
};

// One time step of a single box.  odd selects the AA-pattern parity (0: own
// slots, 1: neighbour slots), bc the boundary kind (BC_*), force the source
// terms, mode one of the MODE_* collision modes (common.cuh).
cudaError_t launch_step(int precision, int odd, int bc, int force, int mode, const StepArgs<double>& a64,
                        const StepArgs<float>& a32, const StepLaunch& cfg, cudaStream_t st);

// Auxiliary kernels (aux_kernels.cu).  All fields double.
struct BoxGeom {
    void* buf;
    unsigned stride;
    unsigned ncells;
    int nx, ny, nz;
    int walls;  // 0: periodic, 1: bounce-back walls at y = -1/2, ny - 1/2, 2: on all six faces,
                // 3: half channel (wall at y = -1/2, specular symmetry plane at y = ny - 1/2)
    FastDiv div_nx, div_nxny;
};

// populations <- equilibrium of (rho, u) for cells [c0, c0 + n)
cudaError_t launch_init_eq(int precision, const BoxGeom& b, const double* rho, const double* ux, const double* uy,
                           const double* uz, unsigned c0, unsigned n, cudaStream_t st);
// rho, u (Step 7 with half force) of cells [c0, c0+n); parity = steps & 1; null outputs skipped
cudaError_t launch_moments(int precision, const BoxGeom& b, int parity, double Fx, double Fy, double Fz, double* rho,
                           double* ux, double* uy, double* uz, unsigned c0, unsigned n, cudaStream_t st);
// full populations in paper alpha order: out[alpha * ld + (c - c0)]
cudaError_t launch_get_pops(int precision, const BoxGeom& b, int parity, double* out, unsigned ld, unsigned c0,
                            unsigned n, cudaStream_t st);
// full populations of listed cells: out[alpha * n + i] for cells[i]
cudaError_t launch_get_pops_at(int precision, const BoxGeom& b, int parity, const unsigned* cells, unsigned n,
                               double* out, cudaStream_t st);
// populations <- in[alpha * ld + (c - c0)] (full f, paper alpha order), natural parity
cudaError_t launch_set_pops(int precision, const BoxGeom& b, const double* in, unsigned ld, unsigned c0, unsigned n,
                            cudaStream_t st);
// fp64 diagnostics: partial sums of (rho, rho u, rho |u|^2 / 2) per block of
// diag_blocks(ncells) into part[5 * k], then one pass over all partials.
int diag_blocks(unsigned ncells);
cudaError_t launch_diag_partial(int precision, const BoxGeom& b, int parity, double Fx, double Fy, double Fz,
                                double* part, cudaStream_t st);
cudaError_t launch_diag_final(const double* part, int nparts, double* out, cudaStream_t st);

// Paper alpha order -> tensor slot (host table, filled from the velocity list).
extern const int kSlotOfAlpha[27];

}  // namespace fpc
