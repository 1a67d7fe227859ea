// common.cuh -- shared definitions of the libfpclbm CUDA sources (sm_103a).
//
// Memory layout of the populations (one buffer, in place, AA pattern):
//   buf[s * stride + cell],  s = (ex+1) + 3 (ey+1) + 9 (ez+1)  (tensor order),
//   cell = x + nx (y + ny z).  Each entry stores the deviation g = f - w_s from
//   the rest state w_s = w1(ex) w1(ey) w1(ez), w1 = (1/6, 2/3, 1/6) (the
//   equilibrium at rho = 1, u = 0 of the D3Q27 lattice, Sec. 3).  The
//   opposite of slot s is 26 - s.  stride is the cell count rounded up to a
//   multiple of 64 so that every slot row starts 128-byte aligned.
#pragma once
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace fpc {

// Attractor modes of the collision: FP diffusion tensor, Maxwellian (MCM),
// FP with the learned shear-rate correction, FP with the Smagorinsky eddy
// viscosity (van Driest damped) in the shear rates.  MODE_FP_R1 and
// MODE_EQ_R1 are the FP and MCM modes in the paper's default setting, every
// rate of order >= 3 equal to 1: the post-collision moments of orders 3-6 are
// then their attractors plus half their sources (kappa + 1 (kappa^Mv - kappa)
// + (1 - 1/2) sigma), with no grouping; without force the pre-collision
// moments of those orders are not formed at all.
// MODE_LEARNED_R1 is the learned mode with the unit rates of orders 3-6.
enum { MODE_FP = 0, MODE_EQ = 1, MODE_LEARNED = 2, MODE_SMAG = 3, MODE_FP_R1 = 4, MODE_EQ_R1 = 5, MODE_LEARNED_R1 = 6 };

// FP or MCM attractors with the full register-cap / pipelined / paired variant set.
__host__ __device__ constexpr bool plain_mode(int m) { return m == MODE_FP || m == MODE_EQ || m == MODE_FP_R1 || m == MODE_EQ_R1; }
__host__ __device__ constexpr bool eq_mode(int m) { return m == MODE_EQ || m == MODE_EQ_R1; }
__host__ __device__ constexpr bool r1_mode(int m) { return m == MODE_FP_R1 || m == MODE_EQ_R1 || m == MODE_LEARNED_R1; }
__host__ __device__ constexpr bool learned_mode(int m) { return m == MODE_LEARNED || m == MODE_LEARNED_R1; }

// Boundary kinds of the step kernel: periodic box; half-way bounce-back walls
// at y = -1/2 and ny - 1/2 (x, z periodic); the same with the wall at
// y = ny - 1/2 moving; closed box (bounce-back on all six faces) whose wall
// at y = ny - 1/2 moves (lid-driven cavity; the lid may be at rest); half
// channel: bounce-back wall at y = -1/2, specular-reflection symmetry plane
// at y = ny - 1/2 (x, z periodic).
enum { BC_PERIODIC = 0, BC_WALLS_Y = 1, BC_WALLS_Y_LID = 2, BC_BOX_LID = 3, BC_HALF_CHANNEL = 4 };

// Boundary kinds whose walls rest and that have the register-cap variants.
__host__ __device__ constexpr bool bc_fixed(int bc) { return bc == BC_PERIODIC || bc == BC_WALLS_Y || bc == BC_HALF_CHANNEL; }

// Unsigned division by a runtime constant d < 2^31 for numerators n < 2^31:
// q = (umulhi(n, m) + n) >> s with s = ceil(log2 d), m = floor(2^32 (2^s - d) / d) + 1
// (Granlund & Montgomery, "Division by invariant integers using multiplication", 1994).
struct FastDiv {
    unsigned d, m, s;
};

inline FastDiv make_fastdiv(unsigned d)
{
    FastDiv f;
    f.d = d;
    unsigned s = 0;
    while ((1ull << s) < d) ++s;
    f.s = s;
    f.m = (unsigned)(((1ull << 32) * ((1ull << s) - d)) / d + 1ull);
    return f;
}

__device__ __forceinline__ unsigned fdiv(unsigned n, const FastDiv& f)
{
    return (__umulhi(n, f.m) + n) >> f.s;
}

// Relaxation data of one box: omega_j, 1 - omega_j, 1 - omega_j / 2 in the
// numbering of Appendix D Step 3 (0:000 ... 26:222).  Entries 0..3 (the
// conserved moments) are not read by the kernels: they cancel in exact
// arithmetic (see collide.cuh, order 1).
template <typename R>
struct Rates {
    R om[27];
    R keep[27];
    R src[27];
};

// Arguments of one single-box step launch.
template <typename R>
struct StepArgs {
    void* buf;            // populations, storage type
    unsigned stride;      // elements between slot rows
    unsigned ncells;      // nx * ny * nz
    int nx, ny, nz;
    FastDiv div_nx, div_nxny;
    R Fx, Fy, Fz;         // body force
    R lid6x, lid6z;       // 2 / cs^2 = 6 times the velocity of the wall y = ny - 1/2 (BC_*_LID)
    Rates<R> rates;
    int* flag;            // set to 1 by any cell with rho <= 0 or non-finite
    const float* closure; // packed MLP weights (learned mode), else null
    const R* smag;        // (C_s Delta D(y))^2 per row y (Smagorinsky mode), else null
};

// Storage traits: load as compute type R, store from R with round-to-nearest.
template <typename S>
struct Store;
template <>
struct Store<double> {
    __device__ __forceinline__ static double ld(const double* p) { return *p; }
    __device__ __forceinline__ static void st(double* p, double v) { *p = v; }
    __device__ __forceinline__ static double ldd(const double* p) { return *p; }
    __device__ __forceinline__ static double fromd(double v) { return v; }
};
template <>
struct Store<float> {
    __device__ __forceinline__ static float ld(const float* p) { return *p; }
    __device__ __forceinline__ static void st(float* p, float v) { *p = v; }
    __device__ __forceinline__ static double ldd(const float* p) { return (double)*p; }
    __device__ __forceinline__ static float fromd(double v) { return (float)v; }
};
template <>
struct Store<__half> {
    __device__ __forceinline__ static float ld(const __half* p) { return __half2float(*p); }
    __device__ __forceinline__ static void st(__half* p, float v) { *p = __float2half_rn(v); }
    __device__ __forceinline__ static double ldd(const __half* p) { return (double)__half2float(*p); }
    __device__ __forceinline__ static __half fromd(double v) { return __double2half(v); }
};
template <>
struct Store<__nv_bfloat16> {
    __device__ __forceinline__ static float ld(const __nv_bfloat16* p) { return __bfloat162float(*p); }
    __device__ __forceinline__ static void st(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }
    __device__ __forceinline__ static double ldd(const __nv_bfloat16* p) { return (double)__bfloat162float(*p); }
    __device__ __forceinline__ static __nv_bfloat16 fromd(double v) { return __double2bfloat16(v); }
};

// 1D rest weights at e = -1, 0, +1 and rest central moments (1, 0, cs^2) per axis.
__host__ __device__ constexpr double w1(int i) { return i == 1 ? 2.0 / 3.0 : 1.0 / 6.0; }
__host__ __device__ constexpr double r1(int k) { return k == 0 ? 1.0 : (k == 1 ? 0.0 : 1.0 / 3.0); }

// Rest weight of tensor slot s.
__host__ __device__ constexpr double wslot(int s) { return w1(s % 3) * w1((s / 3) % 3) * w1(s / 9); }

}  // namespace fpc
