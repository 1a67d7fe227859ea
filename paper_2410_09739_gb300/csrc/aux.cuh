// aux.cuh -- readers of a box's populations at the current time, shared by the
// off-hot-path kernels (field export, diagnostics, closure data).
#pragma once
#include <type_traits>

#include "internal.h"

namespace fpc {

__device__ __forceinline__ void cell_xyz(const BoxGeom& b, unsigned cell, unsigned& x, unsigned& y, unsigned& z)
{
    z = fdiv(cell, b.div_nxny);
    const unsigned rem = cell - z * (unsigned)(b.nx * b.ny);
    y = fdiv(rem, b.div_nx);
    x = rem - y * b.nx;
}

// One stored deviation as T: fp64 (exact for every storage type) or fp32
// (exact for fp32 and the 16-bit types).
template <typename T, typename S>
__device__ __forceinline__ T load_as(const S* p)
{
    if constexpr (std::is_same<T, double>::value)
        return Store<S>::ldd(p);
    else
        return (T)Store<S>::ld(p);
}

// Deviations g_s(x) at the current time, whatever the AA parity.
// parity 0: buf[s][x]; parity 1: buf[26-s][x - e_s], or buf[s][x] when the
// source lies in a wall (see cell.cuh).
template <typename S, typename T>
__device__ __forceinline__ void load_cell(const BoxGeom& b, int parity, unsigned cell, T g[27])
{
    const S* buf = static_cast<const S*>(b.buf);
    if (parity == 0) {
#pragma unroll
        for (int s = 0; s < 27; ++s) g[s] = load_as<T>(buf + (size_t)s * b.stride + cell);
        return;
    }
    unsigned x, y, z;
    cell_xyz(b, cell, x, y, z);
    const int nx = b.nx, ny = b.ny, nz = b.nz;
#pragma unroll
    for (int s = 0; s < 27; ++s) {
        const int ex = s % 3 - 1, ey = (s / 3) % 3 - 1, ez = s / 9 - 1;
        const int sx0 = (int)x - ex, sy = (int)y - ey, sz0 = (int)z - ez;
        if (b.walls == 3 && sy >= ny) {  // half channel: specular through the symmetry plane
            const int mx = (sx0 + nx) % nx, mz = (sz0 + nz) % nz;
            g[s] = load_as<T>(buf + (size_t)(20 - s) * b.stride + (size_t)mx + (size_t)nx * ((size_t)y + (size_t)ny * mz));
            continue;
        }
        const bool out_y = b.walls >= 1 && (sy < 0 || sy >= ny);
        const bool out_xz = b.walls == 2 && (sx0 < 0 || sx0 >= nx || sz0 < 0 || sz0 >= nz);
        if (out_y || out_xz) {
            g[s] = load_as<T>(buf + (size_t)s * b.stride + cell);
            continue;
        }
        const int sx = ((int)x - ex + nx) % nx, syw = (sy + ny) % ny, sz = ((int)z - ez + nz) % nz;
        const size_t src = (size_t)sx + (size_t)nx * ((size_t)syw + (size_t)ny * sz);
        g[s] = load_as<T>(buf + (size_t)(26 - s) * b.stride + src);
    }
}

// Compensated fp32 summation: s + c carries the running sum of the added terms
// with the rounding error of every addition captured in c (Knuth's TwoSum
// error-free transformation, accumulated as in Ogita, Rump & Oishi, "Accurate
// sum and dot product", SIAM J. Sci. Comput. 26 (2005), Algorithm 4.4).  The
// result is as accurate as a sum in twice the working precision, which for 27
// deviations keeps the fp64 value of the sum in all but the last bits.  The
// round-to-nearest intrinsics keep the compiler from contracting or
// reassociating the error terms.
__device__ __forceinline__ void sum2_add(float& s, float& c, float x)
{
    const float t = __fadd_rn(s, x);
    const float bp = __fsub_rn(t, s);
    const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(x, bp));
    s = t;
    c = __fadd_rn(c, err);
}

// Density and half-force velocity (Appendix D Step 7) from deviations.
__device__ __forceinline__ void fields_of(const double g[27], double Fx, double Fy, double Fz, double& rho, double& ux,
                                          double& uy, double& uz)
{
    double dr = 0, jx = 0, jy = 0, jz = 0;
#pragma unroll
    for (int s = 0; s < 27; ++s) {
        dr += g[s];
        jx += (s % 3 - 1) * g[s];
        jy += ((s / 3) % 3 - 1) * g[s];
        jz += (s / 9 - 1) * g[s];
    }
    rho = 1.0 + dr;
    ux = (jx + 0.5 * Fx) / rho;
    uy = (jy + 0.5 * Fy) / rho;
    uz = (jz + 0.5 * Fz) / rho;
}

}  // namespace fpc
