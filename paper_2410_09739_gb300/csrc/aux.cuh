// aux.cuh -- fp64 readers of a box's populations at the current time, shared by
// the off-hot-path kernels (field export, diagnostics, closure data).
#pragma once
#include "internal.h"

namespace fpc {

__device__ __forceinline__ void cell_xyz(const BoxGeom& b, unsigned cell, unsigned& x, unsigned& y, unsigned& z)
{
    z = fdiv(cell, b.div_nxny);
    const unsigned rem = cell - z * (unsigned)(b.nx * b.ny);
    y = fdiv(rem, b.div_nx);
    x = rem - y * b.nx;
}

// Deviations g_s(x) at the current time, whatever the AA parity.
// parity 0: buf[s][x]; parity 1: buf[26-s][x - e_s], or buf[s][x] when the
// source lies in a wall (see cell.cuh).
template <typename S>
__device__ void load_cell(const BoxGeom& b, int parity, unsigned cell, double g[27])
{
    const S* buf = static_cast<const S*>(b.buf);
    if (parity == 0) {
        for (int s = 0; s < 27; ++s) g[s] = Store<S>::ldd(buf + (size_t)s * b.stride + cell);
        return;
    }
    unsigned x, y, z;
    cell_xyz(b, cell, x, y, z);
    const int nx = b.nx, ny = b.ny, nz = b.nz;
    for (int s = 0; s < 27; ++s) {
        const int ex = s % 3 - 1, ey = (s / 3) % 3 - 1, ez = s / 9 - 1;
        const int sx0 = (int)x - ex, sy = (int)y - ey, sz0 = (int)z - ez;
        if (b.walls == 3 && sy >= ny) {  // half channel: specular through the symmetry plane
            const int mx = (sx0 + nx) % nx, mz = (sz0 + nz) % nz;
            g[s] = Store<S>::ldd(buf + (size_t)(20 - s) * b.stride + (size_t)mx + (size_t)nx * ((size_t)y + (size_t)ny * mz));
            continue;
        }
        const bool out_y = b.walls >= 1 && (sy < 0 || sy >= ny);
        const bool out_xz = b.walls == 2 && (sx0 < 0 || sx0 >= nx || sz0 < 0 || sz0 >= nz);
        if (out_y || out_xz) {
            g[s] = Store<S>::ldd(buf + (size_t)s * b.stride + cell);
            continue;
        }
        const int sx = ((int)x - ex + nx) % nx, syw = (sy + ny) % ny, sz = ((int)z - ez + nz) % nz;
        const size_t src = (size_t)sx + (size_t)nx * ((size_t)syw + (size_t)ny * sz);
        g[s] = Store<S>::ldd(buf + (size_t)(26 - s) * b.stride + src);
    }
}

// Density and half-force velocity (Appendix D Step 7) from deviations.
__device__ __forceinline__ void fields_of(const double g[27], double Fx, double Fy, double Fz, double& rho, double& ux,
                                          double& uy, double& uz)
{
    double dr = 0, jx = 0, jy = 0, jz = 0;
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
