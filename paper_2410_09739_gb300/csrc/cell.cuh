// cell.cuh -- one cell's fused AA-pattern update: load 27, collide, store 27.
//
// AA pattern, one buffer updated in place:
//   even step: read own slots buf[s][x], collide, write buf[26-s][x]
//              (post-collision values parked in the opposite slot);
//   odd step:  read buf[26-s][x - e_s] (the streamed value of Step 6),
//              collide, write buf[s][x + e_s].
// Each thread reads and writes the same 27 addresses in both parities, so
// the update is race-free without a second buffer.  Half-way bounce-back on
// y walls: an odd-step read whose source x - e_s lies in a wall takes
// buf[s][x] (the reflected post-collision value parked there by the even
// step), and an odd-step write whose destination x + e_s lies in a wall goes
// to buf[26-s][x], where the next even step reads it as the reflected
// population.  Periodic wrap in x, z (and y without walls).
//
// Traffic per cell update: 27 reads + 27 writes of the storage type.
#pragma once
#include "closure.cuh"
#include "collide.cuh"

namespace fpc {

struct CellGeom {
    unsigned stride;  // elements between slot rows
    int nx, ny, nz;
    FastDiv div_nx, div_nxny;
};

template <typename S, typename R, bool ODD, bool WALLS, bool FORCE, int MODE>
__device__ __forceinline__ void update_cell(S* __restrict__ buf, const CellGeom& G, unsigned cell,
                                            const Rates<R>& rt, R Fx, R Fy, R Fz, R om4, R om5, R om6, R om8,
                                            R om9, const float* closure, int* flag)
{
    const unsigned stride = G.stride;
    R g[27];
    unsigned xs[3], yr[3], zp[3];  // source column, row offset, plane offset for e = -1, 0, +1
    bool yin[3];                   // source row inside the fluid (walls)
    if (ODD) {
        const unsigned nx = G.nx, ny = G.ny, nz = G.nz, nxny = nx * ny;
        const unsigned z = fdiv(cell, G.div_nxny);
        const unsigned rem = cell - z * nxny;
        const unsigned y = fdiv(rem, G.div_nx);
        const unsigned x = rem - y * nx;
        // source of slot component e is x - e
        xs[0] = (x + 1 == nx) ? 0u : x + 1;
        xs[1] = x;
        xs[2] = (x == 0) ? nx - 1 : x - 1;
        const unsigned yp = (y + 1 == ny) ? 0u : y + 1, ym = (y == 0) ? ny - 1 : y - 1;
        yr[0] = yp * nx;
        yr[1] = y * nx;
        yr[2] = ym * nx;
        yin[0] = WALLS ? (y + 1 < ny) : true;
        yin[1] = true;
        yin[2] = WALLS ? (y > 0) : true;
        const unsigned zpp = (z + 1 == nz) ? 0u : z + 1, zmm = (z == 0) ? nz - 1 : z - 1;
        zp[0] = zpp * nxny;
        zp[1] = z * nxny;
        zp[2] = zmm * nxny;
#pragma unroll
        for (int s = 0; s < 27; ++s) {
            const int ix = s % 3, iy = (s / 3) % 3, iz = s / 9;
            if (WALLS && !yin[iy])
                g[s] = Store<S>::ld(buf + (size_t)(s * stride + cell));
            else
                g[s] = Store<S>::ld(buf + (size_t)((26 - s) * stride + xs[ix] + yr[iy] + zp[iz]));
        }
    } else {
#pragma unroll
        for (int s = 0; s < 27; ++s) g[s] = Store<S>::ld(buf + (size_t)(s * stride + cell));
    }

    const bool ok = collide_cell<R, FORCE, MODE>(g, rt, Fx, Fy, Fz, om4, om5, om6, om8, om9, closure);
    if (!ok) atomicOr(flag, 1);

    if (ODD) {
        // destination of slot component e is x + e: the source of -e
#pragma unroll
        for (int s = 0; s < 27; ++s) {
            const int ix = s % 3, iy = (s / 3) % 3, iz = s / 9;
            if (WALLS && !yin[2 - iy])
                Store<S>::st(buf + (size_t)((26 - s) * stride + cell), g[s]);
            else
                Store<S>::st(buf + (size_t)(s * stride + xs[2 - ix] + yr[2 - iy] + zp[2 - iz]), g[s]);
        }
    } else {
#pragma unroll
        for (int s = 0; s < 27; ++s) Store<S>::st(buf + (size_t)((26 - s) * stride + cell), g[s]);
    }
}

}  // namespace fpc
