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

// Neighbour coordinates of a cell for the odd step: column, row offset and
// plane offset of x - e for e = -1, 0, +1 (index 0, 1, 2), and whether the
// source row lies inside the fluid (y walls).
struct Nbr {
    unsigned xs[3], yr[3], zp[3];
    bool yin[3];
};

template <bool WALLS>
__device__ __forceinline__ Nbr make_nbr(const CellGeom& G, unsigned cell)
{
    Nbr n;
    const unsigned nx = G.nx, ny = G.ny, nz = G.nz, nxny = nx * ny;
    const unsigned z = fdiv(cell, G.div_nxny);
    const unsigned rem = cell - z * nxny;
    const unsigned y = fdiv(rem, G.div_nx);
    const unsigned x = rem - y * nx;
    n.xs[0] = (x + 1 == nx) ? 0u : x + 1;
    n.xs[1] = x;
    n.xs[2] = (x == 0) ? nx - 1 : x - 1;
    const unsigned yp = (y + 1 == ny) ? 0u : y + 1, ym = (y == 0) ? ny - 1 : y - 1;
    n.yr[0] = yp * nx;
    n.yr[1] = y * nx;
    n.yr[2] = ym * nx;
    n.yin[0] = WALLS ? (y + 1 < ny) : true;
    n.yin[1] = true;
    n.yin[2] = WALLS ? (y > 0) : true;
    const unsigned zpp = (z + 1 == nz) ? 0u : z + 1, zmm = (z == 0) ? nz - 1 : z - 1;
    n.zp[0] = zpp * nxny;
    n.zp[1] = z * nxny;
    n.zp[2] = zmm * nxny;
    return n;
}

// Address read for slot s (the population that streams into the cell).  The
// slot row base buf + row * stride is the same for the whole warp, so it is
// formed separately from the per-thread cell offset (uniform-register base).
template <typename S, bool ODD, bool WALLS>
__device__ __forceinline__ S* load_ptr(S* buf, int s, const Nbr& n, unsigned stride, unsigned cell)
{
    if (!ODD) return buf + (size_t)s * stride + cell;
    const int ix = s % 3, iy = (s / 3) % 3, iz = s / 9;
    if (WALLS && !n.yin[iy]) return buf + (size_t)s * stride + cell;
    return buf + (size_t)(26 - s) * stride + (n.xs[ix] + n.yr[iy] + n.zp[iz]);
}

// Address written for slot s (the destination of the post-collision value).
template <typename S, bool ODD, bool WALLS>
__device__ __forceinline__ S* store_ptr(S* buf, int s, const Nbr& n, unsigned stride, unsigned cell)
{
    if (!ODD) return buf + (size_t)(26 - s) * stride + cell;
    const int ix = s % 3, iy = (s / 3) % 3, iz = s / 9;
    if (WALLS && !n.yin[2 - iy]) return buf + (size_t)(26 - s) * stride + cell;
    return buf + (size_t)s * stride + (n.xs[2 - ix] + n.yr[2 - iy] + n.zp[2 - iz]);
}

template <typename S, typename R, bool ODD, bool WALLS, bool FORCE, int MODE>
__device__ __forceinline__ void update_cell(S* __restrict__ buf, const CellGeom& G, unsigned cell,
                                            const Rates<R>& rt, R Fx, R Fy, R Fz, R om4, R om5, R om6, R om8,
                                            R om9, const float* closure, int* flag)
{
    const unsigned stride = G.stride;
    R g[27];
    Nbr n;
    if (ODD) n = make_nbr<WALLS>(G, cell);
#pragma unroll
    for (int s = 0; s < 27; ++s) g[s] = Store<S>::ld(load_ptr<S, ODD, WALLS>(buf, s, n, stride, cell));

    const bool ok = collide_cell<R, FORCE, MODE>(g, rt, Fx, Fy, Fz, om4, om5, om6, om8, om9, closure);
    if (!ok) atomicOr(flag, 1);

#pragma unroll
    for (int s = 0; s < 27; ++s) Store<S>::st(store_ptr<S, ODD, WALLS>(buf, s, n, stride, cell), g[s]);
}

}  // namespace fpc
