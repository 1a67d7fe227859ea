// cell.cuh -- one cell's fused AA-pattern update: load 27, collide, store 27.
//
// AA pattern, one buffer updated in place:
//   even step: read own slots buf[s][x], collide, write buf[26-s][x]
//              (post-collision values parked in the opposite slot);
//   odd step:  read buf[26-s][x - e_s] (the streamed value of Step 6),
//              collide, write buf[s][x + e_s].
// Each thread reads and writes the same 27 addresses in both parities, so
// the update is race-free without a second buffer.  Half-way bounce-back
// (y walls, or all six faces of a closed box): an odd-step read whose source
// x - e_s lies in a wall takes buf[s][x] (the reflected post-collision value
// parked there by the even step), and an odd-step write whose destination
// x + e_s lies in a wall goes to buf[26-s][x], where the next even step reads
// it as the reflected population.  Periodic wrap on the other axes.
//
// Symmetry plane y = ny - 1/2 of the half channel (Sec. 4, turbulent channel):
// a population leaving the top row along (ex, +1, ez) comes back along
// (ex, -1, ez) at x + (ex, 0, ez) (specular reflection).  Only the odd step
// sees it: the read of slot s (e_y = -1) of a top-row cell takes the value
// parked by the even step at x - (ex, 0, ez) in slot 20 - s (the opposite of
// the mirror image of s), and the write of slot s (e_y = +1) goes to slot
// s - 6 (its mirror image) at x + (ex, 0, ez), the address the receiving
// thread read for that slot, so the in-place update stays race-free.
//
// Moving wall y = ny - 1/2 (Sec. 4, cubic cavity): a post-collision value of
// a top-row cell with e_y = +1 is reflected by that wall in either parity, so
// the momentum correction -2 w_s rho (e_s . u_w) / cs^2 is applied to it just
// before it is stored, with rho the cell's density.
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
// source lies inside the fluid on each axis (walls).
struct Nbr {
    unsigned xs[3], yz[3][3];  // column of x - e_x; row + plane offset of (y - e_y, z - e_z)
    bool xin[3], yin[3], zin[3];
};

template <int BC>
__device__ __forceinline__ Nbr make_nbr(const CellGeom& G, unsigned cell)
{
    constexpr bool WY = BC != BC_PERIODIC, WXZ = BC == BC_BOX_LID;  // half channel: rows tested like walls
    Nbr n;
    const unsigned nx = G.nx, ny = G.ny, nz = G.nz, nxny = nx * ny;
    const unsigned z = fdiv(cell, G.div_nxny);
    const unsigned rem = cell - z * nxny;
    const unsigned y = fdiv(rem, G.div_nx);
    const unsigned x = rem - y * nx;
    n.xs[0] = (x + 1 == nx) ? 0u : x + 1;
    n.xs[1] = x;
    n.xs[2] = (x == 0) ? nx - 1 : x - 1;
    n.xin[0] = WXZ ? (x + 1 < nx) : true;
    n.xin[1] = true;
    n.xin[2] = WXZ ? (x > 0) : true;
    const unsigned yp = (y + 1 == ny) ? 0u : y + 1, ym = (y == 0) ? ny - 1 : y - 1;
    const unsigned yr[3] = {yp * nx, y * nx, ym * nx};
    n.yin[0] = WY ? (y + 1 < ny) : true;
    n.yin[1] = true;
    n.yin[2] = WY ? (y > 0) : true;
    n.zin[0] = WXZ ? (z + 1 < nz) : true;
    n.zin[1] = true;
    n.zin[2] = WXZ ? (z > 0) : true;
    const unsigned zpp = (z + 1 == nz) ? 0u : z + 1, zmm = (z == 0) ? nz - 1 : z - 1;
    const unsigned zp[3] = {zpp * nxny, z * nxny, zmm * nxny};
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int k = 0; k < 3; ++k) n.yz[j][k] = yr[j] + zp[k];
    return n;
}

// Address read for slot s (the population that streams into the cell).  The
// slot row base buf + row * stride is the same for the whole warp, so it is
// formed separately from the per-thread cell offset (uniform-register base).
// Whether the point x - e (index i = e + 1 per axis) lies inside the fluid.
template <int BC>
__device__ __forceinline__ bool inside(const Nbr& n, int ix, int iy, int iz)
{
    if (BC == BC_PERIODIC) return true;
    if (BC == BC_BOX_LID) return n.xin[ix] && n.yin[iy] && n.zin[iz];
    return n.yin[iy];
}

template <typename S, bool ODD, int BC>
__device__ __forceinline__ S* load_ptr(S* buf, int s, const Nbr& n, unsigned stride, unsigned cell)
{
    if (!ODD) return buf + (size_t)s * stride + cell;
    const int ix = s % 3, iy = (s / 3) % 3, iz = s / 9;
    if (BC == BC_HALF_CHANNEL && iy == 0 && !n.yin[0])  // specular, through the symmetry plane
        return buf + (size_t)(20 - s) * stride + (n.xs[ix] + n.yz[1][iz]);
    if (!inside<BC>(n, ix, iy, iz)) return buf + (size_t)s * stride + cell;
    return buf + (size_t)(26 - s) * stride + (n.xs[ix] + n.yz[iy][iz]);
}

// Address written for slot s (the destination of the post-collision value).
template <typename S, bool ODD, int BC>
__device__ __forceinline__ S* store_ptr(S* buf, int s, const Nbr& n, unsigned stride, unsigned cell)
{
    if (!ODD) return buf + (size_t)(26 - s) * stride + cell;
    const int ix = s % 3, iy = (s / 3) % 3, iz = s / 9;
    if (BC == BC_HALF_CHANNEL && iy == 2 && !n.yin[0])  // specular, through the symmetry plane
        return buf + (size_t)(s - 6) * stride + (n.xs[2 - ix] + n.yz[1][2 - iz]);
    if (!inside<BC>(n, 2 - ix, 2 - iy, 2 - iz)) return buf + (size_t)(26 - s) * stride + cell;
    return buf + (size_t)s * stride + (n.xs[2 - ix] + n.yz[2 - iy][2 - iz]);
}

// Moving-wall correction of the post-collision values of a top-row cell:
// g_s -= w_s rho (e_s . u_w) 2 / cs^2 for the nine slots with e_y = +1.
template <typename R>
__device__ __forceinline__ void lid_correct(R g[27], R lid6x, R lid6z)
{
    R rho = R(1);
#pragma unroll
    for (int s = 0; s < 27; ++s) rho += g[s];
#pragma unroll
    for (int s = 6; s < 9; ++s) {  // e_y = +1, e_z = -1
        const R ex = R(s % 3 - 1);
        g[s] -= R(wslot(s)) * rho * (ex * lid6x - lid6z);
        g[s + 9] -= R(wslot(s + 9)) * rho * (ex * lid6x);
        g[s + 18] -= R(wslot(s + 18)) * rho * (ex * lid6x + lid6z);
    }
}

// Whether a cell lies in the top row y = ny - 1 (the moving wall's neighbours).
__device__ __forceinline__ bool top_row(const CellGeom& G, unsigned cell)
{
    const unsigned y = fdiv(cell - fdiv(cell, G.div_nxny) * (unsigned)(G.nx * G.ny), G.div_nx);
    return y + 1 == (unsigned)G.ny;
}

// The moving-wall correction for the lanes of a pair whose cell lies in the
// top row: the other lane's wall velocity is masked to zero, which leaves its
// values unchanged (g - 0 = g).
template <int BC>
__device__ __forceinline__ void lid_correct_pair(f2 (&g)[27], const CellGeom& G, unsigned ca, unsigned cb, f2 lid6x,
                                                 f2 lid6z)
{
    if constexpr (BC == BC_WALLS_Y_LID || BC == BC_BOX_LID) {
        const bool ta = top_row(G, ca), tb = top_row(G, cb);
        if (ta || tb) {
            const f2 m(ta ? 1.f : 0.f, tb ? 1.f : 0.f);
            lid_correct(g, lid6x * m, lid6z * m);
        }
    }
}

// active = false: the lane only takes part in warp-collective work (learned
// mode); it reads a valid cell but writes nothing.
template <typename S, typename R, bool ODD, int BC, bool FORCE, int MODE>
__device__ __forceinline__ void update_cell(S* __restrict__ buf, const CellGeom& G, unsigned cell,
                                            const Rates<R>& rt, R Fx, R Fy, R Fz, R om4, R om5, R om6, R om8,
                                            R om9, const float* closure, int* flag, bool active = true,
                                            R lid6x = R(0), R lid6z = R(0), const R* smag = nullptr)
{
    const unsigned stride = G.stride;
    R g[27];
    Nbr n;
    if (ODD) n = make_nbr<BC>(G, cell);
#pragma unroll
    for (int s = 0; s < 27; ++s) g[s] = Store<S>::ld(load_ptr<S, ODD, BC>(buf, s, n, stride, cell));

    R c2 = R(0);  // Smagorinsky: (C_s Delta D(y))^2 of this cell's row
    if (MODE == MODE_SMAG) c2 = smag[fdiv(cell - fdiv(cell, G.div_nxny) * (unsigned)(G.nx * G.ny), G.div_nx)];
    const bool ok = collide_cell<R, FORCE, MODE>(g, rt, Fx, Fy, Fz, om4, om5, om6, om8, om9, closure, c2);
    if (!ok && active) atomicOr(flag, 1);

    // rebuild the store addresses (and the odd step's neighbour table) instead of keeping
    // the load addresses live through the collision: the empty asm hides that cell is
    // unchanged, so the compiler cannot keep the old copies in registers
    asm volatile("" : "+r"(cell));
    if (ODD) n = make_nbr<BC>(G, cell);
    if (!active) return;
    if (BC == BC_WALLS_Y_LID || BC == BC_BOX_LID) {
        const unsigned y = fdiv(cell - fdiv(cell, G.div_nxny) * (unsigned)(G.nx * G.ny), G.div_nx);
        if (y + 1 == (unsigned)G.ny) lid_correct(g, lid6x, lid6z);
    }
#pragma unroll
    for (int s = 0; s < 27; ++s) Store<S>::st(store_ptr<S, ODD, BC>(buf, s, n, stride, cell), g[s]);
}

// Two cells per thread (see pair.cuh): cells c1 and c2 = c1 + half (c2 only
// when it is below ncells) are loaded into the lanes of f2 values, collided
// with packed fp32 arithmetic and stored back, each cell at its own AA
// addresses.  c2 is recomputed after the collision (from the uniform half)
// rather than kept live through it.  Every boundary kind; the moving-wall
// correction is applied per lane.
template <typename S, bool ODD, int BC, bool FORCE, int MODE>
__device__ __forceinline__ void update_pair(S* __restrict__ buf, const CellGeom& G, unsigned c1, unsigned half,
                                            unsigned ncells, const Rates<f2>& rt, f2 Fx, f2 Fy, f2 Fz, f2 om4,
                                            f2 om5, f2 om6, f2 om8, f2 om9, int* flag, f2 lid6x = f2(0.0),
                                            f2 lid6z = f2(0.0), const float* closure = nullptr, bool active = true)
{
    const unsigned stride = G.stride;
    f2 g[27];
    {
        const unsigned c2 = c1 + half < ncells ? c1 + half : c1;
        Nbr n;
        if (ODD) n = make_nbr<BC>(G, c1);
#pragma unroll
        for (int s = 0; s < 27; ++s) g[s].v.x = Store<S>::ld(load_ptr<S, ODD, BC>(buf, s, n, stride, c1));
        if (ODD) n = make_nbr<BC>(G, c2);
#pragma unroll
        for (int s = 0; s < 27; ++s) g[s].v.y = Store<S>::ld(load_ptr<S, ODD, BC>(buf, s, n, stride, c2));
    }
    const bool ok = collide_cell<f2, FORCE, MODE>(g, rt, Fx, Fy, Fz, om4, om5, om6, om8, om9, closure);
    if (!active) return;  // a tail lane of the warp-collective learned mode: nothing to write
    if (!ok) atomicOr(flag, 1);
    asm volatile("" : "+r"(c1));  // rebuild the store addresses (see update_cell)
    lid_correct_pair<BC>(g, G, c1, c1 + half < ncells ? c1 + half : c1, lid6x, lid6z);
    Nbr n;
    if (ODD) n = make_nbr<BC>(G, c1);
#pragma unroll
    for (int s = 0; s < 27; ++s) Store<S>::st(store_ptr<S, ODD, BC>(buf, s, n, stride, c1), g[s].v.x);
    const unsigned c2 = c1 + half;
    if (c2 < ncells) {
        if (ODD) n = make_nbr<BC>(G, c2);
#pragma unroll
        for (int s = 0; s < 27; ++s) Store<S>::st(store_ptr<S, ODD, BC>(buf, s, n, stride, c2), g[s].v.y);
    }
}

// Two neighbouring entries of one slot row (index c even, so the pair is 4- or
// 8-byte aligned: every slot row starts 128-byte aligned) as one vector access.
template <typename S>
struct Store2;
template <>
struct Store2<float> {
    __device__ __forceinline__ static f2 ld(const float* p) { return f2(*reinterpret_cast<const float2*>(p)); }
    __device__ __forceinline__ static void st(float* p, f2 v) { *reinterpret_cast<float2*>(p) = v.v; }
};
template <>
struct Store2<__half> {
    __device__ __forceinline__ static f2 ld(const __half* p)
    {
        return f2(__half22float2(*reinterpret_cast<const __half2*>(p)));
    }
    __device__ __forceinline__ static void st(__half* p, f2 v) { *reinterpret_cast<__half2*>(p) = __float22half2_rn(v.v); }
};
template <>
struct Store2<__nv_bfloat16> {
    __device__ __forceinline__ static f2 ld(const __nv_bfloat16* p)
    {
        return f2(__bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(p)));
    }
    __device__ __forceinline__ static void st(__nv_bfloat16* p, f2 v)
    {
        *reinterpret_cast<__nv_bfloat162*>(p) = __float22bfloat162_rn(v.v);
    }
};

// Even step of the paired kernel with neighbouring cells c = 2t and c + 1 in
// the two lanes: every access of the even step is to the cell's own slots, so
// the two cells' values of a slot are adjacent and move as one vector load or
// store (and, for 16-bit storage, one packed conversion).  A thread whose
// second cell lies past the end (odd cell count) updates c alone.  Which
// thread updates which cell is free within a step (each cell touches only its
// own addresses), so the odd step keeps its own pairing.
template <typename S, int BC, bool FORCE, int MODE>
__device__ __forceinline__ void update_pair_even(S* __restrict__ buf, const CellGeom& G, unsigned t, unsigned ncells,
                                                 const Rates<f2>& rt, f2 Fx, f2 Fy, f2 Fz, f2 om4, f2 om5, f2 om6,
                                                 f2 om8, f2 om9, int* flag, f2 lid6x = f2(0.0), f2 lid6z = f2(0.0),
                                                 const float* closure = nullptr, bool active = true)
{
    const unsigned stride = G.stride;
    unsigned c = 2 * t;
    const bool two = c + 1 < ncells;
    f2 g[27];
    if (two) {
#pragma unroll
        for (int s = 0; s < 27; ++s) g[s] = Store2<S>::ld(buf + (size_t)s * stride + c);
    } else {
#pragma unroll
        for (int s = 0; s < 27; ++s) {
            const float v = Store<S>::ld(buf + (size_t)s * stride + c);
            g[s] = f2(v, v);
        }
    }
    const bool ok = collide_cell<f2, FORCE, MODE>(g, rt, Fx, Fy, Fz, om4, om5, om6, om8, om9, closure);
    if (!active) return;
    if (!ok) atomicOr(flag, 1);
    asm volatile("" : "+r"(c));  // rebuild the store addresses (see update_cell)
    lid_correct_pair<BC>(g, G, c, two ? c + 1 : c, lid6x, lid6z);
    if (two) {
#pragma unroll
        for (int s = 0; s < 27; ++s) Store2<S>::st(buf + (size_t)(26 - s) * stride + c, g[s]);
    } else {
#pragma unroll
        for (int s = 0; s < 27; ++s) Store<S>::st(buf + (size_t)(26 - s) * stride + c, g[s].v.x);
    }
}

// Odd step of the paired kernel for boxes with nx even: neighbouring cells
// c = 2t (x even) and c + 1 share y and z, hence the neighbour table.  For the
// nine slots with e_x = 0 their two values (neighbour reads, bounce-back
// redirects to their own slots, and writes) sit side by side, 2-element
// aligned: one vector access per slot.  For the other eighteen slots the
// second cell's address is the first one's plus 1, minus nx where the
// second cell's neighbour column wraps (x + 2 = nx for a neighbour at x + 1
// of the first cell, x = 0 for one at x - 1); a bounce-back redirect stays
// within the cells' own slots (plus 1).  In the closed box the x walls give
// the two cells different tests for e_x != 0, so there the second cell's
// address is formed from its own test.  Not for the half channel.
template <typename S, int BC, bool FORCE, int MODE>
__device__ __forceinline__ void update_pair_odd_adj(S* __restrict__ buf, const CellGeom& G, unsigned t,
                                                    const Rates<f2>& rt, f2 Fx, f2 Fy, f2 Fz, f2 om4, f2 om5,
                                                    f2 om6, f2 om8, f2 om9, int* flag, f2 lid6x = f2(0.0),
                                                    f2 lid6z = f2(0.0), const float* closure = nullptr,
                                                    bool active = true)
{
    static_assert(BC == BC_PERIODIC || BC == BC_WALLS_Y || BC == BC_WALLS_Y_LID || BC == BC_BOX_LID,
                  "no symmetry plane");
    const unsigned stride = G.stride;
    unsigned c = 2 * t;
    f2 g[27];
    {
        const Nbr n = make_nbr<BC>(G, c);
        const int x = (int)n.xs[1];
        const int wp = x + 2 == G.nx ? -G.nx : 0;  // second cell's column x + 2 wraps
        const int wm = x == 0 ? -G.nx : 0;         // first cell's column x - 1 wrapped
#pragma unroll
        for (int s = 0; s < 27; ++s) {
            const int ix = s % 3, iy = (s / 3) % 3, iz = s / 9;
            S* p = load_ptr<S, true, BC>(buf, s, n, stride, c);
            if (ix == 1) {
                g[s] = Store2<S>::ld(p);
            } else {  // the read is at x - e_x: x + 1 for ix = 0, x - 1 for ix = 2
                g[s].v.x = Store<S>::ld(p);
                if constexpr (BC == BC_BOX_LID) {  // x walls: the second cell's source has its own test
                    const int x2 = ix == 0 ? x + 2 : x;
                    const bool in2 = n.yin[iy] && n.zin[iz] && x2 < G.nx;
                    g[s].v.y = Store<S>::ld(in2 ? buf + (size_t)(26 - s) * stride + ((unsigned)x2 + n.yz[iy][iz])
                                                : buf + (size_t)s * stride + (c + 1));
                } else {
                    const int w = inside<BC>(n, ix, iy, iz) ? (ix == 0 ? wp : wm) : 0;
                    g[s].v.y = Store<S>::ld(p + 1 + w);
                }
            }
        }
    }
    const bool ok = collide_cell<f2, FORCE, MODE>(g, rt, Fx, Fy, Fz, om4, om5, om6, om8, om9, closure);
    if (!active) return;
    if (!ok) atomicOr(flag, 1);
    asm volatile("" : "+r"(c));  // rebuild the store addresses (see update_cell)
    lid_correct_pair<BC>(g, G, c, c + 1, lid6x, lid6z);
    const Nbr n = make_nbr<BC>(G, c);
    const int x = (int)n.xs[1];
    const int wp = x + 2 == G.nx ? -G.nx : 0;
    const int wm = x == 0 ? -G.nx : 0;
#pragma unroll
    for (int s = 0; s < 27; ++s) {
        const int ix = s % 3, iy = (s / 3) % 3, iz = s / 9;
        S* p = store_ptr<S, true, BC>(buf, s, n, stride, c);
        if (ix == 1) {
            Store2<S>::st(p, g[s]);
        } else {  // the write is at x + e_x: x + 1 for ix = 2, x - 1 for ix = 0
            Store<S>::st(p, g[s].v.x);
            if constexpr (BC == BC_BOX_LID) {
                const int x2 = ix == 2 ? x + 2 : x;  // the second cell writes to x + 1 + e_x
                const bool in2 = n.yin[2 - iy] && n.zin[2 - iz] && x2 < G.nx;
                Store<S>::st(in2 ? buf + (size_t)s * stride + ((unsigned)x2 + n.yz[2 - iy][2 - iz])
                                 : buf + (size_t)(26 - s) * stride + (c + 1),
                             g[s].v.y);
            } else {
                const int w = inside<BC>(n, 2 - ix, 2 - iy, 2 - iz) ? (ix == 2 ? wp : wm) : 0;
                Store<S>::st(p + 1 + w, g[s].v.y);
            }
        }
    }
}

}  // namespace fpc
