// collide.cuh -- per-cell FPC-LBM collision (Appendix D Steps 7, 1-5) in registers.
//
// The 27 populations of a cell arrive as deviations g[s] = f_s - w_s in tensor
// slot order s = (ex+1) + 3 (ey+1) + 9 (ez+1).  The central-moment transform
// kappa = C(u) f (Steps 1+2) factorises over the axes because the D3Q27
// velocities are a tensor product: three passes of a 3-point transform, each
// along one axis, turn the slot array into d[m + 3n + 9p], the deviation of
// kappa_mnp from the rest-state central moments r_m r_n r_p, r = (1, 0, cs^2).
// Working with deviations keeps every intermediate small, so that fp32
// arithmetic (and 16-bit storage) loses no digits to O(1) cancellations.
//
// A 3-point line (a, b, c) at e = (-1, 0, +1) whose rest values are
// K (1/6, 2/3, 1/6) maps to
//   d0 = a + b + c
//   d1 = (c - a) - u (K + d0)
//   d2 = (a + c) - 2u (c - a) + u^2 (K + d0)
// i.e. the moments sum v (e-u)^k minus their rest values (K, 0, K/3); the
// inverse map follows from raw moments m0 = K + d0, m1 = d1 + u m0,
// m2 = K/3 + d2 + 2u d1 + u^2 m0 and a = (m2-m1)/2, b = m0-m2, c = (m2+m1)/2.
//
// The collision relaxes the grouped moments of Step 3 in the chain order
// 2 -> 3 -> 4 -> 5 -> 6 toward the attractors of Eq. (Mvcmattractor3D) with
// D' of Eq. (diffusion-tensor-parameter-3D), adds the body-force sources of
// Eq. (cmupdatesourceD3Q27) with weight (1 - omega/2), and maps back.
// Readings: first-order moments enter attractors and sources as 0; sources
// use pre-collision moments; attractors of orders 4-6 use post-collision
// lower moments; kappa^Mv_122 carries Pi_110 Pi_012 (continuous form).
// In the modes *_R1 (rates of orders 3-6 equal to 1) the moments of orders 3-6
// are set to their attractors plus half their sources, kappa~ = kappa^Mv +
// sigma / 2, with no grouping.  Without force the third- and fifth-order
// moments then vanish (attractors built from odd moments that are zero after
// the collision), and the unused pre-collision moments of orders 3-6 drop out
// of the forward transform.
#pragma once
#include "common.cuh"
#include "pair.cuh"

namespace fpc {

#define FPC_D(m, n, p) g[(m) + 3 * (n) + 9 * (p)]

template <typename R>
__device__ __forceinline__ R fmaR(R a, R b, R c) { return fma(a, b, c); }
template <typename R>
__device__ __forceinline__ R fminR(R a, R b) { return fmin(a, b); }
template <typename R>
__device__ __forceinline__ R fmaxR(R a, R b) { return fmax(a, b); }

// Forward 3-point central-moment transform in deviation form (see header).
template <typename R, bool K0>
__device__ __forceinline__ void fwd3(R& a, R& b, R& c, R u, R u2, R tu, R K)
{
    const R P = a + c, D = c - a, S = P + b;
    const R U = K0 ? S : K + S;
    a = S;
    b = fmaR(-u, U, D);
    c = fmaR(u2, U, fmaR(-tu, D, P));
}

// Inverse of fwd3.
template <typename R, bool K0>
__device__ __forceinline__ void inv3(R& k0, R& k1, R& k2, R u, R u2, R tu, R K)
{
    const R U = K0 ? k0 : K + k0;
    const R M1 = fmaR(u, U, k1);
    const R M2 = fmaR(u2, U, fmaR(tu, k1, k2));
    // (M2 -/+ M1) / 2 with both halvings exact: the same roundings as 0.5 M2 -/+ 0.5 M1, and no
    // separate negation (which costs an instruction in packed f2 arithmetic)
    const R h2 = R(0.5) * M2;
    const R lo = fmaR(R(-0.5), M1, h2);
    const R hi = fmaR(R(0.5), M1, h2);
    const R mid = k0 - M2;
    k0 = lo;
    k1 = mid;
    k2 = hi;
}

// inv3 for a line some of whose inputs are known to be zero (Z0, Z1, Z2 for
// k0, k1, k2): the terms they would feed are left out.  Used in the unit-rate
// modes, where the moments of orders 3 and 5 are exactly zero after the
// collision.  A line with K0 && Z0 && Z1 && Z2 does not occur.
template <typename R, bool K0, bool Z0, bool Z1, bool Z2>
__device__ __forceinline__ void inv3z(R& k0, R& k1, R& k2, R u, R u2, R tu, R K)
{
    constexpr bool UZ = K0 && Z0;  // U = K + k0 vanishes
    R U = R(0);
    if constexpr (!UZ) {
        if constexpr (K0) U = k0;
        else if constexpr (Z0) U = K;
        else U = K + k0;
    }
    R M1;
    if constexpr (UZ) M1 = k1;
    else if constexpr (Z1) M1 = u * U;
    else M1 = fmaR(u, U, k1);
    R M2;
    if constexpr (Z1 && Z2) {
        M2 = u2 * U;
    } else {
        R t;
        if constexpr (Z1) t = k2;
        else if constexpr (Z2) t = tu * k1;
        else t = fmaR(tu, k1, k2);
        if constexpr (UZ) M2 = t;
        else M2 = fmaR(u2, U, t);
    }
    const R h2 = R(0.5) * M2;
    const R lo = fmaR(R(-0.5), M1, h2);
    const R hi = fmaR(R(0.5), M1, h2);
    R mid;
    if constexpr (Z0) mid = -M2;
    else mid = k0 - M2;
    k0 = lo;
    k1 = mid;
    k2 = hi;
}

// Rest constants of the three passes (axis z first, then y, then x).
// Pass A (z lines at fixed (ix, iy)): K = w1(ix) w1(iy)
// Pass B (y lines at fixed (ix, p)):  K = w1(ix) r1(p)
// Pass C (x lines at fixed (n, p)):   K = r1(n) r1(p)
#define FPC_PASS_B(OP)                                                                   \
    {                                                                                    \
        _Pragma("unroll") for (int p = 0; p < 3; ++p)                                    \
            _Pragma("unroll") for (int ix = 0; ix < 3; ++ix)                             \
        {                                                                                \
            const double Kd = w1(ix) * r1(p);                                            \
            if (Kd == 0.0)                                                               \
                OP<R, true>(g[ix + 9 * p], g[ix + 3 + 9 * p], g[ix + 6 + 9 * p], uy, uy2, tuy, R(0)); \
            else                                                                         \
                OP<R, false>(g[ix + 9 * p], g[ix + 3 + 9 * p], g[ix + 6 + 9 * p], uy, uy2, tuy, R(Kd)); \
        }                                                                                \
    }
#define FPC_PASS_C(OP)                                                                   \
    {                                                                                    \
        _Pragma("unroll") for (int p = 0; p < 3; ++p)                                    \
            _Pragma("unroll") for (int n = 0; n < 3; ++n)                                \
        {                                                                                \
            const double Kd = r1(n) * r1(p);                                             \
            if (Kd == 0.0)                                                               \
                OP<R, true>(g[3 * n + 9 * p], g[1 + 3 * n + 9 * p], g[2 + 3 * n + 9 * p], ux, ux2, tux, R(0)); \
            else                                                                         \
                OP<R, false>(g[3 * n + 9 * p], g[1 + 3 * n + 9 * p], g[2 + 3 * n + 9 * p], ux, ux2, tux, R(Kd)); \
        }                                                                                \
    }

// Per-cell learned correction of the shear rates (mode LEARNED): MLP
// 9 -> 64 -> 64 -> 1 with tanh hidden layers on the tensor cores, weights
// packed by fpclbm_set_closure.  Warp-collective; implemented in closure.cuh.
template <typename R>
__device__ R closure_delta_omega(const uint32_t* P, const R in[9]);

// Collide one cell in place.  rt: rates of Step 3; Fx, Fy, Fz: body force;
// om4..om9: the five shear rates (110, 101, 011, 2d1, 2d2), given separately
// because ensembles carry one shear rate per box; closure: MLP weights
// (learned mode only); c2 = (C_s Delta D)^2 of the cell (Smagorinsky mode
// only).  Returns false when rho <= 0 or not finite.
template <typename R, bool FORCE, int MODE>
__device__ __forceinline__ bool collide_cell(R (&g)[27], const Rates<R>& rt, R Fx, R Fy, R Fz, R om4, R om5, R om6,
                                             R om8, R om9, const float* closure, R c2 = R(0))
{
    constexpr bool R1 = r1_mode(MODE);
    constexpr bool ODD0 = R1 && !FORCE;  // moments of orders 3 and 5 exactly zero after the collision
    // ---- Step 7 and the first pass (z lines), sharing the line sums ----
    R S[9], Dz[9], Pz[9];
#pragma unroll
    for (int l = 0; l < 9; ++l) {
        const R lo = g[l], mid = g[l + 9], hi = g[l + 18];
        Pz[l] = lo + hi;
        Dz[l] = hi - lo;
        S[l] = Pz[l] + mid;
    }
    const R drho = ((S[0] + S[1] + S[2]) + (S[3] + S[4] + S[5])) + (S[6] + S[7] + S[8]);
    const R jx = ((S[2] - S[0]) + (S[5] - S[3])) + (S[8] - S[6]);
    const R jy = ((S[6] - S[0]) + (S[7] - S[1])) + (S[8] - S[2]);
    const R jz = ((Dz[0] + Dz[1] + Dz[2]) + (Dz[3] + Dz[4] + Dz[5])) + (Dz[6] + Dz[7] + Dz[8]);
    const R rho = R(1) + drho;
    const R inv_rho = R(1) / rho;
    const bool ok = (rho > R(0)) && (rho < R(1e30));
    R ux, uy, uz;
    if (FORCE) {
        ux = fmaR(R(0.5), Fx, jx) * inv_rho;
        uy = fmaR(R(0.5), Fy, jy) * inv_rho;
        uz = fmaR(R(0.5), Fz, jz) * inv_rho;
    } else {
        ux = jx * inv_rho;
        uy = jy * inv_rho;
        uz = jz * inv_rho;
    }
    const R ux2 = ux * ux, uy2 = uy * uy, uz2 = uz * uz;
    const R tux = R(2) * ux, tuy = R(2) * uy, tuz = R(2) * uz;

#pragma unroll
    for (int l = 0; l < 9; ++l) {
        const double Kd = w1(l % 3) * w1(l / 3);
        const R U = R(Kd) + S[l];
        g[l] = S[l];
        g[l + 9] = fmaR(-uz, U, Dz[l]);
        g[l + 18] = fmaR(uz2, U, fmaR(-tuz, Dz[l], Pz[l]));
    }
    FPC_PASS_B(fwd3)
    FPC_PASS_C(fwd3)
    // now g[m + 3n + 9p] = kappa_mnp - r_m r_n r_p

    // ---- Step 3: relaxation toward the Markovian attractors ----
    const R third = R(1.0 / 3.0), ninth = R(1.0 / 9.0);
    R fx = R(0), fy = R(0), fz = R(0);
    if (FORCE) {
        fx = Fx * inv_rho;
        fy = Fy * inv_rho;
        fz = Fz * inv_rho;
    }

    // shear rates, possibly corrected by the learned closure
    if constexpr (learned_mode(MODE)) {
        R in[9];
        in[0] = FPC_D(2, 0, 0) - third * drho;  // kappa_200 - cs^2 rho
        in[1] = FPC_D(0, 2, 0) - third * drho;
        in[2] = FPC_D(0, 0, 2) - third * drho;
        in[3] = FPC_D(1, 1, 0);
        in[4] = FPC_D(1, 0, 1);
        in[5] = FPC_D(0, 1, 1);
        in[6] = ux;
        in[7] = uy;
        in[8] = uz;
        // the correction adds an eddy viscosity nu_t >= 0 (the training label's definition), so it
        // only lowers the rates: omega + min(delta omega, 0), kept above 0.02
        const R dw = fminR(closure_delta_omega<R>(reinterpret_cast<const uint32_t*>(closure), in), R(0));
        const R lo = R(0.02);
        om4 = fmaxR(om4 + dw, lo);
        om5 = fmaxR(om5 + dw, lo);
        om6 = fmaxR(om6 + dw, lo);
        om8 = fmaxR(om8 + dw, lo);
        om9 = fmaxR(om9 + dw, lo);
    }

    // Smagorinsky eddy viscosity (Sec. 4, turbulent channel LES): nu_t = c2 |S|, the strain rate
    // from the deviatoric non-equilibrium second moments Pi^d at the effective time tau,
    // S = -Pi^d / (2 rho cs^2 tau), tau = tau0 + nu_t / cs^2; the positive root of
    // tau^2 - tau0 tau - c2 |Pi^d| / (2 rho cs^4) = 0 replaces all five shear rates.
    if constexpr (MODE == MODE_SMAG) {
        const R p0 = FPC_D(2, 0, 0) - third * drho, p1 = FPC_D(0, 2, 0) - third * drho;
        const R p2 = FPC_D(0, 0, 2) - third * drho;
        const R tr = third * ((p0 + p1) + p2);
        const R q0 = p0 - tr, q1 = p1 - tr, q2 = p2 - tr;
        const R o1 = FPC_D(1, 1, 0), o2 = FPC_D(1, 0, 1), o3 = FPC_D(0, 1, 1);
        const R pp = fmaR(q0, q0, fmaR(q1, q1, q2 * q2)) + R(2) * fmaR(o1, o1, fmaR(o2, o2, o3 * o3));
        const R Pn = sqrt(R(2) * pp);
        const R tau0 = R(1) / om4;
        const R te = R(0.5) * (tau0 + sqrt(fmaR(tau0, tau0, R(18) * c2 * Pn * inv_rho)));
        const R w = R(1) / te;
        om4 = om5 = om6 = om8 = om9 = w;
    }

    // order 1 (attractor 0, source F).  In exact arithmetic kappa_100 = -F_x/2 and
    // kappa~_100 = F_x/2 whatever omega_1..3 are, so they are applied here as 0:
    // kappa~_100 = kappa_100 + F_x keeps the rounding residual j - rho u of the forward
    // transform, and the back transform then rebuilds the momentum j + F to the last
    // bit instead of rho * round(j / rho) (whose error repeats every step in a slowly
    // varying flow and would accumulate linearly in fp32).
    if (FORCE) {
        FPC_D(1, 0, 0) += Fx;
        FPC_D(0, 1, 0) += Fy;
        FPC_D(0, 0, 1) += Fz;
    }

    // sources of order 3 from the pre-collision second moments
    R s120 = 0, s102 = 0, s210 = 0, s012 = 0, s201 = 0, s021 = 0, s111 = 0;
    if (FORCE) {
        const R k200 = third + FPC_D(2, 0, 0), k020 = third + FPC_D(0, 2, 0), k002 = third + FPC_D(0, 0, 2);
        const R k110 = FPC_D(1, 1, 0), k101 = FPC_D(1, 0, 1), k011 = FPC_D(0, 1, 1);
        s120 = fx * k020 + R(2) * fy * k110;
        s102 = fx * k002 + R(2) * fz * k101;
        s210 = R(2) * fx * k110 + fy * k200;
        s012 = fy * k002 + R(2) * fz * k011;
        s201 = R(2) * fx * k101 + fz * k200;
        s021 = R(2) * fy * k011 + fz * k020;
        s111 = fx * k011 + fy * k101 + fz * k110;
    }

    // order 2: off-diagonal (attractor 0, no source), 2s1 (attractor 3 cs^2 rho),
    // 2d1, 2d2 (attractor 0)
    FPC_D(1, 1, 0) = (R(1) - om4) * FPC_D(1, 1, 0);
    FPC_D(1, 0, 1) = (R(1) - om5) * FPC_D(1, 0, 1);
    FPC_D(0, 1, 1) = (R(1) - om6) * FPC_D(0, 1, 1);
    {
        const R d200 = FPC_D(2, 0, 0), d020 = FPC_D(0, 2, 0), d002 = FPC_D(0, 0, 2);
        const R y2s = (d200 + d020) + d002;
        const R y2d1 = d200 - d020, y2d2 = d200 - d002;
        const R t2s = fmaR(rt.om[7], drho, rt.keep[7] * y2s);  // attractor deviation: drho
        const R t2d1 = (R(1) - om8) * y2d1;
        const R t2d2 = (R(1) - om9) * y2d2;
        FPC_D(2, 0, 0) = third * ((t2s + t2d1) + t2d2);
        FPC_D(0, 2, 0) = third * (fmaR(R(-2), t2d1, t2s) + t2d2);
        FPC_D(0, 0, 2) = third * (fmaR(R(-2), t2d2, t2s) + t2d1);
    }

    // sources of order 4 from the pre-collision third moments
    R s220 = 0, s202 = 0, s022 = 0, s211 = 0, s121 = 0, s112 = 0;
    if (FORCE) {
        s220 = R(2) * (fx * FPC_D(1, 2, 0) + fy * FPC_D(2, 1, 0));
        s202 = R(2) * (fx * FPC_D(1, 0, 2) + fz * FPC_D(2, 0, 1));
        s022 = R(2) * (fy * FPC_D(0, 1, 2) + fz * FPC_D(0, 2, 1));
        s211 = R(2) * fx * FPC_D(1, 1, 1) + fy * FPC_D(2, 0, 1) + fz * FPC_D(2, 1, 0);
        s121 = fx * FPC_D(0, 2, 1) + R(2) * fy * FPC_D(1, 1, 1) + fz * FPC_D(1, 2, 0);
        s112 = fx * FPC_D(0, 1, 2) + fy * FPC_D(1, 0, 2) + R(2) * fz * FPC_D(1, 1, 1);
    }

    // order 3 (attractors 0): pairs (120,102), (210,012), (201,021), and 111
    if constexpr (ODD0) {
        FPC_D(1, 2, 0) = FPC_D(1, 0, 2) = FPC_D(2, 1, 0) = R(0);
        FPC_D(0, 1, 2) = FPC_D(2, 0, 1) = FPC_D(0, 2, 1) = R(0);
        FPC_D(1, 1, 1) = R(0);
    } else if constexpr (R1) {  // with force: half the sources
        FPC_D(1, 2, 0) = R(0.5) * s120;
        FPC_D(1, 0, 2) = R(0.5) * s102;
        FPC_D(2, 1, 0) = R(0.5) * s210;
        FPC_D(0, 1, 2) = R(0.5) * s012;
        FPC_D(2, 0, 1) = R(0.5) * s201;
        FPC_D(0, 2, 1) = R(0.5) * s021;
        FPC_D(1, 1, 1) = R(0.5) * s111;
    } else {
#define FPC_PAIR3(A, B, sa, sb, j)                                                      \
    {                                                                                   \
        const R ys = A + B, ym = A - B;                                                 \
        R ts = rt.keep[j] * ys, tm = rt.keep[j + 1] * ym;                               \
        if (FORCE) {                                                                    \
            ts = fmaR(rt.src[j], sa + sb, ts);                                          \
            tm = fmaR(rt.src[j + 1], sa - sb, tm);                                      \
        }                                                                               \
        A = R(0.5) * (ts + tm);                                                         \
        B = R(0.5) * (ts - tm);                                                         \
    }
    FPC_PAIR3(FPC_D(1, 2, 0), FPC_D(1, 0, 2), s120, s102, 10)
    FPC_PAIR3(FPC_D(2, 1, 0), FPC_D(0, 1, 2), s210, s012, 12)
    FPC_PAIR3(FPC_D(2, 0, 1), FPC_D(0, 2, 1), s201, s021, 14)
#undef FPC_PAIR3
    FPC_D(1, 1, 1) = rt.keep[16] * FPC_D(1, 1, 1);
    if (FORCE) FPC_D(1, 1, 1) = fmaR(rt.src[16], s111, FPC_D(1, 1, 1));
    }

    // sources of order 5 from the pre-collision fourth moments
    R s122 = 0, s212 = 0, s221 = 0;
    if (FORCE) {
        const R k022 = ninth + FPC_D(0, 2, 2), k202 = ninth + FPC_D(2, 0, 2), k220 = ninth + FPC_D(2, 2, 0);
        s122 = fx * k022 + R(2) * (fy * FPC_D(1, 1, 2) + fz * FPC_D(1, 2, 1));
        s212 = fy * k202 + R(2) * (fx * FPC_D(1, 1, 2) + fz * FPC_D(2, 1, 1));
        s221 = fz * k220 + R(2) * (fx * FPC_D(1, 2, 1) + fy * FPC_D(2, 1, 1));
    }

    // post-collision second moments used by the attractors of orders 4-6
    const R pa = FPC_D(2, 0, 0), pb = FPC_D(0, 2, 0), pc = FPC_D(0, 0, 2);
    const R o110 = FPC_D(1, 1, 0), o101 = FPC_D(1, 0, 1), o011 = FPC_D(0, 1, 1);

    // order 4: groups 4s1, 4d1, 4d2 and 211, 121, 112
    {
        R A220, A202, A022, A211, A121, A112;
        if constexpr (eq_mode(MODE)) {
            A220 = A202 = A022 = ninth * drho;  // cs^4 rho - 1/9
            A211 = A121 = A112 = R(0);
        } else {
            const R dn = ninth * drho;
            A220 = (fmaR(third, pa + pb, fmaR(pa, pb, R(2) * o110 * o110)) - dn) * inv_rho;
            A202 = (fmaR(third, pa + pc, fmaR(pa, pc, R(2) * o101 * o101)) - dn) * inv_rho;
            A022 = (fmaR(third, pb + pc, fmaR(pb, pc, R(2) * o011 * o011)) - dn) * inv_rho;
            A211 = fmaR(third + pa, o011, R(2) * o110 * o101) * inv_rho;
            A121 = fmaR(third + pb, o101, R(2) * o110 * o011) * inv_rho;
            A112 = fmaR(third + pc, o110, R(2) * o011 * o101) * inv_rho;
        }
        if constexpr (R1) {
            if constexpr (FORCE) {
                FPC_D(2, 2, 0) = fmaR(R(0.5), s220, A220);
                FPC_D(2, 0, 2) = fmaR(R(0.5), s202, A202);
                FPC_D(0, 2, 2) = fmaR(R(0.5), s022, A022);
                FPC_D(2, 1, 1) = fmaR(R(0.5), s211, A211);
                FPC_D(1, 2, 1) = fmaR(R(0.5), s121, A121);
                FPC_D(1, 1, 2) = fmaR(R(0.5), s112, A112);
            } else {
                FPC_D(2, 2, 0) = A220;
                FPC_D(2, 0, 2) = A202;
                FPC_D(0, 2, 2) = A022;
                FPC_D(2, 1, 1) = A211;
                FPC_D(1, 2, 1) = A121;
                FPC_D(1, 1, 2) = A112;
            }
        } else {
        const R d220 = FPC_D(2, 2, 0), d202 = FPC_D(2, 0, 2), d022 = FPC_D(0, 2, 2);
        const R y4s = (d220 + d202) + d022, y4d1 = (d220 + d202) - d022, y4d2 = d220 - d202;
        const R a4s = (A220 + A202) + A022, a4d1 = (A220 + A202) - A022, a4d2 = A220 - A202;
        R t4s = fmaR(rt.om[17], a4s, rt.keep[17] * y4s);
        R t4d1 = fmaR(rt.om[18], a4d1, rt.keep[18] * y4d1);
        R t4d2 = fmaR(rt.om[19], a4d2, rt.keep[19] * y4d2);
        if (FORCE) {
            t4s = fmaR(rt.src[17], (s220 + s202) + s022, t4s);
            t4d1 = fmaR(rt.src[18], (s220 + s202) - s022, t4d1);
            t4d2 = fmaR(rt.src[19], s220 - s202, t4d2);
        }
        FPC_D(2, 2, 0) = R(0.25) * fmaR(R(2), t4d2, t4s + t4d1);
        FPC_D(2, 0, 2) = R(0.25) * fmaR(R(-2), t4d2, t4s + t4d1);
        FPC_D(0, 2, 2) = R(0.5) * (t4s - t4d1);
        R t211 = fmaR(rt.om[20], A211, rt.keep[20] * FPC_D(2, 1, 1));
        R t121 = fmaR(rt.om[21], A121, rt.keep[21] * FPC_D(1, 2, 1));
        R t112 = fmaR(rt.om[22], A112, rt.keep[22] * FPC_D(1, 1, 2));
        if (FORCE) {
            t211 = fmaR(rt.src[20], s211, t211);
            t121 = fmaR(rt.src[21], s121, t121);
            t112 = fmaR(rt.src[22], s112, t112);
        }
        FPC_D(2, 1, 1) = t211;
        FPC_D(1, 2, 1) = t121;
        FPC_D(1, 1, 2) = t112;
        }
    }

    // source of order 6 from the pre-collision fifth moments
    R s222 = 0;
    if (FORCE) s222 = R(2) * ((fx * FPC_D(1, 2, 2) + fy * FPC_D(2, 1, 2)) + fz * FPC_D(2, 2, 1));

    // order 5: attractors from post-collision second and third moments
    if constexpr (ODD0) {
        FPC_D(1, 2, 2) = FPC_D(2, 1, 2) = FPC_D(2, 2, 1) = R(0);
    } else {
        R A122 = R(0), A212 = R(0), A221 = R(0);
        if constexpr (!eq_mode(MODE)) {
            const R K200 = third + pa, K020 = third + pb, K002 = third + pc;
            const R k111 = FPC_D(1, 1, 1);
            const R c = R(0.4) * inv_rho;
            A122 = c * (fmaR(K020, FPC_D(1, 0, 2), K002 * FPC_D(1, 2, 0)) +
                        fmaR(R(4) * o011, k111, R(2) * fmaR(o101, FPC_D(0, 2, 1), o110 * FPC_D(0, 1, 2))));
            A212 = c * (fmaR(K200, FPC_D(0, 1, 2), K002 * FPC_D(2, 1, 0)) +
                        fmaR(R(4) * o101, k111, R(2) * fmaR(o110, FPC_D(1, 0, 2), o011 * FPC_D(2, 0, 1))));
            A221 = c * (fmaR(K200, FPC_D(0, 2, 1), K020 * FPC_D(2, 0, 1)) +
                        fmaR(R(4) * o110, k111, R(2) * fmaR(o011, FPC_D(2, 1, 0), o101 * FPC_D(1, 2, 0))));
        }
        if constexpr (R1) {  // with force (ODD0 handled above)
            FPC_D(1, 2, 2) = fmaR(R(0.5), s122, A122);
            FPC_D(2, 1, 2) = fmaR(R(0.5), s212, A212);
            FPC_D(2, 2, 1) = fmaR(R(0.5), s221, A221);
        } else {
            R t122 = fmaR(rt.om[23], A122, rt.keep[23] * FPC_D(1, 2, 2));
            R t212 = fmaR(rt.om[24], A212, rt.keep[24] * FPC_D(2, 1, 2));
            R t221 = fmaR(rt.om[25], A221, rt.keep[25] * FPC_D(2, 2, 1));
            if (FORCE) {
                t122 = fmaR(rt.src[23], s122, t122);
                t212 = fmaR(rt.src[24], s212, t212);
                t221 = fmaR(rt.src[25], s221, t221);
            }
            FPC_D(1, 2, 2) = t122;
            FPC_D(2, 1, 2) = t212;
            FPC_D(2, 2, 1) = t221;
        }
    }

    // order 6: attractor from post-collision second and fourth moments
    {
        R A222;
        if constexpr (eq_mode(MODE)) {
            A222 = R(1.0 / 27.0) * drho;  // cs^6 rho - 1/27
        } else {
            const R q220 = FPC_D(2, 2, 0), q202 = FPC_D(2, 0, 2), q022 = FPC_D(0, 2, 2);
            R t = fmaR(ninth, (pa + pb) + pc, third * ((q022 + q202) + q220));
            t = fmaR(pa, q022, fmaR(pb, q202, fmaR(pc, q220, t)));
            t = fmaR(R(4), fmaR(o110, FPC_D(1, 1, 2), fmaR(o101, FPC_D(1, 2, 1), o011 * FPC_D(2, 1, 1))), t);
            A222 = (t - ninth * drho) * (third * inv_rho);
        }
        if constexpr (R1) {
            FPC_D(2, 2, 2) = FORCE ? fmaR(R(0.5), s222, A222) : A222;
        } else {
            R t222 = fmaR(rt.om[26], A222, rt.keep[26] * FPC_D(2, 2, 2));
            if (FORCE) t222 = fmaR(rt.src[26], s222, t222);
            FPC_D(2, 2, 2) = t222;
        }
    }

    // ---- Steps 4+5: back to populations (passes in reverse order) ----
    if constexpr (ODD0) {
        // x lines at fixed (n, p); inputs of total order 3 or 5 are zero
#define FPC_INVC(n, p, Z0, Z1, Z2)                                                                        \
    inv3z<R, r1(n) * r1(p) == 0.0, Z0, Z1, Z2>(g[3 * (n) + 9 * (p)], g[1 + 3 * (n) + 9 * (p)],           \
                                               g[2 + 3 * (n) + 9 * (p)], ux, ux2, tux, R(r1(n) * r1(p)))
        FPC_INVC(0, 0, false, false, false);
        FPC_INVC(1, 0, false, false, true);
        FPC_INVC(2, 0, false, true, false);
        FPC_INVC(0, 1, false, false, true);
        FPC_INVC(1, 1, false, true, false);
        FPC_INVC(2, 1, true, false, true);
        FPC_INVC(0, 2, false, true, false);
        FPC_INVC(1, 2, true, false, true);
        FPC_INVC(2, 2, false, true, false);
#undef FPC_INVC
    } else {
        FPC_PASS_C(inv3)
    }
    FPC_PASS_B(inv3)
#pragma unroll
    for (int l = 0; l < 9; ++l) {
        const double Kd = w1(l % 3) * w1(l / 3);
        inv3<R, false>(g[l], g[l + 9], g[l + 18], uz, uz2, tuz, R(Kd));
    }
    return ok;
}

#undef FPC_PASS_B
#undef FPC_PASS_C

}  // namespace fpc
