/*
 * fpc_oracle.c -- slow, literal FP64 CPU statement of the D3Q27 FPC-LBM.
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the test suite, the smoke
 * check in __graft_entry__.py and the CPU-baseline leg of bench.py load this
 * library.  The product library (libfpclbm.so) never links, loads or calls
 * it, and this file shares no code, header, table or constant with the CUDA
 * path.
 *
 * What it computes (Schupbach & Premnath, "Fokker-Planck central moment
 * lattice Boltzmann method", arXiv 2410.09739):
 *   - lattice: D3Q27 velocities in the order of Sec. 3 ("Construction of 3D
 *     FPC-LBM", the |e_x>,|e_y>,|e_z> lists);
 *   - central moments kappa_mnp = sum_a f_a (e_ax-u_x)^m (e_ay-u_y)^n
 *     (e_az-u_z)^p in the order of the vector m^c (Sec. 3, discrete central
 *     moments), built as ONE explicit 27x27 matrix C(u) = F(u) P and applied
 *     by a plain matrix-vector product; the way back is a numerical LU solve
 *     with partial pivoting (Golub & Van Loan, Alg. 3.4.1), never the
 *     binomial chain of Appendix D Steps 2/4;
 *   - Markovian attractors from the GENERIC formula Eq. (Mvcmattractor3D),
 *     with the diffusion tensor of Eq. (diffusion-tensor-parameter-3D):
 *     D' = cs^2 delta for order <= 2, D' = kappa~_ij / rho for order > 2;
 *   - source moments Eq. (cmupdatesourceD3Q27);
 *   - the relaxation chain and moment groups of Appendix D Step 3, with the
 *     grouping applied as a 27x27 matrix G and undone by its numerical
 *     inverse;
 *   - half-force velocity of Appendix D Step 7, push streaming of Step 6
 *     (Eq. LBMsteps), half-way bounce-back on y-walls or on all six faces of
 *     a closed box, with the moving-wall momentum correction on the wall
 *     y = ny-1/2 (Sec. 4 cubic cavity), or a half channel closed by a
 *     specular-reflection symmetry plane (Sec. 4 turbulent channel);
 *   - the Smagorinsky subgrid model with van Driest wall damping (Sec. 4
 *     turbulent channel LES).
 *
 * Readings where the paper is silent or self-contradictory (each one is
 * listed with its reason in the design notes of the repository):
 *   R1  first-order central moments enter attractors and sources as 0 (their
 *       continuous values, Eq. solvability conditions of Appendix C and the
 *       zero third-order attractors listed in Step 3);
 *   R2  lower moments in the attractors of orders 4, 5, 6 are the current
 *       post-collision values (Sec. 3 text after the boxed attractor list);
 *   R3  equilibrium / MCM mode: D' = cs^2 delta at every order and the lower
 *       moments are themselves at their attractors (Maxwellian central
 *       moments);
 *   R4  initial populations are f = C(u)^-1 kappa^eq(rho,u) with kappa^eq the
 *       MCM attractors (no non-equilibrium part);
 *   R5  sources of order >= 3 use the pre-collision central moments;
 *   R6  moving wall: the density in the momentum correction is that of the
 *       fluid cell the population leaves, and the moving wall is the whole
 *       layer y = ny, so links through its edges and corners are corrected
 *       too;
 *   R7  Smagorinsky model: the strain rate comes from the deviatoric part of
 *       the non-equilibrium second-order central moments, the force's
 *       contribution to them is neglected, Delta = 1, and the eddy viscosity
 *       replaces all five shear rates; van Driest damping uses the distance
 *       of the cell centre to the nearest wall and the nominal friction
 *       velocity u*.
 *
 * Layout of population arrays: f[a][z][y][x], a = 0..26 (alpha-major), full
 * populations (not deviations), fp64.
 *
 * Compile: plain C99, -ffp-contract=off so that x86 and Arm give the same
 * roundings; OpenMP over z-planes only.
 */
#include <math.h>
#include <stddef.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define Q 27
#define CS2 (1.0 / 3.0)

/* D3Q27 velocity set, Sec. 3 (Construction of 3D FPC-LBM), alpha = 0..26. */
static const int EX[Q] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1,
                          0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1};
static const int EY[Q] = {0, 0, 0, 1, -1, 0, 0, 1, 1, -1, -1, 0, 0, 0, 0,
                          1, -1, 1, -1, 1, 1, -1, -1, 1, 1, -1, -1};
static const int EZ[Q] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, 1, -1, -1,
                          1, 1, -1, -1, 1, 1, 1, 1, -1, -1, -1, -1};

/* Exponents (m,n,p) of the central-moment vector m^c, Sec. 3, in order. */
static const int MNP[Q][3] = {
    {0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {1, 1, 0}, {1, 0, 1},
    {0, 1, 1}, {2, 0, 0}, {0, 2, 0}, {0, 0, 2}, {1, 2, 0}, {1, 0, 2},
    {2, 1, 0}, {0, 1, 2}, {2, 0, 1}, {0, 2, 1}, {1, 1, 1}, {2, 2, 0},
    {2, 0, 2}, {0, 2, 2}, {2, 1, 1}, {1, 2, 1}, {1, 1, 2}, {1, 2, 2},
    {2, 1, 2}, {2, 2, 1}, {2, 2, 2}};

/* Position of moment (m,n,p) in m^c, filled by index_of(). */
static int index_of(int m, int n, int p)
{
    for (int i = 0; i < Q; ++i)
        if (MNP[i][0] == m && MNP[i][1] == n && MNP[i][2] == p) return i;
    return -1;
}

static double ipow(double b, int e)
{
    double r = 1.0;
    for (int k = 0; k < e; ++k) r *= b;
    return r;
}

/* ------------------------------------------------------------------------ */
/* Matrices                                                                   */
/* ------------------------------------------------------------------------ */

/* C(u)[i][a] = (e_ax-u_x)^m_i (e_ay-u_y)^n_i (e_az-u_z)^p_i: the definition of
 * the discrete central moments (Sec. 3).  With u = 0 it is the raw-moment
 * projection P of Sec. 3 (rows |e_x^m e_y^n e_z^p>). */
void orc_central_matrix(const double u[3], double C[Q][Q])
{
    for (int i = 0; i < Q; ++i)
        for (int a = 0; a < Q; ++a)
            C[i][a] = ipow(EX[a] - u[0], MNP[i][0]) *
                      ipow(EY[a] - u[1], MNP[i][1]) *
                      ipow(EZ[a] - u[2], MNP[i][2]);
}

/* Group index j (the subscript of omega_j in Appendix D Step 3):
 *  0:000 1:100 2:010 3:001 4:110 5:101 6:011 7:2s1 8:2d1 9:2d2
 * 10:3s1 11:3m1 12:3s2 13:3m2 14:3s3 15:3m3 16:111 17:4s1 18:4d1 19:4d2
 * 20:211 21:121 22:112 23:122 24:212 25:221 26:222
 * G[j][i]: y_j = sum_i G[j][i] kappa_i, the combinations of Step 3. */
void orc_grouping_matrix(double G[Q][Q])
{
    memset(G, 0, sizeof(double) * Q * Q);
    for (int j = 0; j < 7; ++j) G[j][j] = 1.0; /* 000 .. 011 unchanged */
    const int k200 = index_of(2, 0, 0), k020 = index_of(0, 2, 0), k002 = index_of(0, 0, 2);
    G[7][k200] = 1; G[7][k020] = 1; G[7][k002] = 1;  /* 2s1 */
    G[8][k200] = 1; G[8][k020] = -1;                 /* 2d1 */
    G[9][k200] = 1; G[9][k002] = -1;                 /* 2d2 */
    const int k120 = index_of(1, 2, 0), k102 = index_of(1, 0, 2);
    const int k210 = index_of(2, 1, 0), k012 = index_of(0, 1, 2);
    const int k201 = index_of(2, 0, 1), k021 = index_of(0, 2, 1);
    G[10][k120] = 1; G[10][k102] = 1;   /* 3s1 */
    G[11][k120] = 1; G[11][k102] = -1;  /* 3m1 */
    G[12][k210] = 1; G[12][k012] = 1;   /* 3s2 */
    G[13][k210] = 1; G[13][k012] = -1;  /* 3m2 */
    G[14][k201] = 1; G[14][k021] = 1;   /* 3s3 */
    G[15][k201] = 1; G[15][k021] = -1;  /* 3m3 */
    G[16][index_of(1, 1, 1)] = 1;       /* 111 */
    const int k220 = index_of(2, 2, 0), k202 = index_of(2, 0, 2), k022 = index_of(0, 2, 2);
    G[17][k220] = 1; G[17][k202] = 1; G[17][k022] = 1;   /* 4s1 */
    G[18][k220] = 1; G[18][k202] = 1; G[18][k022] = -1;  /* 4d1 */
    G[19][k220] = 1; G[19][k202] = -1;                   /* 4d2 */
    G[20][index_of(2, 1, 1)] = 1;
    G[21][index_of(1, 2, 1)] = 1;
    G[22][index_of(1, 1, 2)] = 1;
    G[23][index_of(1, 2, 2)] = 1;
    G[24][index_of(2, 1, 2)] = 1;
    G[25][index_of(2, 2, 1)] = 1;
    G[26][index_of(2, 2, 2)] = 1;
}

/* Moment order of group j. */
static int group_order(int j)
{
    if (j == 0) return 0;
    if (j <= 3) return 1;
    if (j <= 9) return 2;
    if (j <= 16) return 3;
    if (j <= 22) return 4;
    if (j <= 25) return 5;
    return 6;
}

/* LU factorisation with partial pivoting, in place (Golub & Van Loan 3.4.1).
 * Returns 0, or -1 if a pivot is exactly zero. */
static int lu_factor(double A[Q][Q], int piv[Q])
{
    for (int k = 0; k < Q; ++k) {
        int p = k;
        double best = fabs(A[k][k]);
        for (int i = k + 1; i < Q; ++i)
            if (fabs(A[i][k]) > best) { best = fabs(A[i][k]); p = i; }
        piv[k] = p;
        if (best == 0.0) return -1;
        if (p != k)
            for (int c = 0; c < Q; ++c) { double t = A[k][c]; A[k][c] = A[p][c]; A[p][c] = t; }
        for (int i = k + 1; i < Q; ++i) {
            A[i][k] /= A[k][k];
            for (int c = k + 1; c < Q; ++c) A[i][c] -= A[i][k] * A[k][c];
        }
    }
    return 0;
}

/* Solve (LU) x = b in place, b -> x. */
static void lu_solve(double LU[Q][Q], const int piv[Q], double b[Q])
{
    for (int k = 0; k < Q; ++k) {
        int p = piv[k];
        if (p != k) { double t = b[k]; b[k] = b[p]; b[p] = t; }
    }
    for (int i = 1; i < Q; ++i)
        for (int c = 0; c < i; ++c) b[i] -= LU[i][c] * b[c];
    for (int i = Q - 1; i >= 0; --i) {
        for (int c = i + 1; c < Q; ++c) b[i] -= LU[i][c] * b[c];
        b[i] /= LU[i][i];
    }
}

/* x = A^-1 b via LU; returns 0 on success. */
int orc_solve(const double A[Q][Q], const double b[Q], double x[Q])
{
    double LU[Q][Q];
    int piv[Q];
    memcpy(LU, A, sizeof(LU));
    if (lu_factor(LU, piv) != 0) return -1;
    memcpy(x, b, sizeof(double) * Q);
    lu_solve(LU, piv, x);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Attractors and sources                                                     */
/* ------------------------------------------------------------------------ */

/* Eq. (Mvcmattractor3D): attractor of moment (m,n,p) of order s = m+n+p > 0
 * from the moments Pi of order s-2 and the diffusion tensor D (symmetric
 * 3x3, D[0][0] = D'_200, D[0][1] = D'_110, ...).  Pi is indexed [m][n][p]. */
double orc_attractor_generic(int m, int n, int p, const double Pi[27], const double D[9])
{
#define PI(a, b, c) Pi[((a) * 3 + (b)) * 3 + (c)]
#define DD(a, b) D[(a) * 3 + (b)]
    const int s = m + n + p;
    double r = 0.0;
    if (s == 0) return PI(0, 0, 0);
    if (m >= 2) r += DD(0, 0) * m * (m - 1) * PI(m - 2, n, p);
    if (n >= 2) r += DD(1, 1) * n * (n - 1) * PI(m, n - 2, p);
    if (p >= 2) r += DD(2, 2) * p * (p - 1) * PI(m, n, p - 2);
    if (m >= 1 && n >= 1) r += 2.0 * DD(0, 1) * m * n * PI(m - 1, n - 1, p);
    if (n >= 1 && p >= 1) r += 2.0 * DD(1, 2) * n * p * PI(m, n - 1, p - 1);
    if (m >= 1 && p >= 1) r += 2.0 * DD(0, 2) * m * p * PI(m - 1, n, p - 1);
    return r / s;
#undef PI
#undef DD
}

/* Maxwellian central moments (reading R3): the attractor chain with
 * D' = cs^2 delta at every order and lower moments at their own attractors.
 * Output M indexed [m][n][p]. */
void orc_maxwell_moments(double rho, double M[27])
{
    double D[9] = {CS2, 0, 0, 0, CS2, 0, 0, 0, CS2};
    memset(M, 0, sizeof(double) * 27);
    M[0] = rho;
    for (int s = 1; s <= 6; ++s)
        for (int m = 0; m < 3; ++m)
            for (int n = 0; n < 3; ++n)
                for (int p = 0; p < 3; ++p)
                    if (m + n + p == s)
                        M[(m * 3 + n) * 3 + p] = orc_attractor_generic(m, n, p, M, D);
}

/* ------------------------------------------------------------------------ */
/* Collision of one cell                                                      */
/* ------------------------------------------------------------------------ */

/* Appendix D Steps 7, 1-5 for one cell.
 *   f      pre-collision populations (27)
 *   F      body force (Fx,Fy,Fz)
 *   omega  relaxation rates omega_0..omega_26 (Step 3 numbering)
 *   mode   0: FP diffusion tensor (Eq. diffusion-tensor-parameter-3D)
 *          1: Maxwellian central moments at every order (MCM, reading R3)
 *   ft     post-collision populations (27)
 * Returns 0, or -1 if C(u) is singular (never for finite u). */
int orc_collide(const double f[Q], const double F[3], const double omega[Q], int mode,
                double ft[Q])
{
    /* Step 7 (hydrodynamic fields of the incoming populations). */
    double rho = 0, jx = 0, jy = 0, jz = 0;
    for (int a = 0; a < Q; ++a) {
        rho += f[a];
        jx += f[a] * EX[a];
        jy += f[a] * EY[a];
        jz += f[a] * EZ[a];
    }
    const double u[3] = {(jx + 0.5 * F[0]) / rho, (jy + 0.5 * F[1]) / rho, (jz + 0.5 * F[2]) / rho};

    /* Steps 1+2 as their definition: kappa = C(u) f. */
    double C[Q][Q], kap[Q];
    orc_central_matrix(u, C);
    for (int i = 0; i < Q; ++i) {
        double s = 0;
        for (int a = 0; a < Q; ++a) s += C[i][a] * f[a];
        kap[i] = s;
    }

    /* Pre-collision moments in [m][n][p] form; first order set to 0 for the
     * sources (reading R1). */
    double K[27];
    for (int i = 0; i < Q; ++i) K[(MNP[i][0] * 3 + MNP[i][1]) * 3 + MNP[i][2]] = kap[i];
    double Ks[27];
    memcpy(Ks, K, sizeof(Ks));
    Ks[(1 * 3 + 0) * 3 + 0] = 0; Ks[(0 * 3 + 1) * 3 + 0] = 0; Ks[(0 * 3 + 0) * 3 + 1] = 0;

    /* Eq. (cmupdatesourceD3Q27): sigma_mnp from moments one order lower. */
    double sig[Q];
    for (int i = 0; i < Q; ++i) {
        const int m = MNP[i][0], n = MNP[i][1], p = MNP[i][2];
        double s = 0;
        if (m >= 1) s += m * (F[0] / rho) * Ks[((m - 1) * 3 + n) * 3 + p];
        if (n >= 1) s += n * (F[1] / rho) * Ks[(m * 3 + (n - 1)) * 3 + p];
        if (p >= 1) s += p * (F[2] / rho) * Ks[(m * 3 + n) * 3 + (p - 1)];
        sig[i] = s;
    }

    /* Grouping of Step 3: y = G kappa, s = G sigma. */
    double G[Q][Q], y[Q], sg[Q];
    orc_grouping_matrix(G);
    for (int j = 0; j < Q; ++j) {
        double a = 0, b = 0;
        for (int i = 0; i < Q; ++i) { a += G[j][i] * kap[i]; b += G[j][i] * sig[i]; }
        y[j] = a;
        sg[j] = b;
    }

    /* Post-collision moments, [m][n][p]; filled stage by stage. */
    double Pt[27];
    memset(Pt, 0, sizeof(Pt));
    double Meq[27];
    orc_maxwell_moments(rho, Meq);

    /* Stages of the chain: orders {0,1,2}, then 3, 4, 5, 6. */
    static const int stage_lo[5] = {0, 3, 4, 5, 6};
    static const int stage_hi[5] = {2, 3, 4, 5, 6};
    double yt[Q];
    memcpy(yt, y, sizeof(yt));
    for (int st = 0; st < 5; ++st) {
        const int lo = stage_lo[st], hi = stage_hi[st];
        /* Attractors of every moment in this stage. */
        double att[Q];
        memset(att, 0, sizeof(att));
        double D[9];
        double Pi[27];
        if (mode == 1 || hi <= 2) {
            /* D' = cs^2 delta; for orders <= 2 in FP mode the lower moment is
             * rho (order 0), which is the same in both tables. */
            D[0] = CS2; D[1] = 0; D[2] = 0; D[3] = 0; D[4] = CS2; D[5] = 0; D[6] = 0; D[7] = 0; D[8] = CS2;
            memcpy(Pi, Meq, sizeof(Pi));
        } else {
            /* D' = kappa~_ij / rho (post-collision second order). */
            D[0] = Pt[(2 * 3 + 0) * 3 + 0] / rho; D[4] = Pt[(0 * 3 + 2) * 3 + 0] / rho;
            D[8] = Pt[(0 * 3 + 0) * 3 + 2] / rho;
            D[1] = D[3] = Pt[(1 * 3 + 1) * 3 + 0] / rho;
            D[2] = D[6] = Pt[(1 * 3 + 0) * 3 + 1] / rho;
            D[5] = D[7] = Pt[(0 * 3 + 1) * 3 + 1] / rho;
            memcpy(Pi, Pt, sizeof(Pi));
            /* Reading R1: first-order moments are 0 inside attractors. */
            Pi[(1 * 3 + 0) * 3 + 0] = 0; Pi[(0 * 3 + 1) * 3 + 0] = 0; Pi[(0 * 3 + 0) * 3 + 1] = 0;
            Pi[0] = rho;
        }
        for (int i = 0; i < Q; ++i) {
            const int m = MNP[i][0], n = MNP[i][1], p = MNP[i][2];
            const int s = m + n + p;
            if (s < lo || s > hi) continue;
            att[i] = orc_attractor_generic(m, n, p, Pi, D);
        }
        /* Group the attractors and relax each group of this stage. */
        for (int j = 0; j < Q; ++j) {
            const int o = group_order(j);
            if (o < lo || o > hi) continue;
            double ya = 0;
            for (int i = 0; i < Q; ++i) ya += G[j][i] * att[i];
            yt[j] = y[j] + omega[j] * (ya - y[j]) + (1.0 - 0.5 * omega[j]) * sg[j];
        }
        /* Undo the grouping with the numerical inverse of G and keep the
         * moments of this stage as post-collision values. */
        double kt[Q];
        if (orc_solve((const double(*)[Q])G, yt, kt) != 0) return -1;
        for (int i = 0; i < Q; ++i) {
            const int s = MNP[i][0] + MNP[i][1] + MNP[i][2];
            if (s >= lo && s <= hi) Pt[(MNP[i][0] * 3 + MNP[i][1]) * 3 + MNP[i][2]] = kt[i];
        }
    }

    /* Steps 4+5 as their definition: f~ = C(u)^-1 kappa~. */
    double kt[Q];
    for (int i = 0; i < Q; ++i) kt[i] = Pt[(MNP[i][0] * 3 + MNP[i][1]) * 3 + MNP[i][2]];
    return orc_solve((const double(*)[Q])C, kt, ft);
}

/* Reading R4: equilibrium populations f = C(u)^-1 kappa^eq(rho,u). */
int orc_equilibrium(double rho, const double u[3], double feq[Q])
{
    double C[Q][Q], M[27], k[Q];
    orc_central_matrix(u, C);
    orc_maxwell_moments(rho, M);
    for (int i = 0; i < Q; ++i) k[i] = M[(MNP[i][0] * 3 + MNP[i][1]) * 3 + MNP[i][2]];
    return orc_solve((const double(*)[Q])C, k, feq);
}

/* ------------------------------------------------------------------------ */
/* Lattice-level operations                                                   */
/* ------------------------------------------------------------------------ */

static int opposite(int a)
{
    for (int b = 0; b < Q; ++b)
        if (EX[b] == -EX[a] && EY[b] == -EY[a] && EZ[b] == -EZ[a]) return b;
    return -1;
}

static long wrap(long i, long n) { return ((i % n) + n) % n; }

/* Fill f (alpha-major) with equilibria of the fields rho, ux, uy, uz
 * (x-fastest, idx = x + nx*(y + ny*z)). */
int orc_init_equilibrium(int nx, int ny, int nz, const double* rho, const double* ux,
                         const double* uy, const double* uz, double* f)
{
    const long N = (long)nx * ny * nz;
    int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad)
    for (long c = 0; c < N; ++c) {
        double u[3] = {ux[c], uy[c], uz[c]}, fe[Q];
        if (orc_equilibrium(rho[c], u, fe) != 0) bad |= 1;
        for (int a = 0; a < Q; ++a) f[a * N + c] = fe[a];
    }
    return bad ? -1 : 0;
}

/* ------------------------------------------------------------------------ */
/* Smagorinsky subgrid model with van Driest damping (Sec. 4, turbulent     */
/* channel; the paper names the model and cites it, the formulas below are   */
/* the standard definitions, reading R7)                                     */
/* ------------------------------------------------------------------------ */

/* Effective shear relaxation time of one cell:
 *   nu_t = c2 |S|,  |S| = sqrt(2 S_ij S_ij),  c2 = (C_s Delta D)^2, Delta = 1,
 *   S_ij = -Pi^d_ij / (2 rho cs^2 tau),  tau = tau0 + nu_t / cs^2,
 * with Pi_ij = kappa_ij - cs^2 rho delta_ij the non-equilibrium second-order
 * central moments of the incoming populations (at the half-force velocity)
 * and Pi^d its deviatoric part (the trace belongs to the bulk rate, which the
 * model leaves alone).  tau is the root of the defining relation, found by
 * bisection. */
double orc_smagorinsky_tau(const double f[Q], const double F[3], double tau0, double c2)
{
    double rho = 0, j[3] = {0, 0, 0};
    for (int a = 0; a < Q; ++a) {
        rho += f[a];
        j[0] += f[a] * EX[a];
        j[1] += f[a] * EY[a];
        j[2] += f[a] * EZ[a];
    }
    const double u[3] = {(j[0] + 0.5 * F[0]) / rho, (j[1] + 0.5 * F[1]) / rho, (j[2] + 0.5 * F[2]) / rho};
    double P[3][3] = {{0}};
    for (int a = 0; a < Q; ++a) {
        const double c[3] = {EX[a] - u[0], EY[a] - u[1], EZ[a] - u[2]};
        for (int i = 0; i < 3; ++i)
            for (int k = 0; k < 3; ++k) P[i][k] += f[a] * c[i] * c[k];
    }
    for (int i = 0; i < 3; ++i) P[i][i] -= CS2 * rho;
    const double tr = (P[0][0] + P[1][1] + P[2][2]) / 3.0;
    for (int i = 0; i < 3; ++i) P[i][i] -= tr;
    double pp = 0;
    for (int i = 0; i < 3; ++i)
        for (int k = 0; k < 3; ++k) pp += P[i][k] * P[i][k];
    const double Pn = sqrt(2.0 * pp); /* |Pi^d| = sqrt(2 Pi^d : Pi^d) */
    /* g(tau) = tau - tau0 - c2 |S(tau)| / cs^2 is increasing on tau >= tau0 */
    double lo = tau0, hi = tau0 + c2 * Pn / (2.0 * rho * CS2 * tau0) / CS2;
    for (int it = 0; it < 200 && hi > lo; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        const double g = mid - tau0 - c2 * (Pn / (2.0 * rho * CS2 * mid)) / CS2;
        if (g > 0) hi = mid; else lo = mid;
    }
    return 0.5 * (lo + hi);
}

/* Distance of cell row y (cell centre) to the nearest wall of boundary kind
 * bc along y, or a negative value when there is none (bc 0; bc 2 uses all
 * three axes and is handled by the caller). */
static double wall_distance_y(int bc, int y, int ny)
{
    if (bc == 1) { const double a = y + 0.5, b = ny - 0.5 - y; return a < b ? a : b; }
    if (bc == 3) return y + 0.5;
    return -1.0;
}

/* van Driest damping D = 1 - exp(-y+ / A+), y+ = y_w u* / nu. */
static double van_driest(double yw, double u_star, double nu, double a_plus)
{
    if (yw < 0 || u_star <= 0 || a_plus <= 0) return 1.0;
    return 1.0 - exp(-(yw * u_star / nu) / a_plus);
}

/* One time step: collision (Steps 7,1-5) then push streaming (Step 6).
 * bc = 0: periodic in x, y, z;
 * bc = 1: half-way bounce-back walls at y = -1/2 and y = ny-1/2, periodic in
 *         x and z (channel);
 * bc = 2: closed box, half-way bounce-back walls at -1/2 and n-1/2 on all
 *         three axes (the cubic cavity of Sec. 4);
 * bc = 3: half channel (Sec. 4, turbulent channel): bounce-back wall at
 *         y = -1/2 and a specular-reflection symmetry plane at y = ny-1/2: a
 *         population leaving the top row along (ex, +1, ez) comes back along
 *         (ex, -1, ez) into the top row, shifted by (ex, ez) in x and z.
 * uw is the velocity of the wall at y = ny-1/2 (bc 1 and 2; it must be
 * tangential, uw[1] = 0).  The population that leaves cell x along e_a
 * towards a solid point is reflected into the opposite direction at x; when
 * that point lies in the layer y = ny (every link with e_ay = +1 out of the
 * top row, edges and corners included) it carries the moving-wall momentum
 * correction of half-way bounce-back that Sec. 4 applies to the cavity lid
 * (Ladd's form):
 *   f_opp(a)(x, t+1) = ft_a(x, t) - 2 w_a rho(x, t) (e_a . uw) / cs^2,
 * with w_a the rest weights (equilibrium at rho = 1, u = 0) and rho(x, t)
 * the density of the fluid cell.
 * les (optional, NULL for none) = {C_s, u*, A+}: Smagorinsky model with van
 * Driest damping; every cell's shear rates omega_4,5,6,8,9 become
 * 1 / orc_smagorinsky_tau(f, F, 1/omega_4, (C_s D)^2). */
int orc_step_les(int nx, int ny, int nz, int bc, const double* fin, double* fout,
                 const double F[3], const double omega[Q], int mode, const double uw[3],
                 const double* les)
{
    const long N = (long)nx * ny * nz;
    if (bc < 0 || bc > 3 || ((bc == 0 || bc == 3) && (uw[0] != 0 || uw[2] != 0)) || uw[1] != 0) return -2;
    int opp[Q], mir[Q];
    for (int a = 0; a < Q; ++a) {
        opp[a] = opposite(a);
        for (int b = 0; b < Q; ++b)
            if (EX[b] == EX[a] && EY[b] == -EY[a] && EZ[b] == EZ[a]) mir[a] = b;
    }
    double w[Q];
    const double zero[3] = {0, 0, 0};
    if (orc_equilibrium(1.0, zero, w) != 0) return -1;
    const double tau0 = 1.0 / omega[4], nu0 = CS2 * (tau0 - 0.5);
    int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad)
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                const long c = x + (long)nx * (y + (long)ny * z);
                double f[Q], ft[Q], rho = 0;
                for (int a = 0; a < Q; ++a) {
                    f[a] = fin[a * N + c];
                    rho += f[a];
                }
                const double* om = omega;
                double om_les[Q];
                if (les) {
                    double yw = wall_distance_y(bc, y, ny);
                    if (bc == 2) {
                        const double d[6] = {x + 0.5, nx - 0.5 - x, y + 0.5, ny - 0.5 - y, z + 0.5, nz - 0.5 - z};
                        yw = d[0];
                        for (int k = 1; k < 6; ++k) if (d[k] < yw) yw = d[k];
                    }
                    const double cd = les[0] * van_driest(yw, les[1], nu0, les[2]);
                    const double te = orc_smagorinsky_tau(f, F, tau0, cd * cd);
                    memcpy(om_les, omega, sizeof(om_les));
                    om_les[4] = om_les[5] = om_les[6] = om_les[8] = om_les[9] = 1.0 / te;
                    om = om_les;
                }
                if (orc_collide(f, F, om, mode, ft) != 0) bad |= 1;
                for (int a = 0; a < Q; ++a) {
                    const long xd = x + EX[a], yd = y + EY[a], zd = z + EZ[a];
                    if (bc == 3 && yd >= ny) { /* specular reflection at the symmetry plane */
                        const long xw = wrap(xd, nx), zw = wrap(zd, nz);
                        fout[mir[a] * N + xw + nx * ((long)(ny - 1) + (long)ny * zw)] = ft[a];
                        continue;
                    }
                    const int out_y = bc >= 1 && (yd < 0 || yd >= ny);
                    const int out_xz = bc == 2 && (xd < 0 || xd >= nx || zd < 0 || zd >= nz);
                    if (out_y || out_xz) { /* half-way bounce-back */
                        double v = ft[a];
                        if (yd == ny) v -= 2.0 * w[a] * rho * (EX[a] * uw[0] + EZ[a] * uw[2]) / CS2;
                        fout[opp[a] * N + c] = v;
                        continue;
                    }
                    const long xw = wrap(xd, nx), yw = wrap(yd, ny), zw = wrap(zd, nz);
                    fout[a * N + xw + nx * (yw + (long)ny * zw)] = ft[a];
                }
            }
    return bad ? -1 : 0;
}

int orc_step_bc(int nx, int ny, int nz, int bc, const double* fin, double* fout,
                const double F[3], const double omega[Q], int mode, const double uw[3])
{
    return orc_step_les(nx, ny, nz, bc, fin, fout, F, omega, mode, uw, NULL);
}

/* orc_step_bc with resting walls. */
int orc_step(int nx, int ny, int nz, int bc, const double* fin, double* fout,
             const double F[3], const double omega[Q], int mode)
{
    const double still[3] = {0, 0, 0};
    return orc_step_bc(nx, ny, nz, bc, fin, fout, F, omega, mode, still);
}

/* n time steps; f is updated in place, work is scratch of the same size. */
int orc_run_les(int nx, int ny, int nz, int bc, double* f, double* work, const double F[3],
                const double omega[Q], int mode, long nsteps, const double uw[3], const double* les)
{
    const long N = (long)nx * ny * nz;
    double *a = f, *b = work;
    int rc = 0;
    for (long t = 0; t < nsteps && rc == 0; ++t) {
        rc = orc_step_les(nx, ny, nz, bc, a, b, F, omega, mode, uw, les);
        double* tmp = a; a = b; b = tmp;
    }
    if (a != f) memcpy(f, a, sizeof(double) * Q * N);
    return rc;
}

int orc_run_bc(int nx, int ny, int nz, int bc, double* f, double* work, const double F[3],
               const double omega[Q], int mode, long nsteps, const double uw[3])
{
    return orc_run_les(nx, ny, nz, bc, f, work, F, omega, mode, nsteps, uw, NULL);
}

int orc_run(int nx, int ny, int nz, int bc, double* f, double* work, const double F[3],
            const double omega[Q], int mode, long nsteps)
{
    const double still[3] = {0, 0, 0};
    return orc_run_bc(nx, ny, nz, bc, f, work, F, omega, mode, nsteps, still);
}

/* Step 7: rho and u (with half force) of every cell. */
void orc_moments(int nx, int ny, int nz, const double* f, const double F[3], double* rho,
                 double* ux, double* uy, double* uz)
{
    const long N = (long)nx * ny * nz;
#pragma omp parallel for schedule(static)
    for (long c = 0; c < N; ++c) {
        double r = 0, jx = 0, jy = 0, jz = 0;
        for (int a = 0; a < Q; ++a) {
            const double v = f[a * N + c];
            r += v; jx += v * EX[a]; jy += v * EY[a]; jz += v * EZ[a];
        }
        rho[c] = r;
        ux[c] = (jx + 0.5 * F[0]) / r;
        uy[c] = (jy + 0.5 * F[1]) / r;
        uz[c] = (jz + 0.5 * F[2]) / r;
    }
}

/* Relaxation rates from (tau, drift) (Appendix C Eq. transportcoeff3DFPCLBM,
 * Sec. 3 omega_mnp = (m+n+p) omega_FP, Sec. 4 remark on unit rates):
 *   omega_4,5,6,8,9 = 1/tau (shear), omega_7 = 1 (bulk), omega_0..3 = 1 (no
 *   effect), orders >= 3: drift > 0 ? order*drift : 1. */
void orc_rates(double tau, double drift, double omega[Q])
{
    for (int j = 0; j < Q; ++j) {
        const int o = group_order(j);
        if (o <= 1) omega[j] = 1.0;
        else if (o == 2) omega[j] = 1.0 / tau;
        else omega[j] = drift > 0 ? o * drift : 1.0;
    }
    omega[7] = 1.0;
}

/* Introspection for the tests. */
void orc_velocity_set(int* ex, int* ey, int* ez)
{
    for (int a = 0; a < Q; ++a) { ex[a] = EX[a]; ey[a] = EY[a]; ez[a] = EZ[a]; }
}
void orc_moment_exponents(int* mnp)
{
    for (int i = 0; i < Q; ++i) { mnp[3 * i] = MNP[i][0]; mnp[3 * i + 1] = MNP[i][1]; mnp[3 * i + 2] = MNP[i][2]; }
}

/* Timing of the oracle as a CPU baseline: threads of the parallel loops (n >= 1; no effect
 * without OpenMP), and the count the runtime will use. */
void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n >= 1) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
