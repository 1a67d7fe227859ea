/*
 * fpc2d_oracle.c -- slow, literal FP64 CPU statement of the D2Q9 FPC-LBM.
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE (see fpc_oracle.c; compiled into the
 * same oracle library, sharing nothing with the CUDA path).
 *
 * What it computes (Schupbach & Premnath, arXiv 2410.09739, Sec. 2 and the
 * appendix on the 2D algorithm):
 *   - D2Q9 velocities in the order of Sec. 2 (Construction of 2D FPC-LBM);
 *   - central moments kappa_mn = sum_a f_a (e_ax-u_x)^m (e_ay-u_y)^n in the
 *     order of m^c = (00,10,01,20,02,11,21,12,22), built as one explicit 9x9
 *     matrix and undone by a numerical LU solve;
 *   - attractors from the generic formula Eq. (Mvcmattractor2D) with the
 *     diffusion tensor of Sec. 2 (choice of diffusion tensor parameter):
 *     D' = cs^2 delta for order <= 2, D' = kappa~_ij / rho above;
 *   - sources Eq. (forcing:2D) / (sourceCM2D) with first-order moments 0 and
 *     pre-collision kappa (readings R1, R5 of fpc_oracle.c);
 *   - the 2D Step 3 grouping (2s = 20 + 02, 2d = 20 - 02) as a 9x9 matrix and
 *     its numerical inverse, rates omega_0..omega_8 in the 2D numbering
 *     (3: 2s bulk, 4: 2d and 5: 11 shear, 6: 21, 7: 12, 8: 22);
 *   - chain order: orders <= 2, then 3, then 4 (the fourth-order attractor
 *     uses post-collision second moments, reading R2);
 *   - half-force velocity of Step 7, push streaming of Step 6, periodic or in
 *     a closed square box with half-way bounce-back and a moving lid (the 2D
 *     lid-driven cavity of Sec. 4).
 * mode 1 (MCM): Maxwellian central moments at every order (reading R3).
 *
 * Arrays: f[a][y][x], a = 0..8 (alpha-major), full populations, fp64.
 */
#include <math.h>
#include <string.h>

#define Q2 9
#define CS2_2D (1.0 / 3.0)

static const int EX2[Q2] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int EY2[Q2] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const int MN2[Q2][2] = {{0, 0}, {1, 0}, {0, 1}, {2, 0}, {0, 2}, {1, 1}, {2, 1}, {1, 2}, {2, 2}};

static int idx2(int m, int n)
{
    for (int i = 0; i < Q2; ++i)
        if (MN2[i][0] == m && MN2[i][1] == n) return i;
    return -1;
}

static double pw2(double b, int e)
{
    double r = 1.0;
    for (int k = 0; k < e; ++k) r *= b;
    return r;
}

/* C(u)[i][a] = (e_ax - u_x)^m_i (e_ay - u_y)^n_i; with u = 0 the raw-moment
 * projection P of Sec. 2. */
void orc2_central_matrix(const double u[2], double C[Q2][Q2])
{
    for (int i = 0; i < Q2; ++i)
        for (int a = 0; a < Q2; ++a) C[i][a] = pw2(EX2[a] - u[0], MN2[i][0]) * pw2(EY2[a] - u[1], MN2[i][1]);
}

/* Group index j of the 2D Step 3: 0:00 1:10 2:01 3:2s 4:2d 5:11 6:21 7:12 8:22. */
void orc2_grouping_matrix(double G[Q2][Q2])
{
    memset(G, 0, sizeof(double) * Q2 * Q2);
    G[0][idx2(0, 0)] = 1;
    G[1][idx2(1, 0)] = 1;
    G[2][idx2(0, 1)] = 1;
    G[3][idx2(2, 0)] = 1; G[3][idx2(0, 2)] = 1;
    G[4][idx2(2, 0)] = 1; G[4][idx2(0, 2)] = -1;
    G[5][idx2(1, 1)] = 1;
    G[6][idx2(2, 1)] = 1;
    G[7][idx2(1, 2)] = 1;
    G[8][idx2(2, 2)] = 1;
}

static int order2(int j)
{
    if (j == 0) return 0;
    if (j <= 2) return 1;
    if (j <= 5) return 2;
    if (j <= 7) return 3;
    return 4;
}

/* Solve A x = b (n <= 9) by Gaussian elimination with partial pivoting. */
static int solve_small(int n, const double A_in[Q2][Q2], const double b_in[Q2], double x[Q2])
{
    double A[Q2][Q2], b[Q2];
    memcpy(A, A_in, sizeof(A));
    memcpy(b, b_in, sizeof(b));
    for (int k = 0; k < n; ++k) {
        int p = k;
        for (int i = k + 1; i < n; ++i)
            if (fabs(A[i][k]) > fabs(A[p][k])) p = i;
        if (A[p][k] == 0.0) return -1;
        if (p != k) {
            for (int j = 0; j < n; ++j) { const double t = A[k][j]; A[k][j] = A[p][j]; A[p][j] = t; }
            const double t = b[k]; b[k] = b[p]; b[p] = t;
        }
        for (int i = k + 1; i < n; ++i) {
            const double l = A[i][k] / A[k][k];
            for (int j = k; j < n; ++j) A[i][j] -= l * A[k][j];
            b[i] -= l * b[k];
        }
    }
    for (int i = n - 1; i >= 0; --i) {
        double s = b[i];
        for (int j = i + 1; j < n; ++j) s -= A[i][j] * x[j];
        x[i] = s / A[i][i];
    }
    return 0;
}

/* Eq. (Mvcmattractor2D): Pi[m][n] lower moments (3x3), D = (Dxx, Dyy, Dxy). */
double orc2_attractor_generic(int m, int n, const double Pi[3][3], const double D[3])
{
    if (m + n == 0) return Pi[0][0];
    double s = 0;
    if (m >= 2) s += m * (m - 1) * D[0] * Pi[m - 2][n];
    if (n >= 2) s += n * (n - 1) * D[1] * Pi[m][n - 2];
    if (m >= 1 && n >= 1) s += 2.0 * m * n * D[2] * Pi[m - 1][n - 1];
    return s / (m + n);
}

/* Maxwellian central moments: rho, 0, cs^2 rho (20, 02), cs^4 rho (22). */
static void maxwell2(double rho, double M[3][3])
{
    memset(M, 0, sizeof(double) * 9);
    M[0][0] = rho;
    M[2][0] = M[0][2] = CS2_2D * rho;
    M[2][2] = CS2_2D * CS2_2D * rho;
}

/* Steps 7, 1-5 of the 2D appendix for one cell (mode 0 FP, 1 MCM). */
int orc2_collide(const double f[Q2], const double F[2], const double omega[Q2], int mode, double ft[Q2])
{
    double rho = 0, jx = 0, jy = 0;
    for (int a = 0; a < Q2; ++a) { rho += f[a]; jx += f[a] * EX2[a]; jy += f[a] * EY2[a]; }
    const double u[2] = {(jx + 0.5 * F[0]) / rho, (jy + 0.5 * F[1]) / rho};
    double C[Q2][Q2], kap[Q2];
    orc2_central_matrix(u, C);
    for (int i = 0; i < Q2; ++i) {
        double s = 0;
        for (int a = 0; a < Q2; ++a) s += C[i][a] * f[a];
        kap[i] = s;
    }
    double K[3][3] = {{0}};
    for (int i = 0; i < Q2; ++i) K[MN2[i][0]][MN2[i][1]] = kap[i];
    double Ks[3][3];
    memcpy(Ks, K, sizeof(Ks));
    Ks[1][0] = Ks[0][1] = 0; /* R1 */
    double sig[Q2];
    for (int i = 0; i < Q2; ++i) {
        const int m = MN2[i][0], n = MN2[i][1];
        double s = 0;
        if (m >= 1) s += m * (F[0] / rho) * Ks[m - 1][n];
        if (n >= 1) s += n * (F[1] / rho) * Ks[m][n - 1];
        sig[i] = s;
    }
    double G[Q2][Q2], y[Q2], sg[Q2];
    orc2_grouping_matrix(G);
    for (int j = 0; j < Q2; ++j) {
        double a = 0, b = 0;
        for (int i = 0; i < Q2; ++i) { a += G[j][i] * kap[i]; b += G[j][i] * sig[i]; }
        y[j] = a;
        sg[j] = b;
    }
    double Pt[3][3] = {{0}}, Meq[3][3];
    maxwell2(rho, Meq);
    double yt[Q2];
    memcpy(yt, y, sizeof(yt));
    static const int lo_[3] = {0, 3, 4}, hi_[3] = {2, 3, 4};
    for (int st = 0; st < 3; ++st) {
        const int lo = lo_[st], hi = hi_[st];
        double D[3], Pi[3][3], att[Q2];
        memset(att, 0, sizeof(att));
        if (mode == 1 || hi <= 2) {
            D[0] = CS2_2D; D[1] = CS2_2D; D[2] = 0;
            memcpy(Pi, Meq, sizeof(Pi));
        } else {
            D[0] = Pt[2][0] / rho; D[1] = Pt[0][2] / rho; D[2] = Pt[1][1] / rho;
            memcpy(Pi, Pt, sizeof(Pi));
            Pi[1][0] = Pi[0][1] = 0; /* R1 */
            Pi[0][0] = rho;
        }
        for (int i = 0; i < Q2; ++i) {
            const int s = MN2[i][0] + MN2[i][1];
            if (s >= lo && s <= hi) att[i] = orc2_attractor_generic(MN2[i][0], MN2[i][1], (const double(*)[3])Pi, D);
        }
        for (int j = 0; j < Q2; ++j) {
            const int o = order2(j);
            if (o < lo || o > hi) continue;
            double ya = 0;
            for (int i = 0; i < Q2; ++i) ya += G[j][i] * att[i];
            yt[j] = y[j] + omega[j] * (ya - y[j]) + (1.0 - 0.5 * omega[j]) * sg[j];
        }
        double kt[Q2];
        if (solve_small(Q2, (const double(*)[Q2])G, yt, kt) != 0) return -1;
        for (int i = 0; i < Q2; ++i) {
            const int s = MN2[i][0] + MN2[i][1];
            if (s >= lo && s <= hi) Pt[MN2[i][0]][MN2[i][1]] = kt[i];
        }
    }
    double kt[Q2];
    for (int i = 0; i < Q2; ++i) kt[i] = Pt[MN2[i][0]][MN2[i][1]];
    return solve_small(Q2, (const double(*)[Q2])C, kt, ft);
}

/* Equilibrium f = C(u)^-1 kappa^eq(rho) (reading R4). */
int orc2_equilibrium(double rho, const double u[2], double feq[Q2])
{
    double C[Q2][Q2], M[3][3], k[Q2];
    orc2_central_matrix(u, C);
    maxwell2(rho, M);
    for (int i = 0; i < Q2; ++i) k[i] = M[MN2[i][0]][MN2[i][1]];
    return solve_small(Q2, (const double(*)[Q2])C, k, feq);
}

int orc2_init_equilibrium(int nx, int ny, const double* rho, const double* ux, const double* uy, double* f)
{
    const long N = (long)nx * ny;
    int bad = 0;
    for (long c = 0; c < N; ++c) {
        const double u[2] = {ux[c], uy[c]};
        double fe[Q2];
        if (orc2_equilibrium(rho[c], u, fe) != 0) bad = 1;
        for (int a = 0; a < Q2; ++a) f[a * N + c] = fe[a];
    }
    return bad ? -1 : 0;
}

static long wrap2(long i, long n) { return ((i % n) + n) % n; }

/* One step: collide, then push streaming f_a(x + e_a) = f~_a(x).
 * bc = 0: periodic; bc = 2: closed square box, half-way bounce-back at -1/2
 * and n - 1/2 on both axes, the wall y = ny - 1/2 moving along x at uw (the
 * 2D lid-driven cavity of Sec. 4): a population leaving cell x towards a
 * solid point is reflected into the opposite direction at x, and through the
 * moving wall (destination row y = ny, corners included) it carries the
 * momentum correction -2 w_a rho(x) e_ax uw / cs^2 (as in 3D, reading R6). */
int orc2_step_bc(int nx, int ny, int bc, const double* fin, double* fout, const double F[2], const double omega[Q2],
                 int mode, double uw)
{
    const long N = (long)nx * ny;
    if ((bc != 0 && bc != 2) || (bc == 0 && uw != 0)) return -2;
    int opp[Q2];
    for (int a = 0; a < Q2; ++a)
        for (int b = 0; b < Q2; ++b)
            if (EX2[b] == -EX2[a] && EY2[b] == -EY2[a]) opp[a] = b;
    double w[Q2];
    const double zero[2] = {0, 0};
    if (orc2_equilibrium(1.0, zero, w) != 0) return -1;
    int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad)
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            const long c = x + (long)nx * y;
            double f[Q2], ft[Q2], rho = 0;
            for (int a = 0; a < Q2; ++a) {
                f[a] = fin[a * N + c];
                rho += f[a];
            }
            if (orc2_collide(f, F, omega, mode, ft) != 0) bad |= 1;
            for (int a = 0; a < Q2; ++a) {
                const long xd = x + EX2[a], yd = y + EY2[a];
                if (bc == 2 && (xd < 0 || xd >= nx || yd < 0 || yd >= ny)) {
                    double v = ft[a];
                    if (yd == ny) v -= 2.0 * w[a] * rho * EX2[a] * uw / CS2_2D;
                    fout[opp[a] * N + c] = v;
                    continue;
                }
                fout[a * N + wrap2(xd, nx) + nx * wrap2(yd, ny)] = ft[a];
            }
        }
    return bad ? -1 : 0;
}

int orc2_step(int nx, int ny, const double* fin, double* fout, const double F[2], const double omega[Q2], int mode)
{
    return orc2_step_bc(nx, ny, 0, fin, fout, F, omega, mode, 0.0);
}

int orc2_run_bc(int nx, int ny, int bc, double* f, double* work, const double F[2], const double omega[Q2], int mode,
                long n, double uw)
{
    const long N = (long)nx * ny;
    double *a = f, *b = work;
    int rc = 0;
    for (long t = 0; t < n && rc == 0; ++t) {
        rc = orc2_step_bc(nx, ny, bc, a, b, F, omega, mode, uw);
        double* tmp = a; a = b; b = tmp;
    }
    if (a != f) memcpy(f, a, sizeof(double) * Q2 * N);
    return rc;
}

int orc2_run(int nx, int ny, double* f, double* work, const double F[2], const double omega[Q2], int mode, long n)
{
    return orc2_run_bc(nx, ny, 0, f, work, F, omega, mode, n, 0.0);
}

void orc2_moments(int nx, int ny, const double* f, const double F[2], double* rho, double* ux, double* uy)
{
    const long N = (long)nx * ny;
    for (long c = 0; c < N; ++c) {
        double r = 0, jx = 0, jy = 0;
        for (int a = 0; a < Q2; ++a) {
            const double v = f[a * N + c];
            r += v; jx += v * EX2[a]; jy += v * EY2[a];
        }
        rho[c] = r;
        ux[c] = (jx + 0.5 * F[0]) / r;
        uy[c] = (jy + 0.5 * F[1]) / r;
    }
}

/* Rates (2D Step 3 numbering): shear omega_4 = omega_5 = 1/tau, bulk
 * omega_3 = bulk (> 0) or 1, orders 3 and 4: order * drift when drift > 0,
 * else 1; omega_0..2 = 1. */
void orc2_rates(double tau, double bulk, double drift, double omega[Q2])
{
    for (int j = 0; j < Q2; ++j) omega[j] = 1.0;
    omega[3] = bulk > 0 ? bulk : 1.0;
    omega[4] = omega[5] = 1.0 / tau;
    for (int j = 6; j < Q2; ++j) omega[j] = drift > 0 ? order2(j) * drift : 1.0;
}

void orc2_velocity_set(int* ex, int* ey)
{
    for (int a = 0; a < Q2; ++a) { ex[a] = EX2[a]; ey[a] = EY2[a]; }
}
