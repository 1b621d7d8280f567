/*
 * d2q37_oracle.c -- plain, slow FP64 CPU oracle for the D2Q37 thermal lattice
 * Boltzmann step of Ripesi, Biferale, Schifano & Tripiccione (PRE 89, 043022, 2014).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the package smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no code, header
 * or constant table with the CUDA path: it builds its own velocity set, solves its
 * own quadrature, and evaluates the equilibrium as a generic Hermite tensor
 * contraction (the CUDA path uses a closed form).
 *
 * Every function follows one passage of the paper:
 *   - velocity set and lattice constant r ~ 1.1969 ........ Sec. III.A, Fig. 2 caption
 *   - lattice BGK evolution ................................. Sec. III.A, Eq. (LBE)
 *   - equilibrium with the force shift u+g tau, T+tau(dt-tau)g^2/d ... Sec. III.A
 *   - moments rho, rho u, d rho T ........................... Sec. III.A
 *   - renormalised u^H, T^H ................................. Sec. III.A
 *   - pull propagate, periodic x, bc on rows 0..2, Lz-3..Lz-1 ... Sec. III.B
 *   - three-layer hydrostatic initial state ................. Sec. I, Eq. (seteq), pressure
 *                                                             continuity, Fig. 1 caption
 *   - horizontal mean T(z) and mixing lengths ............... Sec. IV (threshold definition,
 *                                                             tent map, Eq. (3L))
 * Where the paper cites but does not print a formula (weights, Hermite order, wall rule)
 * the reading is stated at the function.  The adjoint functions differentiate the same
 * step (chain rule written out; the Jacobian is formed explicitly per site).
 *
 * Array layout (the paper's structure-of-arrays, column-major, Sec. III.B):
 *   f[l][x][z], z fastest; index ((l*Lx)+x)*Lz+z.
 * Units: Delta t = 1, reference temperature 1, xi_l = r c_l, gravity vector (0,-g);
 * one lattice spacing is r length units, so row k sits at height r (k + 1/2).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define NPOP 37
#define DIM 2

typedef long double ld;

static int    g_setup_done = 0;
static int    VEL[NPOP][2];       /* integer lattice vectors c_l */
static int    OPPO[NPOP];         /* index of -c_l */
static int    SHELL_OF[NPOP];     /* shell index of c_l */
static double XI[NPOP][2];        /* r c_l */
static double WGT[NPOP];          /* quadrature weights */
static double R_LATTICE;
static double WSHELL[8];
static const int SHELL_C2[8] = {0, 1, 2, 4, 5, 8, 9, 10};

/* Hermite tensor polynomials at each xi_l, orders 0..4, all index tuples in {0,1}^n */
static double HERM[5][16][NPOP];

static size_t ix(int Lx, int Lz, int l, int x, int z) {
    return ((size_t)l * Lx + x) * Lz + z;
}

/* ---------------------------------------------------------------------------
 * Velocity set (Sec. III.A, Fig. 2 caption: 37 velocities, speeds up to sqrt(10)
 * in units of the lattice constant r).  Reading: all integer vectors with
 * |c|^2 in {0,1,2,4,5,8,9,10}.  Canonical order: shells by |c|^2, then by
 * polar angle atan2(c_z, c_x) in [0, 2 pi).
 * ------------------------------------------------------------------------- */
static double polar_angle(int cx, int cz) {
    double a = atan2((double)cz, (double)cx);
    if (a < 0) a += 2.0 * M_PI;
    return a;
}

static int cmp_vel(const void *pa, const void *pb) {
    const int *a = (const int *)pa, *b = (const int *)pb;
    int a2 = a[0] * a[0] + a[1] * a[1], b2 = b[0] * b[0] + b[1] * b[1];
    if (a2 != b2) return a2 < b2 ? -1 : 1;
    double ta = polar_angle(a[0], a[1]), tb = polar_angle(b[0], b[1]);
    if (ta == tb) return 0;
    return ta < tb ? -1 : 1;
}

static int build_velocity_set(void) {
    int n = 0;
    for (int cx = -3; cx <= 3; cx++)
        for (int cz = -3; cz <= 3; cz++) {
            int c2 = cx * cx + cz * cz, ok = 0;
            for (int s = 0; s < 8; s++) ok |= (c2 == SHELL_C2[s]);
            if (!ok) continue;
            if (n >= NPOP) return -1;
            VEL[n][0] = cx; VEL[n][1] = cz; n++;
        }
    if (n != NPOP) return -1;
    qsort(VEL, NPOP, sizeof(VEL[0]), cmp_vel);
    for (int l = 0; l < NPOP; l++) {
        int c2 = VEL[l][0] * VEL[l][0] + VEL[l][1] * VEL[l][1];
        for (int s = 0; s < 8; s++) if (SHELL_C2[s] == c2) SHELL_OF[l] = s;
        OPPO[l] = -1;
        for (int m = 0; m < NPOP; m++)
            if (VEL[m][0] == -VEL[l][0] && VEL[m][1] == -VEL[l][1]) OPPO[l] = m;
        if (OPPO[l] < 0) return -1;
    }
    return 0;
}

/* ---------------------------------------------------------------------------
 * Quadrature (Sec. III.A; the paper cites the D2Q37 construction and prints only
 * r ~ 1.1969).  Reading: the shell weights w_s and r make the discrete moments
 * sum_l w_l xi_x^a xi_z^b equal those of the unit 2-D Gaussian for the nine even
 * monomials (a,b) = (0,0),(2,0),(4,0),(2,2),(6,0),(4,2),(8,0),(6,2),(4,4).
 * Solved here as: for fixed r the eight equations other than (2,0) are linear in
 * the weights; r is then the root of the (2,0) residual, found by bisection in
 * long double on [1.1, 1.3].
 * ------------------------------------------------------------------------- */
static ld gauss_moment_1d(int a) {          /* E[x^a], x ~ N(0,1) */
    if (a % 2) return 0.0L;
    ld m = 1.0L;
    for (int k = a - 1; k > 0; k -= 2) m *= (ld)k;
    return m;
}

static const int QEQ[9][2] = {{0,0},{2,0},{4,0},{2,2},{6,0},{4,2},{8,0},{6,2},{4,4}};

static ld ipow(ld b, int e) { ld p = 1.0L; for (int i = 0; i < e; i++) p *= b; return p; }

static void quad_matrix(ld r, ld A[9][8], ld rhs[9]) {
    for (int e = 0; e < 9; e++) {
        rhs[e] = gauss_moment_1d(QEQ[e][0]) * gauss_moment_1d(QEQ[e][1]);
        for (int s = 0; s < 8; s++) A[e][s] = 0.0L;
        for (int l = 0; l < NPOP; l++)
            A[e][SHELL_OF[l]] += ipow(r * VEL[l][0], QEQ[e][0]) * ipow(r * VEL[l][1], QEQ[e][1]);
    }
}

/* Gaussian elimination with partial pivoting on an n x n long double system. */
static int solve_ld(int n, ld M[8][9]) {
    for (int c = 0; c < n; c++) {
        int p = c;
        for (int i = c + 1; i < n; i++) if (fabsl(M[i][c]) > fabsl(M[p][c])) p = i;
        if (M[p][c] == 0.0L) return -1;
        if (p != c) for (int j = 0; j <= n; j++) { ld t = M[c][j]; M[c][j] = M[p][j]; M[p][j] = t; }
        for (int i = 0; i < n; i++) {
            if (i == c) continue;
            ld f = M[i][c] / M[c][c];
            for (int j = c; j <= n; j++) M[i][j] -= f * M[c][j];
        }
    }
    for (int i = 0; i < n; i++) M[i][n] /= M[i][i];
    return 0;
}

static int weights_for_r(ld r, ld w[8], ld *resid) {
    ld A[9][8], rhs[9], M[8][9];
    quad_matrix(r, A, rhs);
    int row = 0;
    for (int e = 0; e < 9; e++) {
        if (e == 1) continue;                 /* (2,0) is the residual equation */
        for (int s = 0; s < 8; s++) M[row][s] = A[e][s];
        M[row][8] = rhs[e];
        row++;
    }
    if (solve_ld(8, M)) return -1;
    ld res = -rhs[1];
    for (int s = 0; s < 8; s++) { w[s] = M[s][8]; res += A[1][s] * w[s]; }
    *resid = res;
    return 0;
}

static int solve_quadrature(void) {
    ld lo = 1.1L, hi = 1.3L, w[8], flo, fhi, fm;
    if (weights_for_r(lo, w, &flo) || weights_for_r(hi, w, &fhi)) return -2;
    if (!((flo > 0) != (fhi > 0))) return -3;
    for (int it = 0; it < 200; it++) {
        ld mid = 0.5L * (lo + hi);
        if (weights_for_r(mid, w, &fm)) return -2;
        if ((fm > 0) == (flo > 0)) { lo = mid; flo = fm; } else { hi = mid; }
        if (hi - lo < 1e-19L) break;
    }
    ld r = 0.5L * (lo + hi);
    if (weights_for_r(r, w, &fm)) return -2;
    R_LATTICE = (double)r;
    for (int s = 0; s < 8; s++) { WSHELL[s] = (double)w[s]; if (w[s] <= 0) return -4; }
    for (int l = 0; l < NPOP; l++) {
        WGT[l] = WSHELL[SHELL_OF[l]];
        XI[l][0] = (double)(r * VEL[l][0]);
        XI[l][1] = (double)(r * VEL[l][1]);
    }
    return 0;
}

/* ---------------------------------------------------------------------------
 * Generic "sum over partial pairings" of an index tuple (i_1..i_n):
 *     S = sum over sets M of disjoint index pairs of
 *         pw^{|M|} * prod_{(a,b) in M} delta(i_a,i_b) * prod_{unpaired k} v[i_k]
 * With pw = -1 and v = xi this is the Hermite tensor polynomial H^(n)(xi); with
 * pw = theta and v = u it is the n-th Hermite coefficient of the Maxwellian of mean u
 * and temperature 1 + theta (the equilibrium expansion the paper cites in Sec. III.A).
 * dv_i (optional) returns dS/dv_i, dpw the derivative with respect to pw.
 * ------------------------------------------------------------------------- */
static void pairing_sum(int n, const int *idx, const double *v, double pw,
                        double *S, double dS_dv[2], double *dS_dpw) {
    double s = 0.0, dv0 = 0.0, dv1 = 0.0, dp = 0.0;
    /* enumerate matchings by recursion on an explicit stack: n <= 4 so at most 10 */
    /* list all matchings for n <= 4 explicitly by pairing masks */
    int pairs[16][2][2]; int npairs_of[16]; int nm = 0;
    /* empty matching */
    npairs_of[nm] = 0; nm++;
    for (int a = 0; a < n; a++)
        for (int b = a + 1; b < n; b++) {
            npairs_of[nm] = 1; pairs[nm][0][0] = a; pairs[nm][0][1] = b; nm++;
        }
    if (n == 4) {
        int P[3][2][2] = {{{0,1},{2,3}}, {{0,2},{1,3}}, {{0,3},{1,2}}};
        for (int k = 0; k < 3; k++) {
            npairs_of[nm] = 2;
            pairs[nm][0][0] = P[k][0][0]; pairs[nm][0][1] = P[k][0][1];
            pairs[nm][1][0] = P[k][1][0]; pairs[nm][1][1] = P[k][1][1];
            nm++;
        }
    }
    for (int m = 0; m < nm; m++) {
        int used[4] = {0, 0, 0, 0};
        double term = 1.0;
        for (int p = 0; p < npairs_of[m]; p++) {
            int a = pairs[m][p][0], b = pairs[m][p][1];
            used[a] = used[b] = 1;
            term *= (idx[a] == idx[b]) ? 1.0 : 0.0;
        }
        if (term == 0.0) continue;
        double pwk = 1.0, dpwk = 0.0;
        for (int p = 0; p < npairs_of[m]; p++) { dpwk = dpwk * pw + pwk; pwk *= pw; }
        double prod = 1.0;
        int free_idx[4], nf = 0;
        for (int k = 0; k < n; k++) if (!used[k]) { free_idx[nf++] = idx[k]; prod *= v[idx[k]]; }
        s += pwk * prod;
        dp += dpwk * prod;
        for (int q = 0; q < nf; q++) {       /* product rule over the unpaired factors */
            double pr = 1.0;
            for (int k = 0; k < nf; k++) if (k != q) pr *= v[free_idx[k]];
            if (free_idx[q] == 0) dv0 += pwk * pr; else dv1 += pwk * pr;
        }
    }
    *S = s;
    if (dS_dv) { dS_dv[0] = dv0; dS_dv[1] = dv1; }
    if (dS_dpw) *dS_dpw = dp;
}

static void tuple_of(int n, int t, int *idx) { for (int k = 0; k < n; k++) idx[k] = (t >> k) & 1; }

static void build_hermite_tables(void) {
    for (int l = 0; l < NPOP; l++)
        for (int n = 0; n <= 4; n++)
            for (int t = 0; t < (1 << n); t++) {
                int idx[4]; double h;
                tuple_of(n, t, idx);
                pairing_sum(n, idx, XI[l], -1.0, &h, NULL, NULL);
                HERM[n][t][l] = h;
            }
}

int oracle_setup(void) {
    if (g_setup_done) return 0;
    if (build_velocity_set()) return -1;
    int rc = solve_quadrature();
    if (rc) return rc;
    build_hermite_tables();
    g_setup_done = 1;
    return 0;
}

int oracle_velocities(int *c, int *opp) {
    if (oracle_setup()) return -1;
    for (int l = 0; l < NPOP; l++) { c[2 * l] = VEL[l][0]; c[2 * l + 1] = VEL[l][1]; opp[l] = OPPO[l]; }
    return NPOP;
}

int oracle_weights(double *w, double *r) {
    if (oracle_setup()) return -1;
    for (int l = 0; l < NPOP; l++) w[l] = WGT[l];
    *r = R_LATTICE;
    return NPOP;
}

/* ---------------------------------------------------------------------------
 * Equilibrium (Sec. III.A).  Reading: the 4th-order Hermite expansion of the
 * Maxwellian, f^eq_l = w_l rho sum_{n<=4} (1/n!) a^(n)(u, theta) : H^(n)(xi_l),
 * theta = T - 1, evaluated by explicit tensor contraction over all index tuples.
 * Optional outputs: derivatives with respect to u_x, u_z and T.
 * ------------------------------------------------------------------------- */
static const double INV_FACT[5] = {1.0, 1.0, 0.5, 1.0 / 6.0, 1.0 / 24.0};

static void equilibrium_with_derivs(double rho, double ux, double uz, double T,
                                    double *feq, double (*dfdu)[2], double *dfdT) {
    double u[2] = {ux, uz}, th = T - 1.0;
    double acoef[5][16], adu[5][16][2], adth[5][16];
    for (int n = 0; n <= 4; n++)
        for (int t = 0; t < (1 << n); t++) {
            int idx[4];
            tuple_of(n, t, idx);
            pairing_sum(n, idx, u, th, &acoef[n][t], adu[n][t], &adth[n][t]);
        }
    for (int l = 0; l < NPOP; l++) {
        double s = 0.0, su0 = 0.0, su1 = 0.0, sth = 0.0;
        for (int n = 0; n <= 4; n++)
            for (int t = 0; t < (1 << n); t++) {
                double h = HERM[n][t][l] * INV_FACT[n];
                s += acoef[n][t] * h;
                su0 += adu[n][t][0] * h;
                su1 += adu[n][t][1] * h;
                sth += adth[n][t] * h;
            }
        feq[l] = WGT[l] * rho * s;
        if (dfdu) { dfdu[l][0] = WGT[l] * rho * su0; dfdu[l][1] = WGT[l] * rho * su1; }
        if (dfdT) dfdT[l] = WGT[l] * rho * sth;
    }
}

void oracle_equilibrium(double rho, double ux, double uz, double T, double *feq) {
    oracle_setup();
    equilibrium_with_derivs(rho, ux, uz, T, feq, NULL, NULL);
}

/* ---------------------------------------------------------------------------
 * Moments at one site (Sec. III.A): rho = sum f, rho u = sum xi f,
 * D rho T = sum |xi - u|^2 f.
 * ------------------------------------------------------------------------- */
static void site_moments(const double *fs, double *rho, double *ux, double *uz, double *T) {
    double r = 0.0, jx = 0.0, jz = 0.0;
    for (int l = 0; l < NPOP; l++) { r += fs[l]; jx += XI[l][0] * fs[l]; jz += XI[l][1] * fs[l]; }
    double vx = jx / r, vz = jz / r, e = 0.0;
    for (int l = 0; l < NPOP; l++) {
        double dx = XI[l][0] - vx, dz = XI[l][1] - vz;
        e += (dx * dx + dz * dz) * fs[l];
    }
    *rho = r; *ux = vx; *uz = vz; *T = e / (DIM * r);
}

void oracle_site_moments(const double *fs, double *out4) {
    oracle_setup();
    site_moments(fs, &out4[0], &out4[1], &out4[2], &out4[3]);
}

/* ---------------------------------------------------------------------------
 * Propagate (Sec. III.B, "pull"): g_l(x,z) = f_l((x - c_lx) mod Lx, z - c_lz)
 * for every destination whose source row lies inside the lattice.  Periodic x is
 * the index wrap (the paper's pbc step).  Destinations whose source row is
 * outside [0, Lz) are left untouched here and filled by oracle_bc.
 * ------------------------------------------------------------------------- */
void oracle_propagate(int Lx, int Lz, const double *f, double *g) {
    oracle_setup();
    #pragma omp parallel for schedule(static)
    for (int x = 0; x < Lx; x++)
        for (int l = 0; l < NPOP; l++)
            for (int z = 0; z < Lz; z++) {
                int zs = z - VEL[l][1];
                if (zs < 0 || zs >= Lz) continue;
                int xs = ((x - VEL[l][0]) % Lx + Lx) % Lx;
                g[ix(Lx, Lz, l, x, z)] = f[ix(Lx, Lz, l, xs, zs)];
            }
}

/* ---------------------------------------------------------------------------
 * Wall boundary condition (Sec. III.B names the rows z = 0,1,2 and Lz-3..Lz-1 but
 * not the rule).  Reading: adiabatic no-slip half-way bounce-back with walls at
 * z = -1/2 and z = Lz - 1/2, same column: a destination (l, x, k) whose pull source
 * row k - c_lz is below 0 takes f_opp(l)(x, c_lz - 1 - k); one whose source row is
 * at or above Lz takes f_opp(l)(x, 2 Lz - 1 - k + c_lz).
 * ------------------------------------------------------------------------- */
void oracle_bc(int Lx, int Lz, const double *f, double *g) {
    oracle_setup();
    #pragma omp parallel for schedule(static)
    for (int x = 0; x < Lx; x++)
        for (int l = 0; l < NPOP; l++)
            for (int z = 0; z < Lz; z++) {
                int zs = z - VEL[l][1];
                if (zs >= 0 && zs < Lz) continue;
                int zb = (zs < 0) ? (VEL[l][1] - 1 - z) : (2 * Lz - 1 - z + VEL[l][1]);
                g[ix(Lx, Lz, l, x, z)] = f[ix(Lx, Lz, OPPO[l], x, zb)];
            }
}

/* ---------------------------------------------------------------------------
 * Thermal-wall variant of the bc (Sec. III.B names only the rows).  Reading: each wall is
 * an isothermal no-slip wall at temperature T_w, realised by three ghost rows beyond it
 * (z = -1, -2, -3 below the bottom, Lz, Lz+1, Lz+2 above the top) that hold the
 * equilibrium at rest f^eq(rho_w(x), 0, T_w).  A destination whose pull source row lies
 * in a ghost row takes that ghost population.  The ghost density of each ghost column x
 * balances the mass through the wall in the step:
 *   out(x) = sum of the populations f_l(x', z) whose move z + c_lz, x' + c_lx (mod Lx)
 *            lands in a ghost row of column x;
 *   in(x)  = rho_w(x) * sum over ghost rows zg and velocities l of f^eq_l(1, 0, T_w) for
 *            which zg + c_lz lies inside the lattice;
 *   rho_w(x) = out(x) / in(x) at rho_w = 1,
 * so the total mass is conserved exactly and the wall sends the fluid a Maxwellian at
 * its own temperature.
 * ------------------------------------------------------------------------- */
static void thermal_wall(int Lx, int Lz, const double *f, double *g, double Tw, int top) {
    double feq1[NPOP];
    equilibrium_with_derivs(1.0, 0.0, 0.0, Tw, feq1, NULL, NULL);
    const int g0 = top ? Lz : -3;                       /* ghost rows g0 .. g0 + 2 */
    double in1 = 0.0;                                   /* inflow per unit ghost density */
    for (int zg = g0; zg < g0 + 3; zg++)
        for (int l = 0; l < NPOP; l++) {
            int zd = zg + VEL[l][1];
            if (zd >= 0 && zd < Lz) in1 += feq1[l];
        }
    double *out = calloc((size_t)Lx, sizeof(double));
    for (int x = 0; x < Lx; x++)
        for (int z = 0; z < Lz; z++)
            for (int l = 0; l < NPOP; l++) {
                int zd = z + VEL[l][1];
                if (zd >= g0 && zd < g0 + 3) {
                    int xd = ((x + VEL[l][0]) % Lx + Lx) % Lx;
                    out[xd] += f[ix(Lx, Lz, l, x, z)];
                }
            }
    for (int x = 0; x < Lx; x++)
        for (int l = 0; l < NPOP; l++)
            for (int z = 0; z < Lz; z++) {
                int zs = z - VEL[l][1];
                if (zs < g0 || zs >= g0 + 3) continue;
                int xs = ((x - VEL[l][0]) % Lx + Lx) % Lx;
                g[ix(Lx, Lz, l, x, z)] = out[xs] / in1 * feq1[l];
            }
    free(out);
}

void oracle_bc_thermal(int Lx, int Lz, const double *f, double *g, double T_bot, double T_top) {
    oracle_setup();
    thermal_wall(Lx, Lz, f, g, T_bot, 0);
    thermal_wall(Lx, Lz, f, g, T_top, 1);
}

/* One full step with the thermal walls: f <- collide(bc_thermal(propagate(f))). */
void oracle_step_thermal(int Lx, int Lz, double tau, double grav, int nsteps, double *f, double *work,
                         double T_bot, double T_top);

/* ---------------------------------------------------------------------------
 * Collide (Sec. III.A, Eq. (LBE) right-hand side with the shifted equilibrium):
 *   f'_l = g_l - (1/tau) [g_l - f^eq_l(rho, u + tau gvec, T + tau (1 - tau) g^2 / D)]
 * with rho, u, T the moments of the post-propagate g, gvec = (0, -grav), dt = 1.
 * ------------------------------------------------------------------------- */
void oracle_collide(int Lx, int Lz, double tau, double grav, const double *g, double *fout) {
    oracle_setup();
    #pragma omp parallel for schedule(static)
    for (int x = 0; x < Lx; x++)
        for (int z = 0; z < Lz; z++) {
            double gs[NPOP], feq[NPOP], rho, ux, uz, T;
            for (int l = 0; l < NPOP; l++) gs[l] = g[ix(Lx, Lz, l, x, z)];
            site_moments(gs, &rho, &ux, &uz, &T);
            double usx = ux + tau * 0.0, usz = uz + tau * (-grav);
            double Ts = T + tau * (1.0 - tau) * grav * grav / DIM;
            equilibrium_with_derivs(rho, usx, usz, Ts, feq, NULL, NULL);
            for (int l = 0; l < NPOP; l++)
                fout[ix(Lx, Lz, l, x, z)] = gs[l] - (gs[l] - feq[l]) / tau;
        }
}

/* One full time step f <- collide(bc(propagate(f))); work must hold 37*Lx*Lz doubles. */
void oracle_step(int Lx, int Lz, double tau, double grav, int nsteps, double *f, double *work) {
    oracle_setup();
    for (int s = 0; s < nsteps; s++) {
        oracle_propagate(Lx, Lz, f, work);
        oracle_bc(Lx, Lz, f, work);
        oracle_collide(Lx, Lz, tau, grav, work, f);
    }
}

void oracle_step_thermal(int Lx, int Lz, double tau, double grav, int nsteps, double *f, double *work,
                         double T_bot, double T_top) {
    oracle_setup();
    for (int s = 0; s < nsteps; s++) {
        oracle_propagate(Lx, Lz, f, work);
        oracle_bc_thermal(Lx, Lz, f, work, T_bot, T_top);
        oracle_collide(Lx, Lz, tau, grav, work, f);
    }
}

/* ---------------------------------------------------------------------------
 * Initial state (Sec. I, Eq. (seteq), pressure continuity, Fig. 1 caption).
 * Heights are in sites with row k at z = k + 1/2 (physical height r z).
 *   interfaces  z_lo(x) = zlo0 + sum_k A^lo_k cos(2 pi k x / Lx + phi^lo_k), k = 1..K,
 *               z_hi(x) likewise;
 *   pressure    isothermal hydrostatic in each layer, continuous at z_lo and z_hi:
 *               p = rho_ref T_d exp(-g r z / T_d) below z_lo, then exp(-g r (z - z_lo)/T_m),
 *               then exp(-g r (z - z_hi)/T_u);
 *   temperature T_u + (T_m - T_u) (1 - tanh((z - z_hi)/w))/2 + (T_d - T_m)(1 - tanh((z - z_lo)/w))/2;
 *   density     rho = p / T;   populations f = f^eq(rho, gvec/2, T) (renormalised velocity 0).
 * ------------------------------------------------------------------------- */
static double interface_height(double z0, int K, const double *amp, const double *ph, int x, int Lx) {
    double z = z0;
    for (int k = 0; k < K; k++) z += amp[k] * cos(2.0 * M_PI * (k + 1) * x / (double)Lx + ph[k]);
    return z;
}

static void layer_state(double z, double zl, double zh, double grav, double Tu, double Tm, double Td,
                        double rho_ref, double wt, double *p, double *T) {
    double r = R_LATTICE;
    double plo = rho_ref * Td * exp(-grav * r * zl / Td);
    double phi = plo * exp(-grav * r * (zh - zl) / Tm);
    if (z < zl)       *p = rho_ref * Td * exp(-grav * r * z / Td);
    else if (z < zh)  *p = plo * exp(-grav * r * (z - zl) / Tm);
    else              *p = phi * exp(-grav * r * (z - zh) / Tu);
    *T = Tu + (Tm - Tu) * 0.5 * (1.0 - tanh((z - zh) / wt)) + (Td - Tm) * 0.5 * (1.0 - tanh((z - zl) / wt));
}

/* Column x of the Lx-column initial state into column j of an ncol-column array. */
static void init_column(int Lx, int Lz, double grav, double Tu, double Tm, double Td,
                        double zlo0, double zhi0, double rho_ref, double wt, int K,
                        const double *amp_lo, const double *ph_lo,
                        const double *amp_hi, const double *ph_hi, int x, int ncol, int j, double *f) {
    double zl = interface_height(zlo0, K, amp_lo, ph_lo, x, Lx);
    double zh = interface_height(zhi0, K, amp_hi, ph_hi, x, Lx);
    for (int k = 0; k < Lz; k++) {
        double p, T, feq[NPOP];
        layer_state(k + 0.5, zl, zh, grav, Tu, Tm, Td, rho_ref, wt, &p, &T);
        equilibrium_with_derivs(p / T, 0.0, -0.5 * grav, T, feq, NULL, NULL);
        for (int l = 0; l < NPOP; l++) f[ix(ncol, Lz, l, j, k)] = feq[l];
    }
}

void oracle_init_layers(int Lx, int Lz, double grav, double Tu, double Tm, double Td,
                        double zlo0, double zhi0, double rho_ref, double wt, int K,
                        const double *amp_lo, const double *ph_lo,
                        const double *amp_hi, const double *ph_hi, double *f) {
    oracle_setup();
    for (int x = 0; x < Lx; x++)
        init_column(Lx, Lz, grav, Tu, Tm, Td, zlo0, zhi0, rho_ref, wt, K, amp_lo, ph_lo, amp_hi, ph_hi,
                    x, Lx, x, f);
}

/* The same state restricted to the listed columns cols[0..ncol-1] of the Lx-column lattice
 * (f: 37 x ncol x Lz), so that single columns of a large lattice can be checked. */
void oracle_init_columns(int Lx, int Lz, double grav, double Tu, double Tm, double Td,
                         double zlo0, double zhi0, double rho_ref, double wt, int K,
                         const double *amp_lo, const double *ph_lo,
                         const double *amp_hi, const double *ph_hi,
                         int ncol, const int *cols, double *f) {
    oracle_setup();
    for (int j = 0; j < ncol; j++)
        init_column(Lx, Lz, grav, Tu, Tm, Td, zlo0, zhi0, rho_ref, wt, K, amp_lo, ph_lo, amp_hi, ph_hi,
                    cols[j], ncol, j, f);
}

/* ---------------------------------------------------------------------------
 * Macroscopic fields of the stored populations (Sec. III.A).  renorm = 0: raw
 * rho, u, T; renorm = 1: the renormalised fields.  The stored populations are
 * post-collision, whose velocity exceeds the pre-collision one by gvec, so the
 * paper's u^H = u_pre + gvec/2 is u_stored - gvec/2; T^H = T + g^2/(4 D).
 * ------------------------------------------------------------------------- */
void oracle_moments(int Lx, int Lz, double grav, const double *f, double *rho, double *ux,
                    double *uz, double *T, int renorm) {
    oracle_setup();
    for (int x = 0; x < Lx; x++)
        for (int z = 0; z < Lz; z++) {
            double fs[NPOP], r, vx, vz, t;
            for (int l = 0; l < NPOP; l++) fs[l] = f[ix(Lx, Lz, l, x, z)];
            site_moments(fs, &r, &vx, &vz, &t);
            size_t s = (size_t)x * Lz + z;
            rho[s] = r; ux[s] = vx; uz[s] = vz; T[s] = t;
            if (renorm) { uz[s] = vz + 0.5 * grav; T[s] = t + grav * grav / (4.0 * DIM); }
        }
}

/* Horizontal mean T(z) = (1/Lx) sum_x T(x,z) of the raw temperature (Sec. IV). */
void oracle_row_mean_T(int Lx, int Lz, const double *f, double *Tbar) {
    oracle_setup();
    for (int z = 0; z < Lz; z++) {
        double s = 0.0;
        for (int x = 0; x < Lx; x++) {
            double fs[NPOP], r, vx, vz, t;
            for (int l = 0; l < NPOP; l++) fs[l] = f[ix(Lx, Lz, l, x, z)];
            site_moments(fs, &r, &vx, &vz, &t);
            s += t;
        }
        Tbar[z] = s / Lx;
    }
}

/* ---------------------------------------------------------------------------
 * Threshold mixing widths (Sec. IV: the region where the mean profile lies between
 * 5% and 95% of the jump; the paper's "(1+a)T_u, a = 0.05 (T_d - T_u)" is read as
 * T_u + 0.05 dT).  Upper front: b = (Tbar - T_u)/(T_m - T_u), rows scanned from the
 * top down; z_a = first crossing of 0.05, z_b = next crossing of 0.95, L_u = z_a - z_b.
 * Lower front: b = (Tbar - T_m)/(T_d - T_m), rows scanned from the bottom up;
 * z_c = first crossing of 0.95, z_d = next crossing of 0.05, L_d = z_d - z_c.
 * A crossing between consecutive scanned rows p (before) and q (after) with
 * b_p < thr <= b_q (rising) or b_p > thr >= b_q (falling) sits at
 * z = z_p + (z_q - z_p) (thr - b_p)/(b_q - b_p).  If the first scanned row already
 * satisfies the condition, the crossing is that row.  Returns 0, or -1 when a crossing
 * is missing.  dL (optional, length Lz) receives d(L_u + L_d)/d Tbar(z).
 * ------------------------------------------------------------------------- */
static int find_crossing(const double *b, int Lz, int start, int dir, double thr, int rising,
                         double *zc, int *next, double dzdb[2], int rows[2]) {
    int p = start;
    int hit0 = rising ? (b[p] >= thr) : (b[p] <= thr);
    if (hit0) { *zc = p; *next = p; dzdb[0] = dzdb[1] = 0.0; rows[0] = rows[1] = p; return 0; }
    for (int q = start + dir; q >= 0 && q < Lz; q += dir) {
        int hit = rising ? (b[q] >= thr) : (b[q] <= thr);
        if (hit) {
            double db = b[q] - b[p], t = (thr - b[p]) / db;
            *zc = p + (q - p) * t;
            /* dz/db_p and dz/db_q */
            dzdb[0] = (q - p) * (-(1.0) / db + (thr - b[p]) / (db * db));
            dzdb[1] = (q - p) * (-(thr - b[p]) / (db * db));
            rows[0] = p; rows[1] = q;
            *next = q;
            return 0;
        }
        p = q;
    }
    return -1;
}

int oracle_widths(int Lz, const double *Tbar, double Tu, double Tm, double Td, double *out2, double *dL) {
    double *bu = (double *)malloc(sizeof(double) * Lz), *bd = (double *)malloc(sizeof(double) * Lz);
    if (!bu || !bd) { free(bu); free(bd); return -2; }
    for (int z = 0; z < Lz; z++) { bu[z] = (Tbar[z] - Tu) / (Tm - Tu); bd[z] = (Tbar[z] - Tm) / (Td - Tm); }
    double za, zb, zc, zd, g1[2], g2[2], g3[2], g4[2];
    int r1[2], r2[2], r3[2], r4[2], nx, rc = 0;
    rc |= find_crossing(bu, Lz, Lz - 1, -1, 0.05, 1, &za, &nx, g1, r1);
    if (!rc) rc |= find_crossing(bu, Lz, nx, -1, 0.95, 1, &zb, &nx, g2, r2);
    if (!rc) rc |= find_crossing(bd, Lz, 0, +1, 0.95, 0, &zc, &nx, g3, r3);
    if (!rc) rc |= find_crossing(bd, Lz, nx, +1, 0.05, 0, &zd, &nx, g4, r4);
    if (rc) { free(bu); free(bd); return -1; }
    out2[0] = za - zb;
    out2[1] = zd - zc;
    if (dL) {
        for (int z = 0; z < Lz; z++) dL[z] = 0.0;
        double su = 1.0 / (Tm - Tu), sd = 1.0 / (Td - Tm);
        for (int k = 0; k < 2; k++) {
            dL[r1[k]] += g1[k] * su;  dL[r2[k]] -= g2[k] * su;
            dL[r4[k]] += g4[k] * sd;  dL[r3[k]] -= g3[k] * sd;
        }
    }
    free(bu); free(bd);
    return 0;
}

/* Tent-map mixing lengths, Sec. IV Eq. (3L): L = sum_z Theta[b(z)] (one row = one site),
 * Theta[b] = 2b on (0,1/2), 2(1-b) on (1/2,1), 0 elsewhere.  out2 = {L_u, L_d}. */
static double tent(double b) {
    if (b > 0.0 && b < 0.5) return 2.0 * b;
    if (b >= 0.5 && b < 1.0) return 2.0 * (1.0 - b);
    return 0.0;
}
void oracle_tent_widths(int Lz, const double *Tbar, double Tu, double Tm, double Td, double *out2) {
    double lu = 0.0, ldd = 0.0;
    for (int z = 0; z < Lz; z++) {
        lu += tent((Tbar[z] - Tu) / (Tm - Tu));
        ldd += tent((Tbar[z] - Tm) / (Td - Tm));
    }
    out2[0] = lu; out2[1] = ldd;
}

/* ---------------------------------------------------------------------------
 * Adjoint of one step f_{t+1} = C(P f_t) (P = propagate + bc, C = collide):
 *   lam_t = P^T J_C(P f_t)^T lam_{t+1}.
 * J_C is formed explicitly per site by the chain rule through (rho, u, T):
 *   J_lm = (1 - 1/tau) delta_lm + (1/tau) [ df^eq_l/drho
 *          + sum_i df^eq_l/du_i (xi_mi - u_i)/rho + df^eq_l/dT (|xi_m - u|^2 - D T)/(D rho) ],
 * the derivatives taken at the shifted (u_s, T_s) (the shift is a constant offset).
 * P^T is applied through the explicit permutation obtained by running oracle_propagate
 * and oracle_bc on an array of source indices.
 * ------------------------------------------------------------------------- */
/* mu = J_C(g)^T lam_next at every site: the transpose of the collide's Jacobian, by the chain
 * rule through rho, u, T of the shifted equilibrium (Sec. III.A). */
static void collide_adjoint_sites(int Lx, int Lz, double tau, double grav, const double *g,
                                  const double *lam_next, double *mu) {
    double om = 1.0 / tau;
    for (int x = 0; x < Lx; x++)
        for (int z = 0; z < Lz; z++) {
            double gs[NPOP], feq[NPOP], dfdu[NPOP][2], dfdT[NPOP], lam[NPOP], rho, ux, uz, T;
            for (int l = 0; l < NPOP; l++) { gs[l] = g[ix(Lx, Lz, l, x, z)]; lam[l] = lam_next[ix(Lx, Lz, l, x, z)]; }
            site_moments(gs, &rho, &ux, &uz, &T);
            double Ts = T + tau * (1.0 - tau) * grav * grav / DIM;
            equilibrium_with_derivs(rho, ux, uz - tau * grav, Ts, feq, dfdu, dfdT);
            for (int m = 0; m < NPOP; m++) {
                double dx = XI[m][0] - ux, dz = XI[m][1] - uz;
                double drho = 1.0, dux = dx / rho, duz = dz / rho;
                double dT = (dx * dx + dz * dz - DIM * T) / (DIM * rho);
                double acc = 0.0;
                for (int l = 0; l < NPOP; l++) {
                    double J = ((l == m) ? (1.0 - om) : 0.0)
                             + om * (feq[l] / rho * drho + dfdu[l][0] * dux + dfdu[l][1] * duz + dfdT[l] * dT);
                    acc += J * lam[l];
                }
                mu[ix(Lx, Lz, m, x, z)] = acc;
            }
        }
}

void oracle_adjoint_step(int Lx, int Lz, double tau, double grav, const double *f_t,
                         const double *lam_next, double *lam_out) {
    oracle_setup();
    size_t n = (size_t)NPOP * Lx * Lz;
    double *g = (double *)malloc(n * sizeof(double));
    double *mu = (double *)malloc(n * sizeof(double));
    double *src = (double *)malloc(n * sizeof(double));
    double *idxf = (double *)malloc(n * sizeof(double));
    oracle_propagate(Lx, Lz, f_t, g);
    oracle_bc(Lx, Lz, f_t, g);
    collide_adjoint_sites(Lx, Lz, tau, grav, g, lam_next, mu);
    /* P^T of the permutation propagate + bc: each destination's mu goes back to its source */
    for (size_t i = 0; i < n; i++) idxf[i] = (double)i;
    oracle_propagate(Lx, Lz, idxf, src);
    oracle_bc(Lx, Lz, idxf, src);
    for (size_t i = 0; i < n; i++) lam_out[(size_t)src[i]] = mu[i];
    free(g); free(mu); free(src); free(idxf);
}

/* The adjoint step with the thermal walls of oracle_bc_thermal.  Propagate + thermal bc is
 * linear but no longer a permutation: a destination pulled from a lattice entry passes its mu
 * back to that entry; a destination pulled from a ghost row passes mu * f^eq_l(1,0,T_w) / in_w
 * to the ghost column's density, which was out(x) / in_w, and so to every entry that the step
 * moves into that ghost column (coefficient 1 in out(x)).  No destination pulls those
 * entries, so they receive only the ghost column's sum. */
static void thermal_wall_transpose(int Lx, int Lz, const double *mu, double *lam_out, double Tw, int top) {
    double feq1[NPOP];
    equilibrium_with_derivs(1.0, 0.0, 0.0, Tw, feq1, NULL, NULL);
    const int g0 = top ? Lz : -3;
    double in1 = 0.0;
    for (int zg = g0; zg < g0 + 3; zg++)
        for (int l = 0; l < NPOP; l++) {
            int zd = zg + VEL[l][1];
            if (zd >= 0 && zd < Lz) in1 += feq1[l];
        }
    double *omega = calloc((size_t)Lx, sizeof(double));
    for (int x = 0; x < Lx; x++)
        for (int l = 0; l < NPOP; l++)
            for (int z = 0; z < Lz; z++) {
                int zs = z - VEL[l][1];
                if (zs < g0 || zs >= g0 + 3) continue;
                int xs = ((x - VEL[l][0]) % Lx + Lx) % Lx;
                omega[xs] += mu[ix(Lx, Lz, l, x, z)] * feq1[l] / in1;
            }
    for (int x = 0; x < Lx; x++)
        for (int z = 0; z < Lz; z++)
            for (int l = 0; l < NPOP; l++) {
                int zd = z + VEL[l][1];
                if (zd >= g0 && zd < g0 + 3) {
                    int xd = ((x + VEL[l][0]) % Lx + Lx) % Lx;
                    lam_out[ix(Lx, Lz, l, x, z)] += omega[xd];
                }
            }
    free(omega);
}

void oracle_adjoint_step_thermal(int Lx, int Lz, double tau, double grav, const double *f_t,
                                 const double *lam_next, double *lam_out, double T_bot, double T_top) {
    oracle_setup();
    size_t n = (size_t)NPOP * Lx * Lz;
    double *g = (double *)malloc(n * sizeof(double));
    double *mu = (double *)malloc(n * sizeof(double));
    oracle_propagate(Lx, Lz, f_t, g);
    oracle_bc_thermal(Lx, Lz, f_t, g, T_bot, T_top);
    collide_adjoint_sites(Lx, Lz, tau, grav, g, lam_next, mu);
    memset(lam_out, 0, n * sizeof(double));
    /* lattice-to-lattice pulls */
    for (int x = 0; x < Lx; x++)
        for (int l = 0; l < NPOP; l++)
            for (int z = 0; z < Lz; z++) {
                int zs = z - VEL[l][1];
                if (zs < 0 || zs >= Lz) continue;
                int xs = ((x - VEL[l][0]) % Lx + Lx) % Lx;
                lam_out[ix(Lx, Lz, l, xs, zs)] += mu[ix(Lx, Lz, l, x, z)];
            }
    thermal_wall_transpose(Lx, Lz, mu, lam_out, T_bot, 0);
    thermal_wall_transpose(Lx, Lz, mu, lam_out, T_top, 1);
    free(g); free(mu);
}

/* Adjoint of the loss readout: lam_N(l,x,z) = dL/dTbar(z) / Lx * dT(x,z)/df_l with
 * dT/df_l = (|xi_l - u|^2 - D T)/(D rho) (raw moments of the stored f_N). */
void oracle_loss_adjoint(int Lx, int Lz, const double *f, const double *dL_dTbar, double *lam) {
    oracle_setup();
    for (int x = 0; x < Lx; x++)
        for (int z = 0; z < Lz; z++) {
            double fs[NPOP], r, vx, vz, t;
            for (int l = 0; l < NPOP; l++) fs[l] = f[ix(Lx, Lz, l, x, z)];
            site_moments(fs, &r, &vx, &vz, &t);
            for (int l = 0; l < NPOP; l++) {
                double dx = XI[l][0] - vx, dz = XI[l][1] - vz;
                lam[ix(Lx, Lz, l, x, z)] = dL_dTbar[z] / Lx * (dx * dx + dz * dz - DIM * t) / (DIM * r);
            }
        }
}

/* Adjoint of the initial state with respect to the mode amplitudes:
 *   dL/dA^lo_k = sum_x cos(2 pi k x/Lx + phi^lo_k) sum_{z,l} lam0 df0/dz_lo(x),  same for hi.
 * df0/dz_lo = df^eq/drho drho/dz_lo + df^eq/dT dT/dz_lo, rho = p/T; p depends on z_lo
 * above z_lo through p(z_lo), continuity making the layer boundaries themselves contribute
 * nothing. */
/* dL/dz_lo(x) and dL/dz_hi(x) for every column: the adjoint of the initial state (a function
 * of the interface heights of the column) applied to lam0 = dL/df_0. */
static void init_adjoint_columns(int Lx, int Lz, double grav, double Tu, double Tm, double Td,
                                 double zlo0, double zhi0, double rho_ref, double wt, int K,
                                 const double *amp_lo, const double *ph_lo,
                                 const double *amp_hi, const double *ph_hi,
                                 const double *lam0, double *gcol_lo, double *gcol_hi) {
    double r = R_LATTICE;
    for (int x = 0; x < Lx; x++) {
        double zl = interface_height(zlo0, K, amp_lo, ph_lo, x, Lx);
        double zh = interface_height(zhi0, K, amp_hi, ph_hi, x, Lx);
        double gl = 0.0, gh = 0.0;
        for (int kr = 0; kr < Lz; kr++) {
            double z = kr + 0.5, p, T, feq[NPOP], dfdT[NPOP];
            layer_state(z, zl, zh, grav, Tu, Tm, Td, rho_ref, wt, &p, &T);
            double rho = p / T;
            equilibrium_with_derivs(rho, 0.0, -0.5 * grav, T, feq, NULL, dfdT);
            double dp_dzl = 0.0, dp_dzh = 0.0;
            if (z >= zl) dp_dzl = p * (-grav * r / Td + grav * r / Tm);
            if (z >= zh) dp_dzh = p * (-grav * r / Tm + grav * r / Tu);
            double sl = 1.0 / cosh((z - zl) / wt), sh = 1.0 / cosh((z - zh) / wt);
            double dT_dzl = (Td - Tm) * 0.5 * sl * sl / wt;
            double dT_dzh = (Tm - Tu) * 0.5 * sh * sh / wt;
            double drho_dzl = dp_dzl / T - p * dT_dzl / (T * T);
            double drho_dzh = dp_dzh / T - p * dT_dzh / (T * T);
            for (int l = 0; l < NPOP; l++) {
                double lamv = lam0[ix(Lx, Lz, l, x, kr)];
                gl += lamv * (feq[l] / rho * drho_dzl + dfdT[l] * dT_dzl);
                gh += lamv * (feq[l] / rho * drho_dzh + dfdT[l] * dT_dzh);
            }
        }
        gcol_lo[x] = gl;
        gcol_hi[x] = gh;
    }
}

/* dL/dA_k = sum_x dL/dz(x) cos(2 pi k x / Lx + phi_k) (the interface heights of Sec. I). */
void oracle_init_adjoint(int Lx, int Lz, double grav, double Tu, double Tm, double Td,
                         double zlo0, double zhi0, double rho_ref, double wt, int K,
                         const double *amp_lo, const double *ph_lo,
                         const double *amp_hi, const double *ph_hi,
                         const double *lam0, double *dA_lo, double *dA_hi) {
    oracle_setup();
    double *gl = malloc((size_t)Lx * sizeof(double)), *gh = malloc((size_t)Lx * sizeof(double));
    init_adjoint_columns(Lx, Lz, grav, Tu, Tm, Td, zlo0, zhi0, rho_ref, wt, K, amp_lo, ph_lo, amp_hi, ph_hi,
                         lam0, gl, gh);
    for (int k = 0; k < K; k++) { dA_lo[k] = 0.0; dA_hi[k] = 0.0; }
    for (int x = 0; x < Lx; x++)
        for (int k = 0; k < K; k++) {
            dA_lo[k] += gl[x] * cos(2.0 * M_PI * (k + 1) * x / (double)Lx + ph_lo[k]);
            dA_hi[k] += gh[x] * cos(2.0 * M_PI * (k + 1) * x / (double)Lx + ph_hi[k]);
        }
    free(gl); free(gh);
}

/* dL/dphi_k = -A_k sum_x dL/dz(x) sin(2 pi k x / Lx + phi_k). */
void oracle_init_adjoint_phases(int Lx, int Lz, double grav, double Tu, double Tm, double Td,
                                double zlo0, double zhi0, double rho_ref, double wt, int K,
                                const double *amp_lo, const double *ph_lo,
                                const double *amp_hi, const double *ph_hi,
                                const double *lam0, double *dph_lo, double *dph_hi) {
    oracle_setup();
    double *gl = malloc((size_t)Lx * sizeof(double)), *gh = malloc((size_t)Lx * sizeof(double));
    init_adjoint_columns(Lx, Lz, grav, Tu, Tm, Td, zlo0, zhi0, rho_ref, wt, K, amp_lo, ph_lo, amp_hi, ph_hi,
                         lam0, gl, gh);
    for (int k = 0; k < K; k++) { dph_lo[k] = 0.0; dph_hi[k] = 0.0; }
    for (int x = 0; x < Lx; x++)
        for (int k = 0; k < K; k++) {
            dph_lo[k] -= amp_lo[k] * gl[x] * sin(2.0 * M_PI * (k + 1) * x / (double)Lx + ph_lo[k]);
            dph_hi[k] -= amp_hi[k] * gh[x] * sin(2.0 * M_PI * (k + 1) * x / (double)Lx + ph_hi[k]);
        }
    free(gl); free(gh);
}
