// lattice.cuh -- the D2Q37 velocity set and its quadrature, as used by the CUDA path.
//
// Sec. III.A (and the caption of the D2Q37 velocity-set figure) fixes 37 velocities with
// speeds up to sqrt(10) lattice units and a lattice constant r ~ 1.1969.  The set is the
// 37 integer vectors with |c|^2 in {0,1,2,4,5,8,9,10}; the shell weights and r are the
// solution of the moment conditions that make the discrete moments of all monomials of
// degree <= 8 equal those of the unit two-dimensional Gaussian.  This file solves that
// system with Newton's method on all nine unknowns (8 shell weights and r) in long
// double, starting from r = 1.2 and the least-squares weights at that r.
#pragma once
#include <cmath>
#include <cstdint>

namespace lbm {

constexpr int Q = 37;
constexpr int NSHELL = 8;

struct VelTable {
    int x[Q];
    int z[Q];
};

// Canonical order: (0,0), then shells |c|^2 = 1,2,4,5,8,9,10, each by polar angle in [0, 2 pi).
__host__ __device__ constexpr VelTable vel_table() {
    return VelTable{
        {0, 1, 0, -1, 0, 1, -1, -1, 1, 2, 0, -2, 0, 2, 1, -1, -2, -2, -1, 1, 2, 2, -2, -2, 2,
         3, 0, -3, 0, 3, 1, -1, -3, -3, -1, 1, 3},
        {0, 0, 1, 0, -1, 1, 1, -1, -1, 0, 2, 0, -2, 1, 2, 2, 1, -1, -2, -2, -1, 2, 2, -2, -2,
         0, 3, 0, -3, 1, 3, 3, 1, -1, -3, -3, -1}};
}
__host__ __device__ constexpr int cx(int l) { return vel_table().x[l]; }
__host__ __device__ constexpr int cz(int l) { return vel_table().z[l]; }
__host__ __device__ constexpr int c2(int l) { return cx(l) * cx(l) + cz(l) * cz(l); }
__host__ __device__ constexpr int opp(int l) {
    int o = -1;
    for (int m = 0; m < Q; m++)
        if (cx(m) == -cx(l) && cz(m) == -cz(l)) o = m;
    return o;
}
__host__ __device__ constexpr int shell_c2(int s) {
    return s == 0 ? 0 : s == 1 ? 1 : s == 2 ? 2 : s == 3 ? 4 : s == 4 ? 5 : s == 5 ? 8 : s == 6 ? 9 : 10;
}
__host__ __device__ constexpr int shell_of(int l) {
    int s = -1;
    for (int k = 0; k < NSHELL; k++)
        if (shell_c2(k) == c2(l)) s = k;
    return s;
}
// The 18 opposite pairs (a, opp(a)): a is the first member of each pair in canonical order.
__host__ __device__ constexpr int pair_first(int k) {
    int n = 0, found = -1;
    for (int l = 1; l < Q; l++)
        if (opp(l) > l) {
            if (n == k) found = l;
            n++;
        }
    return found;
}
constexpr int NPAIR = 18;

static_assert(opp(0) == 0, "rest population is its own opposite");
static_assert(pair_first(NPAIR - 1) > 0 && pair_first(NPAIR) == -1, "18 opposite pairs");

// Lattice constants in device constant memory, filled once per device.
struct DevLattice {
    double w[NSHELL];      // shell weights
    double r, r2;          // lattice constant and its square
    double r2_half;        // r^2 / 2
    float r_hi, r2_hi;     // FP32 r and r^2 (FP32 collide)
    float wf[NSHELL];      // FP32 weights
    // constants of the float-float collide as three FP32 terms each (no representation
    // error that would bias every step): r, and 6 r^2, 12 r^2, 3 r^4 of the coefficients of 24 P(s)
    float r3[3], r2x6[3], r2x12[3], r4x3[3];
};

// ----------------------------------------------------------------------------------
// Host quadrature solve (Newton on the 9 x 9 moment system).
// Equations: sum_l w_l (r c_lx)^a (r c_lz)^b = m(a) m(b), m(a) = (a-1)!! for even a,
// for (a,b) in (0,0),(2,0),(4,0),(2,2),(6,0),(4,2),(8,0),(6,2),(4,4).
// ----------------------------------------------------------------------------------
struct Quadrature {
    double w_shell[NSHELL];
    double r;
    int ok;
};

// Host helpers of the quadrature solve (plain functions: a lambda would also be compiled for
// the device, where long double is not available).
// Moment of order a of the unit Gaussian: (a - 1)!! for even a, 0 for odd a.
inline long double quad_gauss_moment(int a) {
    if (a % 2) return 0.0L;
    long double m = 1.0L;
    for (int k = a - 1; k > 0; k -= 2) m *= k;
    return m;
}
inline long double quad_ipow(long double b, int e) {
    long double p = 1.0L;
    for (int i = 0; i < e; i++) p *= b;
    return p;
}
// The nine moment exponents (e_x, e_z) the quadrature must reproduce.
constexpr int QUAD_E[9][2] = {{0, 0}, {2, 0}, {4, 0}, {2, 2}, {6, 0}, {4, 2}, {8, 0}, {6, 2}, {4, 4}};
// A[e][s](r) = sum over shell s of xi_x^ex xi_z^ez, dA/dr and the Gaussian moments rhs[e].
inline void quad_system(long double r, long double A[9][NSHELL], long double dA[9][NSHELL], long double rhs[9]) {
    for (int e = 0; e < 9; e++) {
        rhs[e] = quad_gauss_moment(QUAD_E[e][0]) * quad_gauss_moment(QUAD_E[e][1]);
        for (int s = 0; s < NSHELL; s++) { A[e][s] = 0; dA[e][s] = 0; }
        const int deg = QUAD_E[e][0] + QUAD_E[e][1];
        for (int l = 0; l < Q; l++) {
            const long double mono = quad_ipow((long double)cx(l), QUAD_E[e][0]) * quad_ipow((long double)cz(l), QUAD_E[e][1]);
            A[e][shell_of(l)] += mono * quad_ipow(r, deg);
            if (deg > 0) dA[e][shell_of(l)] += mono * deg * quad_ipow(r, deg - 1);
        }
    }
}
// Gauss-Jordan with partial pivoting on an n x (n+1) augmented matrix; false if singular.
inline bool quad_solve(int n, long double M[9][10]) {
    for (int c = 0; c < n; c++) {
        int p = c;
        for (int i = c + 1; i < n; i++) if (fabsl(M[i][c]) > fabsl(M[p][c])) p = i;
        if (M[p][c] == 0) return false;
        for (int j = 0; j <= n; j++) { const long double t = M[c][j]; M[c][j] = M[p][j]; M[p][j] = t; }
        for (int i = 0; i < n; i++) {
            if (i == c) continue;
            const long double f = M[i][c] / M[c][c];
            for (int j = c; j <= n; j++) M[i][j] -= f * M[c][j];
        }
    }
    for (int i = 0; i < n; i++) M[i][n] /= M[i][i];
    return true;
}

inline Quadrature solve_quadrature_host() {
    typedef long double ld;
    const auto build = quad_system;
    const auto solve = quad_solve;
    Quadrature q{};
    ld r = 1.2L, w[NSHELL];
    ld A[9][NSHELL], dA[9][NSHELL], rhs[9];
    build(r, A, dA, rhs);
    {   // start: least-squares weights at r = 1.2 (normal equations, 8 x 8)
        ld N[9][10];
        for (int i = 0; i < NSHELL; i++) {
            for (int j = 0; j < NSHELL; j++) {
                ld s = 0;
                for (int e = 0; e < 9; e++) s += A[e][i] * A[e][j];
                N[i][j] = s;
            }
            ld s = 0;
            for (int e = 0; e < 9; e++) s += A[e][i] * rhs[e];
            N[i][NSHELL] = s;
        }
        if (!solve(NSHELL, N)) return q;
        for (int s = 0; s < NSHELL; s++) w[s] = N[s][NSHELL];
    }
    for (int it = 0; it < 60; it++) {
        build(r, A, dA, rhs);
        ld M[9][10], res = 0;
        for (int e = 0; e < 9; e++) {
            ld F = -rhs[e], dFdr = 0;
            for (int s = 0; s < NSHELL; s++) { F += A[e][s] * w[s]; dFdr += dA[e][s] * w[s]; M[e][s] = A[e][s]; }
            M[e][NSHELL] = dFdr;
            M[e][9] = -F;
            res += fabsl(F);
        }
        if (res < 1e-18L) break;
        if (!solve(9, M)) return q;
        for (int s = 0; s < NSHELL; s++) w[s] += M[s][9];
        r += M[NSHELL][9];
    }
    build(r, A, dA, rhs);
    ld worst = 0;
    for (int e = 0; e < 9; e++) {
        ld F = -rhs[e];
        for (int s = 0; s < NSHELL; s++) F += A[e][s] * w[s];
        if (fabsl(F) > worst) worst = fabsl(F);
    }
    q.r = (double)r;
    for (int s = 0; s < NSHELL; s++) q.w_shell[s] = (double)w[s];
    q.ok = (worst < 1e-15L) && (r > 1.1L) && (r < 1.3L);
    for (int s = 0; s < NSHELL; s++) if (!(w[s] > 0)) q.ok = 0;
    return q;
}

}  // namespace lbm
