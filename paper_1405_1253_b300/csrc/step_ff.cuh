// step_ff.cuh -- fused propagate + bc + collide with IEEE binary64 storage and the
// collide in float-float arithmetic on the FP32 pipes.
//
// B300 issues FP64 at about 1/64 of the FP32 rate, far below what a 37-population
// collide needs to keep up with HBM.  This kernel keeps the FP64 layout and bytes of
// k_step_f64 but evaluates the same closed-form collide (step_f64.cuh) with pairs of
// FP32 numbers (ff.cuh), which carry a 48-bit significand.
#pragma once
#include "common.cuh"
#include "ff.cuh"

namespace lbm {

struct StepParamsFF {
    int Lx, Lz, plane;
    ff omega, one_m_omega, us_z, T_shift;
    ff c24, c6;              // 1/24 and 1/6 as float-float
};

__device__ __forceinline__ void collide_ff(const ff (&g)[Q], ff (&fo)[Q], const StepParamsFF& p) {
    const ff r = ff_make(d_lat.r_hi, d_lat.r_lo);
    const ff r2 = ff_make(d_lat.r2_hi, d_lat.r2_lo);
    ff pp[NPAIR], mm[NPAIR];
    static_for<NPAIR>([&](auto k) {
        constexpr int A = pair_first(decltype(k)::value), B = opp(A);
        pp[k.value] = ff_add(g[A], g[B]);
        mm[k.value] = ff_sub(g[A], g[B]);
    });
    ff rho = g[0], Jx = ff_make(0.f, 0.f), Jz = ff_make(0.f, 0.f);
    ff S[NSHELL];
#pragma unroll
    for (int s = 0; s < NSHELL; s++) S[s] = ff_make(0.f, 0.f);
    static_for<NPAIR>([&](auto k) {
        constexpr int A = pair_first(decltype(k)::value);
        rho = ff_add(rho, pp[k.value]);
        if constexpr (cx(A) != 0) Jx = ff_add(Jx, ff_mul_f(mm[k.value], (float)cx(A)));
        if constexpr (cz(A) != 0) Jz = ff_add(Jz, ff_mul_f(mm[k.value], (float)cz(A)));
        S[shell_of(A)] = ff_add(S[shell_of(A)], pp[k.value]);
    });
    ff E = ff_make(0.f, 0.f);
    static_for<NSHELL>([&](auto s) {
        if constexpr (decltype(s)::value > 0)
            E = ff_add(E, ff_mul_f(S[s.value], (float)shell_c2(decltype(s)::value)));
    });
    const ff inv = ff_rcp(rho);
    const ff rinv = ff_mul(r, inv);
    const ff ux = ff_mul(Jx, rinv), uz = ff_mul(Jz, rinv);
    const ff uu = ff_add(ff_mul(ux, ux), ff_mul(uz, uz));
    const ff T = ff_mul_f(ff_sub(ff_mul(ff_mul(r2, E), inv), uu), 0.5f);
    const ff usz = ff_add(uz, p.us_z);
    const ff th = ff_add(ff_add_f(T, -1.0f), p.T_shift);
    const ff u2 = ff_add(ff_mul(ux, ux), ff_mul(usz, usz));
    const ff u4 = ff_mul(u2, u2), thu2 = ff_mul(th, u2), th2 = ff_mul(th, th);
    // k00 = 1 - u2/2 - th + u4/8 + th u2 + th^2
    ff k00 = ff_add_f(ff_mul_f(u2, -0.5f), 1.0f);
    k00 = ff_add(k00, ff_neg(th));
    k00 = ff_add(k00, ff_mul_f(u4, 0.125f));
    k00 = ff_add(k00, thu2);
    k00 = ff_add(k00, th2);
    // k01 = r2 (th/2 - th u2/4 - th^2), k02 = r2^2 th^2 / 8
    const ff k01 = ff_mul(r2, ff_add(ff_add(ff_mul_f(th, 0.5f), ff_mul_f(thu2, -0.25f)), ff_neg(th2)));
    const ff k02 = ff_mul(ff_mul(r2, r2), ff_mul_f(th2, 0.125f));
    const ff k10 = ff_add(ff_add_f(ff_mul_f(u2, -0.5f), 1.0f), ff_mul_f(th, -2.0f));
    const ff k11 = ff_mul(r2, ff_mul_f(th, 0.5f));
    const ff k20 = ff_add(ff_add_f(ff_mul_f(u2, -0.25f), 0.5f), ff_mul_f(th, -1.5f));
    const ff k21 = ff_mul(r2, ff_mul_f(th, 0.25f));
    const ff a = ff_mul(r, ux), b = ff_mul(r, usz);
    const ff orho = ff_mul(p.omega, rho);
    fo[0] = ff_add(ff_mul(p.one_m_omega, g[0]), ff_mul(ff_mul(orho, ff_make(d_lat.wf_hi[0], d_lat.wf_lo[0])), k00));
    const ff c24 = p.c24, c6 = p.c6;
    static_for<NPAIR>([&](auto k) {
        constexpr int A = pair_first(decltype(k)::value), B = opp(A);
        constexpr int SH = shell_of(A);
        constexpr float C2 = (float)c2(A);
        const ff K0 = ff_add(ff_mul_f(ff_add(ff_mul_f(k02, C2), k01), C2), k00);
        const ff K1 = ff_add(ff_mul_f(k11, C2), k10);
        const ff K2 = ff_add(ff_mul_f(k21, C2), k20);
        ff s;
        if constexpr (cx(A) == 0) s = ff_mul_f(b, (float)cz(A));
        else if constexpr (cz(A) == 0) s = ff_mul_f(a, (float)cx(A));
        else s = ff_add(ff_mul_f(a, (float)cx(A)), ff_mul_f(b, (float)cz(A)));
        const ff s2 = ff_mul(s, s);
        const ff Ev = ff_add(ff_mul(s2, ff_add(ff_mul(s2, c24), K2)), K0);
        const ff Od = ff_mul(s, ff_add(ff_mul(s2, c6), K1));
        const ff W = ff_mul(orho, ff_make(d_lat.wf_hi[SH], d_lat.wf_lo[SH]));
        const ff Pa = ff_mul(W, Ev), Pb = ff_mul(W, Od);
        fo[A] = ff_add(ff_mul(p.one_m_omega, g[A]), ff_add(Pa, Pb));
        fo[B] = ff_add(ff_mul(p.one_m_omega, g[B]), ff_sub(Pa, Pb));
    });
}

__global__ void __launch_bounds__(BLOCK_Z)
k_step_ff(const double* __restrict__ fin, double* __restrict__ fout, StepParamsFF p) {
    const int z = blockIdx.x * BLOCK_Z + threadIdx.x;
    const int x = blockIdx.y;
    if (z >= p.Lz) return;
    int col[7];
#pragma unroll
    for (int k = 0; k < 7; k++) col[k] = wrap_x(x + k - 3, p.Lx) * p.Lz;
    ff g[Q], fo[Q];
    const int z0 = blockIdx.x * BLOCK_Z;
    const bool interior = (z0 >= 3) && (z0 + BLOCK_Z + 3 <= p.Lz);
    if (interior) {
        static_for<Q>([&](auto l) { g[l.value] = ff_from_double(__ldg(fin + pull_index_interior<decltype(l)::value>(z, col, p.plane))); });
    } else {
        static_for<Q>([&](auto l) { g[l.value] = ff_from_double(__ldg(fin + pull_index<decltype(l)::value>(x, z, col, p.Lz, p.plane))); });
    }
    collide_ff(g, fo, p);
    const int o = x * p.Lz + z;
#pragma unroll
    for (int l = 0; l < Q; l++) fout[l * p.plane + o] = ff_to_double(fo[l]);
}

inline ff ff_host(double v) {
    ff r;
    r.hi = (float)v;
    r.lo = (float)(v - (double)r.hi);
    return r;
}

inline void launch_step_ff(const double* fin, double* fout, const StepParams& p, cudaStream_t st) {
    StepParamsFF q;
    q.Lx = p.Lx; q.Lz = p.Lz; q.plane = p.plane;
    q.omega = ff_host(p.omega);
    q.one_m_omega = ff_host(p.one_m_omega);
    q.us_z = ff_host(p.us_z);
    q.T_shift = ff_host(p.T_shift);
    q.c24 = ff_host(1.0 / 24.0);
    q.c6 = ff_host(1.0 / 6.0);
    dim3 grid((p.Lz + BLOCK_Z - 1) / BLOCK_Z, p.Lx);
    k_step_ff<<<grid, BLOCK_Z, 0, st>>>(fin, fout, q);
}

}  // namespace lbm
