// step_ff.cuh -- fused propagate + bc + collide with IEEE binary64 storage and an
// FP64-accurate collide that stays off B300's slow FP64 pipe for all per-population work.
//
// B300 issues FP64 at about 1/64 of the FP32 rate (and every FP64 conversion at the same
// rate), far below what 37 populations per site need at HBM speed.  Per site:
//   1. the 37 pulled binary64 values are taken apart with integer instructions into
//      a 64-bit fixed-point copy (unit 2^-60) and a float-float copy (ff.cuh);
//   2. rho, J = sum c f and E = sum |c|^2 f are summed EXACTLY in 64-bit integers;
//   3. the few per-site scalars (1/rho, u, T, the force shift) are formed in native FP64
//      (about 30 FP64 instructions per site) and split into float-float;
//   4. the Hermite polynomial P(s) = K0 + K1 s + K2 s^2 + s^3/6 + s^4/24 (step_f64.cuh) and
//      the relaxation f' = (1 - w) g + w w_l rho P are evaluated in float-float, opposite
//      velocities sharing the even part;
//   5. each result is assembled back into a binary64 pattern with integer instructions.
#pragma once
#include "common.cuh"
#include "ff.cuh"

namespace lbm {

struct StepParamsFF {
    int Lx, Lz, plane;
    double omega, us_z, T_shift;   // FP64 per-site stage
    ff one_m_omega;                // float-float per-population stage
    ff c24, c6;                    // 1/24 and 1/6
};

// Split a double into float-float with integer instructions.
__device__ __forceinline__ ff dsplit(double x) {
    return bits_to_ff((uint32_t)__double2hiint(x), (uint32_t)__double2loint(x));
}

__device__ __forceinline__ void collide_ff1(const uint32_t (&H)[Q], const uint32_t (&L)[Q], double (&out)[Q],
                                            const StepParamsFF& p) {
    // -- exact moments in 64-bit fixed point ------------------------------------------
    int64_t R, Jx = 0, Jz = 0, E = 0;
    int64_t S[NSHELL] = {0, 0, 0, 0, 0, 0, 0, 0};
    R = bits_to_fix60(H[0], L[0]);
    static_for<NPAIR>([&](auto k) {
        constexpr int A = pair_first(decltype(k)::value), B = opp(A);
        const int64_t fa = bits_to_fix60(H[A], L[A]);
        const int64_t fb = bits_to_fix60(H[B], L[B]);
        const int64_t ps = fa + fb, ms = fa - fb;
        S[shell_of(A)] += ps;
        if constexpr (cx(A) != 0) Jx += (int64_t)cx(A) * ms;
        if constexpr (cz(A) != 0) Jz += (int64_t)cz(A) * ms;
    });
    static_for<NSHELL>([&](auto s) {
        constexpr int SS = decltype(s)::value;
        if constexpr (SS > 0) {
            R += S[SS];
            E += (int64_t)shell_c2(SS) * S[SS];
        }
    });
    // -- per-site scalars in FP64 (the 2^60 scale cancels in the ratios) -----------------
    const double r = d_lat.r;
    const double rho_i = (double)R;
    const double inv = 1.0 / rho_i;
    const double ux = r * ((double)Jx * inv);
    const double uz = r * ((double)Jz * inv);
    const double T = 0.5 * (d_lat.r2 * ((double)E * inv) - (ux * ux + uz * uz));
    const double usz = uz + p.us_z;
    const double thd = (T - 1.0) + p.T_shift;
    const double u2d = fma(ux, ux, usz * usz);
    const double orhod = p.omega * (rho_i * 0x1p-60);
    const ff a = dsplit(r * ux), b = dsplit(r * usz);
    const ff th = dsplit(thd), u2 = dsplit(u2d), orho = dsplit(orhod);
    // -- polynomial coefficients in float-float ---------------------------------------
    const ff r2 = ff_make(d_lat.r2_hi, d_lat.r2_lo);
    const ff thu2 = ff_mul(th, u2), th2 = ff_mul(th, th), u4 = ff_mul(u2, u2);
    // k00 = 1 - u2/2 - th + u4/8 + th u2 + th^2
    ff k00 = ff_add(ff_make(1.0f, 0.0f), ff_mul_f_u(u2, -0.5f));
    k00 = ff_add(k00, ff_add(ff_neg(th), ff_add(ff_mul_f_u(u4, 0.125f), ff_add(thu2, th2))));
    // |c|^2 coefficients (|xi|^2 = r^2 |c|^2)
    const ff k01 = ff_mul(r2, ff_add(ff_mul_f_u(th, 0.5f), ff_neg(ff_add(ff_mul_f_u(thu2, 0.25f), th2))));
    const ff k02 = ff_mul(ff_mul(r2, r2), ff_mul_f_u(th2, 0.125f));
    const ff k10 = ff_add(ff_add(ff_make(1.0f, 0.0f), ff_mul_f_u(u2, -0.5f)), ff_mul_f_u(th, -2.0f));
    const ff k11 = ff_mul(r2, ff_mul_f_u(th, 0.5f));
    const ff k20 = ff_add(ff_add(ff_make(0.5f, 0.0f), ff_mul_f_u(u2, -0.25f)), ff_mul_f_u(th, -1.5f));
    const ff k21 = ff_mul(r2, ff_mul_f_u(th, 0.25f));
    const ff a3 = ff_renorm(ff_mul_f_u(a, 3.0f)), b3 = ff_renorm(ff_mul_f_u(b, 3.0f));
    const ff om = p.one_m_omega;
    // rest population: f' = (1-w) g + w rho w_0 k00
    {
        const ff g0 = bits_to_ff(H[0], L[0]);
        const ff W0 = ff_mul(orho, ff_make(d_lat.wf_hi[0], d_lat.wf_lo[0]));
        out[0] = ff_to_double_bits(ff_add(ff_mul_u(om, g0), ff_mul_u(W0, k00)));
    }
    // per-shell coefficients (general float-float sums: no ordering assumed)
    ff K0[NSHELL], K1[NSHELL], K2[NSHELL], W[NSHELL];
    static_for<NSHELL>([&](auto sh) {
        constexpr int SS = decltype(sh)::value;
        constexpr float C2 = (float)shell_c2(SS);
        K0[SS] = ff_add(k00, ff_mul_f_u(ff_add(k01, ff_mul_f_u(k02, C2)), C2));
        K1[SS] = ff_add(k10, ff_mul_f_u(k11, C2));
        K2[SS] = ff_add(k20, ff_mul_f_u(k21, C2));
        W[SS] = ff_mul(orho, ff_make(d_lat.wf_hi[SS], d_lat.wf_lo[SS]));
    });
    static_for<NPAIR>([&](auto k) {
        constexpr int A = pair_first(decltype(k)::value), B = opp(A);
        constexpr int SH = shell_of(A);
        constexpr int CX = cx(A), CZ = cz(A);
        // s = xi_A . u_s = c_x a + c_z b
        auto mult = [&](const ff& v, const ff& v3, int c) -> ff {
            const int m = c < 0 ? -c : c;
            ff t = (m == 1) ? v : (m == 2) ? ff{2.f * v.hi, 2.f * v.lo} : v3;
            return c < 0 ? ff_neg(t) : t;
        };
        ff s;
        if constexpr (CX == 0) s = mult(b, b3, CZ);
        else if constexpr (CZ == 0) s = mult(a, a3, CX);
        else s = ff_add(mult(a, a3, CX), mult(b, b3, CZ));
        const ff q = ff_mul_u(s, s);
        // |K0| ~ 1 > |q K2|, |K2| ~ 1/2 > q/24, |K1| ~ 1 > q/6 and |Ev| > |Od| for |u| < 0.3
        const ff Ev = ff_add_big_u(K0[SH], ff_mul_u(q, ff_add_big_u(K2[SH], ff_mul_u(q, p.c24))));
        const ff Od = ff_mul_u(s, ff_add_big_u(K1[SH], ff_mul_u(q, p.c6)));
        const ff Pa = ff_mul_u(W[SH], Ev), Pb = ff_mul_u(W[SH], Od);
        const ff Xp = ff_add_big_u(Pa, Pb), Xm = ff_add_big_u(Pa, ff_neg(Pb));
        const ff ga = bits_to_ff(H[A], L[A]), gb = bits_to_ff(H[B], L[B]);
        out[A] = ff_to_double_bits(ff_add(ff_mul_u(om, ga), Xp));
        out[B] = ff_to_double_bits(ff_add(ff_mul_u(om, gb), Xm));
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
    uint32_t H[Q], L[Q];
    const int z0 = blockIdx.x * BLOCK_Z;
    const bool interior = (z0 >= 3) && (z0 + BLOCK_Z + 3 <= p.Lz);
    if (interior) {
        static_for<Q>([&](auto l) {
            const double v = __ldg(fin + pull_index_interior<decltype(l)::value>(z, col, p.plane));
            H[l.value] = (uint32_t)__double2hiint(v);
            L[l.value] = (uint32_t)__double2loint(v);
        });
    } else {
        static_for<Q>([&](auto l) {
            const double v = __ldg(fin + pull_index<decltype(l)::value>(x, z, col, p.Lz, p.plane));
            H[l.value] = (uint32_t)__double2hiint(v);
            L[l.value] = (uint32_t)__double2loint(v);
        });
    }
    double out[Q];
    collide_ff1(H, L, out, p);
    const int o = x * p.Lz + z;
#pragma unroll
    for (int l = 0; l < Q; l++) fout[l * p.plane + o] = out[l];
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
    q.omega = p.omega;
    q.us_z = p.us_z;
    q.T_shift = p.T_shift;
    q.one_m_omega = ff_host(p.one_m_omega);
    q.c24 = ff_host(1.0 / 24.0);
    q.c6 = ff_host(1.0 / 6.0);
    dim3 grid((p.Lz + BLOCK_Z - 1) / BLOCK_Z, p.Lx);
    k_step_ff<<<grid, BLOCK_Z, 0, st>>>(fin, fout, q);
}

}  // namespace lbm
