// step_f64.cuh -- fused propagate + bc + collide in native FP64 (IEEE binary64 storage).
//
// One thread per site.  The 37 pulled populations (Sec. III.B "pull": misaligned reads,
// aligned writes) are gathered straight from HBM with the periodic-x wrap and the wall
// bounce-back folded into the index; the collide (Sec. III.A Eq. (LBE) with the shifted
// equilibrium) runs in registers; the 37 results are stored coalesced into the other
// lattice copy.  The equilibrium is the 4th-order Hermite form collapsed to a polynomial
// in s = xi.u_s per velocity shell:
//   P(s) = K0 + K1 s + K2 s^2 + s^3/6 + s^4/24,
//   K0 = 1 - u^2/2 + th (c2-2)/2 + u^4/8 - th u^2 (c2-4)/4 + th^2 (c2^2 - 8 c2 + 8)/8,
//   K1 = 1 - u^2/2 + th (c2-4)/2,   K2 = 1/2 - u^2/4 + th (c2-6)/4,
// with u = u_s, th = T_s - 1, c2 = |xi|^2 = r^2 |c|^2 (D = 2); opposite velocities share
// the even part and flip the odd part.
#pragma once
#include "common.cuh"
#include "moments_fix.cuh"

namespace lbm {

// Per-site collide in FP64: g = post-propagate populations, fo = post-collide.
__device__ __forceinline__ void collide_f64(const double (&g)[Q], double (&fo)[Q], const StepParams& p) {
    const double r = d_lat.r;
    // rho, J = sum c g, E = sum |c|^2 g summed exactly in 64-bit fixed point (unit 2^-60,
    // moments_fix.cuh) with integer instructions: B300's FP64 pipe, which binds this kernel,
    // is left the per-site scalars and the equilibrium (about a quarter of its instructions
    // were these sums).  The scale 2^60 cancels in the ratios and is folded into omega rho.
    const MomentsFix m = moments_fix(SrcArray{g});
    const double R = __ll2double_rn(m.R);
    const double inv = 1.0 / R;
    const double rinv = r * inv;
    const double ux = __ll2double_rn(m.Jx) * rinv, uz = __ll2double_rn(m.Jz) * rinv;
    // T - 1 = (r^2 E / 2 - rho) / rho - |u|^2 / 2: the O(1) difference in one FMA on the sums
    const double tm1 = fma(d_lat.r2_half, __ll2double_rn(m.E), -R) * inv - 0.5 * (ux * ux + uz * uz);
    // force shift (Sec. III.A): u_s = u + tau g, T_s = T + tau (1 - tau) g^2 / D
    const double usz = uz + p.us_z;
    const double th = tm1 + p.T_shift;
    const double u2 = ux * ux + usz * usz;
    // K0, K1, K2 as polynomials in the integer |c|^2 (|xi|^2 = r^2 |c|^2)
    const double r2 = d_lat.r2;
    const double k00 = 1.0 - 0.5 * u2 - th + 0.125 * u2 * u2 + th * u2 + th * th;
    const double k01 = r2 * (0.5 * th - 0.25 * th * u2 - th * th);
    const double k02 = r2 * r2 * 0.125 * th * th;
    const double k10 = 1.0 - 0.5 * u2 - 2.0 * th, k11 = r2 * 0.5 * th;
    const double k20 = 0.5 - 0.25 * u2 - 1.5 * th, k21 = r2 * 0.25 * th;
    const double a = r * ux, b = r * usz;          // s_l = c_x a + c_z b
    const double orho = p.omega * 0x1p-60 * R;
    fo[0] = fma(p.one_m_omega, g[0], orho * d_lat.w[0] * k00);    // rest population
    // The shell factor W = w omega rho is folded into each shell's coefficients (formed once
    // per shell), so that a pair costs s, s^2, two Horner steps per part and the relaxation.
    static_for<NPAIR>([&](auto k) {
        constexpr int A = pair_first(decltype(k)::value), B = opp(A);
        constexpr int SH = shell_of(A);
        constexpr double C2 = (double)c2(A);
        const double W = orho * d_lat.w[SH];
        const double WK0 = W * fma(C2, fma(C2, k02, k01), k00);
        const double WK1 = W * fma(C2, k11, k10);
        const double WK2 = W * fma(C2, k21, k20);
        const double W24 = W * (1.0 / 24.0), W6 = W * (1.0 / 6.0);
        double s;
        if constexpr (cx(A) == 0) s = (double)cz(A) * b;
        else if constexpr (cz(A) == 0) s = (double)cx(A) * a;
        else s = fma((double)cx(A), a, (double)cz(A) * b);
        const double s2 = s * s;
        const double Pa = fma(s2, fma(s2, W24, WK2), WK0);             // W x even part
        const double Pb = s * fma(s2, W6, WK1);                         // W x odd part
        fo[A] = fma(p.one_m_omega, g[A], Pa + Pb);
        fo[B] = fma(p.one_m_omega, g[B], Pa - Pb);
    });
}

// One site: pull form (PUSH = false: gather the pulled populations, store at the site) or
// push form (PUSH = true: the site's own populations, stored where they move to).
template <bool WALL, class LD, bool PUSH>
__device__ __forceinline__ void site_f64(const double* __restrict__ fin, double* __restrict__ fout,
                                        const SiteAddr& ad, const StepParams& p) {
    double g[Q], fo[Q];
    load_site<PUSH, WALL, LD>(fin, ad, g);
    collide_f64(g, fo, p);
    store_site<PUSH, WALL>(fout, ad, fo);
}

// One BLOCK_Z-thread tile b of the lattice tiling t.
template <class LD, bool PUSH = false>
__device__ __forceinline__ void tile_f64(const double* __restrict__ fin, double* __restrict__ fout,
                                        const StepParams& p, Tiling t, int b) {
    SiteAddr ad;
    bool wall;
    if (!ad.setup(p.Lx, p.Lz, p.plane, t, b, wall)) return;
    if (wall) site_f64<true, LD, PUSH>(fin, fout, ad, p);
    else site_f64<false, LD, PUSH>(fin, fout, ad, p);
}

__global__ void __launch_bounds__(BLOCK_Z)
k_step_f64(const double* __restrict__ fin, double* __restrict__ fout, StepParams p, Tiling t) {
    tile_f64<LoadNC>(fin, fout, p, t, blockIdx.x);
}

__global__ void __launch_bounds__(BLOCK_Z)
k_step_f64_push(const double* __restrict__ fin, double* __restrict__ fout, StepParams p, Tiling t) {
    tile_f64<LoadNC, true>(fin, fout, p, t, blockIdx.x);
}

// One step over the columns of tiling t (the whole lattice when t = make_tiling(Lx, Lz, BLOCK_Z)).
inline void launch_step_f64(const double* fin, double* fout, const StepParams& p, const Tiling& t, cudaStream_t st) {
    k_step_f64<<<tiling_blocks(t), BLOCK_Z, 0, st>>>(fin, fout, p, t);
}
inline void launch_step_f64_push(const double* fin, double* fout, const StepParams& p, const Tiling& t,
                                 cudaStream_t st) {
    k_step_f64_push<<<tiling_blocks(t), BLOCK_Z, 0, st>>>(fin, fout, p, t);
}

}  // namespace lbm
