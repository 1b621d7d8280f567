// step_f32.cuh -- fused propagate + bc + collide with FP32 storage and FP32 arithmetic.
//
// Same structure as the FP64 kernel (step_f64.cuh).  To keep FP32 rounding off the
// O(1) parts, the equilibrium is evaluated as P - 1 (the deviation of the Hermite
// polynomial from its rest value) and the relaxation as
//   f' = g + w (w_l rho (1 + (P - 1)) - g),
// and the moment sums use compensated (two-sum) accumulation.
#pragma once
#include "common.cuh"

namespace lbm {

struct StepParamsF {
    int Lx, Lz, plane;
    float omega, us_z, T_shift;
};

// s + e = a + b exactly (Knuth two-sum).
__device__ __forceinline__ void two_sum_f(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

__device__ __forceinline__ void collide_f32(const float (&g)[Q], float (&fo)[Q], const StepParamsF& p) {
    const float r = d_lat.r_hi;
    // compensated moment sums
    float rho = g[0], rho_c = 0.f, Jx = 0.f, Jz = 0.f, E = 0.f, E_c = 0.f;
    static_for<NPAIR>([&](auto k) {
        constexpr int A = pair_first(decltype(k)::value), B = opp(A);
        float ps, pe;
        two_sum_f(g[A], g[B], ps, pe);
        const float m = g[A] - g[B];
        float s, e;
        two_sum_f(rho, ps, s, e);
        rho = s;
        rho_c += e + pe;
        if constexpr (cx(A) != 0) Jx = fmaf((float)cx(A), m, Jx);
        if constexpr (cz(A) != 0) Jz = fmaf((float)cz(A), m, Jz);
        two_sum_f(E, (float)c2(A) * ps, s, e);
        E = s;
        E_c += e + (float)c2(A) * pe;
    });
    rho += rho_c;
    E += E_c;
    const float inv = 1.f / rho;
    const float ux = r * Jx * inv, uz = r * Jz * inv;
    const float T = 0.5f * (d_lat.r2_hi * E * inv - (ux * ux + uz * uz));
    const float usz = uz + p.us_z;
    const float th = (T - 1.f) + p.T_shift;
    const float u2 = ux * ux + usz * usz;
    const float r2 = d_lat.r2_hi;
    // K0 - 1, K1, K2 as polynomials in the integer |c|^2
    const float d00 = -0.5f * u2 - th + 0.125f * u2 * u2 + th * u2 + th * th;
    const float k01 = r2 * (0.5f * th - 0.25f * th * u2 - th * th);
    const float k02 = r2 * r2 * 0.125f * th * th;
    const float k10 = 1.f - 0.5f * u2 - 2.f * th, k11 = r2 * 0.5f * th;
    const float k20 = 0.5f - 0.25f * u2 - 1.5f * th, k21 = r2 * 0.25f * th;
    const float a = r * ux, b = r * usz;
    const float orho = p.omega * rho;
    {
        const float W = orho * d_lat.wf[0];
        fo[0] = fmaf(W, d00, W) - p.omega * g[0];                  // update D_0 (finished below)
    }
    // Conservation repair.  The update D_l = f'_l - g_l is small, so its moments are summed
    // accurately in plain FP32; the collide must change them by exactly
    //   sum D = 0,  sum c D = rho gvec / r,  sum |c|^2 D = rho (2 u.gvec + g^2) / r^2
    // (mass kept, momentum + rho g, internal energy kept).  FP32 rounding of the weights and
    // of the equilibrium misses these by ~1e-8 per step, with the same sign across a smooth
    // region; the residual (d0, d1, d2) is put on the rest and the four |c| = 1 populations:
    //   rest: d0 - d2;  (+-1, 0): d2/4 +- d1x/2;  (0, +-1): d2/4 +- d1z/2.
    // All other populations are final as soon as their update is known.
    float S0 = fo[0], S1x = 0.f, S1z = 0.f, S2 = 0.f;
    float D1[4];   // updates of the |c| = 1 populations 1..4, finished after the repair
    static_for<NPAIR>([&](auto k) {
        constexpr int A = pair_first(decltype(k)::value), B = opp(A);
        constexpr int SH = shell_of(A);
        constexpr float C2 = (float)c2(A);
        const float D0v = fmaf(C2, fmaf(C2, k02, k01), d00);     // K0 - 1
        const float K1 = fmaf(C2, k11, k10);
        const float K2 = fmaf(C2, k21, k20);
        float sv;
        if constexpr (cx(A) == 0) sv = (float)cz(A) * b;
        else if constexpr (cz(A) == 0) sv = (float)cx(A) * a;
        else sv = fmaf((float)cx(A), a, (float)cz(A) * b);
        const float s2 = sv * sv;
        const float Ev = fmaf(s2, fmaf(s2, 1.f / 24.f, K2), D0v);  // even part - 1
        const float Od = sv * fmaf(s2, 1.f / 6.f, K1);
        const float W = orho * d_lat.wf[SH];
        const float Da = fmaf(W, Ev + Od, W) - p.omega * g[A];     // f' = g + (W (1 + Ev +- Od) - w g)
        const float Db = fmaf(W, Ev - Od, W) - p.omega * g[B];
        const float sp = Da + Db, dm = Da - Db;
        S0 += sp;
        S2 = fmaf(C2, sp, S2);
        if constexpr (cx(A) != 0) S1x = fmaf((float)cx(A), dm, S1x);
        if constexpr (cz(A) != 0) S1z = fmaf((float)cz(A), dm, S1z);
        if constexpr (SH == 1) {
            D1[A - 1] = Da;
            D1[B - 1] = Db;
        } else {
            fo[A] = g[A] + Da;
            fo[B] = g[B] + Db;
        }
    });
    static_assert(pair_first(0) == 1 && pair_first(1) == 2 && opp(1) == 3 && opp(2) == 4, "shell 1 layout");
    const float ir = 1.f / r, ir2 = ir * ir;
    const float gz = p.us_z * p.omega;                             // gvec_z = -g (us_z = -tau g)
    const float d0 = -S0;
    const float d1x = -S1x;
    const float d1z = rho * gz * ir - S1z;
    const float d2 = rho * (2.f * uz * gz + gz * gz) * ir2 - S2;
    fo[0] = g[0] + (fo[0] + (d0 - d2));
    fo[1] = g[1] + (D1[0] + fmaf(0.5f, d1x, 0.25f * d2));
    fo[3] = g[3] + (D1[2] + fmaf(-0.5f, d1x, 0.25f * d2));
    fo[2] = g[2] + (D1[1] + fmaf(0.5f, d1z, 0.25f * d2));
    fo[4] = g[4] + (D1[3] + fmaf(-0.5f, d1z, 0.25f * d2));
}

// One site, pull (PUSH = false) or push (PUSH = true) form (see site_f64).
template <bool WALL, class LD, bool PUSH>
__device__ __forceinline__ void site_f32(const float* __restrict__ fin, float* __restrict__ fout,
                                        const SiteAddr& ad, const StepParamsF& p) {
    float g[Q], fo[Q];
    load_site<PUSH, WALL, LD>(fin, ad, g);
    collide_f32(g, fo, p);
    store_site<PUSH, WALL>(fout, ad, fo);
}

template <class LD, bool PUSH = false>
__device__ __forceinline__ void tile_f32(const float* __restrict__ fin, float* __restrict__ fout,
                                        const StepParamsF& p, Tiling t, int b) {
    SiteAddr ad;
    bool wall;
    if (!ad.setup(p.Lx, p.Lz, p.plane, t, b, wall)) return;
    if (wall) site_f32<true, LD, PUSH>(fin, fout, ad, p);
    else site_f32<false, LD, PUSH>(fin, fout, ad, p);
}

// Launched as a programmatic dependent of the previous kernel in its stream (as k_step_ff):
// the next step's blocks may be scheduled once all of this step's blocks have started, and
// every thread waits for the previous grid to complete before it reads or writes populations.
__global__ void __launch_bounds__(BLOCK_Z)
k_step_f32(const float* __restrict__ fin, float* __restrict__ fout, StepParamsF p, Tiling t) {
    pdl_allow_next();
    pdl_wait();
    tile_f32<LoadNC>(fin, fout, p, t, blockIdx.x);
}

__global__ void __launch_bounds__(BLOCK_Z)
k_step_f32_push(const float* __restrict__ fin, float* __restrict__ fout, StepParamsF p, Tiling t) {
    tile_f32<LoadNC, true>(fin, fout, p, t, blockIdx.x);
}

inline StepParamsF f32_params(const StepParams& p) {
    StepParamsF q;
    q.Lx = p.Lx; q.Lz = p.Lz; q.plane = p.plane;
    q.omega = (float)p.omega;
    q.us_z = (float)p.us_z;
    q.T_shift = (float)p.T_shift;
    return q;
}

// One step over the columns of tiling t (the whole lattice when t = make_tiling(Lx, Lz, BLOCK_Z)).
inline void launch_step_f32(const float* fin, float* fout, const StepParams& p, const Tiling& t, cudaStream_t st) {
    const StepParamsF q = f32_params(p);
    launch_pdl(k_step_f32, tiling_blocks(t), BLOCK_Z, st, fin, fout, q, t);
}
inline void launch_step_f32_push(const float* fin, float* fout, const StepParams& p, const Tiling& t,
                                 cudaStream_t st) {
    const StepParamsF q = f32_params(p);
    k_step_f32_push<<<tiling_blocks(t), BLOCK_Z, 0, st>>>(fin, fout, q, t);
}

}  // namespace lbm
