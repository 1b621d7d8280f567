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
//   4. w f^eq_l = w w_l rho P(s), P(s) = K0 + K1 s + K2 s^2 + s^3/6 + s^4/24 (step_f64.cuh),
//      is evaluated in float-float, opposite velocities sharing the even part, and
//      assembled into a binary64 pattern with integer instructions;
//   5. a second read of the populations (served by L1/L2, so DRAM sees each byte once)
//      gives f' = (1 - w) g + w f^eq with one FP64 FMA per population.
#pragma once
#include "common.cuh"
#include "ff.cuh"

namespace lbm {

struct StepParamsFF {
    int Lx, Lz, plane;
    double omega, us_z, T_shift;   // FP64 per-site stage
    double one_m_omega_d;          // the final f' = (1 - w) g + w f^eq is one FP64 FMA
    ff c24, c6;                    // 1/24 and 1/6
};

// Split a double into float-float with integer instructions.
__device__ __forceinline__ ff dsplit(double x) {
    return bits_to_ff((uint32_t)__double2hiint(x), (uint32_t)__double2loint(x));
}

template <bool WALL>
__device__ __forceinline__ int pull_src(const SiteAddr& ad, const int* sbase, int l, int lop, int vx, int vz) {
    if constexpr (WALL) return ad.template src_rt<true>(l, lop, vx, vz);
    else return sbase[l] + ad.z;
}

template <bool WALL, class LD>
__device__ __forceinline__ void site_ff(const double* __restrict__ fin, double* __restrict__ fout,
                                       const SiteAddr& ad, const int* sbase, const StepParamsFF& p) {
    // -- pass 1: exact moments in 64-bit fixed point (all 37 loads in flight) -----------
    auto src1 = [&](auto tag) -> int {
        constexpr int L = decltype(tag)::value;
        if constexpr (WALL) return ad.template src<L, true>();
        else return sbase[L] + ad.z;
    };
    // pair sums by shell, pair differences grouped by |c_x| and |c_z| (no multiplies)
    int64_t R, Jx, Jz, E = 0;
    int64_t S[NSHELL] = {0, 0, 0, 0, 0, 0, 0, 0};
    int64_t GX[4] = {0, 0, 0, 0}, GZ[4] = {0, 0, 0, 0};
    {
        const double v0 = LD::ld(fin + src1(Tag<0>{}));
        R = bits_to_fix60((uint32_t)__double2hiint(v0), (uint32_t)__double2loint(v0));
    }
    static_for<NPAIR>([&](auto k) {
        constexpr int A = pair_first(decltype(k)::value), B = opp(A);
        const double va = LD::ld(fin + src1(Tag<A>{}));
        const double vb = LD::ld(fin + src1(Tag<B>{}));
        const int64_t fa = bits_to_fix60((uint32_t)__double2hiint(va), (uint32_t)__double2loint(va));
        const int64_t fb = bits_to_fix60((uint32_t)__double2hiint(vb), (uint32_t)__double2loint(vb));
        S[shell_of(A)] += fa + fb;
        constexpr int AX = cx(A) < 0 ? -cx(A) : cx(A), AZ = cz(A) < 0 ? -cz(A) : cz(A);
        if constexpr (cx(A) > 0) GX[AX] += fa - fb;
        if constexpr (cx(A) < 0) GX[AX] += fb - fa;
        if constexpr (cz(A) > 0) GZ[AZ] += fa - fb;
        if constexpr (cz(A) < 0) GZ[AZ] += fb - fa;
    });
    static_for<NSHELL>([&](auto s) {
        constexpr int SS = decltype(s)::value;
        if constexpr (SS > 0) {
            R += S[SS];
            E += (int64_t)shell_c2(SS) * S[SS];
        }
    });
    Jx = GX[1] + 2 * GX[2] + 3 * GX[3];
    Jz = GZ[1] + 2 * GZ[2] + 3 * GZ[3];
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
    // k00 = 1 - u2/2 - th + u4/8 + th u2 + th^2; the |c|^2 coefficients carry r^2
    ff k00 = ff_add(ff_make(1.0f, 0.0f), ff_mul_f_u(u2, -0.5f));
    k00 = ff_add(k00, ff_add(ff_neg(th), ff_add(ff_mul_f_u(u4, 0.125f), ff_add(thu2, th2))));
    const ff k01 = ff_mul(r2, ff_add(ff_mul_f_u(th, 0.5f), ff_neg(ff_add(ff_mul_f_u(thu2, 0.25f), th2))));
    const ff k02 = ff_mul(ff_mul(r2, r2), ff_mul_f_u(th2, 0.125f));
    const ff k10 = ff_add(ff_add(ff_make(1.0f, 0.0f), ff_mul_f_u(u2, -0.5f)), ff_mul_f_u(th, -2.0f));
    const ff k11 = ff_mul(r2, ff_mul_f_u(th, 0.5f));
    const ff k20 = ff_add(ff_add(ff_make(0.5f, 0.0f), ff_mul_f_u(u2, -0.25f)), ff_mul_f_u(th, -1.5f));
    const ff k21 = ff_mul(r2, ff_mul_f_u(th, 0.25f));
    const int o = ad.dst();
    // -- pass 2: relaxation; rolled loops over shells and their pairs keep the code in
    //    the instruction cache, the shell coefficients are formed once per shell -------
    {
        const double v0 = LD::ld_again(fin + src1(Tag<0>{}));
        const ff W0 = ff_mul(orho, ff_make(d_lat.wf_hi[0], d_lat.wf_lo[0]));
        fout[o] = fma(p.one_m_omega_d, v0, ff_to_double_bits(ff_renorm(ff_mul_u(W0, k00))));
    }
    // Loop over the shells; each shell (2 or 4 pairs) is processed two pairs at a time, so
    // two independent dependency chains are in flight per thread.  The shell coefficients
    // are formed once per shell; loops stay rolled to keep the code in the I-cache.
    auto pair_out = [&](const PairInfo& pi, const ff& K0, const ff& K1, const ff& K2, const ff& W,
                        double va, double vb) {
        // s = xi_A . u_s = c_x a + c_z b (left unnormalised)
        const ff sx = ff_mul_f_u(a, pi.fcx), sz = ff_mul_f_u(b, pi.fcz);
        const ff st = two_sum(sx.hi, sz.hi);
        const ff s = ff_make(st.hi, st.lo + (sx.lo + sz.lo));
        const ff q = ff_mul_u(s, s);
        // |K0| ~ 1 > |q K2|, |K2| ~ 1/2 > q/24, |K1| ~ 1 > q/6 and |Ev| > |Od| for |u| < 0.3
        const ff Ev = ff_add_big_u(K0, ff_mul_u(q, ff_add_big_u(K2, ff_mul_u(q, p.c24))));
        const ff Od = ff_mul_u(s, ff_add_big_u(K1, ff_mul_u(q, p.c6)));
        const ff Pa = ff_mul_u(W, Ev), Pb = ff_mul_u(W, Od);
        // w f^eq of the pair in binary64, then f' = (1 - w) g + w f^eq by one FP64 FMA each
        const double Xp = ff_to_double_bits(ff_renorm(ff_add_big_u(Pa, Pb)));
        const double Xm = ff_to_double_bits(ff_renorm(ff_add_big_u(Pa, ff_neg(Pb))));
        fout[pi.A * p.plane + o] = fma(p.one_m_omega_d, va, Xp);
        fout[pi.B * p.plane + o] = fma(p.one_m_omega_d, vb, Xm);
    };
#pragma unroll 1
    for (int sh = 1; sh < NSHELL; sh++) {
        const int k0 = d_shell_first[sh], k1 = k0 + d_shell_npair[sh];
        const float C2 = d_pairs[k0].fc2;
        const ff K0 = ff_add_u(k00, ff_mul_f_u(ff_add_u(k01, ff_mul_f_u(k02, C2)), C2));
        const ff K1 = ff_add_u(k10, ff_mul_f_u(k11, C2));
        const ff K2 = ff_add_u(k20, ff_mul_f_u(k21, C2));
        const ff W = ff_mul(orho, ff_make(d_lat.wf_hi[sh], d_lat.wf_lo[sh]));
#pragma unroll 1
        for (int k = k0; k < k1; k += 2) {            // every shell has an even number of pairs
            const PairInfo p0 = d_pairs[k], p1 = d_pairs[k + 1];
            const double v0a = LD::ld_again(fin + pull_src<WALL>(ad, sbase, p0.A, p0.B, p0.cx, p0.cz));
            const double v0b = LD::ld_again(fin + pull_src<WALL>(ad, sbase, p0.B, p0.A, -p0.cx, -p0.cz));
            const double v1a = LD::ld_again(fin + pull_src<WALL>(ad, sbase, p1.A, p1.B, p1.cx, p1.cz));
            const double v1b = LD::ld_again(fin + pull_src<WALL>(ad, sbase, p1.B, p1.A, -p1.cx, -p1.cz));
            pair_out(p0, K0, K1, K2, W, v0a, v0b);
            pair_out(p1, K0, K1, K2, W, v1a, v1b);
        }
    }
}

// One tile b of the lattice tiling t; sbase: Q ints of shared memory.  All threads of the
// block must call this (it synchronises once after filling sbase).
template <class LD>
__device__ __forceinline__ void tile_ff(const double* __restrict__ fin, double* __restrict__ fout,
                                       const StepParamsFF& p, Tiling t, int b, int* sbase) {
    const bool wall_tile = tile_is_wall(t, b);
    if (!wall_tile) {
        fill_pull_bases(sbase, tile_column(t, b), p.Lx, p.Lz, p.plane);
        __syncthreads();
    }
    SiteAddr ad;
    bool wall;
    if (!ad.setup(p.Lx, p.Lz, p.plane, t, b, wall)) return;
    if (wall) site_ff<true, LD>(fin, fout, ad, sbase, p);
    else site_ff<false, LD>(fin, fout, ad, sbase, p);
}

// 7 resident blocks per SM (72 registers, 28 warps): measured best; 8 spills
__global__ void __launch_bounds__(BLOCK_Z, 7)
k_step_ff(const double* __restrict__ fin, double* __restrict__ fout, StepParamsFF p, Tiling t) {
    __shared__ int sbase[Q];
    tile_ff<LoadNC>(fin, fout, p, t, blockIdx.x, sbase);
}

inline ff ff_host(double v) {
    ff r;
    r.hi = (float)v;
    r.lo = (float)(v - (double)r.hi);
    return r;
}

inline StepParamsFF ff_params(const StepParams& p) {
    StepParamsFF q;
    q.Lx = p.Lx; q.Lz = p.Lz; q.plane = p.plane;
    q.omega = p.omega;
    q.us_z = p.us_z;
    q.T_shift = p.T_shift;
    q.one_m_omega_d = p.one_m_omega;
    q.c24 = ff_host(1.0 / 24.0);
    q.c6 = ff_host(1.0 / 6.0);
    return q;
}

inline void launch_step_ff(const double* fin, double* fout, const StepParams& p, cudaStream_t st) {
    const StepParamsFF q = ff_params(p);
    const Tiling t = make_tiling(p.Lx, p.Lz, BLOCK_Z);
    k_step_ff<<<tiling_blocks(t, p.Lx), BLOCK_Z, 0, st>>>(fin, fout, q, t);
}

}  // namespace lbm
