// step_ff.cuh -- fused propagate + bc + collide with IEEE binary64 storage and an
// FP64-accurate collide that keeps B300's slow FP64 pipe for one FMA per population.
//
// B300 issues FP64 at about 1/64 of the FP32 rate (and every FP64 conversion at the same
// rate), far below what 37 populations per site need at HBM speed.  Per site:
//   1. the 37 pulled binary64 values are taken apart with integer instructions into a
//      64-bit fixed-point copy (unit 2^-60, ff.cuh);
//   2. rho, J = sum c f and E = sum |c|^2 f are summed in 64-bit integers;
//   3. the per-site scalars (1/rho, u, T, the force shift) are formed in float-float from
//      the four sums (four FP64 conversions and one FP64 FMA for T - 1, everything else on
//      the FP32 pipes);
//   4. 24 P(s), P(s) = K0 + K1 s + K2 s^2 + s^3/6 + s^4/24 (step_f64.cuh), is evaluated in
//      float-float with the factor 24 folded into the coefficients (so the s^3 and s^4 terms
//      need no constant), opposite velocities sharing the even part, two velocity pairs at a
//      time in the lanes of packed FP32 (f32x2) registers; w f^eq_l = (w w_l / 24)
//      rho * 24 P(s), the constant held in three FP32 terms so that no representation error
//      of it biases every step, is assembled into a binary64 pattern with integer instructions;
//   5. a second read of the populations (served by L1/L2, so DRAM sees each byte once)
//      gives f' = (1 - w) g + w f^eq with one FP64 FMA per population.
#pragma once
#include "common.cuh"
#include "ff.cuh"
#include "moments_fix.cuh"

namespace lbm {

struct StepParamsFF {
    int Lx, Lz, plane;
    double one_m_omega_d;   // the final f' = (1 - w) g + w f^eq is one FP64 FMA
    ff3 wsh[NSHELL];        // w w_shell / 24 * 2^-60 (rho arrives in units of 2^-60)
    ff us_z;                // tau (-g): velocity shift of the equilibrium
    ff T_shift;             // tau (1 - tau) g^2 / D
    int off[Q];             // pull offsets (pull_offsets) for the columns off the periodic seam
    int poff[Q];            // push offsets (push_offsets), likewise
};

// Split a double into float-float with integer instructions.
__device__ __forceinline__ ff dsplit(double x) {
    return bits_to_ff((uint32_t)__double2hiint(x), (uint32_t)__double2loint(x));
}
// 64-bit integer -> float-float (one FP64 conversion, then the integer split).
__device__ __forceinline__ ff i64_to_ff(int64_t v) { return dsplit(__ll2double_rn(v)); }

// Pull sources of one site, read from global memory (interior sites through the pull bases
// of the tile, wall sites through the bounce-back rule).  KEEP (the step, which reads every
// value twice): the first reads are kept in L2 for the second pass, and those of the shells
// |c|^2 <= 5, which the second pass reads first, in L1 too (shells 1-4: +0.7%; all shells:
// +0.4%; the others marked evict-first: -3.5%).  ONCE (the adjoint's gather, the only read):
// evict-first.
template <bool WALL, class LD, bool KEEP = false, bool ONCE = false>
struct SrcGlobal {
    const double* __restrict__ fin;
    const SiteAddr& ad;
    const int* sbase;     // interior pull bases: the tile's table (fill_pull_bases) or the offsets
    int zoff;             // added to sbase[l]: the row z, or the site x Lz + z with the offsets
    template <int L>
    __device__ __forceinline__ int idx() const {
        if constexpr (WALL) return LBM_IDX((ad.template src<L, true>()), Q * ad.plane);
        else return LBM_IDX(sbase[L] + zoff, Q * ad.plane);
    }
    template <int L>
    __device__ __forceinline__ double first() const {
        if constexpr (KEEP && shell_of(L) >= 1 && shell_of(L) <= 4) return LD::ld_keep(fin + idx<L>());
        else if constexpr (KEEP) return LD::ld_first(fin + idx<L>());
        else if constexpr (ONCE) return LD::ld_once(fin + idx<L>());
        else return LD::ld(fin + idx<L>());
    }
    // second reads (the step's last use of each value)
    template <int L>
    __device__ __forceinline__ double again() const { return LD::ld_last(fin + idx<L>()); }
    __device__ __forceinline__ void pair(const PairInfo& pi, double& va, double& vb) const {
        if constexpr (WALL) {
            va = LD::ld_last(fin + LBM_IDX((ad.template src_rt<true>(pi.A, pi.B, pi.cx, pi.cz)), Q * ad.plane));
            vb = LD::ld_last(fin + LBM_IDX((ad.template src_rt<true>(pi.B, pi.A, -pi.cx, -pi.cz)), Q * ad.plane));
        } else {
            va = LD::ld_last(fin + LBM_IDX(sbase[pi.A] + zoff, Q * ad.plane));   // one 32-bit add, one address add
            vb = LD::ld_last(fin + LBM_IDX(sbase[pi.B] + zoff, Q * ad.plane));
        }
    }
};

// The site's own populations (push form: collide first, then move); the first reads are kept
// in L2 for the second pass and the results stored streaming, as in the pull form (push step
// 0.2769 -> 0.2667 ms on 1024 x 2048).
template <class LD>
struct SrcOwn {
    const double* __restrict__ fin;
    int o, plane;
    template <int L>
    __device__ __forceinline__ double first() const { return LD::ld_first(fin + LBM_IDX(L * plane + o, Q * plane)); }
    template <int L>
    __device__ __forceinline__ double again() const { return LD::ld_last(fin + LBM_IDX(L * plane + o, Q * plane)); }
    __device__ __forceinline__ void pair(const PairInfo& pi, double& va, double& vb) const {
        va = LD::ld_last(fin + LBM_IDX(pi.A * plane + o, Q * plane));
        vb = LD::ld_last(fin + LBM_IDX(pi.B * plane + o, Q * plane));
    }
};

// Where the results go.  Pull form: every population at the site, fout[l * plane + o].
struct DstSite {
    double* __restrict__ fout;
    int o, plane;
    template <int L>
    __device__ __forceinline__ void put(double v) const { st_stream(fout + LBM_IDX(L * plane + o, Q * plane), v); }
    __device__ __forceinline__ void pair(const PairInfo& pi, double va, double vb) const {
        st_stream(fout + LBM_IDX(pi.A * plane + o, Q * plane), va);
        st_stream(fout + LBM_IDX(pi.B * plane + o, Q * plane), vb);
    }
};

// Push form: each population where it moves to (interior sites through the push bases of
// the tile, wall sites through the mirrored bounce-back rule).
template <bool WALL>
struct DstPush {
    double* __restrict__ fout;
    const SiteAddr& ad;
    const int* pbase;     // interior push bases (fill_push_bases) or the push offsets
    int zoff;             // the row z, or the site x Lz + z with the offsets
    template <int L>
    __device__ __forceinline__ void put(double v) const {
        if constexpr (WALL) st_stream(fout + LBM_IDX((ad.template push_dst<L, true>()), Q * ad.plane), v);
        else st_stream(fout + LBM_IDX(pbase[L] + zoff, Q * ad.plane), v);
    }
    __device__ __forceinline__ void pair(const PairInfo& pi, double va, double vb) const {
        if constexpr (WALL) {
            st_stream(fout + LBM_IDX((ad.template push_dst_rt<true>(pi.A, pi.B, pi.cx, pi.cz)), Q * ad.plane), va);
            st_stream(fout + LBM_IDX((ad.template push_dst_rt<true>(pi.B, pi.A, -pi.cx, -pi.cz)), Q * ad.plane), vb);
        } else {
            st_stream(fout + LBM_IDX(pbase[pi.A] + zoff, Q * ad.plane), va);
            st_stream(fout + LBM_IDX(pbase[pi.B] + zoff, Q * ad.plane), vb);
        }
    }
};


// The rest of the collide of one site from its moments m: per-site scalars, equilibrium,
// relaxation; src.again / src.pair give the populations g again, dst takes the results.
template <class SRC, class DST>
__device__ __forceinline__ void collide_ff(const MomentsFix& m, const SRC& src, const DST& dst, const StepParamsFF& p) {
    const int64_t R = m.R, Jx = m.Jx, Jz = m.Jz, E = m.E;
    // -- per-site scalars in float-float (the 2^60 scale cancels in the ratios) -----------
    const double Rd = __ll2double_rn(R);
    const ff rho = dsplit(Rd), jx = i64_to_ff(Jx), jz = i64_to_ff(Jz);
    // T - 1 = (r^2 E / 2 - rho) / rho - |u|^2 / 2 (unshifted u).  The difference of the two
    // O(1) terms is one FP64 FMA on the integer sums, so T - 1 keeps its relative accuracy
    // (the K coefficients multiply it by up to ~|xi|^2 / 2).
    const ff dT = dsplit(fma(d_lat.r2_half, __ll2double_rn(E), -Rd));
    const ff inv = ff_rcp(rho);
    const ff3 r = ff3_of(d_lat.r3);
    const ff rinv = ff_mul_c3(inv, r);
    const ff ux = ff_mul(jx, rinv), uz = ff_mul(jz, rinv);
    const ff usz = ff_add(uz, p.us_z);                       // u_s = u + tau g
    const ff ux2 = ff_mul_u(ux, ux);
    const ff u2 = ff_add(ux2, ff_mul_u(usz, usz));
    // th = T_s - 1 = T - 1 + T_shift
    const ff th = ff_add(ff_sub(ff_mul_u(dT, inv), ff_mul_pow2(ff_add_u(ux2, ff_mul_u(uz, uz)), 0.5f)), p.T_shift);
    const ff a = ff_mul_c3(ux, r), b = ff_mul_c3(usz, r);   // s_l = c_x a + c_z b
    // -- coefficients of 24 K0, 24 K1, 24 K2 as polynomials in |c|^2 ------------------------
    //    (pairs of coefficients of the same form are formed together in the two lanes of
    //    packed FP32 registers, each lane with the operations of the scalar form)
    const ff th2 = ff_mul(th, th), thu2 = ff_mul(th, u2), u4 = ff_mul_u(u2, u2);
    // 24 k00 = 24 - 12 u2 + 3 u4 + 24 (th u2 + th^2 - th)
    const ff k00 = ff_add(ff_add(ff_make(24.0f, 0.0f), ff_mul_f_u(u2, -12.0f)),
                          ff_add(ff_mul_f_u(u4, 3.0f), ff_mul_f_u(ff_add(thu2, ff_sub(th2, th)), 24.0f)));
    // 24 k01 = 6 r^2 (2 th - th u2 - 4 th^2),  24 k02 = 3 r^4 th^2 (lanes 0, 1)
    const ff k01v = ff_sub(ff_mul_pow2(th, 2.0f), ff_add(thu2, ff_mul_pow2(th2, 4.0f)));
    const ffx2 k012 = ffx2_mul_c3(ffx2{x2_pack(k01v.hi, th2.hi), x2_pack(k01v.lo, th2.lo)},
                                  ff3_of(d_lat.r2x6), ff3_of(d_lat.r4x3));
    const ff k01 = ffx2_lane0(k012), k02 = ffx2_lane1(k012);
    // 24 k10 = 24 - 12 u2 - 48 th,  24 k20 = 12 - 6 u2 - 36 th (lanes 0, 1)
    const ffx2 u2b = ffx2_both(u2), thb = ffx2_both(th);
    const ffx2 k1020 = ffx2_add(ffx2{x2_pack(24.0f, 12.0f), x2_pack(0.0f, 0.0f)},
                                ffx2_add(ffx2_mul_f_u(u2b, x2_pack(-12.0f, -6.0f)),
                                         ffx2_mul_f_u(thb, x2_pack(-48.0f, -36.0f))));
    const ff k10 = ffx2_lane0(k1020), k20 = ffx2_lane1(k1020);
    // 24 k11 = 12 r^2 th,  24 k21 = 6 r^2 th = 24 k11 / 2 (the three-term constant of 12 r^2 is
    // twice that of 6 r^2, so the halving is exact and equals the product with 6 r^2)
    const ff k11 = ff_mul_c3(th, ff3_of(d_lat.r2x12));
    const ff k21 = ff_mul_pow2(k11, 0.5f);
    // -- pass 2: relaxation; rolled loops over shells and their pairs keep the code in
    //    the instruction cache, the shell coefficients are formed once per shell -------
    {
        const double v0 = src.template again<0>();
        const ff W0 = ff_mul_c3(rho, p.wsh[0]);
        dst.template put<0>(fma(p.one_m_omega_d, v0, ff_to_double_bits(ff_renorm(ff_mul_u(W0, k00)))));
    }
    // Loop over the shells; each shell (2 or 4 pairs) is processed two pairs at a time, the
    // float-float arithmetic of the two pairs in the two lanes of packed FP32 registers
    // (ffx2: one f32x2 add, sub or mul for both; the same operations per lane as the scalar
    // forms, so the results are those of ff.cuh's scalar functions).
    const ffx2 A = ffx2_both(a), B = ffx2_both(b);
    auto pairs_out = [&](const PairInfo& p0, const PairInfo& p1, const ffx2& K0, const ffx2& K1, const ffx2& K2,
                         const ffx2& W) {
        double v0a, v0b, v1a, v1b;
        src.pair(p0, v0a, v0b);
        src.pair(p1, v1a, v1b);
        // s = xi_A . u_s = c_x a + c_z b (left unnormalised)
        const ffx2 sx = ffx2_mul_f_u(A, x2_pack(p0.fcx, p1.fcx)), sz = ffx2_mul_f_u(B, x2_pack(p0.fcz, p1.fcz));
        const ffx2 st = ffx2_two_sum(sx.hi, sz.hi);
        const ffx2 s{st.hi, x2_add(st.lo, x2_add(sx.lo, sz.lo))};
        const ffx2 q = ffx2_mul_u(s, s);
        // 24 P = [24 K0 + q (24 K2 + q)] + s [24 K1 + 4 q]; |24 K0| ~ 24 > q |24 K2 + q|,
        // |24 K2| ~ 12 > q, |24 K1| ~ 24 > 4 q and the even part exceeds the odd one for |u| < 0.3
        const ffx2 Ev = ffx2_add_big_u(K0, ffx2_mul_u(q, ffx2_add_big_u(K2, q)));
        const ffx2 Od = ffx2_mul_u(s, ffx2_add_big_u_x4(K1, q));
        const ffx2 Pa = ffx2_mul_u(W, Ev), Pb = ffx2_mul_u(W, Od);
        // w f^eq of both populations of each pair in binary64, then f' = (1 - w) g + w f^eq
        // by one FP64 FMA each
        const ffx2 Xp = ffx2_renorm(ffx2_add_big_u(Pa, Pb)), Xm = ffx2_renorm(ffx2_sub_big_u(Pa, Pb));
        dst.pair(p0, fma(p.one_m_omega_d, v0a, ff_to_double_bits(ffx2_lane0(Xp))),
                 fma(p.one_m_omega_d, v0b, ff_to_double_bits(ffx2_lane0(Xm))));
        dst.pair(p1, fma(p.one_m_omega_d, v1a, ff_to_double_bits(ffx2_lane1(Xp))),
                 fma(p.one_m_omega_d, v1b, ff_to_double_bits(ffx2_lane1(Xm))));
    };
    // Shells are taken in the groups of d_groups: the coefficients of two shells are formed
    // together, one shell per lane, and each iteration takes one pair of each.
    const ffx2 k00b = ffx2_both(k00), k01b = ffx2_both(k01), k02b = ffx2_both(k02);
    const ffx2 k10b = ffx2_both(k10), k11b = ffx2_both(k11), k20b = ffx2_both(k20), k21b = ffx2_both(k21);
    const ffx2 rhob = ffx2_both(rho);
#pragma unroll 1
    for (int g = 0; g < NGROUP; g++) {
        const ShellGroup sg = d_groups[g];
        const f32x2 C2 = x2_pack(sg.c2a, sg.c2b);
        const ffx2 K0 = ffx2_add_u(k00b, ffx2_mul_f_u(ffx2_add_u(k01b, ffx2_mul_f_u(k02b, C2)), C2));
        const ffx2 K1 = ffx2_add_u(k10b, ffx2_mul_f_u(k11b, C2));
        const ffx2 K2 = ffx2_add_u(k20b, ffx2_mul_f_u(k21b, C2));
        const ffx2 W = ffx2_mul_c3(rhob, p.wsh[sg.sa], p.wsh[sg.sb]);
#pragma unroll 1
        for (int k = 0; k < sg.n; k++)
            pairs_out(d_pairs[sg.k0 + k], d_pairs[sg.k1 + k], K0, K1, K2, W);
    }
}

// Where a step leaves each site's fixed-point moments: nowhere (the step), or four planes of
// int64 (R, Jx, Jz, E at site o; the adjoint of that step needs only these, not the state).
struct NoMoments {
    __device__ __forceinline__ void put(const MomentsFix&, int) const {}
};
struct MomentsOut {
    int64_t* __restrict__ m;
    int plane;
    __device__ __forceinline__ void put(const MomentsFix& v, int o) const {
        m[LBM_IDX(o, 4 * plane)] = v.R;
        m[LBM_IDX(plane + o, 4 * plane)] = v.Jx;
        m[LBM_IDX(2 * plane + o, 4 * plane)] = v.Jz;
        m[LBM_IDX(3 * plane + o, 4 * plane)] = v.E;
    }
};

// The collide of one site: src gives its 37 populations g, dst takes the 37 results; mo
// records the moments of the site (index o).
template <class SRC, class DST, class MOUT = NoMoments>
__device__ __forceinline__ void site_ff(const SRC& src, const DST& dst, const StepParamsFF& p,
                                        const MOUT& mo = MOUT{}, int o = 0) {
    const MomentsFix m = moments_fix(src);
    mo.put(m, o);
    collide_ff(m, src, dst, p);
}

// Lattice shape of one tile's lattice, apart from the physics in StepParamsFF (the ensemble
// runs lattices of several shapes under one parameter block; copying that block to change
// its shape would put its per-shell constants, indexed at run time, into local memory).
struct Shape {
    int Lx, Lz, plane;
};

// One tile b of the lattice tiling t, pulled from global memory; sbase: Q ints of shared
// memory.  All threads of the block must call this (an interior tile synchronises once after
// filling sbase).  The tile kind is block-uniform, so wall and interior tiles take separate
// paths, each with its own instance of the site code (measured 2% faster than choosing the
// pull rule per site inside one path).
//
// PDL: the kernel was launched as a programmatic dependent of the previous kernel in its
// stream; every thread waits for that grid to complete (griddepcontrol.wait) before its first
// access to the populations, so only the pull-base fill overlaps the previous step.
// OFFS: interior tiles off the periodic seam take their pull sources from p.off (the lattice
// of p; p must then be a __grid_constant__ kernel parameter) instead of a per-tile table, with
// no fill and no block barrier (measured 1.35% faster on 1024 x 2048); tiles on the seam, and
// every tile when OFFS is false (the ensemble, whose lattices differ in shape), fill sbase.
template <class LD, class MOUT = NoMoments, bool PDL = false, bool OFFS = false>
__device__ __forceinline__ void tile_ff(const double* __restrict__ fin, double* __restrict__ fout,
                                       const StepParamsFF& p, Shape sh, Tiling t, int b, int* sbase,
                                       const MOUT& mo = MOUT{}) {
    SiteAddr ad;
    bool wall;
    if (tile_is_wall(t, b)) {
        if constexpr (PDL) pdl_wait();
        if (!ad.setup(sh.Lx, sh.Lz, sh.plane, t, b, wall)) return;
        site_ff(SrcGlobal<true, LD, true>{fin, ad, sbase, 0}, DstSite{fout, ad.dst(), sh.plane}, p, mo, ad.dst());
        return;
    }
    const int x = tile_column(t, b);
    if (OFFS && off_seam(x, sh.Lx)) {               // block-uniform
        if constexpr (PDL) pdl_wait();
        if (!ad.setup(sh.Lx, sh.Lz, sh.plane, t, b, wall)) return;
        site_ff(SrcGlobal<false, LD, true>{fin, ad, p.off, ad.dst()}, DstSite{fout, ad.dst(), sh.plane}, p, mo,
                ad.dst());
        return;
    }
    fill_pull_bases(sbase, x, sh.Lx, sh.Lz, sh.plane);
    __syncthreads();
    if constexpr (PDL) pdl_wait();
    if (!ad.setup(sh.Lx, sh.Lz, sh.plane, t, b, wall)) return;
    site_ff(SrcGlobal<false, LD, true>{fin, ad, sbase, ad.z}, DstSite{fout, ad.dst(), sh.plane}, p, mo, ad.dst());
}
template <class LD>
__device__ __forceinline__ void tile_ff(const double* __restrict__ fin, double* __restrict__ fout,
                                       const StepParamsFF& p, Tiling t, int b, int* sbase) {
    tile_ff<LD>(fin, fout, p, Shape{p.Lx, p.Lz, p.plane}, t, b, sbase);
}

// Push form of one tile: aligned reads of the site's own populations, results written
// where they move to; pbase: Q ints of shared memory (push bases of interior tiles).
template <class LD, bool PDL = false>
__device__ __forceinline__ void tile_ff_push(const double* __restrict__ fin, double* __restrict__ fout,
                                            const StepParamsFF& p, Tiling t, int b, int* pbase) {
    SiteAddr ad;
    bool wall;
    if (tile_is_wall(t, b)) {                       // separate block-uniform paths, as tile_ff
        if constexpr (PDL) pdl_wait();
        if (!ad.setup(p.Lx, p.Lz, p.plane, t, b, wall)) return;
        site_ff(SrcOwn<LD>{fin, ad.dst(), p.plane}, DstPush<true>{fout, ad, pbase, 0}, p);
        return;
    }
    const int x = tile_column(t, b);
    if (off_seam(x, p.Lx)) {                        // push offsets from p (block-uniform), as tile_ff
        if constexpr (PDL) pdl_wait();
        if (!ad.setup(p.Lx, p.Lz, p.plane, t, b, wall)) return;
        site_ff(SrcOwn<LD>{fin, ad.dst(), p.plane}, DstPush<false>{fout, ad, p.poff, ad.dst()}, p);
        return;
    }
    fill_push_bases(pbase, x, p.Lx, p.Lz, p.plane);
    __syncthreads();
    if constexpr (PDL) pdl_wait();
    if (!ad.setup(p.Lx, p.Lz, p.plane, t, b, wall)) return;
    site_ff(SrcOwn<LD>{fin, ad.dst(), p.plane}, DstPush<false>{fout, ad, pbase, ad.z}, p);
}

// 8 resident blocks per SM (64 registers, 32 warps; a 4-byte spill): measured best with the
// packed pair loop (7 blocks at 72 registers is 1.5-3% slower).  Launched as a programmatic
// dependent of the previous kernel in the stream (launch_step_ff): each block allows the next
// step's blocks to be scheduled as soon as all of this step's blocks have started, which
// hides the next launch and its pull-base fills under this step's last wave (+0.7%).
__global__ void __launch_bounds__(BLOCK_Z, 8)
k_step_ff(const double* __restrict__ fin, double* __restrict__ fout, const __grid_constant__ StepParamsFF p,
          Tiling t) {
    __shared__ int sbase[Q];
    pdl_allow_next();
    tile_ff<LoadNC, NoMoments, true, true>(fin, fout, p, Shape{p.Lx, p.Lz, p.plane}, t, blockIdx.x, sbase);
}

// One step that also records every site's moments (for the adjoint of this step); 8 blocks
// per SM and programmatic dependent launch as k_step_ff.
__global__ void __launch_bounds__(BLOCK_Z, 8)
k_step_ff_moments(const double* __restrict__ fin, double* __restrict__ fout, const __grid_constant__ StepParamsFF p,
                  Tiling t, int64_t* __restrict__ mom) {
    __shared__ int sbase[Q];
    pdl_allow_next();
    tile_ff<LoadNC, MomentsOut, true, true>(fin, fout, p, Shape{p.Lx, p.Lz, p.plane}, t, blockIdx.x, sbase,
                                            MomentsOut{mom, p.plane});
}

inline ff ff_host(double v) {
    ff r;
    r.hi = (float)v;
    r.lo = (float)(v - (double)r.hi);
    return r;
}

inline ff3 ff3_host(long double v) {
    ff3 r;
    r.hi = (float)v;
    r.lo = (float)(v - (long double)r.hi);
    r.lo2 = (float)(v - (long double)r.hi - (long double)r.lo);
    return r;
}

// w_shell: the shell weights (binary64).
inline StepParamsFF ff_params(const StepParams& p, const double* w_shell) {
    StepParamsFF q;
    q.Lx = p.Lx; q.Lz = p.Lz; q.plane = p.plane;
    q.one_m_omega_d = p.one_m_omega;
    for (int sh = 0; sh < NSHELL; sh++) q.wsh[sh] = ff3_host((long double)p.omega * w_shell[sh] / 24.0L * 0x1p-60L);
    q.us_z = ff_host(p.us_z);
    q.T_shift = ff_host(p.T_shift);
    pull_offsets(p.Lz, p.plane, q.off);
    push_offsets(p.Lz, p.plane, q.poff);
    return q;
}

__global__ void __launch_bounds__(BLOCK_Z, 8)      // 8 blocks per SM: 2% faster than 7
k_step_ff_push(const double* __restrict__ fin, double* __restrict__ fout, const __grid_constant__ StepParamsFF p,
               Tiling t) {
    __shared__ int pbase[Q];
    pdl_allow_next();                   // launched with launch_pdl, as k_step_ff
    tile_ff_push<LoadNC, true>(fin, fout, p, t, blockIdx.x, pbase);
}

inline void launch_step_ff_push(const double* fin, double* fout, const StepParams& p, const double* w_shell,
                                const Tiling& t, cudaStream_t st) {
    const StepParamsFF q = ff_params(p, w_shell);
    launch_pdl(k_step_ff_push, tiling_blocks(t), BLOCK_Z, st, fin, fout, q, t);
}

// One step over the columns of tiling t (the whole lattice when t = make_tiling(Lx, Lz, BLOCK_Z)).
// k_step_ff waits for the previous grid before touching memory (launch_pdl).
inline void launch_step_ff(const double* fin, double* fout, const StepParams& p, const double* w_shell,
                           const Tiling& t, cudaStream_t st) {
    const StepParamsFF q = ff_params(p, w_shell);
    launch_pdl(k_step_ff, tiling_blocks(t), BLOCK_Z, st, fin, fout, q, t);
}


}  // namespace lbm
