// adjoint_ff.cuh -- the adjoint step lam_t = P^T J_C(g)^T lam_{t+1} (adjoint.cuh) with
// binary64 storage and an FP64-accurate float-float evaluation, the transpose of the
// float-float collide of step_ff.cuh.
//
// Per site, with D = 2, u the velocity and T the temperature of the pulled g = P f_t,
// u_s = u + tau g_vec, th = T_s - 1 (the shifted equilibrium of Sec. III.A), and
// P(s) = K0 + K1 s + K2 s^2 + s^3/6 + s^4/24 the equilibrium polynomial of one velocity
// (s = xi . u_s, K0..K2 polynomials in |u_s|^2, th and C2 = |xi|^2):
//   A  = sum_l w_l lam_l P_l,          B  = sum_l w_l lam_l dP/ds_l xi_l,
//   Bu = sum_l w_l lam_l dP/du2_l,     Cs = sum_l w_l lam_l dP/dth_l,
//   Bt = B + 2 Bu u_s,   A' = A - Bt . u + Cs (|u|^2 / 2 - T),   B' = Bt - Cs u,   C' = Cs / 2,
//   lam_t(source of l) = (1 - w) lam_l + w (A' + B' . xi_l + C' |xi_l|^2)
// (rho cancels between df^eq/dM and dM/dg).  The even/odd split of a velocity pair
// (ls = lam_A + lam_B, ld = lam_A - lam_B) and dP/du2 = -(K1 + s + q/2) / 2 (q = s^2;
// K1 = -2 dK0/du2) give, with the factor 24 of step_ff.cuh folded into the K:
//   24 A        = sum w [ls (24K0 + q (24K2 + q)) + ld s (24K1 + 4 q)]
//   24 B / r    = sum w c [ld (24K1 + 12 q) + 2 ls s (24K2 + 2 q)]
//   -48 Bu      = sum w [ls (24K1 + 12 q) + 24 ld s]
//   4 Cs        = sum w [ls (4 H0 + (C2 - 6) q) + 2 (C2 - 4) ld s],  H0 = dK0/dth.
// Numerics: lam_{t+1} is taken apart into float-float with integer instructions after
// scaling by the site's block exponent (the largest exponent among its 37 values), so the
// relative accuracy does not depend on the magnitude of lam; the moments of g come from the
// 64-bit fixed-point sums of step_ff.cuh; the result A' + B'.xi + C'|xi|^2 (scaled back by
// the block exponent) enters the binary64 output through FP64 adds and one FP64 FMA per
// population.  FP64 instructions per site: 37 FMAs, 36 adds, the five moment conversions.
// The float-float work of the two velocity pairs of each loop iteration runs in the two lanes
// of packed FP32 registers (ffx2, ff.cuh), with each lane's terms added to the sums in pair
// order: the results are those of the scalar form, bit for bit.
#pragma once
#include "step_ff.cuh"

namespace lbm {

struct AdjParamsFF {
    int Lx, Lz, plane;
    double one_m_omega_d;
    ff3 wsh[NSHELL];       // omega w_shell
    ff us_z, T_shift;      // tau (-g), tau (1 - tau) g^2 / D
    ff3 r2, r4;            // r^2, r^4
    ff3 r_24, inv24;       // r / 24, 1 / 24
    ff c6[NSHELL];         // r^2 |c|^2 - 6 of each shell
    ff c4[NSHELL];         // 2 (r^2 |c|^2 - 4)
    int off[Q];            // pull offsets (pull_offsets) for the columns off the periodic seam
};

// a * c, not renormalised.
__device__ __forceinline__ ff ff_mul_c3_u(ff a, const ff3& c) {
    const float p = __fmul_rn(a.hi, c.hi);
    float e = fmaf(a.hi, c.hi, -p);
    e = fmaf(a.hi, c.lo2, e);
    e = fmaf(a.hi, c.lo, e);
    e = fmaf(a.lo, c.hi, e);
    return ff{p, e};
}

// a + 2 b when |a| >= |2 b| is known, not renormalised.
__device__ __forceinline__ ff ff_add_big_u_x2(ff a, ff b) {
    const float s = fmaf(2.0f, b.hi, a.hi);
    const float e = fmaf(2.0f, b.hi, -(s - a.hi));
    return ff{s, e + fmaf(2.0f, b.lo, a.lo)};
}

// Renormalisation without an ordering assumption (the sum may have cancelled).
__device__ __forceinline__ ff ff_renorm2(ff a) { return two_sum(a.hi, a.lo); }

// Packed two-lane forms of the adjoint's float-float operations (lane-wise the operations of
// the scalar functions, so the results are the same bits; ffx2_add_u is in ff.cuh).
__device__ __forceinline__ ffx2 ffx2_sub_u(const ffx2& a, const ffx2& b) {            // ff_add_u(a, ff_neg(b))
    const f32x2 s = x2_sub(a.hi, b.hi), bb = x2_sub(s, a.hi);
    const f32x2 e = x2_sub(x2_sub(a.hi, x2_sub(s, bb)), x2_add(b.hi, bb));
    return ffx2{s, x2_add(e, x2_sub(a.lo, b.lo))};
}
__device__ __forceinline__ ffx2 ffx2_mul_c3_u(const ffx2& a, const ff3& c) {          // ff_mul_c3_u
    const f32x2 p = x2_mul(a.hi, x2_pack(c.hi, c.hi));
    const float a0 = x2_lane0(a.hi), a1 = x2_lane1(a.hi);
    float e0 = fmaf(a0, c.hi, -x2_lane0(p)), e1 = fmaf(a1, c.hi, -x2_lane1(p));
    e0 = fmaf(a0, c.lo2, e0); e1 = fmaf(a1, c.lo2, e1);
    e0 = fmaf(a0, c.lo, e0);  e1 = fmaf(a1, c.lo, e1);
    e0 = fmaf(x2_lane0(a.lo), c.hi, e0); e1 = fmaf(x2_lane1(a.lo), c.hi, e1);
    return ffx2{p, x2_pack(e0, e1)};
}
// ff_mul_c3_u with the constant c0 in lane 0 and c1 in lane 1
__device__ __forceinline__ ffx2 ffx2_mul_c3_u2(const ffx2& a, const ff3& c0, const ff3& c1) {
    const f32x2 chi = x2_pack(c0.hi, c1.hi);
    const f32x2 p = x2_mul(a.hi, chi);
    f32x2 e = x2_prod_err(a.hi, chi, p);
    e = x2_fma(a.hi, x2_pack(c0.lo2, c1.lo2), e);
    e = x2_fma(a.hi, x2_pack(c0.lo, c1.lo), e);
    e = x2_fma(a.lo, chi, e);
    return ffx2{p, e};
}
__device__ __forceinline__ ffx2 ffx2_add_big_u_x2(const ffx2& a, const ffx2& b) {     // ff_add_big_u_x2
    const f32x2 two = x2_pack(2.0f, 2.0f);
    const f32x2 s = x2_fma(two, b.hi, a.hi);
    return ffx2{s, x2_add(x2_fma(two, b.hi, x2_sub(a.hi, s)), x2_fma(two, b.lo, a.lo))};
}
__device__ __forceinline__ ffx2 ffx2_scale(const ffx2& a, float k) {                  // exact products (k = 2^n)
    const f32x2 kk = x2_pack(k, k);
    return ffx2{x2_mul(a.hi, kk), x2_mul(a.lo, kk)};
}

// binary64 bit pattern of x -> float-float of x * 2^-(S >> 20), S = (E_block - 1023) << 20 a
// signed shift of the exponent field.  The value after scaling must stay below 2^127 in
// magnitude; values that fall below 2^-74 after scaling come out as 0 (as do zero and the
// subnormals, which have no exponent, as long as E_block >= 75).
__device__ __forceinline__ ff bits_to_ff_scaled(uint32_t H, uint32_t L, int32_t S) {
    const uint32_t sgn = H & 0x80000000u;
    const int32_t Ha = (int32_t)(H & 0x7FFFFFFFu) - S;
    const bool ok = Ha >= (int32_t)(949u << 20);
    const uint32_t Hu = (uint32_t)Ha;
    const uint64_t m = ((((uint64_t)Hu) << 32) | L) + 0x10000000ull;
    const uint32_t hb = (uint32_t)(m >> 29) - 0xC0000000u;
    const int32_t rem = ((int32_t)(L << 3)) >> 3;
    const uint32_t sb = (Hu >> 20) * 0x00800000u + 0x26000000u;
    const float hi = __uint_as_float(ok ? (hb | sgn) : 0u);
    const float lo = (float)rem * __uint_as_float(ok ? (sb | sgn) : 0u);   // sb may be Inf when !ok
    return ff{hi, lo};
}

// Normalised float-float a -> binary64 of a * 2^(S >> 20) (ff_to_double_bits with the
// exponent field moved by S, S >= (75 - 1023) << 20); 0 when |a.hi| < 2^-74, the range in
// which the assembly's scale 2^(52 - e) would leave FP32 (such a result lies below 2^-74 of
// the block scale; every other result lands in the binary64 normal range).
__device__ __forceinline__ double ff_to_double_scaled(ff a, int32_t S) {
    const uint32_t hb = __float_as_uint(a.hi);
    const uint32_t ha = hb & 0x7FFFFFFFu;
    const uint32_t sgn = hb & 0x80000000u;
    const uint32_t PH = (ha >> 3) + (896u << 20) + (uint32_t)S + sgn;
    const uint32_t PL = ha << 29;
    const uint32_t m = (uint32_t)((int32_t)(__float_as_uint(a.lo) ^ hb) >> 31);
    const uint32_t sbits = 0x99000000u - ((hb + m) & 0x7F800000u) + sgn;
    const int32_t k = __float2int_rn(a.lo * __uint_as_float(sbits));
    const uint64_t P = ((((uint64_t)PH) << 32) | PL) + (uint64_t)(int64_t)k;
    return __longlong_as_double(ha >= (53u << 23) ? (long long)P : 0ll);
}

// lam_{t+1} at the site itself: the high words (block exponent) and the values.
struct LamOwn {
    const double* __restrict__ lam;
    int o, plane;
    template <int L>
    __device__ __forceinline__ uint32_t hiword() const {
        uint32_t v;
        const double* p = lam + LBM_IDX(L * plane + o, Q * plane);
        asm("ld.global.nc.L2::cache_hint.L2::256B.u32 %0, [%1], %2;" : "=r"(v) : "l"((const char*)p + 4),
            "l"(LoadNC::pol_keep()));     // lam is read twice more (the sums, the output)
        return v;
    }
    // re-reads; LAST: the output pass, the final use of each value (evict-first in L1)
    template <int L, bool LAST = false>
    __device__ __forceinline__ double again() const {
        const double* q = lam + LBM_IDX(L * plane + o, Q * plane);
        return LAST ? LoadNC::ld_last(q) : LoadNC::ld_again_keep(q);
    }
    template <bool LAST = false>
    __device__ __forceinline__ void pair(const PairInfo& pi, double& va, double& vb) const {
        const double* qa = lam + LBM_IDX(pi.A * plane + o, Q * plane);
        const double* qb = lam + LBM_IDX(pi.B * plane + o, Q * plane);
        va = LAST ? LoadNC::ld_last(qa) : LoadNC::ld_again_keep(qa);
        vb = LAST ? LoadNC::ld_last(qb) : LoadNC::ld_again_keep(qb);
    }
};

// The adjoint's results go to the pull source of each population (P^T: the inverse of the
// gather, unique targets because propagate + bc is a permutation).
template <bool WALL>
struct DstSource {
    double* __restrict__ out;
    const SiteAddr& ad;
    const int* sbase;     // as SrcGlobal: the tile's pull bases or the offsets
    int zoff;             // the row z, or the site x Lz + z with the offsets
    template <int L>
    __device__ __forceinline__ void put(double v) const {
        if constexpr (WALL) st_stream(out + LBM_IDX((ad.template src<L, true>()), Q * ad.plane), v);
        else st_stream(out + LBM_IDX(sbase[L] + zoff, Q * ad.plane), v);
    }
    __device__ __forceinline__ void pair(const PairInfo& pi, double va, double vb) const {
        if constexpr (WALL) {
            st_stream(out + LBM_IDX((ad.template src_rt<true>(pi.A, pi.B, pi.cx, pi.cz)), Q * ad.plane), va);
            st_stream(out + LBM_IDX((ad.template src_rt<true>(pi.B, pi.A, -pi.cx, -pi.cz)), Q * ad.plane), vb);
        } else {
            st_stream(out + LBM_IDX(sbase[pi.A] + zoff, Q * ad.plane), va);
            st_stream(out + LBM_IDX(sbase[pi.B] + zoff, Q * ad.plane), vb);
        }
    }
};

// Running float-float sums (unnormalised) of the pair loop.
struct AdjSums {
    ff A, Bx, Bz, U, C;
};

// The moments of the pulled f_t at the site: gathered and summed (as the step does), or read
// from the record of the forward step (k_step_ff_moments); both give the same int64 sums.
template <class FSRC>
struct MomGather {
    const FSRC& src;
    __device__ __forceinline__ MomentsFix get() const { return moments_fix(src); }
};
struct MomStored {
    const int64_t* __restrict__ m;
    int plane, o;
    __device__ __forceinline__ MomentsFix get() const {
        const long long* q = (const long long*)m;
        return MomentsFix{__ldg(q + LBM_IDX(o, 4 * plane)), __ldg(q + LBM_IDX(plane + o, 4 * plane)),
                          __ldg(q + LBM_IDX(2 * plane + o, 4 * plane)), __ldg(q + LBM_IDX(3 * plane + o, 4 * plane))};
    }
};

template <class MSRC, class DST>
__device__ __forceinline__ void adjoint_site_ff(const MSRC& msrc, const LamOwn& lsrc, const DST& dst,
                                                const AdjParamsFF& p) {
    // -- pass 1: moments of the pulled f_t; block exponent of lam_{t+1} -----------------
    const MomentsFix m = msrc.get();
    uint32_t eb = 75u << 20;      // floor: zero and subnormal lam stay 0 after scaling
    static_for<Q>([&](auto l) { eb = max(eb, lsrc.template hiword<decltype(l)::value>() & 0x7FF00000u); });
    const int32_t S = (int32_t)eb - (int32_t)(1023u << 20);                  // (E_block - 1023) << 20
    // -- per-site scalars in float-float (as in collide_ff) ------------------------------
    const double Rd = __ll2double_rn(m.R);
    const ff rho = dsplit(Rd), jx = i64_to_ff(m.Jx), jz = i64_to_ff(m.Jz);
    const ff dT = dsplit(fma(d_lat.r2_half, __ll2double_rn(m.E), -Rd));
    const ff inv = ff_rcp(rho);
    const ff3 r = ff3_of(d_lat.r3);
    const ff rinv = ff_mul_c3(inv, r);
    const ff ux = ff_mul(jx, rinv), uz = ff_mul(jz, rinv);
    const ff usz = ff_add(uz, p.us_z);
    const ff ux2 = ff_mul_u(ux, ux);
    const ff u2 = ff_add(ux2, ff_mul_u(usz, usz));                         // |u_s|^2
    const ff uu = ff_add(ux2, ff_mul_u(uz, uz));                           // |u|^2
    const ff tm1 = ff_sub(ff_mul_u(dT, inv), ff_mul_pow2(uu, 0.5f));        // T - 1
    const ff th = ff_add(tm1, p.T_shift);
    const ff a = ff_mul_c3(ux, r), b = ff_mul_c3(usz, r);
    // -- 24 K0, 24 K1, 24 K2 and 4 H0 as polynomials in |c|^2 ------------------------------
    const ff th2 = ff_mul(th, th), thu2 = ff_mul(th, u2), u4 = ff_mul_u(u2, u2);
    const ff k00 = ff_add(ff_add(ff_make(24.0f, 0.0f), ff_mul_f_u(u2, -12.0f)),
                          ff_add(ff_mul_f_u(u4, 3.0f), ff_mul_f_u(ff_add(thu2, ff_sub(th2, th)), 24.0f)));
    // (k01, k02) and (k10, k20) in the lanes of packed registers, and k21 = k11 / 2 exactly,
    // as in collide_ff
    const ff k01v = ff_sub(ff_mul_pow2(th, 2.0f), ff_add(thu2, ff_mul_pow2(th2, 4.0f)));
    const ffx2 k012 = ffx2_mul_c3(ffx2{x2_pack(k01v.hi, th2.hi), x2_pack(k01v.lo, th2.lo)},
                                  ff3_of(d_lat.r2x6), ff3_of(d_lat.r4x3));
    const ff k01 = ffx2_lane0(k012), k02 = ffx2_lane1(k012);
    const ffx2 k1020 = ffx2_add(ffx2{x2_pack(24.0f, 12.0f), x2_pack(0.0f, 0.0f)},
                                ffx2_add(ffx2_mul_f_u(ffx2_both(u2), x2_pack(-12.0f, -6.0f)),
                                         ffx2_mul_f_u(ffx2_both(th), x2_pack(-48.0f, -36.0f))));
    const ff k10 = ffx2_lane0(k1020), k20 = ffx2_lane1(k1020);
    const ff k11 = ff_mul_c3(th, ff3_of(d_lat.r2x12));
    const ff k21 = ff_mul_pow2(k11, 0.5f);
    // 4 H0 = (-4 + 4 u2 + 8 th) + r^2 (2 - u2 - 8 th) |c|^2 + r^4 th |c|^4
    const ff h00 = ff_add(ff_make(-4.0f, 0.0f), ff_add(ff_mul_pow2(u2, 4.0f), ff_mul_pow2(th, 8.0f)));
    const ff h01 = ff_mul_c3(ff_sub(ff_make(2.0f, 0.0f), ff_add(u2, ff_mul_pow2(th, 8.0f))), p.r2);
    const ff h02 = ff_mul_c3(th, p.r4);
    // -- pass 2: the sums ------------------------------------------------------------------
    AdjSums sm;
    {
        const double v0 = lsrc.template again<0>();
        const ff l0 = ff_mul_c3_u(bits_to_ff_scaled((uint32_t)__double2hiint(v0), (uint32_t)__double2loint(v0), S),
                                  p.wsh[0]);
        sm.A = ff_mul_u(l0, k00);       // s = 0, |c|^2 = 0
        sm.U = ff_mul_u(l0, k10);
        sm.C = ff_mul_u(l0, h00);
        sm.Bx = ff_make(0.0f, 0.0f);
        sm.Bz = ff_make(0.0f, 0.0f);
    }
    // the two pairs of each iteration in the lanes of packed FP32 registers; each lane's terms
    // are added to the sums, lane 0 first (separate sums per lane need registers that the
    // 96-register budget does not have: measured 3% slower)
    const ffx2 A2 = ffx2_both(a), B2 = ffx2_both(b);
    auto pair2_sums = [&](const PairInfo& p0, const PairInfo& p1, const ffx2& K0, const ffx2& K1, const ffx2& K2,
                          const ffx2& H, const ff3& W0, const ff3& W1, const ffx2& c6, const ffx2& c4) {
        double v0a, v0b, v1a, v1b;
        lsrc.pair(p0, v0a, v0b);
        lsrc.pair(p1, v1a, v1b);
        const ff la0 = bits_to_ff_scaled((uint32_t)__double2hiint(v0a), (uint32_t)__double2loint(v0a), S);
        const ff lb0 = bits_to_ff_scaled((uint32_t)__double2hiint(v0b), (uint32_t)__double2loint(v0b), S);
        const ff la1 = bits_to_ff_scaled((uint32_t)__double2hiint(v1a), (uint32_t)__double2loint(v1a), S);
        const ff lb1 = bits_to_ff_scaled((uint32_t)__double2hiint(v1b), (uint32_t)__double2loint(v1b), S);
        const ffx2 la{x2_pack(la0.hi, la1.hi), x2_pack(la0.lo, la1.lo)};
        const ffx2 lb{x2_pack(lb0.hi, lb1.hi), x2_pack(lb0.lo, lb1.lo)};
        const ffx2 ls = ffx2_mul_c3_u2(ffx2_add_u(la, lb), W0, W1);
        const ffx2 ld = ffx2_mul_c3_u2(ffx2_sub_u(la, lb), W0, W1);
        const f32x2 fcx = x2_pack(p0.fcx, p1.fcx), fcz = x2_pack(p0.fcz, p1.fcz);
        const ffx2 sx = ffx2_mul_f_u(A2, fcx), sz = ffx2_mul_f_u(B2, fcz);
        const ffx2 st = ffx2_two_sum(sx.hi, sz.hi);
        const ffx2 s{st.hi, x2_add(st.lo, x2_add(sx.lo, sz.lo))};
        const ffx2 q = ffx2_mul_u(s, s);
        const ffx2 P1 = ffx2_mul_u(ld, s), P2 = ffx2_mul_u(ls, s);
        const ffx2 ev = ffx2_add_big_u(K0, ffx2_mul_u(q, ffx2_add_big_u(K2, q)));
        const ffx2 od = ffx2_add_big_u_x4(K1, q);
        const ffx2 e1 = ffx2_add_big_u(K1, ffx2_mul_f_u(q, x2_pack(12.0f, 12.0f)));
        const ffx2 t2 = ffx2_add_big_u_x2(K2, q);
        const ffx2 tA = ffx2_add_u(ffx2_mul_u(ls, ev), ffx2_mul_u(P1, od));
        const ffx2 bt = ffx2_add_u(ffx2_mul_u(ld, e1), ffx2_scale(ffx2_mul_u(P2, t2), 2.0f));
        const ffx2 tx = ffx2_mul_f_u(bt, fcx), tz = ffx2_mul_f_u(bt, fcz);
        const ffx2 tU = ffx2_add_u(ffx2_mul_u(ls, e1), ffx2_mul_f_u(P1, x2_pack(24.0f, 24.0f)));
        const ffx2 hq = ffx2_add_big_u(H, ffx2_mul_u(c6, q));
        const ffx2 tC = ffx2_add_u(ffx2_mul_u(ls, hq), ffx2_mul_u(c4, P1));
        sm.A = ff_add_u(sm.A, ffx2_lane0(tA));
        sm.Bx = ff_add_u(sm.Bx, ffx2_lane0(tx));
        sm.Bz = ff_add_u(sm.Bz, ffx2_lane0(tz));
        sm.U = ff_add_u(sm.U, ffx2_lane0(tU));
        sm.C = ff_add_u(sm.C, ffx2_lane0(tC));
        sm.A = ff_add_u(sm.A, ffx2_lane1(tA));
        sm.Bx = ff_add_u(sm.Bx, ffx2_lane1(tx));
        sm.Bz = ff_add_u(sm.Bz, ffx2_lane1(tz));
        sm.U = ff_add_u(sm.U, ffx2_lane1(tU));
        sm.C = ff_add_u(sm.C, ffx2_lane1(tC));
    };
    // shells in the groups of d_groups (step_ff.cuh): the coefficients of two shells are formed
    // together, one shell per lane, and each iteration takes one pair of each
    const ffx2 k00b = ffx2_both(k00), k01b = ffx2_both(k01), k02b = ffx2_both(k02);
    const ffx2 k10b = ffx2_both(k10), k11b = ffx2_both(k11), k20b = ffx2_both(k20), k21b = ffx2_both(k21);
    const ffx2 h00b = ffx2_both(h00), h01b = ffx2_both(h01), h02b = ffx2_both(h02);
#pragma unroll 1
    for (int g = 0; g < NGROUP; g++) {
        const ShellGroup sg = d_groups[g];
        const f32x2 C2 = x2_pack(sg.c2a, sg.c2b);
        const ffx2 K0 = ffx2_add_u(k00b, ffx2_mul_f_u(ffx2_add_u(k01b, ffx2_mul_f_u(k02b, C2)), C2));
        const ffx2 K1 = ffx2_add_u(k10b, ffx2_mul_f_u(k11b, C2));
        const ffx2 K2 = ffx2_add_u(k20b, ffx2_mul_f_u(k21b, C2));
        const ffx2 H = ffx2_add_u(h00b, ffx2_mul_f_u(ffx2_add_u(h01b, ffx2_mul_f_u(h02b, C2)), C2));
        const ff c6a = p.c6[sg.sa], c6b = p.c6[sg.sb], c4a = p.c4[sg.sa], c4b = p.c4[sg.sb];
        const ffx2 c6{x2_pack(c6a.hi, c6b.hi), x2_pack(c6a.lo, c6b.lo)};
        const ffx2 c4{x2_pack(c4a.hi, c4b.hi), x2_pack(c4a.lo, c4b.lo)};
#pragma unroll 1
        for (int k = 0; k < sg.n; k++)
            pair2_sums(d_pairs[sg.k0 + k], d_pairs[sg.k1 + k], K0, K1, K2, H, p.wsh[sg.sa], p.wsh[sg.sb], c6, c4);
    }
    const ff sA = sm.A, sBx = sm.Bx, sBz = sm.Bz, sU = sm.U, sC = sm.C;
    // -- A', B', C' (times omega, in units of the block exponent) ---------------------------
    const ff A = ff_mul_c3(ff_renorm2(sA), p.inv24);
    const ff Bx = ff_mul_c3(ff_renorm2(sBx), p.r_24), Bz = ff_mul_c3(ff_renorm2(sBz), p.r_24);
    const ff Bu = ff_mul_pow2(ff_mul_c3(ff_renorm2(sU), p.inv24), -0.5f);
    const ff Cs = ff_mul_pow2(ff_renorm2(sC), 0.25f);
    const ff Btx = ff_add(Bx, ff_mul_pow2(ff_mul(Bu, ux), 2.0f));
    const ff Btz = ff_add(Bz, ff_mul_pow2(ff_mul(Bu, usz), 2.0f));
    // |u|^2 / 2 - T with T = 1 + tm1
    const ff tq = ff_sub(ff_mul_pow2(uu, 0.5f), ff_add(ff_make(1.0f, 0.0f), tm1));
    const ff Ap = ff_add(ff_sub(A, ff_add(ff_mul(Btx, ux), ff_mul(Btz, uz))), ff_mul(Cs, tq));
    const ff phx = ff_mul_c3(ff_sub(Btx, ff_mul(Cs, ux)), r);                // r B'_x
    const ff phz = ff_mul_c3(ff_sub(Btz, ff_mul(Cs, uz)), r);                // r B'_z
    const ff ph2 = ff_mul_pow2(ff_mul_c3(Cs, p.r2), 0.5f);                   // r^2 C'
    // -- pass 3: lam_t = (1 - w) lam + w (A' + B'.xi + C'|xi|^2), to the pull sources -------
    {
        const double v0 = lsrc.template again<0, true>();
        dst.template put<0>(fma(p.one_m_omega_d, v0, ff_to_double_scaled(Ap, S)));
    }
    const ffx2 PHX = ffx2_both(phx), PHZ = ffx2_both(phz);
    // even part A' + C'|xi|^2 once per shell, odd part B'.xi once per pair, each rounded to
    // binary64; the sum and the relaxation are FP64 (the FP64 pipe has room for the adds,
    // the issue slots of a float-float add and a second assembly per population it saves)
    const ffx2 APb = ffx2_both(Ap), PH2 = ffx2_both(ph2);
#pragma unroll 1
    for (int g = 0; g < NGROUP; g++) {
        const ShellGroup sg = d_groups[g];
        // A' + C'|xi|^2 of the two shells of the group (lanes 0, 1)
        const ffx2 e2 = ffx2_add_u(APb, ffx2_mul_f_u(PH2, x2_pack(sg.c2a, sg.c2b)));
        const ffx2 er = ffx2_two_sum(e2.hi, e2.lo);                                      // ff_renorm2
        const double eva = ff_to_double_scaled(ffx2_lane0(er), S), evb = ff_to_double_scaled(ffx2_lane1(er), S);
#pragma unroll 1
        for (int k = 0; k < sg.n; k++) {
            const PairInfo p0 = d_pairs[sg.k0 + k], p1 = d_pairs[sg.k1 + k];
            double v0a, v0b, v1a, v1b;
            lsrc.template pair<true>(p0, v0a, v0b);
            lsrc.template pair<true>(p1, v1a, v1b);
            // B'.xi of both pairs in the two lanes
            const ffx2 ox = ffx2_mul_f_u(PHX, x2_pack(p0.fcx, p1.fcx)), oz = ffx2_mul_f_u(PHZ, x2_pack(p0.fcz, p1.fcz));
            const ffx2 ot = ffx2_two_sum(ox.hi, oz.hi);
            const ffx2 o = ffx2_two_sum(ot.hi, x2_add(ot.lo, x2_add(ox.lo, oz.lo)));     // ff_renorm2
            const double od0 = ff_to_double_scaled(ffx2_lane0(o), S), od1 = ff_to_double_scaled(ffx2_lane1(o), S);
            dst.pair(p0, fma(p.one_m_omega_d, v0a, eva + od0), fma(p.one_m_omega_d, v0b, eva - od0));
            dst.pair(p1, fma(p.one_m_omega_d, v1a, evb + od1), fma(p.one_m_omega_d, v1b, evb - od1));
        }
    }
}

// One tile b of the tiling t (the step's tiling: wall tiles, then interior columns); the
// moments come from f_t (ft) or, if ft is null, from the record mom.
// PDL: launched with launch_pdl (every thread waits for the previous grid before its first
// global access, as tile_ff).  Interior tiles off the periodic seam take their pull sources
// and scatter targets from p.off (p a __grid_constant__ kernel parameter), as tile_ff.
template <bool PDL = false>
__device__ __forceinline__ void adjoint_tile_ff(const double* __restrict__ ft, const int64_t* __restrict__ mom,
                                                const double* __restrict__ lam_next, double* __restrict__ lam_out,
                                                const AdjParamsFF& p, Tiling t, int b, int* sbase) {
    // wall and interior tiles on separate paths (the tile kind is block-uniform), as tile_ff
    SiteAddr ad;
    bool wall;
    if (tile_is_wall(t, b)) {
        if constexpr (PDL) pdl_wait();
        if (!ad.setup(p.Lx, p.Lz, p.plane, t, b, wall)) return;
        const LamOwn lsrc{lam_next, ad.dst(), p.plane};
        const DstSource<true> dst{lam_out, ad, sbase, 0};
        if (mom) {
            adjoint_site_ff(MomStored{mom, p.plane, ad.dst()}, lsrc, dst, p);
        } else {
            const SrcGlobal<true, LoadNC, false, true> src{ft, ad, sbase, 0};
            adjoint_site_ff(MomGather<SrcGlobal<true, LoadNC, false, true>>{src}, lsrc, dst, p);
        }
        return;
    }
    // an interior tile's sources and targets: through the offsets or the tile's table (two
    // instances of the site code, so that each reads its bases from a known memory space)
    auto interior = [&](const int* bases, int zoff) {
        const LamOwn lsrc{lam_next, ad.dst(), p.plane};
        const DstSource<false> dst{lam_out, ad, bases, zoff};
        if (mom) {
            adjoint_site_ff(MomStored{mom, p.plane, ad.dst()}, lsrc, dst, p);
        } else {
            const SrcGlobal<false, LoadNC, false, true> src{ft, ad, bases, zoff};
            adjoint_site_ff(MomGather<SrcGlobal<false, LoadNC, false, true>>{src}, lsrc, dst, p);
        }
    };
    const int x = tile_column(t, b);
    if (off_seam(x, p.Lx)) {                        // block-uniform
        if constexpr (PDL) pdl_wait();
        if (!ad.setup(p.Lx, p.Lz, p.plane, t, b, wall)) return;
        interior(p.off, ad.dst());
        return;
    }
    fill_pull_bases(sbase, x, p.Lx, p.Lz, p.plane);
    __syncthreads();
    if constexpr (PDL) pdl_wait();
    if (!ad.setup(p.Lx, p.Lz, p.plane, t, b, wall)) return;
    interior(sbase, ad.z);
}

// Two register budgets: 5 resident blocks per SM (96 registers, 20 warps; 4.6% faster than 4
// blocks with 114 registers on large lattices) and 7 (72 registers; with the packed pair loops
// it spills 128-260 bytes and takes about the same total time on large lattices, but it needs
// one wave where the 5-block form needs two, as on 256 x 512).
template <int MINB>
__global__ void __launch_bounds__(BLOCK_Z, MINB)
k_adjoint_ff(const double* __restrict__ ft, const double* __restrict__ lam_next, double* __restrict__ lam_out,
             const __grid_constant__ AdjParamsFF p, Tiling t) {
    __shared__ int sbase[Q];
    pdl_allow_next();
    adjoint_tile_ff<true>(ft, nullptr, lam_next, lam_out, p, t, blockIdx.x, sbase);
}

// The same adjoint with the moments of f_t read from the forward step's record.
template <int MINB>
__global__ void __launch_bounds__(BLOCK_Z, MINB)
k_adjoint_ff_moments(const int64_t* __restrict__ mom, const double* __restrict__ lam_next,
                     double* __restrict__ lam_out, const __grid_constant__ AdjParamsFF p, Tiling t) {
    __shared__ int sbase[Q];
    pdl_allow_next();
    adjoint_tile_ff<true>(nullptr, mom, lam_next, lam_out, p, t, blockIdx.x, sbase);
}

// Relative time per block of the 7-block form (measured on 1024 x 2048: 0.647 vs 0.623 ms).
constexpr double ADJ_FF_COST7 = 1.04;

// Resident slots (SMs x blocks per SM) of the 5- and 7-block forms of one kernel, per device.
struct TwoForms {
    int s5 = 0, s7 = 0, dev = -1;
};

// Whether the 7-block form is expected to finish first: blocks rounded up to whole waves of
// each form's resident slots, weighted by the time per block.
template <class K5, class K7>
inline bool pick_7_blocks(TwoForms& c, int blocks, K5 k5, K7 k7) {
    int d = 0;
    cudaGetDevice(&d);
    if (d != c.dev) {
        int sms = 0, b5 = 0, b7 = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, d);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b5, k5, BLOCK_Z, 0);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b7, k7, BLOCK_Z, 0);
        c.s5 = sms * b5;
        c.s7 = sms * b7;
        c.dev = d;
    }
    if (c.s5 <= 0 || c.s7 <= 0) return false;
    const double padded5 = (double)((blocks + c.s5 - 1) / c.s5) * c.s5;
    const double padded7 = (double)((blocks + c.s7 - 1) / c.s7) * c.s7;
    return padded7 * ADJ_FF_COST7 < padded5;
}

// w_shell: the shell weights; r: the lattice constant (both binary64).
inline AdjParamsFF adj_ff_params(const StepParams& p, const double* w_shell, double r) {
    AdjParamsFF q;
    q.Lx = p.Lx; q.Lz = p.Lz; q.plane = p.plane;
    q.one_m_omega_d = p.one_m_omega;
    const long double rl = r, r2 = rl * rl;
    for (int sh = 0; sh < NSHELL; sh++) {
        q.wsh[sh] = ff3_host((long double)p.omega * w_shell[sh]);
        const long double C2 = r2 * shell_c2(sh);
        q.c6[sh] = ff_host((double)(C2 - 6.0L));
        q.c4[sh] = ff_host((double)(2.0L * (C2 - 4.0L)));
    }
    q.us_z = ff_host(p.us_z);
    q.T_shift = ff_host(p.T_shift);
    pull_offsets(p.Lz, p.plane, q.off);
    q.r2 = ff3_host(r2);
    q.r4 = ff3_host(r2 * r2);
    q.r_24 = ff3_host(rl / 24.0L);
    q.inv24 = ff3_host(1.0L / 24.0L);
    return q;
}

inline void launch_adjoint_ff(const double* ft, const double* lam_next, double* lam_out, const StepParams& p,
                              const double* w_shell, double r, const Tiling& t, cudaStream_t st) {
    const AdjParamsFF q = adj_ff_params(p, w_shell, r);
    const int blocks = tiling_blocks(t);
    static TwoForms forms;
    if (pick_7_blocks(forms, blocks, k_adjoint_ff<5>, k_adjoint_ff<7>))
        launch_pdl(k_adjoint_ff<7>, blocks, BLOCK_Z, st, ft, lam_next, lam_out, q, t);
    else
        launch_pdl(k_adjoint_ff<5>, blocks, BLOCK_Z, st, ft, lam_next, lam_out, q, t);
}

inline void launch_adjoint_ff_moments(const int64_t* mom, const double* lam_next, double* lam_out,
                                      const StepParams& p, const double* w_shell, double r, const Tiling& t,
                                      cudaStream_t st) {
    const AdjParamsFF q = adj_ff_params(p, w_shell, r);
    const int blocks = tiling_blocks(t);
    static TwoForms forms;
    if (pick_7_blocks(forms, blocks, k_adjoint_ff_moments<5>, k_adjoint_ff_moments<7>))
        launch_pdl(k_adjoint_ff_moments<7>, blocks, BLOCK_Z, st, mom, lam_next, lam_out, q, t);
    else
        launch_pdl(k_adjoint_ff_moments<5>, blocks, BLOCK_Z, st, mom, lam_next, lam_out, q, t);
}

}  // namespace lbm
