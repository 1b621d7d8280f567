// adjoint.cuh -- adjoint of the fused step, of the width readout and of the initial state.
//
// Forward step: f_{t+1} = C(P f_t) with P = propagate + bc (a permutation of the
// (l, x, z) entries) and C the pointwise collide.  Its adjoint is
//   lam_t = P^T J_C(g)^T lam_{t+1},   g = P f_t.
// The collide depends on g only through rho, J = sum xi g and E = sum |xi|^2 g, so
//   (J_C^T lam)_m = (1 - w) lam_m + w [ A + B.(xi_m - u)/rho + C (|xi_m - u|^2 - D T)/(D rho) ],
//   A = sum_l lam_l f^eq_l / rho,  B = sum_l lam_l df^eq_l/du_s,  C = sum_l lam_l df^eq_l/dT_s,
// (w = 1/tau; the force shift of u and T is a constant offset).  P^T is a scatter to the
// pull source of each population: every (l, x, z) is the source of exactly one
// destination, so the writes never collide.
#pragma once
#include <type_traits>

#include "common.cuh"
#include "init_diag.cuh"
#include "moments_fix.cuh"

namespace lbm {

// P(s) = K0 + K1 s + K2 s^2 + s^3/6 + s^4/24 and its partial derivatives in s, |u|^2
// and th for one velocity (s = xi.u, C2 = |xi|^2, u2 = |u|^2, th = T - 1, D = 2).
struct PDerivs {
    double P, dPds, dPdu2, dPdth;
};

__device__ __forceinline__ PDerivs hermite_poly(double s, double C2, double u2, double th) {
    const double K0 = 1.0 - 0.5 * u2 + 0.5 * th * (C2 - 2.0) + 0.125 * u2 * u2
                    - 0.25 * th * u2 * (C2 - 4.0) + 0.125 * th * th * (C2 * C2 - 8.0 * C2 + 8.0);
    const double K1 = 1.0 - 0.5 * u2 + 0.5 * th * (C2 - 4.0);
    const double K2 = 0.5 - 0.25 * u2 + 0.25 * th * (C2 - 6.0);
    PDerivs d;
    d.P = K0 + s * (K1 + s * (K2 + s * (1.0 / 6.0 + s * (1.0 / 24.0))));
    d.dPds = K1 + s * (2.0 * K2 + s * (0.5 + s * (1.0 / 6.0)));
    d.dPdu2 = (-0.5 + 0.25 * u2 - 0.25 * th * (C2 - 4.0)) - 0.5 * s - 0.25 * s * s;
    d.dPdth = (0.5 * (C2 - 2.0) - 0.25 * u2 * (C2 - 4.0) + 0.25 * th * (C2 * C2 - 8.0 * C2 + 8.0))
            + s * 0.5 * (C2 - 4.0) + s * s * 0.25 * (C2 - 6.0);
    return d;
}

// Per site, with opposite velocities paired (s -> -s flips the odd parts):
//   P(s) = E + O,            E = K0 + q (K2 + q/24),  O = s (K1 + q/6),        q = s^2,
//   dP/ds = E1 + O1,         E1 = K1 + q/2,           O1 = s (2 K2 + q/6),
//   dP/du2 = G0 - q/4 - s/2, G0 = -1/2 + u2/4 - th (C2 - 4)/4,
//   dP/dth = H0 + q (C2 - 6)/4 + s (C2 - 4)/2,  H0 = (C2-2)/2 - u2 (C2-4)/4 + th (C2^2-8C2+8)/4,
// so that with ls = lam_+ + lam_-, ld = lam_+ - lam_-:
//   A = sum w (ls E + ld O),   B = rho sum w [ xi (ld E1 + ls O1) + 2 u_s (ls (G0 - q/4) - ld s/2) ],
//   C = rho sum w [ ls (H0 + q (C2-6)/4) + ld s (C2-4)/2 ],
// and mu_m = (1 - w) lam_m + w (A' + B'.xi_m + C' |xi_m|^2) with
//   A' = A - B.u/rho + C (|u|^2 - D T)/(D rho),  B' = B/rho - 2 C u/(D rho),  C' = C/(D rho).
// Lattice constants in the kernel's arithmetic type.
template <class T>
struct AdjConst;
template <>
struct AdjConst<double> {
    __device__ static double r() { return d_lat.r; }
    __device__ static double r2() { return d_lat.r2; }
    __device__ static double w(int s) { return d_lat.w[s]; }
};
template <>
struct AdjConst<float> {
    __device__ static float r() { return d_lat.r_hi; }
    __device__ static float r2() { return d_lat.r2_hi; }
    __device__ static float w(int s) { return d_lat.wf[s]; }
};

// T = double: the native FP64 adjoint (LBM_F64 contexts); T = float: FP32 storage and
// arithmetic (LBM_F32 contexts; accurate to FP32 rounding of the moments and the sums).
template <class T>
__device__ __forceinline__ void adjoint_native_site(const T* __restrict__ ft, const T* __restrict__ lam_next,
                                                    T* __restrict__ lam_out, const StepParams& p) {
    using C = AdjConst<T>;
    const int z = blockIdx.x * BLOCK_Z + threadIdx.x;
    const int x = blockIdx.y;
    if (z >= p.Lz) return;
    int col[7];
#pragma unroll
    for (int k = 0; k < 7; k++) col[k] = wrap_x(x + k - 3, p.Lx) * p.Lz;
    T g[Q];
    [[maybe_unused]] const int n = Q * p.plane;      // element count for bounds-checked builds
    static_for<Q>([&](auto l) { g[l.value] = ft[LBM_IDX(pull_index<decltype(l)::value>(x, z, col, p.Lz, p.plane), n)]; });
    const T r = C::r(), r2 = C::r2();
    T R, inv, ux, uz, uu, T_;
    if constexpr (std::is_same<T, double>::value) {
        // FP64: the moments summed exactly in 64-bit fixed point with integer instructions
        // (moments_fix.cuh), off the FP64 pipe that binds this kernel; rho in units of 2^-60
        // is scaled back (the ratios do not see the scale)
        const MomentsFix m = moments_fix(SrcArray{g});
        const double Rs = __ll2double_rn(m.R);
        const double invs = 1.0 / Rs;
        ux = r * __ll2double_rn(m.Jx) * invs;
        uz = r * __ll2double_rn(m.Jz) * invs;
        uu = ux * ux + uz * uz;
        T_ = 1.0 + (fma(d_lat.r2_half, __ll2double_rn(m.E), -Rs) * invs - 0.5 * uu);
        R = 0x1p-60 * Rs;
        inv = 0x1p60 * invs;
    } else {
        T Rs = g[0], Jx = T(0), Jz = T(0), E = T(0);
        static_for<NPAIR>([&](auto k) {
            constexpr int A_ = pair_first(decltype(k)::value), B_ = opp(A_);
            const T ps = g[A_] + g[B_], ms = g[A_] - g[B_];
            Rs += ps;
            if constexpr (cx(A_) != 0) Jx = fma(T(cx(A_)), ms, Jx);
            if constexpr (cz(A_) != 0) Jz = fma(T(cz(A_)), ms, Jz);
            E = fma(T(c2(A_)), ps, E);
        });
        R = Rs;
        inv = T(1) / R;
        ux = r * Jx * inv;
        uz = r * Jz * inv;
        uu = ux * ux + uz * uz;
        T_ = T(0.5) * (r2 * E * inv - uu);
    }
    const T usx = ux, usz = uz + T(p.us_z), th = T_ + T(p.T_shift) - T(1);
    const T u2 = usx * usx + usz * usz;
    const T a = r * usx, b = r * usz;          // s_l = c_x a + c_z b
    const int o = x * p.Lz + z;
    const T lam0 = lam_next[LBM_IDX(o, n)];
    // rest population (s = 0, C2 = 0)
    T A = C::w(0) * lam0 * (T(1) - T(0.5) * u2 - th + T(0.125) * u2 * u2 + th * u2 + th * th);
    T Bx = T(0), Bz = T(0), Bu = C::w(0) * lam0 * (T(-0.5) + T(0.25) * u2 + th);
    T Cs = C::w(0) * lam0 * (T(-1) + u2 + T(2) * th);
    static_for<NPAIR>([&](auto k) {
        constexpr int A_ = pair_first(decltype(k)::value), B_ = opp(A_);
        constexpr int SH = shell_of(A_);
        const T C2 = r2 * T(c2(A_));
        const T K0 = T(1) - T(0.5) * u2 + T(0.5) * th * (C2 - T(2)) + T(0.125) * u2 * u2
                   - T(0.25) * th * u2 * (C2 - T(4)) + T(0.125) * th * th * (C2 * C2 - T(8) * C2 + T(8));
        const T K1 = T(1) - T(0.5) * u2 + T(0.5) * th * (C2 - T(4));
        const T K2 = T(0.5) - T(0.25) * u2 + T(0.25) * th * (C2 - T(6));
        T s;
        if constexpr (cx(A_) == 0) s = T(cz(A_)) * b;
        else if constexpr (cz(A_) == 0) s = T(cx(A_)) * a;
        else s = fma(T(cx(A_)), a, T(cz(A_)) * b);
        const T q = s * s;
        const T Ev = fma(q, fma(q, T(1.0 / 24.0), K2), K0);
        const T Od = s * fma(q, T(1.0 / 6.0), K1);
        const T E1 = fma(q, T(0.5), K1);
        const T O1 = s * fma(q, T(1.0 / 6.0), T(2) * K2);
        const T G0 = T(-0.5) + T(0.25) * u2 - T(0.25) * th * (C2 - T(4));
        const T H0 = T(0.5) * (C2 - T(2)) - T(0.25) * u2 * (C2 - T(4)) + T(0.25) * th * (C2 * C2 - T(8) * C2 + T(8));
        const T la = lam_next[LBM_IDX(A_ * p.plane + o, n)], lb = lam_next[LBM_IDX(B_ * p.plane + o, n)];
        const T w = C::w(SH);
        const T ls = w * (la + lb), ld = w * (la - lb);
        A = fma(ls, Ev, fma(ld, Od, A));
        const T bt = fma(ld, E1, ls * O1);          // coefficient of xi_A
        Bx = fma(r * T(cx(A_)), bt, Bx);
        Bz = fma(r * T(cz(A_)), bt, Bz);
        Bu = fma(ls, fma(q, T(-0.25), G0), fma(ld, T(-0.5) * s, Bu));
        Cs = fma(ls, fma(T(0.25) * (C2 - T(6)), q, H0), fma(ld, T(0.5) * (C2 - T(4)) * s, Cs));
    });
    // dP/du_s = dP/ds xi + 2 dP/du2 u_s, times rho
    const T Bxt = R * (Bx + T(2) * Bu * usx);
    const T Bzt = R * (Bz + T(2) * Bu * usz);
    const T Ct = R * Cs;
    const T Dr = T(DIM) * R;
    const T Ap = A - (Bxt * ux + Bzt * uz) * inv + Ct * (uu - T(DIM) * T_) / Dr;
    const T Bpx = Bxt * inv - T(2) * Ct * ux / Dr;
    const T Bpz = Bzt * inv - T(2) * Ct * uz / Dr;
    const T Cp = Ct / Dr;
    const T om = T(p.omega), omo = T(p.one_m_omega);
    // scatter mu to the pull sources (unique targets: propagate + bc is a permutation)
    lam_out[LBM_IDX(pull_index<0>(x, z, col, p.Lz, p.plane), n)] = fma(omo, lam0, om * Ap);
    static_for<NPAIR>([&](auto k) {
        constexpr int A_ = pair_first(decltype(k)::value), B_ = opp(A_);
        const T ev = fma(Cp, r2 * T(c2(A_)), Ap);
        const T od = fma(Bpx, r * T(cx(A_)), Bpz * (r * T(cz(A_))));
        const T la = lam_next[LBM_IDX(A_ * p.plane + o, n)], lb = lam_next[LBM_IDX(B_ * p.plane + o, n)];
        lam_out[LBM_IDX(pull_index<A_>(x, z, col, p.Lz, p.plane), n)] = fma(omo, la, om * (ev + od));
        lam_out[LBM_IDX(pull_index<B_>(x, z, col, p.Lz, p.plane), n)] = fma(omo, lb, om * (ev - od));
    });
}

// Both native forms are launched with launch_pdl (common.cuh): no prologue to overlap, but the
// next adjoint step is scheduled during this one's last wave.
__global__ void __launch_bounds__(BLOCK_Z)
k_adjoint_native_f64(const double* __restrict__ ft, const double* __restrict__ lam_next, double* __restrict__ lam_out,
                     StepParams p) {
    pdl_allow_next();
    pdl_wait();
    adjoint_native_site(ft, lam_next, lam_out, p);
}

// The FP32 form is held by memory latency: 7 resident blocks per SM (72 registers, a small
// spill) instead of the 4 its unconstrained 118 registers allow (measured: 4 blocks 0.253 ms,
// 6 blocks 0.203, 7 and 8 blocks 0.187 on 1024 x 2048).
__global__ void __launch_bounds__(BLOCK_Z, 7)
k_adjoint_native_f32(const float* __restrict__ ft, const float* __restrict__ lam_next, float* __restrict__ lam_out,
                     StepParams p) {
    pdl_allow_next();
    pdl_wait();
    adjoint_native_site(ft, lam_next, lam_out, p);
}

// lam_N(l,x,z) = dL[z] / Lx * (|xi_l - u|^2 - D T)/(D rho) at the stored state f (storage
// policy S: FP64 or FP32 populations and adjoint; the arithmetic is FP64).
template <class S>
__global__ void k_loss_adjoint(const typename S::T* __restrict__ f, const double* __restrict__ dL,
                               typename S::T* __restrict__ lam, int Lx, int Lz) {
    const int z = blockIdx.x * blockDim.x + threadIdx.x;
    const int x = blockIdx.y;
    if (z >= Lz) return;
    double R, ux, uz, T;
    site_moments<S>(f, x, z, Lz, Lx * Lz, R, ux, uz, T);
    const double scale = dL[z] / (double)Lx / (DIM * R);
    const int o = x * Lz + z;
#pragma unroll
    for (int l = 0; l < Q; l++) {
        const double dx = d_lat.r * cx(l) - ux, dz = d_lat.r * cz(l) - uz;
        S::put(lam, l * Lx * Lz + o, scale * (dx * dx + dz * dz - DIM * T));
    }
}

// Per column x: sum_{z,l} lam0 df0/dz_lo(x) -> colred[x], same for z_hi -> colred[Lx + x].
// f0 = f^eq(rho, (0, -g/2), T), rho = p/T with p and T as in layer_p_T; p is continuous
// across the interfaces, so moving an interface adds no boundary term.
template <class S>
__global__ void __launch_bounds__(128)
k_init_adjoint_columns(const typename S::T* __restrict__ lam0, const double* __restrict__ zc, InitParams ip,
                       double* __restrict__ colred) {
    __shared__ double sm[2][128];
    const int x = blockIdx.x;
    const double zl = zc[x], zh = zc[ip.Lx + x];
    const double gr = ip.grav * d_lat.r;
    const double uz = -0.5 * ip.grav, u2 = uz * uz;
    double gl = 0.0, gh = 0.0;
    for (int k = threadIdx.x; k < ip.Lz; k += 128) {
        const double z = k + 0.5;
        double p, T;
        layer_p_T(z, zl, zh, ip, p, T);
        const double rho = p / T, th = T - 1.0;
        const double dp_dzl = (z >= zl) ? p * (-gr / ip.Td + gr / ip.Tm) : 0.0;
        const double dp_dzh = (z >= zh) ? p * (-gr / ip.Tm + gr / ip.Tu) : 0.0;
        const double sl = 1.0 / cosh((z - zl) / ip.wt), sh = 1.0 / cosh((z - zh) / ip.wt);
        const double dT_dzl = (ip.Td - ip.Tm) * 0.5 * sl * sl / ip.wt;
        const double dT_dzh = (ip.Tm - ip.Tu) * 0.5 * sh * sh / ip.wt;
        const double drl = dp_dzl / T - p * dT_dzl / (T * T);
        const double drh = dp_dzh / T - p * dT_dzh / (T * T);
        double s_feq_rho = 0.0, s_dfdT = 0.0;
#pragma unroll
        for (int l = 0; l < Q; l++) {
            const double s = d_lat.r * cz(l) * uz;
            const PDerivs d = hermite_poly(s, d_lat.r2 * c2(l), u2, th);
            const double lv = S::get(lam0, l * ip.plane + x * ip.Lz + k);
            const double w = d_lat.w[shell_of(l)];
            s_feq_rho += lv * w * d.P;           // f^eq / rho
            s_dfdT += lv * w * rho * d.dPdth;    // df^eq / dT
        }
        gl += s_feq_rho * drl + s_dfdT * dT_dzl;
        gh += s_feq_rho * drh + s_dfdT * dT_dzh;
    }
    sm[0][threadIdx.x] = gl;
    sm[1][threadIdx.x] = gh;
    __syncthreads();
    for (int w = 64; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            sm[0][threadIdx.x] += sm[0][threadIdx.x + w];
            sm[1][threadIdx.x] += sm[1][threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        colred[x] = sm[0][0];
        colred[ip.Lx + x] = sm[1][0];
    }
}

// dL/dA_k = sum_x colred[x] cos(2 pi k x / Lx + phi_k) and
// dL/dphi_k = -A_k sum_x colred[x] sin(2 pi k x / Lx + phi_k), one block per mode; out holds
// dA_lo, dA_hi, dphi_lo, dphi_hi (K each).
__global__ void __launch_bounds__(128)
k_init_adjoint_modes(const double* __restrict__ colred, const double* __restrict__ modes, InitParams ip,
                     double* __restrict__ out) {
    __shared__ double sm[4][128];
    const int k = blockIdx.x;
    const double ph_lo = modes[ip.K + k], ph_hi = modes[3 * ip.K + k];
    double a = 0.0, b = 0.0, c = 0.0, d = 0.0;
    for (int x = threadIdx.x; x < ip.Lx; x += 128) {
        const double arg = 2.0 * M_PI * (double)(k + 1) * (double)x / (double)ip.Lx;
        double s_lo, c_lo, s_hi, c_hi;
        sincos(arg + ph_lo, &s_lo, &c_lo);
        sincos(arg + ph_hi, &s_hi, &c_hi);
        a += colred[x] * c_lo;
        b += colred[ip.Lx + x] * c_hi;
        c += colred[x] * s_lo;
        d += colred[ip.Lx + x] * s_hi;
    }
    sm[0][threadIdx.x] = a;
    sm[1][threadIdx.x] = b;
    sm[2][threadIdx.x] = c;
    sm[3][threadIdx.x] = d;
    __syncthreads();
    for (int w = 64; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int j = 0; j < 4; j++) sm[j][threadIdx.x] += sm[j][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[k] = sm[0][0];
        out[ip.K + k] = sm[1][0];
        out[2 * ip.K + k] = -modes[k] * sm[2][0];
        out[3 * ip.K + k] = -modes[2 * ip.K + k] * sm[3][0];
    }
}

}  // namespace lbm
