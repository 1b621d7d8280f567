// step_f32dev.cuh -- FP32 storage of the deviation from a per-row FP64 reference
// (LBM_F32_DEV): the stored value is d_l(x, z) = f_l(x, z) - fref_l(z), with
//   fref_l(z) = f^eq_l(rho0(z), u0, T0(z)),  u0 = gvec / 2,
// the equilibrium at the horizontal means rho0, T0 of the initial state's rows (the state at
// rest of Sec. I).  The populations near a row's reference state are the bulk of the
// lattice, so d is small there and its FP32 rounding is small against f.
//
// The step (pull form, as step_f32.cuh) works on deviations only; every O(1) quantity comes
// from per-row tables built in FP64 on the host:
//   g_l = gref_l(z) + d_src,  gref_l(z) = fref of the pull source of population l at row z
//         (fref_l(z - c_lz), or fref_opp(l) of the mirrored row at a wall), so
//   f'_l - fref_l(z) = (1 - w) d_src + (1 - w) dref_l(z) + w (f^eq_l - fref_l(z)),
//   dref_l(z) = gref_l(z) - fref_l(z)  (table, FP32; small);
//   the moments are those of gref (per row) plus the FP32 sums of the pulled d;
//   f^eq_l - fref_l(z) = w_l [rho (P - P0) + (rho - rho0) P0], with P the polynomial of
//   step_f64.cuh at (s, |u_s|^2, th_s) and P0 at the reference (s0, |u0|^2, th0), the
//   difference P - P0 formed from the differences of its arguments (Delta s, Delta |u|^2,
//   Delta th), so that FP32 rounds only the small parts.
#pragma once
#include "common.cuh"
#include "init_diag.cuh"

namespace lbm {

// Per-row constants of the reference, RC_N = 8 floats per row (row z at 8 z, read as two
// float4; as eight arrays of Lz floats the step took 3% longer):
//   rho0, th0 = T0 - 1, crho = rho_g - rho0, cT = T_g - T0, eg = E_g / rho_g (lattice units),
//   jgx, jgz = J_g (lattice units, sum c gref), ug2 = |u_g|^2,
// where rho_g, J_g, E_g are the moments of gref at the row and T_g, u_g its temperature and
// velocity.
enum { RC_RHO0 = 0, RC_TH0, RC_CRHO, RC_CT, RC_EG, RC_JGX, RC_JGZ, RC_UG2, RC_N };
static_assert(RC_N == 8, "two float4 per row");

// dref_l(z) depends on l only through its shell and c_z (fref is the equilibrium at a row
// state with no horizontal velocity, and a wall mirrors a population into opp(l) of the same
// shell): it is zero for c_z = 0 (pulled from the same row) and takes 18 values per row for
// the other 28 populations.  dref_slot(l): the table column of population l, -1 for c_z = 0.
struct DrefSlots {
    int slot[Q];
    int n;
};
__host__ __device__ constexpr DrefSlots make_dref_slots() {
    DrefSlots r{};
    int keys[Q] = {};
    int nk = 0;
    for (int l = 0; l < Q; l++) {
        r.slot[l] = -1;
        if (cz(l) == 0) continue;
        const int key = shell_of(l) * 8 + cz(l) + 3;
        for (int j = 0; j < nk; j++)
            if (keys[j] == key) r.slot[l] = j;
        if (r.slot[l] < 0) {
            keys[nk] = key;
            r.slot[l] = nk++;
        }
    }
    r.n = nk;
    return r;
}
__host__ __device__ constexpr int dref_slot(int l) { return make_dref_slots().slot[l]; }
constexpr int NDREF = make_dref_slots().n;
static_assert(NDREF == 18, "18 distinct (shell, c_z) classes with c_z != 0");

struct StepParamsFD {
    int Lx, Lz, plane;
    float omega, one_m_omega, us_z, T_shift, u0z;   // u0z = -g / 2
    const float* __restrict__ dref;   // NDREF * Lz: dref of slot k (dref_slot) at k * Lz + z
    const float* __restrict__ rowc;   // RC_N * Lz, row-major (16-byte aligned)
};

template <bool WALL, class LD>
__device__ __forceinline__ void site_f32dev(const float* __restrict__ fin, float* __restrict__ fout,
                                           const SiteAddr& ad, const StepParamsFD& p) {
    const int z = ad.z, Lz = p.Lz;
    const float* __restrict__ dref = p.dref + z;
    float d[Q];
    load_site<false, WALL, LD>(fin, ad, d);
    // -- moments: the pulled reference's (per row) plus the sums of the pulled deviations --
    float dR = d[0], dJx = 0.f, dJz = 0.f, dE = 0.f;
    static_for<NPAIR>([&](auto k) {
        constexpr int A = pair_first(decltype(k)::value), B = opp(A);
        const float ps = d[A] + d[B], dm = d[A] - d[B];
        dR += ps;
        dE = fmaf((float)c2(A), ps, dE);
        if constexpr (cx(A) != 0) dJx = fmaf((float)cx(A), dm, dJx);
        if constexpr (cz(A) != 0) dJz = fmaf((float)cz(A), dm, dJz);
    });
    // the row's constants: (rho0, th0, crho, cT) and (eg, jgx, jgz, ug2)
    const float4 ra = __ldg((const float4*)p.rowc + 2 * z), rb = __ldg((const float4*)p.rowc + 2 * z + 1);
    const float rho0 = ra.x, th0 = ra.y;
    const float drho = ra.z + dR;                                      // rho - rho0
    const float rho = rho0 + drho;
    const float inv = 1.f / rho;
    const float r = d_lat.r_hi, r2 = d_lat.r2_hi;
    const float ux = r * (rb.y + dJx) * inv;
    const float uz = r * (rb.z + dJz) * inv;
    // T - T0 = (T_g - T0) + [r^2 (dE - e_g dR) / rho - (|u|^2 - |u_g|^2)] / 2
    const float dT = ra.w + 0.5f * (r2 * fmaf(-rb.x, dR, dE) * inv - (fmaf(ux, ux, uz * uz) - rb.w));
    // shifted state against the reference (u0 = (0, u0z), th0): differences
    const float usz = uz + p.us_z;
    const float dth = dT + p.T_shift;                                  // th_s - th0
    const float th = th0 + dth;
    const float duz = usz - p.u0z;
    const float q0 = p.u0z * p.u0z;
    const float dq = fmaf(ux, ux, duz * (usz + p.u0z));                // |u_s|^2 - |u0|^2
    const float q = q0 + dq;
    // coefficients (K0 - 1 = d00 + k01 C2 + k02 C2^2, K1 = k10 + k11 C2, K2 = k20 + k21 C2;
    // C2 the integer |c|^2) of the reference, and their differences
    const float d00_0 = -0.5f * q0 - th0 + 0.125f * q0 * q0 + th0 * q0 + th0 * th0;
    const float k01_0 = r2 * (0.5f * th0 - 0.25f * th0 * q0 - th0 * th0);
    const float k02_0 = r2 * r2 * 0.125f * th0 * th0;
    const float k10_0 = 1.f - 0.5f * q0 - 2.f * th0, k11_0 = 0.5f * r2 * th0;
    const float k20_0 = 0.5f - 0.25f * q0 - 1.5f * th0, k21_0 = 0.25f * r2 * th0;
    const float tq = fmaf(dth, q, th0 * dq);                           // th q - th0 q0
    const float tt = dth * (th + th0);                                 // th^2 - th0^2
    const float e00 = -0.5f * dq - dth + 0.125f * dq * (q + q0) + tq + tt;
    const float e01 = r2 * (0.5f * dth - 0.25f * tq - tt);
    const float e02 = r2 * r2 * 0.125f * tt;
    const float e10 = -0.5f * dq - 2.f * dth, e11 = 0.5f * r2 * dth;
    const float e20 = -0.25f * dq - 1.5f * dth, e21 = 0.25f * r2 * dth;
    const float a = r * ux, b = r * usz, b0 = r * p.u0z, db = r * duz;
    const float W = rho, V = drho;                                     // times w_shell below
    const int o = ad.dst();
    {   // rest population: s = s0 = 0, dref = 0
        const float w0 = d_lat.wf[0];
        const float F = w0 * fmaf(W, e00, V * (1.f + d00_0));
        const float v = fmaf(p.one_m_omega, d[0], p.omega * F);
        fout[LBM_IDX(o, Q * ad.plane)] = v;
    }
    static_for<NPAIR>([&](auto k) {
        constexpr int A = pair_first(decltype(k)::value), B = opp(A);
        constexpr float C2 = (float)c2(A);
        constexpr float CX = (float)cx(A), CZ = (float)cz(A);
        const float dK0 = fmaf(C2, fmaf(C2, e02, e01), e00);
        const float dK1 = fmaf(C2, e11, e10), dK2 = fmaf(C2, e21, e20);
        const float K0_0 = 1.f + fmaf(C2, fmaf(C2, k02_0, k01_0), d00_0);
        const float K1_0 = fmaf(C2, k11_0, k10_0), K2_0 = fmaf(C2, k21_0, k20_0);
        float s, ds;
        if constexpr (cx(A) == 0) { s = CZ * b; ds = CZ * db; }
        else if constexpr (cz(A) == 0) { s = CX * a; ds = CX * a; }
        else { s = fmaf(CX, a, CZ * b); ds = fmaf(CX, a, CZ * db); }
        const float s0 = CZ * b0;
        const float s2 = s * s, s02 = s0 * s0;
        const float D2 = ds * (s + s0);                                // s^2 - s0^2
        // P - P0, even and odd parts in s
        const float dEv = dK0 + dK2 * s2 + K2_0 * D2 + D2 * (s2 + s02) * (1.f / 24.f);
        const float dOd = dK1 * s + K1_0 * ds + ds * (s2 + fmaf(s, s0, s02)) * (1.f / 6.f);
        // P0, even and odd parts
        const float Ev0 = K0_0 + s02 * (K2_0 + s02 * (1.f / 24.f));
        const float Od0 = s0 * (K1_0 + s02 * (1.f / 6.f));
        const float wsh = d_lat.wf[shell_of(A)];
        const float FA = wsh * fmaf(W, dEv + dOd, V * (Ev0 + Od0));
        const float FB = wsh * fmaf(W, dEv - dOd, V * (Ev0 - Od0));
        float gA = d[A], gB = d[B];
        if constexpr (cz(A) != 0) {
            constexpr int SA = dref_slot(A), SB = dref_slot(B);
            gA += dref[SA * Lz];
            gB += dref[SB * Lz];
        }
        const float vA = fmaf(p.one_m_omega, gA, p.omega * FA);
        const float vB = fmaf(p.one_m_omega, gB, p.omega * FB);
        fout[LBM_IDX(A * ad.plane + o, Q * ad.plane)] = vA;
        fout[LBM_IDX(B * ad.plane + o, Q * ad.plane)] = vB;
    });
}

template <class LD>
__device__ __forceinline__ void tile_f32dev(const float* __restrict__ fin, float* __restrict__ fout,
                                           const StepParamsFD& p, Tiling t, int b) {
    SiteAddr ad;
    bool wall;
    if (!ad.setup(p.Lx, p.Lz, p.plane, t, b, wall)) return;
    if (wall) site_f32dev<true, LD>(fin, fout, ad, p);
    else site_f32dev<false, LD>(fin, fout, ad, p);
}

// Launched as a programmatic dependent of the previous kernel (as k_step_f32).  6 resident
// blocks per SM (80 registers).  Measured on 1024 x 2048: with the full 37-column offset
// table, 0.1478 ms at the unconstrained 92 registers (5 blocks), 0.1387 / 0.1364 / 0.1413 at
// 6 / 7 / 8 blocks; the 18-column table then took 7 blocks to 0.1290 (an L1 prefetch of its
// lines at the start of the site: 0.1360), and 6 / 8 blocks give 0.1283 / 0.1334; the row
// constants as two float4 per row, 0.1229 (the 18 offsets likewise as five float4: 0.1234).
__global__ void __launch_bounds__(BLOCK_Z, 6)
k_step_f32dev(const float* __restrict__ fin, float* __restrict__ fout, const __grid_constant__ StepParamsFD p,
              Tiling t) {
    pdl_allow_next();
    pdl_wait();
    tile_f32dev<LoadNC>(fin, fout, p, t, blockIdx.x);
}

inline StepParamsFD fd_params(const StepParams& p, const float* dref, const float* rowc) {
    StepParamsFD q;
    q.Lx = p.Lx; q.Lz = p.Lz; q.plane = p.plane;
    q.omega = (float)p.omega;
    q.one_m_omega = (float)p.one_m_omega;
    q.us_z = (float)p.us_z;
    q.T_shift = (float)p.T_shift;
    q.u0z = (float)(-0.5 * p.grav);
    q.dref = dref;
    q.rowc = rowc;
    return q;
}

// One step over the columns of tiling t.
inline void launch_step_f32dev(const float* fin, float* fout, const StepParamsFD& q, const Tiling& t,
                               cudaStream_t st) {
    launch_pdl(k_step_f32dev, tiling_blocks(t), BLOCK_Z, st, fin, fout, q, t);
}

// ---------------------------------------------------------------------------------
// The reference and the conversions of the deviation storage.
// ---------------------------------------------------------------------------------
// Horizontal means of the initial density and temperature per row (the fields of k_init):
// rowm[z] = mean_x rho(x, z), rowm[Lz + z] = mean_x T(x, z).  One block per row; the sums
// run in a fixed order (strided partial sums, then a tree), so the result is reproducible.
__global__ void k_init_rowmeans(const double* __restrict__ zc, InitParams ip, double* __restrict__ rowm) {
    __shared__ double sr[128], st[128];
    const int z = blockIdx.x;
    double R = 0.0, T = 0.0;
    for (int x = threadIdx.x; x < ip.Lx; x += blockDim.x) {
        double p, TT;
        layer_p_T(z + 0.5, zc[x], zc[ip.Lx + x], ip, p, TT);
        R += p / TT;
        T += TT;
    }
    sr[threadIdx.x] = R;
    st[threadIdx.x] = T;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) {
            sr[threadIdx.x] += sr[threadIdx.x + h];
            st[threadIdx.x] += st[threadIdx.x + h];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        rowm[z] = sr[0] / ip.Lx;
        rowm[ip.Lz + z] = st[0] / ip.Lx;
    }
}

// The initial state as deviations: d_l = (float)(f^eq_l - fref_l(z)), both in FP64.
__global__ void k_init_dev(float* __restrict__ f, const double* __restrict__ zc, InitParams ip,
                           const double* __restrict__ fref) {
    const int z = blockIdx.x * blockDim.x + threadIdx.x;
    const int x = blockIdx.y;
    if (z >= ip.Lz) return;
    double p, T, fe[Q];
    layer_p_T(z + 0.5, zc[x], zc[ip.Lx + x], ip, p, T);
    feq_f64(p / T, 0.0, -0.5 * ip.grav, T, fe);
    const int o = x * ip.Lz + z;
#pragma unroll
    for (int l = 0; l < Q; l++) f[l * ip.plane + o] = (float)(fe[l] - fref[l * ip.Lz + z]);
}

// Elements [first, first + n) of the state (index l * plane + x * Lz + z) as FP64
// populations, fref_l(z) + d, or back as deviations, (float)(f - fref_l(z)).
__global__ void k_to_f64_dev(const float* __restrict__ f, long long first, long long n, int plane, int Lz,
                             const double* __restrict__ fref, double* __restrict__ out) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const long long e = first + i;
    const int l = (int)(e / plane), z = (int)((e - (long long)l * plane) % Lz);
    out[i] = fref[l * Lz + z] + (double)f[e];
}
__global__ void k_from_f64_dev(float* __restrict__ f, long long first, long long n, int plane, int Lz,
                               const double* __restrict__ fref, const double* __restrict__ in) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const long long e = first + i;
    const int l = (int)(e / plane), z = (int)((e - (long long)l * plane) % Lz);
    f[e] = (float)(in[i] - fref[l * Lz + z]);
}

}  // namespace lbm
