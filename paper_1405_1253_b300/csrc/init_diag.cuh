// init_diag.cuh -- three-layer initial state, per-site moments, horizontal means, global
// sums, mixing widths and storage conversions.  All arithmetic FP64.
#pragma once
#include "common.cuh"

namespace lbm {

// ---------------------------------------------------------------------------------
// Storage policies: how a stored population is read as FP64 / written from FP64.
// ---------------------------------------------------------------------------------
struct StoreF64 {
    using T = double;
    __device__ static double get(const double* f, int idx) { return f[idx]; }
    __device__ static void put(double* f, int idx, double v) { f[idx] = v; }
};
struct StoreF32 {
    using T = float;
    __device__ static double get(const float* f, int idx) { return (double)f[idx]; }
    __device__ static void put(float* f, int idx, double v) { f[idx] = (float)v; }
};

// ---------------------------------------------------------------------------------
// FP64 equilibrium, closed form of the 4th-order Hermite expansion (see step_f64.cuh).
// ---------------------------------------------------------------------------------
__device__ __forceinline__ void feq_f64(double rho, double ux, double uz, double T, double (&f)[Q]) {
    const double r = d_lat.r;
    const double th = T - 1.0, u2 = ux * ux + uz * uz;
    const double a = r * ux, b = r * uz;
#pragma unroll
    for (int l = 0; l < Q; l++) {
        const double C2 = d_lat.r2 * c2(l);
        const double s = cx(l) * a + cz(l) * b;
        const double K0 = 1.0 - 0.5 * u2 + 0.5 * th * (C2 - 2.0) + 0.125 * u2 * u2
                        - 0.25 * th * u2 * (C2 - 4.0) + 0.125 * th * th * (C2 * C2 - 8.0 * C2 + 8.0);
        const double K1 = 1.0 - 0.5 * u2 + 0.5 * th * (C2 - 4.0);
        const double K2 = 0.5 - 0.25 * u2 + 0.25 * th * (C2 - 6.0);
        const double P = K0 + s * (K1 + s * (K2 + s * (1.0 / 6.0 + s * (1.0 / 24.0))));
        f[l] = d_lat.w[shell_of(l)] * rho * P;
    }
}

// ---------------------------------------------------------------------------------
// Initial state (Sec. I, Eq. (seteq), pressure continuity, Fig. 1 caption).
// ---------------------------------------------------------------------------------
struct InitParams {
    int Lx, Lz, plane;
    double grav, Tu, Tm, Td, rho_ref, wt, zlo0, zhi0;
    int K;
};

// Interface heights per column: zc[x] = z_lo(x), zc[Lx + x] = z_hi(x).
// modes = [amp_lo | phase_lo | amp_hi | phase_hi], K each.
__global__ void k_interfaces(double* __restrict__ zc, const double* __restrict__ modes, InitParams ip) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= ip.Lx) return;
    const double* amp_lo = modes;
    const double* ph_lo = modes + ip.K;
    const double* amp_hi = modes + 2 * ip.K;
    const double* ph_hi = modes + 3 * ip.K;
    double zl = ip.zlo0, zh = ip.zhi0;
    for (int k = 0; k < ip.K; k++) {
        const double arg = 2.0 * M_PI * (double)(k + 1) * (double)x / (double)ip.Lx;
        zl += amp_lo[k] * cos(arg + ph_lo[k]);
        zh += amp_hi[k] * cos(arg + ph_hi[k]);
    }
    zc[x] = zl;
    zc[ip.Lx + x] = zh;
}

// Pressure and temperature at height z (sites) for interfaces zl < zh.
__device__ __forceinline__ void layer_p_T(double z, double zl, double zh, const InitParams& ip,
                                          double& p, double& T) {
    const double gr = ip.grav * d_lat.r;
    const double plo = ip.rho_ref * ip.Td * exp(-gr * zl / ip.Td);
    if (z < zl) p = ip.rho_ref * ip.Td * exp(-gr * z / ip.Td);
    else if (z < zh) p = plo * exp(-gr * (z - zl) / ip.Tm);
    else p = plo * exp(-gr * (zh - zl) / ip.Tm) * exp(-gr * (z - zh) / ip.Tu);
    T = ip.Tu + (ip.Tm - ip.Tu) * 0.5 * (1.0 - tanh((z - zh) / ip.wt))
              + (ip.Td - ip.Tm) * 0.5 * (1.0 - tanh((z - zl) / ip.wt));
}

template <class S>
__global__ void k_init(typename S::T* __restrict__ f, const double* __restrict__ zc, InitParams ip) {
    const int z = blockIdx.x * blockDim.x + threadIdx.x;
    const int x = blockIdx.y;
    if (z >= ip.Lz) return;
    double p, T, fe[Q];
    layer_p_T(z + 0.5, zc[x], zc[ip.Lx + x], ip, p, T);
    feq_f64(p / T, 0.0, -0.5 * ip.grav, T, fe);
    const int o = x * ip.Lz + z;
#pragma unroll
    for (int l = 0; l < Q; l++) S::put(f, l * ip.plane + o, fe[l]);
}

// ---------------------------------------------------------------------------------
// Moments of the stored populations (Sec. III.A).
// ---------------------------------------------------------------------------------
template <class S>
__device__ __forceinline__ void site_moments(const typename S::T* f, int x, int z,
                                             int Lz, int plane, double& rho, double& ux, double& uz,
                                             double& T) {
    const int o = x * Lz + z;
    double R = 0.0, Jx = 0.0, Jz = 0.0, E = 0.0;
#pragma unroll
    for (int l = 0; l < Q; l++) {
        const double v = S::get(f, l * plane + o);
        R += v;
        Jx += cx(l) * v;
        Jz += cz(l) * v;
        E += c2(l) * v;
    }
    rho = R;
    ux = d_lat.r * Jx / R;
    uz = d_lat.r * Jz / R;
    T = 0.5 * (d_lat.r2 * E / R - (ux * ux + uz * uz));
}

template <class S>
__global__ void k_moments(const typename S::T* __restrict__ f, int Lx, int Lz, double grav, int renorm, double* rho, double* ux, double* uz,
                          double* T) {
    const int z = blockIdx.x * blockDim.x + threadIdx.x;
    const int x = blockIdx.y;
    if (z >= Lz) return;
    double R, U, V, TT;
    site_moments<S>(f, x, z, Lz, Lx * Lz, R, U, V, TT);
    if (renorm) {              // u^H = u_stored - gvec/2, T^H = T + g^2/(4 D)
        V += 0.5 * grav;
        TT += grav * grav / (4.0 * DIM);
    }
    const int o = x * Lz + z;
    if (rho) rho[o] = R;
    if (ux) ux[o] = U;
    if (uz) uz[o] = V;
    if (T) T[o] = TT;
}

// Horizontal mean of T, stage 1: columns [c*nx_per, (c+1)*nx_per) summed into part[c][z].
template <class S>
__global__ void k_rowT_partial(const typename S::T* __restrict__ f, int Lx, int Lz, int nx_per,
                               double* __restrict__ part, int part_n) {
    const int z = blockIdx.x * blockDim.x + threadIdx.x;
    const int c = blockIdx.y;
    if (z >= Lz) return;
    const int x0 = c * nx_per, x1 = min(Lx, x0 + nx_per);
    double s = 0.0;
    for (int x = x0; x < x1; x++) {
        double R, U, V, TT;
        site_moments<S>(f, x, z, Lz, Lx * Lz, R, U, V, TT);
        s += TT;
    }
    part[LBM_IDX(c * Lz + z, part_n)] = s;
}

// Stage 2: Tbar[z] = (sum_c part[c][z]) / Lx, chunks added in order.
__global__ void k_rowT_final(const double* __restrict__ part, int part_n, int nchunk, int Lx, int Lz,
                             double* __restrict__ Tbar) {
    const int z = blockIdx.x * blockDim.x + threadIdx.x;
    if (z >= Lz) return;
    double s = 0.0;
    for (int c = 0; c < nchunk; c++) s += part[LBM_IDX(c * Lz + z, part_n)];
    Tbar[z] = s / (double)Lx;
}

// Per-row statistics over x (Sec. IV fluctuation profiles) of T and of the kinetic energy
// per unit mass E_k = |u^H|^2 / 2 (u^H = u - gvec/2, the renormalised velocity), in two
// passes over columns chunked like k_rowT_partial: mean == nullptr sums q; otherwise
// sums (q - mean)^2 with mean[0..Lz) for T and mean[Lz..2 Lz) for E_k.
// part[(c * 2 + k) * Lz + z], k = 0 (T), 1 (E_k).
template <class S>
__global__ void k_row_stats_partial(const typename S::T* __restrict__ f, int Lx, int Lz, int nx_per,
                                    double grav, const double* __restrict__ mean, double* __restrict__ part) {
    const int z = blockIdx.x * blockDim.x + threadIdx.x;
    const int c = blockIdx.y;
    if (z >= Lz) return;
    const int x0 = c * nx_per, x1 = min(Lx, x0 + nx_per);
    double a = 0.0, b = 0.0;
    for (int x = x0; x < x1; x++) {
        double R, U, V, TT;
        site_moments<S>(f, x, z, Lz, Lx * Lz, R, U, V, TT);
        const double vh = V + 0.5 * grav;
        const double ek = 0.5 * (U * U + vh * vh);
        if (mean) {
            const double dt = TT - mean[z], de = ek - mean[Lz + z];
            a += dt * dt;
            b += de * de;
        } else {
            a += TT;
            b += ek;
        }
    }
    part[(2 * c) * Lz + z] = a;
    part[(2 * c + 1) * Lz + z] = b;
}

// Stage 2: out[k * Lz + z] = (sum_c part[c][k][z]) / Lx, chunks added in order; the
// square root of it when root != 0 (rms of the deviations).
__global__ void k_row_stats_final(const double* __restrict__ part, int nchunk, int Lx, int Lz, int root,
                                  double* __restrict__ out) {
    const int z = blockIdx.x * blockDim.x + threadIdx.x;
    if (z >= Lz) return;
    for (int k = 0; k < 2; k++) {
        double s = 0.0;
        for (int c = 0; c < nchunk; c++) s += part[(2 * c + k) * Lz + z];
        s /= (double)Lx;
        out[k * Lz + z] = root ? sqrt(s) : s;
    }
}

// Tent-map widths, Eq. (3L): L_u = sum_z Theta[(Tbar - T_u)/(T_m - T_u)],
// L_d = sum_z Theta[(Tbar - T_m)/(T_d - T_m)] with Theta[b] = 2b on (0, 1/2),
// 2 (1 - b) on [1/2, 1), 0 elsewhere.  One block, fixed-order tree sum.
__device__ __forceinline__ double tent_map(double b) {
    if (b > 0.0 && b < 0.5) return 2.0 * b;
    if (b >= 0.5 && b < 1.0) return 2.0 * (1.0 - b);
    return 0.0;
}

__global__ void __launch_bounds__(256)
k_tent_widths(const double* __restrict__ Tbar, int Lz, double Tu, double Tm, double Td, double* __restrict__ out) {
    __shared__ double sm[2][256];
    double a = 0.0, b = 0.0;
    for (int z = threadIdx.x; z < Lz; z += 256) {
        a += tent_map((Tbar[z] - Tu) / (Tm - Tu));
        b += tent_map((Tbar[z] - Tm) / (Td - Tm));
    }
    sm[0][threadIdx.x] = a;
    sm[1][threadIdx.x] = b;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            sm[0][threadIdx.x] += sm[0][threadIdx.x + w];
            sm[1][threadIdx.x] += sm[1][threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = sm[0][0];
        out[1] = sm[1][0];
    }
}

// Global mass and energy: per-block partial sums (fixed order), then one final block.
constexpr int RED_THREADS = 256;

template <class S>
__global__ void __launch_bounds__(RED_THREADS)
k_global_partial(const typename S::T* __restrict__ f, int Lx, int Lz, double* __restrict__ part) {
    __shared__ double sm[2][RED_THREADS];
    const int nsite = Lx * Lz;
    double m = 0.0, e = 0.0;
    for (int s = blockIdx.x * RED_THREADS + threadIdx.x; s < nsite; s += gridDim.x * RED_THREADS) {
#pragma unroll
        for (int l = 0; l < Q; l++) {
            const double v = S::get(f, l * nsite + s);
            m += v;
            e += c2(l) * v;
        }
    }
    sm[0][threadIdx.x] = m;
    sm[1][threadIdx.x] = e;
    __syncthreads();
    for (int w = RED_THREADS / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            sm[0][threadIdx.x] += sm[0][threadIdx.x + w];
            sm[1][threadIdx.x] += sm[1][threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = sm[0][0];
        part[2 * blockIdx.x + 1] = 0.5 * d_lat.r2 * sm[1][0];
    }
}

__global__ void __launch_bounds__(RED_THREADS)
k_global_final(const double* __restrict__ part, int nblk, double* __restrict__ out) {
    __shared__ double sm[2][RED_THREADS];
    double m = 0.0, e = 0.0;
    for (int b = threadIdx.x; b < nblk; b += RED_THREADS) {
        m += part[2 * b];
        e += part[2 * b + 1];
    }
    sm[0][threadIdx.x] = m;
    sm[1][threadIdx.x] = e;
    __syncthreads();
    for (int w = RED_THREADS / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            sm[0][threadIdx.x] += sm[0][threadIdx.x + w];
            sm[1][threadIdx.x] += sm[1][threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) { out[0] = sm[0][0]; out[1] = sm[1][0]; }
}

// ---------------------------------------------------------------------------------
// Threshold mixing widths (Sec. IV), one thread: out[0..1] = L_u, L_d, out[2] = status
// (0 ok, -1 missing crossing); dL[Lz] = d(L_u + L_d)/dTbar when dL is not NULL.
// A crossing of level thr between consecutive scanned rows p -> q sits at
// z_p + (z_q - z_p) (thr - b_p)/(b_q - b_p); a first scanned row already past the
// level is the crossing itself.
// ---------------------------------------------------------------------------------
struct Crossing {
    double z;
    int p, q;            // bracketing rows (p == q: no interpolation)
    double dzp, dzq;     // dz/db_p, dz/db_q
    int ok;
};

__device__ Crossing scan_crossing(const double* Tbar, double T0, double T1, int Lz, int start, int dir,
                                  double thr, bool rising) {
    Crossing c{0.0, start, start, 0.0, 0.0, 0};
    const double inv = 1.0 / (T1 - T0);
    const double b0 = (Tbar[start] - T0) * inv;
    if (rising ? (b0 >= thr) : (b0 <= thr)) { c.z = start; c.ok = 1; return c; }
    int p = start;
    double bp = b0;
    for (int q = start + dir; q >= 0 && q < Lz; q += dir) {
        const double bq = (Tbar[q] - T0) * inv;
        if (rising ? (bq >= thr) : (bq <= thr)) {
            const double db = bq - bp, t = (thr - bp) / db, span = (double)(q - p);
            c.z = p + span * t;
            c.p = p; c.q = q;
            c.dzp = span * ((thr - bp) / (db * db) - 1.0 / db);
            c.dzq = -span * (thr - bp) / (db * db);
            c.ok = 1;
            return c;
        }
        p = q;
        bp = bq;
    }
    return c;
}

__global__ void k_widths(const double* __restrict__ Tbar, int Lz, double Tu, double Tm, double Td,
                         double* __restrict__ out, double* __restrict__ dL) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    Crossing a = scan_crossing(Tbar, Tu, Tm, Lz, Lz - 1, -1, 0.05, true);
    Crossing bb = a.ok ? scan_crossing(Tbar, Tu, Tm, Lz, a.q, -1, 0.95, true) : a;
    Crossing c = scan_crossing(Tbar, Tm, Td, Lz, 0, +1, 0.95, false);
    Crossing d = c.ok ? scan_crossing(Tbar, Tm, Td, Lz, c.q, +1, 0.05, false) : c;
    const int ok = a.ok && bb.ok && c.ok && d.ok;
    out[0] = ok ? a.z - bb.z : 0.0;
    out[1] = ok ? d.z - c.z : 0.0;
    out[2] = ok ? 0.0 : -1.0;
    if (dL) {
        for (int k = 0; k < Lz; k++) dL[k] = 0.0;
        if (ok) {
            const double su = 1.0 / (Tm - Tu), sd = 1.0 / (Td - Tm);
            dL[a.p] += a.dzp * su;   dL[a.q] += a.dzq * su;
            dL[bb.p] -= bb.dzp * su; dL[bb.q] -= bb.dzq * su;
            dL[d.p] += d.dzp * sd;   dL[d.q] += d.dzq * sd;
            dL[c.p] -= c.dzp * sd;   dL[c.q] -= c.dzq * sd;
        }
    }
}

// One propagate + bc without collide, fout = P fin (Sec. III.B: the pull gather with the
// periodic wrap and the wall rule).  It maps a pull-form state (post-collision) to the
// matching push-form state (post-propagation).
template <class T>
__global__ void __launch_bounds__(BLOCK_Z)
k_propagate(const T* __restrict__ fin, T* __restrict__ fout, int Lx, int Lz, Tiling t) {
    SiteAddr ad;
    bool wall;
    if (!ad.setup(Lx, Lz, Lx * Lz, t, blockIdx.x, wall)) return;
    const int o = ad.dst();
    [[maybe_unused]] const int n = Q * ad.plane;     // element count for bounds-checked builds
    if (wall) static_for<Q>([&](auto l) {
        fout[LBM_IDX(l.value * ad.plane + o, n)] = fin[LBM_IDX((ad.template src<decltype(l)::value, true>()), n)];
    });
    else static_for<Q>([&](auto l) {
        fout[LBM_IDX(l.value * ad.plane + o, n)] = fin[LBM_IDX((ad.template src<decltype(l)::value, false>()), n)];
    });
}

// ---------------------------------------------------------------------------------
// Storage <-> canonical FP64 conversion of n elements starting at element `first`.
// ---------------------------------------------------------------------------------
template <class S>
__global__ void k_to_f64(const typename S::T* __restrict__ f, long long first, long long n,
                         double* __restrict__ out) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    out[i] = S::get(f, (int)(first + i));
}

template <class S>
__global__ void k_from_f64(typename S::T* __restrict__ f, long long first, long long n,
                           const double* __restrict__ in) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    S::put(f, (int)(first + i), in[i]);
}

}  // namespace lbm
