// walls.cuh -- thermal-wall variant of the bc (rows 0..2 and Lz-3..Lz-1, Sec. III.B, which
// names only the rows): isothermal walls at T_bottom and T_top instead of the adiabatic
// half-way bounce-back.
//
// Each wall has three ghost rows beyond it holding the equilibrium at rest at the wall
// temperature, f^eq_l(rho_w(x), 0, T_w).  A population whose pull source row lies in a ghost
// row takes that ghost value.  The ghost density of each ghost column balances the mass
// through the wall in the step: rho_w(x) = out(x) / in_w, where out(x) is the mass of the
// populations that the step moves from the lattice into the ghost rows of column x, and
// in_w = sum over l entering through the wall of |c_lz| f^eq_l(1, 0, T_w) is the mass one
// unit of ghost density sends into the lattice.  So the ghost value of population l is
// out(x) * q_l, q_l = f^eq_l(1, 0, T_w) / in_w, and the total mass is conserved exactly.
//
// A step with thermal walls is one launch of the kernels below, over the step's tiling: the
// wall tiles come first (so their short, latency-bound work overlaps with the interior tiles)
// and take the ghost rule; the interior tiles run the step's own tile code.  A wall tile
// covers the columns of its threads' sites; it first sums out(x) for those columns and three
// more on each side (the reach of a pull) into shared memory, then gathers, collides and
// stores its sites with the collide of the context's precision.
#pragma once
#include "common.cuh"
#include "step_f32.cuh"
#include "step_f64.cuh"
#include "step_ff.cuh"

namespace lbm {

struct ThermalWall {
    double q[2][Q];     // f^eq_l(1, 0, T_w) / in_w, bottom (0) and top (1) wall
};

constexpr int WALL_COLS = 32;   // columns of one wall block: ceil(BLOCK_Z / 6) + 1 + 6 halo <= 32

// Columns of the wall sites of block b: x_first .. x_last, and the first summed column.
__device__ __forceinline__ int wall_block_first_col(int b) { return (b * BLOCK_Z) / 6; }

// out(x) of both walls for the columns x_first - 3 .. x_first - 3 + ncols - 1 (unwrapped
// numbering; the sums read the wrapped columns), into s_out[wall][k].  Bottom: populations with
// c_z < 0 in rows z < -c_z; top: c_z > 0 in rows z >= Lz - c_z; each read at the column it
// leaves from, x - c_x.
template <class T>
__device__ __forceinline__ void wall_out_sums(const T* __restrict__ fin, int Lx, int Lz, int plane, int x_first,
                                              int ncols, double (*s_out)[WALL_COLS]) {
    for (int i = threadIdx.x; i < 2 * ncols; i += blockDim.x) {
        const int top = i >= ncols;
        const int k = top ? i - ncols : i;
        const int x = wrap_x(x_first - 3 + k, Lx);
        double s = 0.0;
        static_for<Q>([&](auto l) {
            constexpr int L = decltype(l)::value, CX = cx(L), CZ = cz(L);
            if constexpr (CZ != 0) {
                const int xs = wrap_x(x - CX, Lx) * Lz;
                if (!top && CZ < 0) {
#pragma unroll
                    for (int z = 0; z < -CZ; z++) s += (double)fin[LBM_IDX(L * plane + xs + z, Q * plane)];
                }
                if (top && CZ > 0) {
#pragma unroll
                    for (int z = Lz - CZ; z < Lz; z++) s += (double)fin[LBM_IDX(L * plane + xs + z, Q * plane)];
                }
            }
        });
        s_out[top][k] = s;
    }
}

// Pull source values of one wall site with the ghost rule (the block's out sums in s_out,
// columns numbered from xbase = x_first - 3).
template <class T, class LD>
struct ThermalSrc {
    const T* __restrict__ fin;
    const SiteAddr& ad;
    const double (*s_out)[WALL_COLS];
    int xbase;
    const ThermalWall& w;
    __device__ __forceinline__ T rt(int l, int vx, int vz, bool again) const {
        const int zs = ad.z - vz;
        if (zs < 0) return (T)(s_out[0][ad.x - vx - xbase] * w.q[0][l]);
        if (zs >= ad.Lz) return (T)(s_out[1][ad.x - vx - xbase] * w.q[1][l]);
        const int xs = wrap_x(ad.x - vx, ad.Lx);
        const T* p = fin + LBM_IDX(l * ad.plane + xs * ad.Lz + zs, Q * ad.plane);
        if constexpr (sizeof(T) == 8) return again ? LD::ld_last(p) : LD::ld(p);
        else return LD::ld(p);
    }
    template <int L>
    __device__ __forceinline__ T first() const { return rt(L, cx(L), cz(L), false); }
    template <int L>
    __device__ __forceinline__ T again() const { return rt(L, cx(L), cz(L), true); }
    __device__ __forceinline__ void pair(const PairInfo& pi, T& va, T& vb) const {
        va = rt(pi.A, pi.cx, pi.cz, true);
        vb = rt(pi.B, -pi.cx, -pi.cz, true);
    }
};

// Wall tile b of tiling t: sums the out(x) of its columns (the whole block), then sets up
// this thread's wall site; false if it has none.
template <class T>
__device__ __forceinline__ bool thermal_wall_site(const T* __restrict__ fin, int Lx, int Lz, int plane, Tiling t,
                                                  int b, double (*s_out)[WALL_COLS], int& xbase, SiteAddr& ad) {
    const int x_first = t.x0 + wall_block_first_col(b);
    const int x_last = min(t.x0 + (b * BLOCK_Z + BLOCK_Z - 1) / 6, t.x0 + t.nx - 1);
    const int ncols = x_last - x_first + 7;
    wall_out_sums(fin, Lx, Lz, plane, x_first, ncols, s_out);
    __syncthreads();
    xbase = x_first - 3;
    bool wall;
    return ad.setup(Lx, Lz, plane, t, b, wall);
}

template <class T>
__device__ __forceinline__ void thermal_gather(const ThermalSrc<T, LoadNC>& src, T (&g)[Q]) {
    static_for<Q>([&](auto l) { g[l.value] = src.template first<decltype(l)::value>(); });
}

// One step with thermal walls (tiling t = make_tiling: wall tiles first).  7 blocks per SM:
// at 8 the wall code spills 84 bytes and the step is no faster.
__global__ void __launch_bounds__(BLOCK_Z, 7)
k_step_ff_thermal(const double* __restrict__ fin, double* __restrict__ fout, const __grid_constant__ StepParamsFF p,
                  Tiling t, ThermalWall w) {
    __shared__ int sbase[Q];
    __shared__ double s_out[2][WALL_COLS];
    pdl_allow_next();                   // launched with launch_pdl, as k_step_ff
    if (!tile_is_wall(t, blockIdx.x)) {
        tile_ff<LoadNC, NoMoments, true, true>(fin, fout, p, Shape{p.Lx, p.Lz, p.plane}, t, blockIdx.x, sbase);
        return;
    }
    pdl_wait();
    int xbase;
    SiteAddr ad;
    if (!thermal_wall_site(fin, p.Lx, p.Lz, p.plane, t, blockIdx.x, s_out, xbase, ad)) return;
    site_ff(ThermalSrc<double, LoadNC>{fin, ad, s_out, xbase, w}, DstSite{fout, ad.dst(), p.plane}, p);
}

__global__ void __launch_bounds__(BLOCK_Z)
k_step_f64_thermal(const double* __restrict__ fin, double* __restrict__ fout, StepParams p, Tiling t,
                   ThermalWall w) {
    __shared__ double s_out[2][WALL_COLS];
    if (!tile_is_wall(t, blockIdx.x)) {
        tile_f64<LoadNC>(fin, fout, p, t, blockIdx.x);
        return;
    }
    int xbase;
    SiteAddr ad;
    if (!thermal_wall_site(fin, p.Lx, p.Lz, p.plane, t, blockIdx.x, s_out, xbase, ad)) return;
    double g[Q], fo[Q];
    thermal_gather(ThermalSrc<double, LoadNC>{fin, ad, s_out, xbase, w}, g);
    collide_f64(g, fo, p);
    store_site<false, true>(fout, ad, fo);
}

__global__ void __launch_bounds__(BLOCK_Z)
k_step_f32_thermal(const float* __restrict__ fin, float* __restrict__ fout, StepParamsF p, Tiling t,
                   ThermalWall w) {
    __shared__ double s_out[2][WALL_COLS];
    if (!tile_is_wall(t, blockIdx.x)) {
        tile_f32<LoadNC>(fin, fout, p, t, blockIdx.x);
        return;
    }
    int xbase;
    SiteAddr ad;
    if (!thermal_wall_site(fin, p.Lx, p.Lz, p.plane, t, blockIdx.x, s_out, xbase, ad)) return;
    float g[Q], fo[Q];
    thermal_gather(ThermalSrc<float, LoadNC>{fin, ad, s_out, xbase, w}, g);
    collide_f32(g, fo, p);
    store_site<false, true>(fout, ad, fo);
}

// Host: q_l of one wall from the shell weights and r (long double), f^eq at rest:
// f^eq_l(1, 0, T) = w_l [1 + th (C2 - 2)/2 + th^2 (C2^2 - 8 C2 + 8)/8], th = T - 1, C2 = r^2 |c_l|^2.
inline void thermal_wall_q(const double* w_shell, double r, double Tw, int top, double (&q)[Q]) {
    const long double th = (long double)Tw - 1.0L, r2 = (long double)r * r;
    long double feq[Q], in = 0.0L;
    for (int l = 0; l < Q; l++) {
        const long double C2 = r2 * c2(l);
        feq[l] = w_shell[shell_of(l)] * (1.0L + th * (C2 - 2.0L) / 2.0L + th * th * (C2 * C2 - 8.0L * C2 + 8.0L) / 8.0L);
        const int vz = cz(l);
        if (!top && vz > 0) in += vz * feq[l];
        if (top && vz < 0) in += -vz * feq[l];
    }
    for (int l = 0; l < Q; l++) q[l] = (double)(feq[l] / in);
}

}  // namespace lbm
