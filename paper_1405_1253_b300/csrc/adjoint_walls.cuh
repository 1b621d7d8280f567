// adjoint_walls.cuh -- the float-float adjoint step (adjoint_ff.cuh) with the thermal walls of
// walls.cuh.
//
// With thermal walls, propagate + bc is linear but not a permutation: a wall-row destination
// pulling from a ghost row takes out(x_g) q_l, out(x_g) the mass the step moves into ghost
// column x_g and q_l = f^eq_l(1, 0, T_w) / in_w.  Its transpose therefore:
//   * passes the mu of a destination pulled from a lattice entry back to that entry (as the
//     bounce-back adjoint does; unique targets);
//   * collects, for each ghost column, Omega(x_g) = sum of mu q_l over the destinations that
//     pull from it;
//   * gives Omega(x_g) to every entry the step moves into that ghost column (coefficient 1 in
//     out); no destination pulls those entries, so that is all they receive.
// The step kernel runs the interior tiles as the bounce-back adjoint does; its wall tiles take
// their moments through the thermal gather of walls.cuh and leave the mu of ghost pulls in a
// scratch array [wall][l][x][row], which a second kernel sums per ghost column in a fixed
// order (the result does not depend on scheduling) before writing the leaving entries.
#pragma once
#include "adjoint_ff.cuh"
#include "walls.cuh"

namespace lbm {

// Scratch index of the mu of destination (x, row r of the wall's three rows) for population l.
__device__ __forceinline__ int ghost_mu_index(int wall, int l, int x, int r, int Lx) {
    return ((wall * Q + l) * Lx + x) * 3 + r;
}

// Where a wall site's results go: pull sources inside the lattice, or the ghost scratch.
struct DstSourceThermal {
    double* __restrict__ out;
    double* __restrict__ gmu;
    const SiteAddr& ad;
    __device__ __forceinline__ void one(int l, int vx, int vz, double v) const {
        const int zs = ad.z - vz;
        [[maybe_unused]] const int ng = 6 * Q * ad.Lx;     // element count for bounds-checked builds
        if (zs < 0) {
            gmu[LBM_IDX(ghost_mu_index(0, l, ad.x, ad.z, ad.Lx), ng)] = v;
        } else if (zs >= ad.Lz) {
            gmu[LBM_IDX(ghost_mu_index(1, l, ad.x, ad.z - (ad.Lz - 3), ad.Lx), ng)] = v;
        } else {
            const int xs = wrap_x(ad.x - vx, ad.Lx);
            out[LBM_IDX(l * ad.plane + xs * ad.Lz + zs, Q * ad.plane)] = v;
        }
    }
    template <int L>
    __device__ __forceinline__ void put(double v) const { one(L, cx(L), cz(L), v); }
    __device__ __forceinline__ void pair(const PairInfo& pi, double va, double vb) const {
        one(pi.A, pi.cx, pi.cz, va);
        one(pi.B, -pi.cx, -pi.cz, vb);
    }
};

template <int MINB>
__global__ void __launch_bounds__(BLOCK_Z, MINB)
k_adjoint_ff_thermal(const double* __restrict__ ft, const double* __restrict__ lam_next,
                     double* __restrict__ lam_out, const __grid_constant__ AdjParamsFF p, Tiling t, ThermalWall w,
                     double* __restrict__ gmu) {
    __shared__ int sbase[Q];
    __shared__ double s_out[2][WALL_COLS];
    if (!tile_is_wall(t, blockIdx.x)) {
        adjoint_tile_ff(ft, nullptr, lam_next, lam_out, p, t, blockIdx.x, sbase);
        return;
    }
    int xbase;
    SiteAddr ad;
    if (!thermal_wall_site(ft, p.Lx, p.Lz, p.plane, t, blockIdx.x, s_out, xbase, ad)) return;
    const ThermalSrc<double, LoadNC> src{ft, ad, s_out, xbase, w};
    adjoint_site_ff(MomGather<ThermalSrc<double, LoadNC>>{src}, LamOwn{lam_next, ad.dst(), p.plane},
                    DstSourceThermal{lam_out, gmu, ad}, p);
}

// One thread per (wall, ghost column): Omega from the scratch, then the leaving entries.
__global__ void __launch_bounds__(128)
k_adjoint_thermal_ghosts(double* __restrict__ lam_out, const double* __restrict__ gmu, int Lx, int Lz, int plane,
                         ThermalWall w) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 2 * Lx) return;
    const int top = i >= Lx;
    const int xg = top ? i - Lx : i;
    [[maybe_unused]] const int ng = 6 * Q * Lx;
    double om = 0.0;
    // destinations that pull from this ghost column: column xg + c_x, rows whose source lies
    // beyond the wall (bottom: z < c_z; top: z >= Lz + c_z, row r = z - (Lz - 3))
    static_for<Q>([&](auto l) {
        constexpr int L = decltype(l)::value, CX = cx(L), CZ = cz(L);
        if constexpr (CZ != 0) {
            const int x = wrap_x(xg + CX, Lx);
            if (!top && CZ > 0) {
#pragma unroll
                for (int r = 0; r < CZ; r++) om += gmu[LBM_IDX(ghost_mu_index(0, L, x, r, Lx), ng)] * w.q[0][L];
            }
            if (top && CZ < 0) {
#pragma unroll
                for (int r = 3 + CZ; r < 3; r++) om += gmu[LBM_IDX(ghost_mu_index(1, L, x, r, Lx), ng)] * w.q[1][L];
            }
        }
    });
    // the entries the step moves into this ghost column (from column xg - c_x)
    static_for<Q>([&](auto l) {
        constexpr int L = decltype(l)::value, CX = cx(L), CZ = cz(L);
        if constexpr (CZ != 0) {
            const int x = wrap_x(xg - CX, Lx) * Lz;
            if (!top && CZ < 0) {
#pragma unroll
                for (int z = 0; z < -CZ; z++) lam_out[LBM_IDX(L * plane + x + z, Q * plane)] = om;
            }
            if (top && CZ > 0) {
#pragma unroll
                for (int z = Lz - CZ; z < Lz; z++) lam_out[LBM_IDX(L * plane + x + z, Q * plane)] = om;
            }
        }
    });
}

// gmu: 6 Q Lx doubles of scratch.
inline void launch_adjoint_ff_thermal(const double* ft, const double* lam_next, double* lam_out, const StepParams& p,
                                      const double* w_shell, double r, const ThermalWall& w, double* gmu,
                                      cudaStream_t st) {
    const AdjParamsFF q = adj_ff_params(p, w_shell, r);
    const Tiling t = make_tiling(p.Lx, p.Lz, BLOCK_Z);
    const int blocks = tiling_blocks(t);
    static TwoForms forms;
    if (pick_7_blocks(forms, blocks, k_adjoint_ff_thermal<5>, k_adjoint_ff_thermal<7>))
        k_adjoint_ff_thermal<7><<<blocks, BLOCK_Z, 0, st>>>(ft, lam_next, lam_out, q, t, w, gmu);
    else
        k_adjoint_ff_thermal<5><<<blocks, BLOCK_Z, 0, st>>>(ft, lam_next, lam_out, q, t, w, gmu);
    k_adjoint_thermal_ghosts<<<(2 * p.Lx + 127) / 128, 128, 0, st>>>(lam_out, gmu, p.Lx, p.Lz, p.plane, w);
}

}  // namespace lbm
