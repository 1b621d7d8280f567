// common.cuh -- device constants, launch parameters and pull-index helpers.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

#include "lattice.cuh"

namespace lbm {

__constant__ DevLattice d_lat;

constexpr int DIM = 2;
constexpr int BLOCK_Z = 128;      // threads per block along z (one site per thread)

// Parameters of one time step (Sec. III.A: dt = 1, omega = 1/tau, shifted equilibrium).
struct StepParams {
    int Lx, Lz;
    int plane;               // Lx * Lz sites per population array
    double omega;            // 1 / tau
    double one_m_omega;      // 1 - 1 / tau
    double us_z;             // tau * (-g): velocity shift of the equilibrium
    double T_shift;          // tau (1 - tau) g^2 / D
    double grav;             // g >= 0
};

// x index wrapped into [0, Lx) for |k| <= 3 (any Lx >= 1).
__device__ __forceinline__ int wrap_x(int v, int Lx) {
    int t = v % Lx;
    return t < 0 ? t + Lx : t;
}

// Element index of the pull source of population l for destination (x, z)
// (Sec. III.B pull propagate with periodic x; walls by half-way bounce-back on the
// same column: source row z - c_z below 0 -> opp(l) at row c_z - 1 - z; at or above
// Lz -> opp(l) at row 2 Lz - 1 - z + c_z).  col[k] = wrap(x + k - 3) * Lz.
template <int L>
__device__ __forceinline__ int pull_index(int x, int z, const int col[7], int Lz, int plane) {
    constexpr int CX = cx(L), CZ = cz(L), OP = opp(L);
    const int zs = z - CZ;
    if (CZ > 0 && zs < 0) return OP * plane + x * Lz + (CZ - 1 - z);
    if (CZ < 0 && zs >= Lz) return OP * plane + x * Lz + (2 * Lz - 1 - z + CZ);
    return L * plane + col[3 - CX] + zs;
}

// Interior form (3 <= z < Lz - 3 for the whole block): no wall test.
template <int L>
__device__ __forceinline__ int pull_index_interior(int z, const int col[7], int plane) {
    return L * plane + col[3 - cx(L)] + z - cz(L);
}

// Compile-time loop: calls f(Tag<L>{}) for L = 0..N-1.
template <int L>
struct Tag { static constexpr int value = L; };

template <int N, int L = 0, class F>
__device__ __forceinline__ void static_for(F&& f) {
    if constexpr (L < N) {
        f(Tag<L>{});
        static_for<N, L + 1>(f);
    }
}

}  // namespace lbm
