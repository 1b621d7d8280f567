// moments_fix.cuh -- the moments of one site's 37 populations, rho = sum g, J = sum c g and
// E = sum |c|^2 g (Sec. III.A, with the integer lattice vectors c; xi = r c), summed exactly
// in 64-bit fixed point (unit 2^-60) from the binary64 patterns with integer instructions
// (ff.cuh), so that no FP64 instruction is spent on them and the sums do not depend on
// their order.  Used by the float-float and the native FP64 steps and adjoints.
#pragma once
#include "common.cuh"
#include "ff.cuh"

namespace lbm {

// Moments of one site in 64-bit fixed point (unit 2^-60): rho, J = sum c g, E = sum |c|^2 g.
struct MomentsFix {
    int64_t R, Jx, Jz, E;
};

// Pass 1: the moments of the site's 37 populations g (src.first<L>()).
template <class SRC>
__device__ __forceinline__ MomentsFix moments_fix(const SRC& src) {
    // pair sums by shell, pair differences grouped by |c_x| and |c_z| (no multiplies)
    int64_t R, Jx, Jz, E = 0;
    int64_t S[NSHELL] = {0, 0, 0, 0, 0, 0, 0, 0};
    int64_t GX[4] = {0, 0, 0, 0}, GZ[4] = {0, 0, 0, 0};
    {
        const double v0 = src.template first<0>();
        R = bits_to_fix60((uint32_t)__double2hiint(v0), (uint32_t)__double2loint(v0));
    }
    static_for<NPAIR>([&](auto k) {
        constexpr int A = pair_first(decltype(k)::value), B = opp(A);
        const double va = src.template first<A>();
        const double vb = src.template first<B>();
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
    return MomentsFix{R, Jx, Jz, E};
}

// The 37 populations of a site held in an array (registers).
struct SrcArray {
    const double (&g)[Q];
    template <int L>
    __device__ __forceinline__ double first() const { return g[L]; }
};

}  // namespace lbm
