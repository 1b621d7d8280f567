// common.cuh -- device constants, launch parameters and pull-index helpers.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

#include "lattice.cuh"

namespace lbm {

__constant__ DevLattice d_lat;

// The 18 opposite velocity pairs for loops that run over pairs at run time
// (filled from the compile-time tables of lattice.cuh at upload).
struct PairInfo {
    int A, B, cx, cz;
    float fcx, fcz, fc2;        // c_x, c_z and |c|^2 as FP32 (no conversion in the loop)
};
__constant__ PairInfo d_pairs[18];
// Pairs are grouped by shell in canonical order: shell s owns pairs
// [d_shell_first[s], d_shell_first[s] + d_shell_npair[s]).
__constant__ int d_shell_first[8];
__constant__ int d_shell_npair[8];
__constant__ int d_vel[37][2];

// The seven moving shells in four groups whose coefficients a collide forms together, one
// shell per lane of packed FP32 registers: (|c|^2 = 1, 2), (4, 8), (5, 10) pair shells with
// equal pair counts, lane 0 taking pairs k0 .. k0 + n - 1 of shell sa and lane 1 pairs
// k1 .. k1 + n - 1 of shell sb; the last group is shell 9 alone, its two pairs one per lane.
struct ShellGroup {
    int k0, k1, n, sa, sb;
    float c2a, c2b;          // |c|^2 of the two lanes' shells
};
constexpr int NGROUP = 4;
__constant__ ShellGroup d_groups[NGROUP];

// Bounds-checked builds (-DLBM_BOUNDS_CHECK): LBM_IDX(i, n) tests every population index
// against the element count n of its buffer; an index outside [0, n) is counted in
// g_oob_count and replaced by 0, so the access stays in the buffer.  Other builds use i.
#ifdef LBM_BOUNDS_CHECK
__device__ unsigned int g_oob_count;
__device__ __forceinline__ int checked_index(int i, int n) {
    if ((unsigned)i < (unsigned)n) return i;
    atomicAdd(&g_oob_count, 1u);
    return 0;
}
#define LBM_IDX(i, n) checked_index((i), (n))
#else
#define LBM_IDX(i, n) (i)
#endif

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

// x index v = x + k (0 <= x < Lx, |k| <= 3) wrapped into [0, Lx) (any Lx >= 1; one
// compare-and-add for Lx >= 3, a remainder only for the narrower lattices).
__device__ __forceinline__ int wrap_x(int v, int Lx) {
    if (Lx >= 3) return v < 0 ? v + Lx : (v >= Lx ? v - Lx : v);
    const int t = v % Lx;
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

// Tiling of one step launch over the columns [x0, x0 + nx) (1D grid of block-thread tiles):
//   blocks [0, nwall):        wall tiles, one thread per (x, row) over the six rows
//                             0, 1, 2, Lz-3, Lz-2, Lz-1 (half-way bounce-back applies);
//   blocks [nwall, nwall + nzb * nx): interior tiles, column x, rows zb*block + t, aligned
//                             to row 0 so warps store whole sectors; threads outside
//                             3 <= z < Lz - 3 return (no wall test in this path).
// Wall tiles come first so their scattered loads overlap with the interior work.  A whole
// lattice is x0 = 0, nx = Lx; a column range serves the x-slab decomposition (slabs.cuh).
struct Tiling {
    int nwall, nzb;
    int x0, nx;
};
inline Tiling make_tiling_cols(int x0, int nx, int Lz, int block) {
    return Tiling{(6 * nx + block - 1) / block, (Lz + block - 1) / block, x0, nx};
}
inline Tiling make_tiling(int Lx, int Lz, int block) { return make_tiling_cols(0, Lx, Lz, block); }
inline int tiling_blocks(const Tiling& t) { return t.nwall + t.nzb * t.nx; }

struct SiteAddr {
    int x, z, Lz, plane, Lx;
    int col[7];            // wrap(x + k - 3) * Lz
    // Sets x, z for this thread of tile b; false if the thread has no site.  wall: tile kind.
    __device__ __forceinline__ bool setup(int Lx_, int Lz_, int plane_, Tiling t, int b, bool& wall) {
        Lx = Lx_;
        Lz = Lz_;
        plane = plane_;
        wall = b < t.nwall;
        if (wall) {
            const int i = b * blockDim.x + threadIdx.x;
            if (i >= 6 * t.nx) return false;
            const int xi = i / 6;
            const int r = i - 6 * xi;
            x = t.x0 + xi;
            z = r < 3 ? r : Lz - 6 + r;
        } else {
            const int tt = b - t.nwall;
            const int xi = tt / t.nzb;
            x = t.x0 + xi;
            z = (tt - xi * t.nzb) * blockDim.x + threadIdx.x;
            if (z < 3 || z >= Lz - 3) return false;
        }
#pragma unroll
        for (int k = 0; k < 7; k++) col[k] = wrap_x(x + k - 3, Lx) * Lz;
        return true;
    }
    template <int L, bool WALL>
    __device__ __forceinline__ int src() const {
        if constexpr (WALL) return pull_index<L>(x, z, col, Lz, plane);
        else return pull_index_interior<L>(z, col, plane);
    }
    // Runtime-velocity form of src() (population l with lattice vector (vx, vz)).
    template <bool WALL>
    __device__ __forceinline__ int src_rt(int l, int lop, int vx, int vz) const {
        const int zs = z - vz;
        if (WALL) {
            if (zs < 0) return lop * plane + x * Lz + (vz - 1 - z);
            if (zs >= Lz) return lop * plane + x * Lz + (2 * Lz - 1 - z + vz);
        }
        int xs = x - vx;
        xs = xs < 0 ? xs + Lx : (xs >= Lx ? xs - Lx : xs);
        if (Lx < 3) xs = wrap_x(x - vx, Lx);
        return l * plane + xs * Lz + zs;
    }
    __device__ __forceinline__ int dst() const { return x * Lz + z; }
    // Push form (collide, then move): the element population L leaving this site is
    // written to.  The inverse of the pull map: interior (L, x + c_x, z + c_z); a
    // population that would leave through a wall lands reversed on the same column,
    // opp(L) at row -c_z - 1 - z (bottom) or 2 Lz - 1 - z - c_z (top).
    template <int L, bool WALL>
    __device__ __forceinline__ int push_dst() const {
        constexpr int CX = cx(L), CZ = cz(L), OP = opp(L);
        const int zd = z + CZ;
        if (WALL) {
            if (CZ < 0 && zd < 0) return OP * plane + x * Lz + (-CZ - 1 - z);
            if (CZ > 0 && zd >= Lz) return OP * plane + x * Lz + (2 * Lz - 1 - z - CZ);
        }
        return L * plane + col[3 + CX] + zd;
    }
    // Runtime-velocity form of push_dst() (population l with lattice vector (vx, vz)).
    template <bool WALL>
    __device__ __forceinline__ int push_dst_rt(int l, int lop, int vx, int vz) const {
        const int zd = z + vz;
        if (WALL) {
            if (zd < 0) return lop * plane + x * Lz + (-vz - 1 - z);
            if (zd >= Lz) return lop * plane + x * Lz + (2 * Lz - 1 - z - vz);
        }
        int xd = x + vx;
        xd = xd < 0 ? xd + Lx : (xd >= Lx ? xd - Lx : xd);
        if (Lx < 3) xd = wrap_x(x + vx, Lx);
        return l * plane + xd * Lz + zd;
    }
};

// Block-uniform decomposition of a tile: wall flag, and for interior tiles the column x
// and the first row.  Every thread of the block computes the same values.
__device__ __forceinline__ bool tile_is_wall(Tiling t, int b) { return b < t.nwall; }
__device__ __forceinline__ int tile_column(Tiling t, int b) { return t.x0 + (b - t.nwall) / t.nzb; }

// Load policies.  LoadNC: read-only path (populations written by an earlier launch).
// LoadCG: L2-coherent loads, for data written earlier in the same launch by other CTAs
// (the persistent ensemble kernel), which the per-SM L1 could hold stale copies of.
struct LoadNC {
    // first reads: read-only path with an L2 prefetch of the surrounding 256 bytes (a pull
    // row starts up to 3 elements off a sector boundary; measured +0.6-0.8% on the steps)
    template <class T>
    __device__ static __forceinline__ T ld(const T* p) { return __ldg(p); }
    __device__ static __forceinline__ double ld(const double* p) {
        double v;
        asm("ld.global.nc.L2::256B.f64 %0, [%1];" : "=d"(v) : "l"(p));   // no side effect: free to schedule
        return v;
    }
    __device__ static __forceinline__ float ld(const float* p) {
        float v;
        asm("ld.global.nc.L2::256B.f32 %0, [%1];" : "=f"(v) : "l"(p));
        return v;
    }
    // L2 eviction policies: evict-last for values read again later in the same kernel, so that
    // the second reads find them in L2 (the two-pass float-float step and the adjoint read
    // every value twice or three times), evict-first for a value's last read.  With the
    // stores marked streaming (st_stream) the float-float step went from 0.2742 to 0.2655 ms
    // on 1024 x 2048 and its DRAM reads from 684 to ~620 MB (the algorithmic figure).
    __device__ static __forceinline__ uint64_t pol_keep() {
        uint64_t q;
        asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(q));
        return q;
    }
    __device__ static __forceinline__ uint64_t pol_last() {
        uint64_t q;
        asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(q));
        return q;
    }
    // first reads of values read again in the same kernel: kept in L2 in preference
    __device__ static __forceinline__ double ld_first(const double* p) {
        double v;
        asm("ld.global.nc.L2::cache_hint.L2::256B.f64 %0, [%1], %2;" : "=d"(v) : "l"(p), "l"(pol_keep()));
        return v;
    }
    // ... and kept in L1 too (evict-last): the float-float step's second pass reads the inner
    // shells first (measured +0.7%)
    __device__ static __forceinline__ double ld_keep(const double* p) {
        double v;
        asm("ld.global.nc.L1::evict_last.L2::cache_hint.L2::256B.f64 %0, [%1], %2;" : "=d"(v) : "l"(p), "l"(pol_keep()));
        return v;
    }
    // a second read issued as its own instruction (not merged with an earlier one)
    __device__ static __forceinline__ double ld_again(const double* p) {
        double v;
        asm volatile("ld.global.nc.f64 %0, [%1];" : "=d"(v) : "l"(p));
        return v;
    }
    // ... of a value that is read once more later in the kernel (kept in L2)
    __device__ static __forceinline__ double ld_again_keep(const double* p) {
        double v;
        asm volatile("ld.global.nc.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(p), "l"(pol_keep()));
        return v;
    }
    // the only read of a value in the kernel (the adjoint's gather of f_t): evict-first in L1
    // and L2
    __device__ static __forceinline__ double ld_once(const double* p) {
        double v;
        asm("ld.global.nc.L1::evict_first.L2::cache_hint.L2::256B.f64 %0, [%1], %2;" : "=d"(v) : "l"(p), "l"(pol_last()));
        return v;
    }
    // the last read of a value (the step's second pass): evict-first in L1 and L2, so that the
    // line does not displace lines still to be read again (L1: measured +0.7% on the
    // float-float step)
    __device__ static __forceinline__ double ld_last(const double* p) {
        double v;
        asm volatile("ld.global.nc.L1::evict_first.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(p), "l"(pol_last()));
        return v;
    }
};
// Stores of results that no later read of the same kernel needs: streaming (evict-first), so
// that they do not displace the lines the kernel reads twice.
__device__ __forceinline__ void st_stream(double* p, double v) {
    asm volatile("st.global.cs.f64 [%0], %1;" :: "l"(p), "d"(v) : "memory");
}
__device__ __forceinline__ void st_stream(float* p, float v) {
    asm volatile("st.global.cs.f32 [%0], %1;" :: "l"(p), "f"(v) : "memory");
}
struct LoadCG {
    template <class T>
    __device__ static __forceinline__ T ld(const T* p) { return __ldcg(p); }
    __device__ static __forceinline__ double ld_keep(const double* p) { return __ldcg(p); }
    __device__ static __forceinline__ double ld_first(const double* p) { return __ldcg(p); }
    __device__ static __forceinline__ double ld_once(const double* p) { return __ldcg(p); }
    __device__ static __forceinline__ double ld_again(const double* p) {
        double v;
        asm volatile("ld.global.cg.f64 %0, [%1];" : "=d"(v) : "l"(p));
        return v;
    }
    __device__ static __forceinline__ double ld_last(const double* p) { return ld_again(p); }
};

// Interior tiles: sbase[l] = l * plane + wrap(x - c_lx) * Lz - c_lz, so that the pull
// source of population l at row z is sbase[l] + z.  Filled by the block's threads in
// turn (every entry is written for any block size).
__device__ __forceinline__ void fill_pull_bases(int* sbase, int x, int Lx, int Lz, int plane) {
    for (int l = threadIdx.x; l < Q; l += blockDim.x)
        sbase[l] = l * plane + wrap_x(x - d_vel[l][0], Lx) * Lz - d_vel[l][1];
}

// The same bases without a table: away from the periodic seam (3 <= x < Lx - 3, no wrap)
// sbase[l] = x * Lz + off[l] with off[l] = l * plane - c_lx * Lz - c_lz, one set of offsets
// for the whole lattice, which the step kernels take from their parameters (no per-block
// fill, no block barrier).
inline void pull_offsets(int Lz, int plane, int (&off)[Q]) {
    for (int l = 0; l < Q; l++) off[l] = l * plane - cx(l) * Lz - cz(l);
}
// Push form: pbase[l] = x * Lz + poff[l] off the seam, poff[l] = l * plane + c_lx * Lz + c_lz.
inline void push_offsets(int Lz, int plane, int (&poff)[Q]) {
    for (int l = 0; l < Q; l++) poff[l] = l * plane + cx(l) * Lz + cz(l);
}
__device__ __forceinline__ bool off_seam(int x, int Lx) { return x >= 3 && x < Lx - 3; }

// Interior tiles, push form: pbase[l] = l * plane + wrap(x + c_lx) * Lz + c_lz, so that
// population l leaving row z is written at pbase[l] + z.
__device__ __forceinline__ void fill_push_bases(int* pbase, int x, int Lx, int Lz, int plane) {
    for (int l = threadIdx.x; l < Q; l += blockDim.x)
        pbase[l] = l * plane + wrap_x(x + d_vel[l][0], Lx) * Lz + d_vel[l][1];
}

// Programmatic dependent launch.  A kernel launched with launch_pdl may start while the
// previous kernel in its stream is still running (once all of that kernel's blocks have
// called pdl_allow_next or exited); every thread of it must call pdl_wait, which returns when
// the previous grid has completed and its writes are visible, before its first access to
// global memory.  Behind a copy or an event wait the launch is ordered as usual.
__device__ __forceinline__ void pdl_allow_next() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Launch errors are left in the runtime's last-error state, as for a <<<>>> launch.
template <class... KArgs, class... Args>
inline void launch_pdl(void (*kernel)(KArgs...), dim3 grid, int threads, cudaStream_t st, Args... args) {
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    (void)cudaLaunchKernelEx(&cfg, kernel, args...);
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

// Array-form sites (native FP64 and FP32 collides): the 37 inputs of the site, pulled
// (PUSH = false) or its own (PUSH = true) ...
template <bool PUSH, bool WALL, class LD, class T>
__device__ __forceinline__ void load_site(const T* __restrict__ fin, const SiteAddr& ad, T (&g)[Q]) {
    if constexpr (PUSH) {
        const int o = ad.dst();
        static_for<Q>([&](auto l) { g[l.value] = LD::ld(fin + LBM_IDX(l.value * ad.plane + o, Q * ad.plane)); });
    } else {
        static_for<Q>([&](auto l) {
            g[l.value] = LD::ld(fin + LBM_IDX((ad.template src<decltype(l)::value, WALL>()), Q * ad.plane));
        });
    }
}
// ... and the 37 results, stored at the site (PUSH = false) or where they move to.
template <bool PUSH, bool WALL, class T>
__device__ __forceinline__ void store_site(T* __restrict__ fout, const SiteAddr& ad, const T (&fo)[Q]) {
    if constexpr (PUSH) {
        static_for<Q>([&](auto l) {
            fout[LBM_IDX((ad.template push_dst<decltype(l)::value, WALL>()), Q * ad.plane)] = fo[l.value];
        });
    } else {
        const int o = ad.dst();
#pragma unroll
        for (int l = 0; l < Q; l++) fout[LBM_IDX(l * ad.plane + o, Q * ad.plane)] = fo[l];
    }
}

}  // namespace lbm
