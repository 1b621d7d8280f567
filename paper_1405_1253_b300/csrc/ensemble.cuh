// ensemble.cuh -- many independent lattices (the paper's N_conf realisations, Table II)
// advanced together.
//
// Every lattice keeps its own two population buffers and its own tiling (wall tiles, then
// interior tiles, see common.cuh); the tiles of all lattices are numbered consecutively
// (lattice i owns tiles [tile_begin_i, tile_begin_i + ntiles_i)).  Two launch shapes:
//   k_ens_step:       one launch per time step over all tiles of all lattices (the launch
//                     boundary separates the steps);
//   k_ens_persistent: ONE launch for n steps.  Co-resident CTAs (cooperative launch) take
//                     work items (step, ens_item consecutive tiles of one lattice) from a
//                     step-major queue; before an item of step s of lattice i runs, the CTA
//                     waits until all tiles of step s-1 of lattice i are done (per-lattice
//                     step barrier: a completion counter of tiles).
//                     The wait is a bounded spin: past the limit it sets the error word and
//                     the CTA leaves, and every other CTA leaves at its next wait.  Data
//                     written inside the launch is read through L2 (LoadCG), never a stale L1.
// Progress of the persistent kernel: all CTAs are resident and items are handed out in
// increasing order, while every item depends only on items of the previous step (smaller
// numbers), so the smallest blocked item always has all of its dependencies running.
#pragma once
#include <type_traits>

#include "common.cuh"
#include "step_f32.cuh"
#include "step_ff.cuh"

namespace lbm {

struct EnsLattice {
    void* buf[2];
    int Lx, Lz, plane;
    int cur;          // buffer holding the state before the launch's first step
    Tiling t;
    int tile_begin;   // first global tile number
    int ntiles;
    int item_begin;   // first persistent work item of the lattice (ens_item tiles per item)
};

// Tiles per work item of the persistent kernel: one queue fetch, lattice search, barrier wait
// and completion count serve that many consecutive tiles of one lattice (the 48-lattice set,
// 200 steps, FP32: 15,172 MLUPS with one tile per item, 16,264 / 17,063 / 17,524 with 2 / 4 / 8;
// float-float at 28 warps per SM: 6,841 with one, 7,064 / 7,116 / 7,110 with 4 / 8 / 16).
// Consecutive tiles of one column sharing the pull-base table (no refill, no barrier between
// them) were slower while every thread also held the lattice record in registers (6,657 and
// 17,294); with the record in shared memory they are faster (ens_item_tile).
constexpr int ens_item(bool) { return 8; }
// Wall tiles per work item (a lattice's items: its wall tiles in items of ens_wall_item, then
// its interior tiles in items of ens_item).  A float-float wall tile (six scattered rows with
// the bounce-back rule) takes several times an interior tile; eight of them in one item made
// that item the last of its lattice's step, which the next step's items of the lattice wait
// for: wall tiles one per item took 16 lattices of 256x512 from 6,240 to 7,137 MLUPS (48-lattice
// set unchanged, 7,368 / 7,360), two per item to 7,202-7,216 (one per item on the same box:
// 7,063-7,071; the 48-lattice set still unchanged).  FP32 wall tiles are cheap, and single-tile
// items only add queue work there (19,035 -> 18,742 and 19,410 -> 19,270): they keep 8.  Larger
// interior items (12 or 16 tiles) gained 0.2% on the 48-lattice set and lost 13% and 23% on the
// 16 small lattices.
constexpr int ens_wall_item(bool ff) { return ff ? 2 : 8; }
// Work items of a lattice with nwall wall tiles of ntiles.
inline int ens_items(bool ff, int nwall, int ntiles) {
    return (nwall + ens_wall_item(ff) - 1) / ens_wall_item(ff) + (ntiles - nwall + ens_item(ff) - 1) / ens_item(ff);
}

struct EnsControl {   // device words, reset before every persistent launch
    unsigned int queue;
    unsigned int err;
    unsigned int pad[2];
};

// Lattice owning global tile b (binary search over tile_begin; n <= a few hundred).
__device__ __forceinline__ int ens_find(const EnsLattice* __restrict__ lats, int n, int b) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (lats[mid].tile_begin <= b) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}
// Lattice owning persistent work item j of a step (binary search over item_begin).
__device__ __forceinline__ int ens_find_item(const EnsLattice* __restrict__ lats, int n, int j) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (lats[mid].item_begin <= j) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// One tile of one lattice at step s of the launch.  The buffers are chosen by parity with a
// select, not an index into L.buf (a run-time index would put the struct in local memory);
// the physics comes from the launch's parameter block, the shape from the lattice.
template <class LD>
__device__ __forceinline__ void ens_tile(const EnsLattice& L, int local, int s, const StepParamsFF& qf,
                                        int* sbase) {
    const bool odd = (L.cur + s) & 1;
    const double* fin = (const double*)(odd ? L.buf[1] : L.buf[0]);
    double* fout = (double*)(odd ? L.buf[0] : L.buf[1]);
    tile_ff<LD>(fin, fout, qf, Shape{L.Lx, L.Lz, L.plane}, L.t, local, sbase);
}
template <class LD>
__device__ __forceinline__ void ens_tile(const EnsLattice& L, int local, int s, const StepParamsF& qs, int*) {
    const bool odd = (L.cur + s) & 1;
    const float* fin = (const float*)(odd ? L.buf[1] : L.buf[0]);
    float* fout = (float*)(odd ? L.buf[0] : L.buf[1]);
    StepParamsF q = qs;              // no arrays: stays in registers
    q.Lx = L.Lx;
    q.Lz = L.Lz;
    q.plane = L.plane;
    tile_f32<LD>(fin, fout, q, L.t, local);
}

// The same for the tiles of one work item of the persistent kernel, with the item's pull-base
// tables in shared memory shared across its tiles: an interior tile fills a table only when
// its column differs from the previous tile's (consecutive tiles of one column have the same
// bases), alternating between two tables, so that each fill needs one block barrier and no
// barrier separates the tiles (the fill barrier also orders every thread's use of the other
// table, two fills back, before its refill).  col / cur (block-uniform): the column of the
// current table and its index, -1 / 0 at the start of an item.
template <class LD>
__device__ __forceinline__ void ens_item_tile(const EnsLattice& L, int tl, int s, const StepParamsFF& qf,
                                             int (*tabs)[Q], int& col, int& cur) {
    const bool odd = (L.cur + s) & 1;
    const double* fin = (const double*)(odd ? L.buf[1] : L.buf[0]);
    double* fout = (double*)(odd ? L.buf[0] : L.buf[1]);
    SiteAddr ad;
    bool wall;
    if (tile_is_wall(L.t, tl)) {
        if (!ad.setup(L.Lx, L.Lz, L.plane, L.t, tl, wall)) return;
        site_ff(SrcGlobal<true, LD, true>{fin, ad, tabs[0], 0}, DstSite{fout, ad.dst(), L.plane}, qf);
        return;
    }
    const int x = tile_column(L.t, tl);
    if (x != col) {
        cur ^= 1;
        fill_pull_bases(tabs[cur], x, L.Lx, L.Lz, L.plane);
        __syncthreads();
        col = x;
    }
    if (!ad.setup(L.Lx, L.Lz, L.plane, L.t, tl, wall)) return;
    site_ff(SrcGlobal<false, LD, true>{fin, ad, tabs[cur], ad.z}, DstSite{fout, ad.dst(), L.plane}, qf);
}
// FP32 tiles use no shared table.
template <class LD>
__device__ __forceinline__ void ens_item_tile(const EnsLattice& L, int tl, int s, const StepParamsF& qs,
                                             int (*)[Q], int&, int&) {
    ens_tile<LD>(L, tl, s, qs, nullptr);
}

// Resident blocks per SM requested from the compiler for a tile height of TZ threads.  The
// per-step kernel takes the register budgets of the single-lattice kernels: 32 warps per SM
// for the float-float tile (64 registers, as k_step_ff) and 24 for the FP32 tile (80, as
// k_step_f32).  The persistent kernel, which carries its queue and barrier state through
// every tile, is held to 28 warps per SM (72 registers): more resident warps outweigh the
// spills (measured on the 48-lattice set with one tile per work item: 6,468 -> 6,841 / 6,957
// float-float at 28 / 32 warps and 13,030 -> 15,179 FP32 at 28, against 20 warps at 96
// registers; with 8-tile work items 28 warps are best for both: 7,116 against 6,898 float-float
// at 32 and 7,047 at 24).
template <class P, int TZ>
constexpr int ens_step_min_blocks() { return (std::is_same<P, StepParamsFF>::value ? 1024 : 768) / TZ; }
template <class P, int TZ>
constexpr int ens_persistent_min_blocks() { return 896 / TZ; }

template <class P, int TZ>
__global__ void __launch_bounds__(TZ, ens_step_min_blocks<P, TZ>())
k_ens_step(const EnsLattice* __restrict__ lats, int n, P q, int s) {
    __shared__ int sbase[Q];
    const int b = blockIdx.x;
    const int i = ens_find(lats, n, b);
    const EnsLattice L = lats[i];
    ens_tile<LoadNC>(L, b - L.tile_begin, s, q, sbase);
}

// Spin until *ctr >= need (acquire), the error word is set, or the cycle budget runs out
// (then the error word gets bit 0).  Returns true when the count was reached.
__device__ __forceinline__ bool ens_wait(const unsigned int* ctr, unsigned int need, unsigned int* err,
                                         long long limit) {
    const long long t0 = clock64();
    for (;;) {
        unsigned int v;
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(ctr) : "memory");
        if (v >= need) return true;
        if (*(volatile unsigned int*)err) return false;
        if (clock64() - t0 > limit) {
            atomicOr(err, 1u);
            return false;
        }
        __nanosleep(64);
    }
}

// extra_wait > 0 raises every barrier target so that it can never be met (a test of the
// bounded wait: the launch must end with the error word set, not hang).
// Per CTA, thread 0 fetches the next work item while the current tile computes, and keeps
// the last completion count it saw for each lattice (up to ENS_CACHE lattices) so that the
// many tiles of one (lattice, step) need a single acquire load of the global counter.  It
// also finds the item's lattice and leaves its record and tile range in shared memory, which
// the tiles read from there: a copy in every thread's registers, live across the item's
// tiles, had raised the spill at 72 registers from 40 to 128 bytes (float-float) and from 56
// to 140 (FP32); reading it from shared memory took the 48-lattice set from 7,130 to 7,366
// MLUPS float-float and from 17,522 to 19,060 FP32 (200 steps; per-step launches 7,420 and
// 18,490, which the same change left unchanged).  The tiles of an item share their pull-base
// tables (ens_item_tile) and are not separated by block barriers: FP32 19,200 -> 19,530 MLUPS,
// float-float 7,438 -> 7,443 (one barrier per tile with a refill for every tile: 19,520 and
// 7,387).
constexpr int ENS_CACHE = 64;

template <class P, int TZ>
__global__ void __launch_bounds__(TZ, ens_persistent_min_blocks<P, TZ>())
k_ens_persistent(const EnsLattice* __restrict__ lats, int n, P q, int nsteps, int total_items,
                 EnsControl* ctl, unsigned int* done, long long spin_limit, unsigned int extra_wait) {
    __shared__ int tabs[2][Q];                 // pull-base tables of the item's tiles
    __shared__ unsigned int s_item, s_next;
    __shared__ int s_ok;
    __shared__ unsigned int s_seen[ENS_CACHE];
    __shared__ EnsLattice s_L;                 // the item's lattice record
    __shared__ int s_i, s_s, s_t0, s_t1;        // its lattice, step and tile range
    const unsigned int total = (unsigned int)nsteps * (unsigned int)total_items;
    for (int i = threadIdx.x; i < ENS_CACHE; i += blockDim.x) s_seen[i] = 0u;
    if (threadIdx.x == 0) s_next = atomicAdd(&ctl->queue, 1u);
    __syncthreads();
    for (;;) {
        if (threadIdx.x == 0) {
            const unsigned int it = s_next;
            int ok = 1;
            if (it < total) {
                s_next = atomicAdd(&ctl->queue, 1u);        // next item, fetched ahead
                const int s = (int)(it / (unsigned int)total_items);
                const int j = (int)(it % (unsigned int)total_items);
                const int i = ens_find_item(lats, n, j);
                if (s > 0 || extra_wait) {
                    const unsigned int need = (unsigned int)s * (unsigned int)lats[i].ntiles + extra_wait;
                    if (i >= ENS_CACHE || s_seen[i] < need) {
                        ok = ens_wait(&done[i], need, &ctl->err, spin_limit);
                        if (ok && i < ENS_CACHE) s_seen[i] = need;
                    }
                }
            }
            s_item = it;
            s_ok = ok;
            if (it < total && ok) {
                const int s = (int)(it / (unsigned int)total_items);
                const int j = (int)(it % (unsigned int)total_items);
                const int i = ens_find_item(lats, n, j);
                constexpr bool FF = std::is_same<P, StepParamsFF>::value;
                constexpr int KT = ens_item(FF), KW = ens_wall_item(FF);
                s_L = lats[i];
                s_i = i;
                s_s = s;
                const int local = j - s_L.item_begin, nw = s_L.t.nwall, nwi = (nw + KW - 1) / KW;
                s_t0 = local < nwi ? local * KW : nw + (local - nwi) * KT;
                s_t1 = local < nwi ? min(s_t0 + KW, nw) : min(s_t0 + KT, s_L.ntiles);
            }
        }
        __syncthreads();
        if (s_item >= total || !s_ok) break;
        const int s = s_s, t0 = s_t0, t1 = s_t1;
        int col = -1, cur = 0;
        for (int tl = t0; tl < t1; tl++) ens_item_tile<LoadCG>(s_L, tl, s, q, tabs, col, cur);
        __syncthreads();   // all stores of the item issued; s_item, s_L and the tables may be reused
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(&done[s_i], (unsigned int)(t1 - t0));
        }
    }
}

}  // namespace lbm
