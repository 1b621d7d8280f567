// probe.cuh -- throughput of B300's FP64 pipe, the second roof of the FP64-storage kernels:
// their DRAM bytes per site set the HBM roof, their FP64 instructions per site (one FMA per
// population and a few conversions in the float-float step) against this rate set the other.
#pragma once
#include "common.cuh"

namespace lbm {

constexpr int PROBE_CHAINS = 8;          // independent FMA chains per thread (hides the latency)
constexpr int PROBE_THREADS = 256;
constexpr int PROBE_BLOCKS_PER_SM = 8;   // 2,048 threads per SM, the SM's limit

// Each thread runs PROBE_CHAINS chains a <- a m + c of iters FMAs each.  With 0 < m < 1 the
// values move towards c / (1 - m) and stay normal, so no operand is ever subnormal, infinite or
// NaN.  The chains' sum decides whether *out is written (practically never), which keeps every
// FMA live without a store per thread.
__global__ void __launch_bounds__(PROBE_THREADS)
k_probe_dfma(int iters, double m, double c, double* __restrict__ out) {
    double a[PROBE_CHAINS];
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; k++) a[k] = 1.0 + 1e-3 * (threadIdx.x + k);
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int k = 0; k < PROBE_CHAINS; k++) a[k] = fma(a[k], m, c);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; k++) s += a[k];
    if (s == -1.0) out[0] = s;           // the chains stay positive: never taken
}

}  // namespace lbm
