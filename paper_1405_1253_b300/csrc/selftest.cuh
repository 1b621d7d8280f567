// selftest.cuh -- device check that the packed two-lane float-float operations (ffx2, ff.cuh and
// adjoint_ff.cuh) give, in each lane, the bits of the scalar operation they stand for.  The step
// and adjoint kernels rely on this to be bit-identical to their scalar forms.
#pragma once
#include "adjoint_ff.cuh"

namespace lbm {

// Counter-based 64-bit mix (splitmix64 finaliser) of (seed, index, stream).
__device__ __forceinline__ unsigned long long st_mix(unsigned long long seed, unsigned long long i, unsigned s) {
    unsigned long long z = seed + 0x9E3779B97F4A7C15ull * (i * 16 + s + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// A normalised float-float value of either sign with |hi| in [2^(e0), 2^(e0 + span)).
__device__ __forceinline__ ff st_value(unsigned long long seed, unsigned long long i, unsigned s, int e0, int span) {
    const unsigned long long z = st_mix(seed, i, s);
    const unsigned mant = (unsigned)(z & 0x7FFFFFu);
    const int e = e0 + (int)((z >> 23) % (unsigned long long)span);
    const float hi = __uint_as_float(((unsigned)(e + 127) << 23) | mant | (unsigned)((z >> 40) & 1u) << 31);
    // lo: |lo| <= ulp(hi)/2, any sign
    const float r = (float)(int)((z >> 41) & 0xFFFFFu) * 0x1p-20f - 0.5f;
    return ff_renorm(ff{hi, hi * r * 0x1p-24f});
}

__device__ __forceinline__ int st_diff(const ff& x, const ff& y) {
    return (__float_as_uint(x.hi) != __float_as_uint(y.hi)) + (__float_as_uint(x.lo) != __float_as_uint(y.lo));
}
__device__ __forceinline__ int st_diff2(const ffx2& p, const ff& lane0, const ff& lane1) {
    return st_diff(ffx2_lane0(p), lane0) + st_diff(ffx2_lane1(p), lane1);
}

// For each of n index pairs: operands a (|a| ~ 2^-2 .. 2^6), b (|b| below |a| / 16, so that
// the "big" forms' ordering holds also for 4 b), an FP32 factor f and a three-term constant c;
// every packed operation against its scalar form in both lanes.  Adds the number of
// differing words to *bad.
__global__ void k_selftest_ffx2(int n, unsigned long long seed, unsigned long long* bad) {
    int count = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        ff a[2], b[2];
        float f[2];
        for (int k = 0; k < 2; k++) {
            const unsigned long long j = 2ull * i + k;
            a[k] = st_value(seed, j, 0, -2, 8);
            b[k] = st_value(seed, j, 1, -14, 8);
            f[k] = st_value(seed, j, 2, -3, 6).hi;
        }
        const ff cc = st_value(seed, i, 3, -1, 2);
        const ff3 c{cc.hi, cc.lo, cc.lo * 0x1p-23f};
        const ffx2 A{x2_pack(a[0].hi, a[1].hi), x2_pack(a[0].lo, a[1].lo)};
        const ffx2 B{x2_pack(b[0].hi, b[1].hi), x2_pack(b[0].lo, b[1].lo)};
        const f32x2 F = x2_pack(f[0], f[1]);
        count += st_diff2(ffx2_two_sum(A.hi, B.hi), two_sum(a[0].hi, b[0].hi), two_sum(a[1].hi, b[1].hi));
        count += st_diff2(ffx2_renorm(A), ff_renorm(a[0]), ff_renorm(a[1]));
        count += st_diff2(ffx2_add_big_u(A, B), ff_add_big_u(a[0], b[0]), ff_add_big_u(a[1], b[1]));
        count += st_diff2(ffx2_sub_big_u(A, B), ff_add_big_u(a[0], ff_neg(b[0])), ff_add_big_u(a[1], ff_neg(b[1])));
        count += st_diff2(ffx2_mul_u(A, B), ff_mul_u(a[0], b[0]), ff_mul_u(a[1], b[1]));
        count += st_diff2(ffx2_mul_f_u(A, F), ff_mul_f_u(a[0], f[0]), ff_mul_f_u(a[1], f[1]));
        count += st_diff2(ffx2_add_big_u_x4(A, B), ff_add_big_u_x4(a[0], b[0]), ff_add_big_u_x4(a[1], b[1]));
        count += st_diff2(ffx2_add_big_u_x2(A, B), ff_add_big_u_x2(a[0], b[0]), ff_add_big_u_x2(a[1], b[1]));
        count += st_diff2(ffx2_add_u(A, B), ff_add_u(a[0], b[0]), ff_add_u(a[1], b[1]));
        count += st_diff2(ffx2_add_u(B, A), ff_add_u(b[0], a[0]), ff_add_u(b[1], a[1]));
        count += st_diff2(ffx2_sub_u(A, B), ff_add_u(a[0], ff_neg(b[0])), ff_add_u(a[1], ff_neg(b[1])));
        count += st_diff2(ffx2_sub_u(B, A), ff_add_u(b[0], ff_neg(a[0])), ff_add_u(b[1], ff_neg(a[1])));
        count += st_diff2(ffx2_mul_c3_u(A, c), ff_mul_c3_u(a[0], c), ff_mul_c3_u(a[1], c));
        count += st_diff2(ffx2_scale(A, 2.0f), ff_mul_pow2(a[0], 2.0f), ff_mul_pow2(a[1], 2.0f));
        count += st_diff2(ffx2_both(a[0]), a[0], a[0]);
    }
    if (count) atomicAdd(bad, (unsigned long long)count);
}

}  // namespace lbm
