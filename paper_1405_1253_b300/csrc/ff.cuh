// ff.cuh -- float-float ("double-FP32") arithmetic on the FP32 pipes, and exact
// conversions between binary64 bit patterns, float-float pairs and 64-bit fixed point
// done with integer instructions only (B300 runs every FP64 conversion at the FP64 rate).
//
// A value is the unevaluated sum hi + lo of two FP32 numbers with |lo| <= ulp(hi)/2,
// carrying a 48-bit significand.  The building blocks are the error-free transformations
// of Knuth (two-sum) and Dekker (fast two-sum, valid for |a| >= |b|) and the FMA form of
// the exact product a*b = p + e, e = fma(a, b, -p).  The "u" (unnormalised) variants
// below skip the final renormalisation: their result keeps |lo| a few units of 2^-24
// below |hi|, which every consumer here tolerates; their error is a few units of 2^-48
// relative to the operands.
//
// The leading products are written __fmul_rn: the compiler may not contract them into a
// following add (an FMA there would round the sum of the exact product instead of the sum of
// the rounded one the error terms describe), so the transformations stay exact and the
// results do not depend on how a kernel's registers and schedule come out.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

namespace lbm {

struct ff {
    float hi, lo;
};

__device__ __forceinline__ ff ff_make(float hi, float lo) { return ff{hi, lo}; }

__device__ __forceinline__ ff fast_two_sum(float a, float b) {   // requires |a| >= |b|
    const float s = a + b;
    return ff{s, b - (s - a)};
}

__device__ __forceinline__ ff two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    return ff{s, (a - (s - bb)) + (b - bb)};
}

__device__ __forceinline__ ff ff_neg(ff a) { return ff{-a.hi, -a.lo}; }

// General sum (no ordering assumed), renormalised.
__device__ __forceinline__ ff ff_add(ff a, ff b) {
    const ff s = two_sum(a.hi, b.hi);
    return fast_two_sum(s.hi, s.lo + (a.lo + b.lo));
}
__device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, ff_neg(b)); }

// General sum, not renormalised (|lo| stays within a few ulps of hi).
__device__ __forceinline__ ff ff_add_u(ff a, ff b) {
    const ff s = two_sum(a.hi, b.hi);
    return ff{s.hi, s.lo + (a.lo + b.lo)};
}

// Sum when |a| >= |b| is known, not renormalised.
__device__ __forceinline__ ff ff_add_big_u(ff a, ff b) {
    const float s = a.hi + b.hi;
    const float e = b.hi - (s - a.hi);
    return ff{s, e + (a.lo + b.lo)};
}

// Product, not renormalised.
__device__ __forceinline__ ff ff_mul_u(ff a, ff b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return ff{p, e};
}
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
    const ff t = ff_mul_u(a, b);
    return fast_two_sum(t.hi, t.lo);
}

// Product with an FP32 number (exact small integers in particular), not renormalised.
__device__ __forceinline__ ff ff_mul_f_u(ff a, float b) {
    const float p = __fmul_rn(a.hi, b);
    float e = fmaf(a.hi, b, -p);
    e = fmaf(a.lo, b, e);
    return ff{p, e};
}

__device__ __forceinline__ ff ff_renorm(ff a) { return fast_two_sum(a.hi, a.lo); }

// a + 4 b when |a| >= |4 b| is known, not renormalised (4 b is exact, so the fast two-sum
// error 4 b.hi - (s - a.hi) comes out of one FMA).
__device__ __forceinline__ ff ff_add_big_u_x4(ff a, ff b) {
    const float s = fmaf(4.0f, b.hi, a.hi);
    const float e = fmaf(4.0f, b.hi, -(s - a.hi));
    return ff{s, e + fmaf(4.0f, b.lo, a.lo)};
}

// A constant held as three FP32 terms (|hi + lo + lo2 - c| below 2^-70 |c|): products with
// it carry no systematic error from the constant's representation.
struct ff3 {
    float hi, lo, lo2;
};
__device__ __forceinline__ ff3 ff3_of(const float (&t)[3]) { return ff3{t[0], t[1], t[2]}; }

// a * c, renormalised (the a.lo * c.lo term, ~2^-48 relative, is dropped as in ff_mul).
__device__ __forceinline__ ff ff_mul_c3(ff a, const ff3& c) {
    const float p = __fmul_rn(a.hi, c.hi);
    float e = fmaf(a.hi, c.hi, -p);
    e = fmaf(a.hi, c.lo2, e);
    e = fmaf(a.hi, c.lo, e);
    e = fmaf(a.lo, c.hi, e);
    return fast_two_sum(p, e);
}

// Product with a power of two (exact).
__device__ __forceinline__ ff ff_mul_pow2(ff a, float p2) { return ff{a.hi * p2, a.lo * p2}; }

// 1 / a for a normalised a (|a.hi| a normal FP32 number, 1/a.hi too): the FP32 reciprocal y
// refined by one Newton step that keeps the second-order term, 1/a = y (1 + e + e^2 + ...)
// with e = 1 - a y (two FMAs; |e| ~ 2^-23 so e carries ~2^-47 absolute error), then
// renormalised.  Relative error about 2^-47.
__device__ __forceinline__ ff ff_rcp(ff a) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(a.hi));
    float e = fmaf(-a.hi, y, 1.0f);
    e = fmaf(-a.lo, y, e);
    return fast_two_sum(y, __fmul_rn(y, fmaf(e, e, e)));
}

// ---------------------------------------------------------------------------------
// binary64 bit pattern (H = high word, L = low word) -> float-float.
// hi = x rounded to 24 significant bits (half-up on the magnitude, by adding half of the
// dropped 29-bit field to the pattern); lo = x - hi, whose 29-bit integer significand is
// converted to FP32 (rounded) and scaled by 2^(E-1075).  Error <= 2^-49 |x|.
// Valid for 2^-74 <= |x| < 2^127; smaller magnitudes (and zero) give 0.
// ---------------------------------------------------------------------------------
__device__ __forceinline__ ff bits_to_ff(uint32_t H, uint32_t L) {
    const uint32_t sgn = H & 0x80000000u;
    const uint32_t Ha = H & 0x7FFFFFFFu;
    const uint64_t m = ((((uint64_t)Ha) << 32) | L) + 0x10000000ull;
    const uint32_t hb = (uint32_t)(m >> 29) - 0xC0000000u;        // exponent bias 1023 -> 127
    const int32_t rem = ((int32_t)(L << 3)) >> 3;                   // x - hi in units of 2^(E-1075)
    // FP32 bits of 2^(E-1075): (E - 948) << 23, i.e. E * 2^23 - 948 * 2^23 modulo 2^32
    const uint32_t sb = (Ha >> 20) * 0x00800000u + 0x26000000u;
    const bool ok = Ha >= (949u << 20);                              // |x| >= 2^-74
    const float hi = __uint_as_float(ok ? (hb | sgn) : 0u);
    // the scale is selected, not rem: for |x| < 2^-74 the pattern sb is meaningless (in some
    // binades an infinity, whose product with 0 would be a NaN)
    const float lo = (float)rem * __uint_as_float(ok ? (sb | sgn) : 0u);
    return ff{hi, lo};
}

// binary64 bit pattern -> signed 64-bit fixed point with unit 2^-60 (exact for
// 2^-8 <= |x| < 4 and x >= 0; bits below 2^-60 are dropped for smaller |x|).  A negative x
// comes out in one's complement, i.e. one unit (2^-60) below its value, which keeps the
// sign handling to two XORs; |x| >= 4 is not representable.
__device__ __forceinline__ int64_t bits_to_fix60(uint32_t H, uint32_t L) {
    const uint32_t n = 1025u - ((H << 1) >> 21);                    // right shift of mant << 10
    // significand << 10 as two words: top 21 bits + the low word's top 22 bits, low word << 10
    const uint32_t mh = __funnelshift_l(L, (H & 0x000FFFFFu) | 0x00100000u, 10);
    const uint32_t ml = L << 10;
    // (mh:ml) >> n in two clamped funnel shifts: the first moves min(n, 32) bits, the
    // second the rest (n >= 64 leaves nothing)
    const int32_t n2 = max((int32_t)n - 32, 0);
    const uint32_t vl0 = __funnelshift_rc(ml, mh, n);
    const uint32_t vl = __funnelshift_rc(vl0, 0u, (uint32_t)n2);
    const uint32_t vh = __funnelshift_rc(mh, 0u, n);
    const uint32_t s = (uint32_t)((int32_t)H >> 31);
    return (int64_t)((((uint64_t)(vh ^ s)) << 32) | (vl ^ s));
}


// Normalised float-float (|lo| <= ulp(hi)/2, hi a normal FP32 number >= 2^-75 in
// magnitude) -> binary64, rounded to nearest.
// The pattern of (double)hi is built from the FP32 fields; lo is added as an integer count
// of binary64 ulps of hi's binade.  When lo points towards zero the count is taken in the
// ulps of the binade of hi's predecessor, which differs from hi's only when hi is a power
// of two, exactly the case where the sum falls into the binade below.
__device__ __forceinline__ double ff_to_double_bits(ff a) {
    const uint32_t hb = __float_as_uint(a.hi);
    const uint32_t ha = hb & 0x7FFFFFFFu;
    const uint32_t sgn = hb & 0x80000000u;
    const uint32_t PH = (ha >> 3) + (896u << 20) + sgn;
    const uint32_t PL = ha << 29;
    const uint32_t m = (uint32_t)((int32_t)(__float_as_uint(a.lo) ^ hb) >> 31);   // 0 or ~0u
    // scale 2^(52 - e) carrying hi's sign: FP32 bits (306 - E8) << 23 (+ sign)
    const uint32_t sbits = 0x99000000u - ((hb + m) & 0x7F800000u) + sgn;
    const int32_t k = __float2int_rn(a.lo * __uint_as_float(sbits));
    const uint64_t P = ((((uint64_t)PH) << 32) | PL) + (uint64_t)(int64_t)k;
    return __longlong_as_double((long long)P);
}

// ---------------------------------------------------------------------------------
// Two float-float values in the lanes of packed FP32 registers (B300's f32x2 add, sub and
// mul: one instruction for both lanes).  Each lane takes exactly the operations of the
// scalar functions above, so results are bit-identical to them.  The FMAs of the error
// terms stay scalar (two per pair of lanes): a packed FMA takes as long as two scalar ones,
// and the scalar form negates its addend for free, which the packed one cannot.
// ---------------------------------------------------------------------------------
typedef unsigned long long f32x2;       // lane 0 in the low word, lane 1 in the high word

__device__ __forceinline__ f32x2 x2_pack(float l0, float l1) {
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(l0), "f"(l1));
    return r;
}
// (the unpack writes both lanes; the other one goes to a scoped PTX register)
__device__ __forceinline__ float x2_lane0(f32x2 v) {
    float l0;
    asm("{\n\t.reg .f32 t;\n\tmov.b64 {%0, t}, %1;\n\t}" : "=f"(l0) : "l"(v));
    return l0;
}
__device__ __forceinline__ float x2_lane1(f32x2 v) {
    float l1;
    asm("{\n\t.reg .f32 t;\n\tmov.b64 {t, %0}, %1;\n\t}" : "=f"(l1) : "l"(v));
    return l1;
}
__device__ __forceinline__ f32x2 x2_add(f32x2 a, f32x2 b) {
    f32x2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f32x2 x2_sub(f32x2 a, f32x2 b) {
    f32x2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f32x2 x2_mul(f32x2 a, f32x2 b) {
    f32x2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
// fmaf on each lane (a * b + c)
__device__ __forceinline__ f32x2 x2_fma(f32x2 a, f32x2 b, f32x2 c) {
    return x2_pack(fmaf(x2_lane0(a), x2_lane0(b), x2_lane0(c)), fmaf(x2_lane1(a), x2_lane1(b), x2_lane1(c)));
}
// a * b - p on each lane: the error of the rounded product p = a * b
__device__ __forceinline__ f32x2 x2_prod_err(f32x2 a, f32x2 b, f32x2 p) {
    return x2_pack(fmaf(x2_lane0(a), x2_lane0(b), -x2_lane0(p)), fmaf(x2_lane1(a), x2_lane1(b), -x2_lane1(p)));
}

struct ffx2 {
    f32x2 hi, lo;
};
__device__ __forceinline__ ffx2 ffx2_both(ff a) { return ffx2{x2_pack(a.hi, a.hi), x2_pack(a.lo, a.lo)}; }
__device__ __forceinline__ ff ffx2_lane0(const ffx2& a) { return ff{x2_lane0(a.hi), x2_lane0(a.lo)}; }
__device__ __forceinline__ ff ffx2_lane1(const ffx2& a) { return ff{x2_lane1(a.hi), x2_lane1(a.lo)}; }

__device__ __forceinline__ ffx2 ffx2_two_sum(f32x2 a, f32x2 b) {             // two_sum
    const f32x2 s = x2_add(a, b), bb = x2_sub(s, a);
    return ffx2{s, x2_add(x2_sub(a, x2_sub(s, bb)), x2_sub(b, bb))};
}
__device__ __forceinline__ ffx2 ffx2_add_u(const ffx2& a, const ffx2& b) {       // ff_add_u
    const ffx2 s = ffx2_two_sum(a.hi, b.hi);
    return ffx2{s.hi, x2_add(s.lo, x2_add(a.lo, b.lo))};
}
__device__ __forceinline__ ffx2 ffx2_add(const ffx2& a, const ffx2& b) {         // ff_add
    const ffx2 s = ffx2_two_sum(a.hi, b.hi);
    const f32x2 t = x2_add(s.lo, x2_add(a.lo, b.lo));
    const f32x2 h = x2_add(s.hi, t);
    return ffx2{h, x2_sub(t, x2_sub(h, s.hi))};
}
__device__ __forceinline__ ffx2 ffx2_renorm(const ffx2& a) {                  // ff_renorm
    const f32x2 s = x2_add(a.hi, a.lo);
    return ffx2{s, x2_sub(a.lo, x2_sub(s, a.hi))};
}
__device__ __forceinline__ ffx2 ffx2_add_big_u(const ffx2& a, const ffx2& b) {   // ff_add_big_u
    const f32x2 s = x2_add(a.hi, b.hi);
    return ffx2{s, x2_add(x2_sub(b.hi, x2_sub(s, a.hi)), x2_add(a.lo, b.lo))};
}
// ff_add_big_u(a, ff_neg(b)), with the negation folded into subtractions
__device__ __forceinline__ ffx2 ffx2_sub_big_u(const ffx2& a, const ffx2& b) {
    const f32x2 s = x2_sub(a.hi, b.hi);
    return ffx2{s, x2_add(x2_sub(x2_sub(a.hi, s), b.hi), x2_sub(a.lo, b.lo))};
}
__device__ __forceinline__ ffx2 ffx2_mul_u(const ffx2& a, const ffx2& b) {       // ff_mul_u
    const f32x2 p = x2_mul(a.hi, b.hi);
    f32x2 e = x2_prod_err(a.hi, b.hi, p);
    e = x2_fma(a.hi, b.lo, e);
    e = x2_fma(a.lo, b.hi, e);
    return ffx2{p, e};
}
__device__ __forceinline__ ffx2 ffx2_mul_f_u(const ffx2& a, f32x2 b) {           // ff_mul_f_u
    const f32x2 p = x2_mul(a.hi, b);
    return ffx2{p, x2_fma(a.lo, b, x2_prod_err(a.hi, b, p))};
}
// ff_mul_c3 with the constant c0 in lane 0 and c1 in lane 1
__device__ __forceinline__ ffx2 ffx2_mul_c3(const ffx2& a, const ff3& c0, const ff3& c1) {
    const f32x2 chi = x2_pack(c0.hi, c1.hi);
    const f32x2 p = x2_mul(a.hi, chi);
    f32x2 e = x2_prod_err(a.hi, chi, p);
    e = x2_fma(a.hi, x2_pack(c0.lo2, c1.lo2), e);
    e = x2_fma(a.hi, x2_pack(c0.lo, c1.lo), e);
    e = x2_fma(a.lo, chi, e);
    const f32x2 s = x2_add(p, e);
    return ffx2{s, x2_sub(e, x2_sub(s, p))};
}
__device__ __forceinline__ ffx2 ffx2_add_big_u_x4(const ffx2& a, const ffx2& b) {   // ff_add_big_u_x4
    const f32x2 four = x2_pack(4.0f, 4.0f);
    const f32x2 s = x2_fma(four, b.hi, a.hi);
    return ffx2{s, x2_add(x2_fma(four, b.hi, x2_sub(a.hi, s)), x2_fma(four, b.lo, a.lo))};
}

}  // namespace lbm
