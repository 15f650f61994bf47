// Double-float ("df") arithmetic on the FP32 pipe: a value is the
// unevaluated sum hi + lo of two binary32 numbers (about 48 significant
// bits).  Error-free transformations: Knuth's TwoSum and Dekker's Fast2Sum
// for sums, the exact error of a product from one fused multiply-add; a sum
// adds the high parts exactly, adds the low parts and renormalises, a product
// takes the high parts' product with its error and the two cross terms.  All
// operations are round-to-nearest intrinsics, so the compiler neither fuses
// nor reorders them.  Conversions between binary64 and hi/lo pairs use
// integer instructions (the FP64 unit's conversions are slow on this GPU).
// Used where FP64 instructions bound a kernel but ~1e-14 relative accuracy
// is enough: the mixed form's forward transform and the CIC deposit.
#pragma once

#include <cuda_runtime.h>

namespace pp {

struct df {
    float hi, lo;
};

__device__ __forceinline__ df df_norm(float s, float e) {   // Fast2Sum
    const float h = __fadd_rn(s, e);
    return {h, __fsub_rn(e, __fsub_rn(h, s))};
}
__device__ __forceinline__ df df_add(df a, df b) {
    const float s = __fadd_rn(a.hi, b.hi);
    const float v = __fsub_rn(s, a.hi);
    float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, v)), __fsub_rn(b.hi, v));   // TwoSum error
    e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    return df_norm(s, e);
}
__device__ __forceinline__ df df_neg(df a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }
__device__ __forceinline__ df df_negif(df a, bool c) { return c ? df_neg(a) : a; }
// a b + c
__device__ __forceinline__ df df_fma(df a, df b, df c) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);   // exact error of the product
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    const float s = __fadd_rn(p, c.hi);
    const float v = __fsub_rn(s, p);
    float f = __fadd_rn(__fsub_rn(p, __fsub_rn(s, v)), __fsub_rn(c.hi, v));
    f = __fadd_rn(f, __fadd_rn(e, c.lo));
    return df_norm(s, f);
}
__device__ __forceinline__ df df_mul(df a, df b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return df_norm(p, e);
}

// Biased binary64 exponent field of x (0 for zero and subnormals).
__device__ __forceinline__ int exp_field(double x) { return (__double2hiint(x) >> 20) & 0x7ff; }

// x 2^(1023 - emax) split into hi + lo (hi: the leading 24 bits; lo: the next
// bits, rounded to 24), with integer instructions and one conversion.
__device__ __forceinline__ df split_scaled(double x, int emax) {
    const unsigned h = (unsigned)__double2hiint(x), l = (unsigned)__double2loint(x);
    const int e = (int)((h >> 20) & 0x7ffu);
    const int fe = e - emax + 127;   // binary32 exponent field after scaling
    if (e == 0 || fe <= 0) return {0.f, 0.f};
    const unsigned sign = h & 0x80000000u;
    const unsigned mh = h & 0xfffffu;                               // mantissa bits 51..32
    const float hi = __uint_as_float(sign | ((unsigned)fe << 23) | (mh << 3) | (l >> 29));
    // remaining mantissa bits 28..0, worth 2^(fe - 127 - 52) each
    const unsigned r = l & 0x1fffffffu;
    float lo = 0.f;
    const int le = fe - 52;   // binary32 exponent field of 2^(fe - 127 - 52)
    if (r != 0 && le > 0) {
        lo = __fmul_rn(__uint2float_rn(r), __uint_as_float((unsigned)le << 23));
        if (sign) lo = -lo;
    }
    return {hi, lo};
}

// Exact binary64 value of a binary32 number times 2^s (s >= -1000).
__device__ __forceinline__ double f32_times_pow2(float f, int s) {
    const unsigned b = __float_as_uint(f);
    const int e = (int)((b >> 23) & 0xffu);
    if (e == 0) return 0.0;   // zero (the transforms produce no binary32 subnormals of interest)
    const unsigned sign = b & 0x80000000u, m = b & 0x7fffffu;
    const int ed = e - 127 + 1023 + s;
    if (ed <= 0) return __hiloint2double((int)sign, 0);
    if (ed >= 0x7ff) return __hiloint2double((int)(sign | 0x7ff00000u), 0);   // overflow: infinity
    return __hiloint2double((int)(sign | ((unsigned)ed << 20) | (m >> 3)), (int)(m << 29));
}
// (hi + lo) 2^s in binary64.
__device__ __forceinline__ double to_double(df a, int s) { return f32_times_pow2(a.hi, s) + f32_times_pow2(a.lo, s); }

}  // namespace pp
