// Float-float ("df64") arithmetic for FP64-accurate results on the FP32 pipes.
//
// GB300 runs FP64 at 1/64 of its FP32 rate, so FP64-accurate sums and
// products are formed from pairs of floats (h, l), value h + l, with the
// error-free transformations of Knuth (TwoSum), Dekker (FastTwoSum) and the
// FMA-based TwoProd.  A normalised pair carries about 48 significand bits.
// Every helper uses the _rn intrinsics so the compiler cannot contract or
// reorder the compensated operations.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace soptx {

struct df {
    float h, l;
};

__device__ __forceinline__ df df_make(float h, float l) { return df{h, l}; }

// a + b = s + e exactly (Knuth TwoSum)
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// a + b = s + e exactly when |a| >= |b| or a == 0 (Dekker FastTwoSum)
__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}

// Sum of two pairs; the error is below about 2^-46 (|a| + |b|).
__device__ __forceinline__ df df_add(df a, df b)
{
    float s, e;
    two_sum(a.h, b.h, s, e);
    float t = __fadd_rn(__fadd_rn(a.l, b.l), e);
    df r;
    fast_two_sum(s, t, r.h, r.l);
    return r;
}

__device__ __forceinline__ df df_neg(df a) { return df{-a.h, -a.l}; }

// Unnormalised product (h, l) of two pairs: h = round(a.h b.h) and l gathers
// the rounding error of that product (exact, by FMA) and the cross terms.
__device__ __forceinline__ df df_mul_raw(df a, df b)
{
    float p = __fmul_rn(a.h, b.h);
    float e = __fmaf_rn(a.h, b.h, -p);
    e = __fmaf_rn(a.h, b.l, e);
    e = __fmaf_rn(a.l, b.h, e);
    return df{p, e};
}

__device__ __forceinline__ df df_mul(df a, df b)
{
    df r = df_mul_raw(a, b);
    df o;
    fast_two_sum(r.h, r.l, o.h, o.l);
    return o;
}

// Split a double into a normalised pair (FP64 pipe; used outside hot loops).
__device__ __forceinline__ df df_from_double(double x)
{
    float h = __double2float_rn(x);
    float l = __double2float_rn(x - (double)h);
    return df{h, l};
}

// Out-of-line rare paths: keeping them as real calls stops the compiler from
// if-converting them into FP64-pipe work on every element of a hot loop.
static __device__ __noinline__ df df_from_double_slow(double x) { return df_from_double(x); }

// Split a double into a pair with integer operations (no FP64 pipe): h keeps
// the leading 24 significand bits (truncated), l the remaining 29 bits
// rounded to 24.  |x - (h + l)| <= 2^-47 |x|.  Magnitudes outside
// [2^-74, 2^127] and zero take the FP64 pipe.
__device__ __forceinline__ df df_split(double x)
{
    const uint64_t b = (uint64_t)__double_as_longlong(x);
    const uint32_t hi = (uint32_t)(b >> 32), lo = (uint32_t)b;
    const uint32_t E = (hi >> 20) & 0x7ffu;
    if (E < 949u || E > 1150u) return df_from_double_slow(x);
    const uint32_t sign = hi & 0x80000000u;
    const uint32_t hb = sign | ((E - 896u) << 23) | ((hi & 0x000fffffu) << 3) | (lo >> 29);
    const float scale = __uint_as_float(((E - 948u) << 23) | sign);   // +-2^(E - 1075)
    const float l = __fmul_rn(__uint2float_rn(lo & 0x1fffffffu), scale);
    return df{__uint_as_float(hb), l};
}

// df_split with exact zeros (and values below 2^-1022) mapped to (0, 0)
// without the FP64 route, for inputs where zeros are common.
__device__ __forceinline__ df df_split_z(double x)
{
    const uint32_t hi = (uint32_t)(__double_as_longlong(x) >> 32);
    if (((hi >> 20) & 0x7ffu) == 0u) return df{0.f, 0.f};
    return df_split(x);
}

// FP64 value of p + e, where p = round(a b) and e carries the product's
// rounding error and cross terms (|e| <= 8 ulp(p)), built from the bit
// patterns with integer operations: the double of p is exact (widen the
// exponent, shift the mantissa); e is scaled so that one unit is 2^6 ulps of
// that double, rounded to an integer (cvt.rni), and added to the 64-bit
// pattern.  The result is within 2^-46 |p| of p + e.  Below a power of two the
// lower binade has half the ulp, hence the doubled step.  For |p| < 2^-81
// (denormal p included) p and e are first scaled by 2^96, exactly, and the
// exponent is lowered by 96 again; p = 0 gives a signed zero.  No FP64
// instruction and no out-of-line path, so the conversion costs a hot loop no
// registers across a call.
__device__ __forceinline__ double df_to_double(float p, float e)
{
    const bool small = (__float_as_uint(p) & 0x7f800000u) < (46u << 23);
    const float f = small ? 0x1p96f : 1.0f;
    const uint32_t hb = __float_as_uint(__fmul_rn(p, f));
    const float es = __fmul_rn(e, f);
    const uint32_t sign = hb & 0x80000000u;
    const uint32_t mag = hb & 0x7fffffffu;
    const uint32_t hi = mag ? (sign | ((mag >> 3) + (small ? 0x32000000u : 0x38000000u))) : sign;
    const uint32_t lo = mag << 29;
    // scale = 2^(46 - E) with p's sign, E the unbiased exponent of the (scaled) p
    const uint32_t sbits = ((300u << 23) - (mag & 0x7f800000u)) | sign;
    int32_t ci = __float2int_rn(__fmul_rn(es, __uint_as_float(sbits)));
    if ((mag & 0x007fffffu) == 0u && ci < 0) ci *= 2;       // just below a power of two
    const uint64_t bits = (((uint64_t)hi << 32) | lo) + (uint64_t)((int64_t)ci * 64);
    return __longlong_as_double((long long)bits);
}

// The value of df_to_double with integer operations and two FP32 multiplies
// only (no out-of-line path), times 2^k where bias = 0x38000000 + (k << 20)
// (the FP32-to-FP64 exponent rebias plus k).  Valid for |p| < 2^84 and any
// exponent of p: the correction scale 2^(46 - E) is applied as 2^64 * 2^(-18 - E),
// both representable for E >= -126.  p = 0 gives a signed zero (e must be 0);
// a denormal p gives a value within 2^-125 * 2^k of (p + e) 2^k.
__device__ __forceinline__ double df_to_double_biased(float p, float e, uint32_t bias)
{
    const uint32_t hb = __float_as_uint(p);
    const uint32_t sign = hb & 0x80000000u;
    const uint32_t mag = hb & 0x7fffffffu;
    const uint32_t hi = mag ? (sign | ((mag >> 3) + bias)) : sign;
    const uint32_t lo = mag << 29;
    const uint32_t s2 = ((236u << 23) - (mag & 0x7f800000u)) | sign;     // +-2^(-18 - E)
    int32_t ci = __float2int_rn(__fmul_rn(__fmul_rn(e, 0x1p64f), __uint_as_float(s2)));
    if ((mag & 0x007fffffu) == 0u && ci < 0) ci *= 2;                      // just below a power of two
    const uint64_t bits = (((uint64_t)hi << 32) | lo) + (uint64_t)((int64_t)ci * 64);
    return __longlong_as_double((long long)bits);
}

// The exact FP64 value of a float built from its bit pattern with integer
// operations (exponent rebias, mantissa shift): no FP64-pipe conversion.
// Zero and denormal floats give a signed zero (an absolute error below
// 2^-126); x must be finite.
__device__ __forceinline__ double f32_to_f64_bits(float x)
{
    const uint32_t u = __float_as_uint(x), a = u & 0x7fffffffu, sign = u & 0x80000000u;
    const bool normal = a >= 0x00800000u;
    const uint32_t hi = normal ? (((a >> 3) + 0x38000000u) | sign) : sign;
    const uint32_t lo = normal ? (u << 29) : 0u;
    return __hiloint2double((int)hi, (int)lo);
}

// FP64 value of an unnormalised pair s + c (finite): both halves widened
// exactly, then one FP64 addition, so the result is s + c correctly rounded
// (up to the flush of denormal halves).  Costs one FP64-pipe instruction and
// about a dozen integer ones.
__device__ __forceinline__ double pair_to_double(float s, float c)
{
    return __dadd_rn(f32_to_f64_bits(s), f32_to_f64_bits(c));
}

// Sum without the final renormalisation (s, e): enough when the result only
// feeds further pair arithmetic.
__device__ __forceinline__ df df_add_lazy(df a, df b)
{
    float s, e;
    two_sum(a.h, b.h, s, e);
    return df{s, __fadd_rn(__fadd_rn(a.l, b.l), e)};
}

}  // namespace soptx
