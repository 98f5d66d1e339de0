// sgn_df64.cuh - double-word ("float-float") arithmetic on the FP32 pipe.
//
// A df64 value is hi + lo with hi = the float nearest (or next toward zero
// of) the value and |lo| <= ulp(hi): about 48 significant bits, relative
// rounding ~2^-48, with every operation on the FP32 units.  On B300 the FP64
// pipe executes two thread-instructions per SM and clock against 128 for
// FP32, so a stencil evaluated in df64 runs several times faster than in FP64
// at a precision 32 times coarser than FP64's and 2^24 times finer than
// FP32's.
//
// The building blocks are the exact transformations of floating-point
// arithmetic: Knuth's TwoSum (s + e = a + b exactly), Dekker's FastTwoSum
// (the same when |a| >= |b|) and the product error by fused multiply-add
// (p + e = a b exactly); the double-word sum, product and multiply-add follow
// the classical constructions (Dekker 1971; Joldes, Muller and Popescu 2017),
// dropping the lo*lo product and summing the low parts in float.  Every
// operation uses explicitly rounded intrinsics so that the compiler neither
// contracts nor reassociates it.
//
// Conversions to and from double use integer operations on the bit patterns
// (no FP64-pipe instruction) except one double addition per value stored.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace sgn {

struct df64 {
    float hi, lo;
};

__host__ __device__ __forceinline__ constexpr df64 df64_of_float(float x) { return {x, 0.0f}; }

// s + e == a + b exactly
__device__ __forceinline__ float two_sum(float a, float b, float& e) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return s;
}
// s + e == a + b exactly when |a| >= |b| (or a == 0)
__device__ __forceinline__ float fast_two_sum(float a, float b, float& e) {
    const float s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
    return s;
}
// p + e == a b exactly
__device__ __forceinline__ float two_prod(float a, float b, float& e) {
    const float p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
    return p;
}

__device__ __forceinline__ df64 operator-(df64 a) { return {-a.hi, -a.lo}; }

__device__ __forceinline__ df64 add_(df64 a, df64 b) {
    float e;
    const float s = two_sum(a.hi, b.hi, e);
    e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    df64 r;
    r.hi = fast_two_sum(s, e, r.lo);
    return r;
}
__device__ __forceinline__ df64 sub_(df64 a, df64 b) { return add_(a, -b); }

// a - b without the final renormalization: hi = fl(a.hi - b.hi), and lo its
// exact error plus the difference of the low parts, so hi + lo carries the
// difference to the double-word rounding of its operands but |lo| may exceed
// ulp(hi)/2.  The consumers (mul_, fma_, add_) treat hi and lo linearly, so
// an unnormalized pair is as good an input as a normalized one.  For the
// stencil differences f_+ - f_-, whose results only enter products.
__device__ __forceinline__ df64 diff_(df64 a, df64 b) {
    float e;
    const float s = two_sum(a.hi, -b.hi, e);
    return {s, __fadd_rn(e, __fsub_rn(a.lo, b.lo))};
}

__device__ __forceinline__ df64 mul_(df64 a, df64 b) {
    float e;
    const float p = two_prod(a.hi, b.hi, e);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    df64 r;
    r.hi = fast_two_sum(p, e, r.lo);
    return r;
}

// a b + c with the product kept exact to the low part before the sum
__device__ __forceinline__ df64 fma_(df64 a, df64 b, df64 c) {
    float pe;
    const float p = two_prod(a.hi, b.hi, pe);
    pe = __fmaf_rn(a.hi, b.lo, pe);
    pe = __fmaf_rn(a.lo, b.hi, pe);
    float se;
    const float s = two_sum(p, c.hi, se);
    se = __fadd_rn(se, __fadd_rn(pe, c.lo));
    df64 r;
    r.hi = fast_two_sum(s, se, r.lo);
    return r;
}

// 1/h: the float reciprocal of hi refined by one Newton step r = x + x (1 - h x)
// with the residual 1 - h x formed exactly to the low part (about 46 bits).
__device__ __forceinline__ df64 recip_df64(df64 h) {
    float x;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(x) : "f"(h.hi));
    float pe;
    const float p = two_prod(h.hi, x, pe);       // h.hi x = p + pe exactly
    pe = __fmaf_rn(h.lo, x, pe);                 // + h.lo x
    const float t = __fsub_rn(1.0f, p);          // exact: p is within a few ulp of 1
    const float e = __fsub_rn(t, pe);            // 1 - h x
    df64 r;
    r.hi = fast_two_sum(x, __fmul_rn(x, e), r.lo);
    return r;
}

// double -> df64 by integer operations only: hi = the double truncated to 24
// significant bits, lo = the next 24 of the remaining 29 (truncated), so
// hi + lo equals x to within 2^-48 |x|.  Magnitudes below the normal float
// range become +-0; above it (and infinities) +-inf; NaN stays NaN.
__device__ __forceinline__ df64 df64_from_double(double x) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
    const unsigned sign = (unsigned)(bits >> 63) << 31;
    const int E = (int)((bits >> 52) & 0x7ff);
    const int ef = E - 1023 + 127;
    if (ef < 1) return {__uint_as_float(sign), 0.0f};                    // +-0 and tiny
    if (ef > 254) {
        const bool nan = E == 0x7ff && (bits & 0xfffffffffffffull) != 0ull;
        return {__uint_as_float(sign | 0x7f800000u | (nan ? 0x400000u : 0u)), 0.0f};
    }
    const unsigned long long m = bits & 0xfffffffffffffull;
    df64 r;
    r.hi = __uint_as_float(sign | ((unsigned)ef << 23) | (unsigned)(m >> 29));
    const unsigned R = (unsigned)(m & 0x1fffffffull);          // the 29 bits below hi
    if (R == 0) {
        r.lo = 0.0f;
        return r;
    }
    const int p = 31 - __clz(R);                              // leading bit of R
    const int elf = ef - 52 + p;                              // lo = 1.f x 2^(E-1023-52+p)
    if (elf < 1) {
        r.lo = 0.0f;                                          // below the float range: < 2^-126
        return r;
    }
    const unsigned mant = p >= 23 ? (R >> (p - 23)) : (R << (23 - p));
    r.lo = __uint_as_float(sign | ((unsigned)elf << 23) | (mant & 0x7fffffu));
    return r;
}

// float -> double by integer operations only (exact for normal floats;
// subnormal floats, below 2^-126, become +-0; infinities and NaN keep their
// class).
__device__ __forceinline__ double double_of_float_bits(float f) {
    const unsigned b = __float_as_uint(f);
    const unsigned long long sign = (unsigned long long)(b >> 31) << 63;
    const unsigned e = (b >> 23) & 0xff;
    const unsigned long long m = (unsigned long long)(b & 0x7fffffu) << 29;
    unsigned long long d;
    if (e == 0) d = sign;                                          // +-0 and subnormal
    else if (e == 0xff) d = sign | 0x7ff0000000000000ull | m;      // inf, NaN
    else d = sign | ((unsigned long long)(e - 127 + 1023) << 52) | m;
    return __longlong_as_double((long long)d);
}

// double -> float rounded to nearest (ties to even) by integer operations only:
// the same value as the conversion instruction for results in the normal
// float range; magnitudes below it become +-0, above it +-inf (NaN stays NaN).
__device__ __forceinline__ float float_of_double_rn(double x) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
    const unsigned sign = (unsigned)(bits >> 63) << 31;
    const int E = (int)((bits >> 52) & 0x7ff);
    const int ef = E - 1023 + 127;
    if (ef < 1) return __uint_as_float(sign);
    if (ef > 254) {
        const bool nan = E == 0x7ff && (bits & 0xfffffffffffffull) != 0ull;
        return __uint_as_float(sign | 0x7f800000u | (nan ? 0x400000u : 0u));
    }
    const unsigned long long m = bits & 0xfffffffffffffull;
    unsigned body = ((unsigned)ef << 23) | (unsigned)(m >> 29);     // exponent and 23 fraction bits
    const unsigned rest = (unsigned)(m & 0x1fffffffull);              // the 29 dropped bits
    const unsigned half = 0x10000000u;
    body += (rest > half || (rest == half && (body & 1u))) ? 1u : 0u; // a carry may reach the exponent
    return __uint_as_float(sign | body);
}

// df64 -> double: the two parts exactly, then one rounded double addition.
__device__ __forceinline__ double double_of_df64(df64 a) {
    return __dadd_rn(double_of_float_bits(a.hi), double_of_float_bits(a.lo));
}

}  // namespace sgn
