// Double-float arithmetic: a value is the unevaluated sum hi + lo of two
// FP32 numbers (|lo| <= ulp(hi)/2), about 48 significant bits.  Built from
// the error-free transformations two-sum (Knuth) and two-product (exact with
// FMA), after Dekker (1971).  Used for the FP64-grade q0 of the FP32-mixed
// form: GB300 issues 64 FP32 FMAs for every FP64 FMA.
#pragma once
#include <cuda_runtime.h>

namespace vdwgb {

struct dfl {
    float hi, lo;
};

// split a double constant into hi + lo (constant-folded for literals)
__host__ __device__ constexpr dfl DF(double x) {
    return dfl{(float)x, (float)(x - (double)(float)x)};
}

__device__ __forceinline__ dfl df_quick(float s, float e) {   // |s| >= |e|
    const float h = s + e;
    return dfl{h, e - (h - s)};
}

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

__device__ __forceinline__ dfl df_from(double x) {
    const float h = (float)x;
    return dfl{h, (float)(x - (double)h)};
}
__device__ __forceinline__ double df_to(dfl a) { return (double)a.hi + (double)a.lo; }

// Split a double into hi + lo on the integer and FP32 pipes only (GB300's FP64
// pipe, which also converts, runs at 1/64 of the FP32 rate): hi keeps the top
// 24 significand bits (truncated), lo the next bits rounded to FP32, then one
// renormalising fast two-sum.  Outside the normal FP32 range of hi the result
// is a signed zero (|x| below 2^-126, about 1.2e-38), a signed infinity (|x|
// of 2^128 or more) or a NaN (x a NaN), all without the FP64 pipe.
__device__ __forceinline__ dfl df_from_bits(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int ed = (int)((b >> 52) & 0x7ff);
    const int ef = ed - 1023 + 127;          // FP32 biased exponent of hi
    const int el = ed - 1075 + 127;          // FP32 biased exponent of the unit of the low 29 bits
    const unsigned sign = (unsigned)(b >> 63) << 31;
    if (ef < 1) return dfl{__uint_as_float(sign), 0.f};
    if (ef > 254) {
        const bool nan = ed == 0x7ff && (b & 0xfffffffffffffull) != 0ull;
        return dfl{__uint_as_float(sign | 0x7f800000u | (nan ? 0x400000u : 0u)), 0.f};
    }
    const float hi = __uint_as_float(sign | ((unsigned)ef << 23) | (unsigned)((b >> 29) & 0x7fffffu));
    // lo = rem 2^(el - 127), scaled in two exact steps: 2^-30, then
    // 2^(el - 97) >= 2^-148 (a normal or subnormal power of two, as ef >= 1)
    const int k = el - 97;
    const float unit = k >= -126 ? __uint_as_float((unsigned)(k + 127) << 23) : __uint_as_float(1u << (k + 149));
    const float lmag = (__uint2float_rn((unsigned)(b & 0x1fffffffu)) * 9.31322574615478515625e-10f) * unit;
    return df_quick(hi, sign ? -lmag : lmag);
}

// Widen an FP32 value to FP64 exactly on the integer pipe: normal values by
// re-biasing the exponent, subnormal ones by normalising the significand
// (leading-zero count), zero, infinities and NaNs by their bit patterns.
__device__ __forceinline__ double f2d_bits(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned e = (u >> 23) & 0xffu;
    const unsigned m = u & 0x7fffffu;
    const unsigned long long sg = (unsigned long long)(u >> 31) << 63;
    unsigned long long b;
    if (e == 255u) {
        b = sg | (0x7ffull << 52) | ((unsigned long long)m << 29);
    } else if (e != 0u) {
        b = sg | ((unsigned long long)(e - 127u + 1023u) << 52) | ((unsigned long long)m << 29);
    } else if (m == 0u) {
        b = sg;
    } else {
        // value m 2^-149 with the top set bit of m at position p (0..22)
        const int p = 31 - __clz((int)m);
        const unsigned long long frac = ((unsigned long long)m << (52 - p)) & 0xfffffffffffffull;
        b = sg | ((unsigned long long)(p - 149 + 1023) << 52) | frac;
    }
    return __longlong_as_double((long long)b);
}

__device__ __forceinline__ dfl df_add(dfl a, dfl b) {
    float s, e, t, f;
    two_sum(a.hi, b.hi, s, e);
    two_sum(a.lo, b.lo, t, f);
    e += t;
    dfl r = df_quick(s, e);
    r.lo += f;
    return df_quick(r.hi, r.lo);
}

__device__ __forceinline__ dfl df_neg(dfl a) { return dfl{-a.hi, -a.lo}; }
__device__ __forceinline__ dfl df_sub(dfl a, dfl b) { return df_add(a, df_neg(b)); }

__device__ __forceinline__ dfl df_mul(dfl a, dfl b) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return df_quick(p, e);
}

__device__ __forceinline__ dfl df_mulf(dfl a, float b) {
    const float p = a.hi * b;
    float e = fmaf(a.hi, b, -p);
    e = fmaf(a.lo, b, e);
    return df_quick(p, e);
}

// a / b with two correction steps
__device__ __forceinline__ dfl df_div(dfl a, dfl b) {
    const float rb = 1.0f / b.hi;
    const float q1 = a.hi * rb;
    dfl r = df_sub(a, df_mulf(b, q1));
    const float q2 = r.hi * rb;
    r = df_sub(r, df_mulf(b, q2));
    const float q3 = r.hi * rb;
    dfl q = df_quick(q1, q2);
    return df_add(q, dfl{q3, 0.f});
}

__device__ __forceinline__ dfl df_rcp(dfl b) { return df_div(dfl{1.f, 0.f}, b); }

// Newton corrections from FP32 seeds (one step doubles the ~24 good bits)
__device__ __forceinline__ dfl df_sqrt(dfl a) {
    const float x = sqrtf(a.hi);
    const float p = x * x;
    const float e = fmaf(x, x, -p);
    const dfl r = df_sub(a, dfl{p, e});
    return df_quick(x, r.hi / (2.f * x));
}

__device__ __forceinline__ dfl df_cbrt(dfl a) {
    const float y = cbrtf(a.hi);
    const float p = y * y;
    const float e = fmaf(y, y, -p);
    const dfl y3 = df_mulf(dfl{p, e}, y);
    const dfl r = df_sub(a, y3);
    return df_quick(y, r.hi / (3.f * p));
}

__device__ __forceinline__ bool df_lt(dfl a, dfl b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }

}  // namespace vdwgb
