// dfloat.cuh -- compensated FP32 pairs ("double-float"): a value is hi + lo with |lo| <=
// half an ulp of hi, about 44 significant bits.  Built from two error-free transformations:
// Knuth's two-sum (TAOCP vol. 2, 4.2.2) and the FMA form of Dekker's two-product (Dekker,
// "A floating-point technique for extending the available precision", 1971), combined as
// in the double-double algorithms of Hida, Li and Bailey (2001).  Used where the FP64
// pipe (1/64 of the FP32 rate on GB300) would otherwise carry bulk work whose result is
// only needed to FP32 precision, so that it rounds like the FP64 computation would.
#pragma once

#include <cuda_runtime.h>

namespace sbr {

struct df {
    float hi, lo;
};

__device__ __forceinline__ df df_of(float x) { return {x, 0.0f}; }

// s + e = a + b exactly (Knuth)
__device__ __forceinline__ df two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

// s + e = a + b exactly when |a| >= |b| (Dekker)
__device__ __forceinline__ df fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

// p + e = a * b exactly (FMA)
__device__ __forceinline__ df two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ df df_add(df x, df y) {
    df s = two_sum(x.hi, y.hi);
    const df t = two_sum(x.lo, y.lo);
    s.lo = __fadd_rn(s.lo, t.hi);
    s = fast_two_sum(s.hi, s.lo);
    s.lo = __fadd_rn(s.lo, t.lo);
    return fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ df df_neg(df x) { return {-x.hi, -x.lo}; }
__device__ __forceinline__ df df_sub(df x, df y) { return df_add(x, df_neg(y)); }

__device__ __forceinline__ df df_mul(df x, df y) {
    df p = two_prod(x.hi, y.hi);
    p.lo = __fmaf_rn(x.hi, y.lo, __fmaf_rn(x.lo, y.hi, p.lo));
    return fast_two_sum(p.hi, p.lo);
}

// exact scaling by a power of two
__device__ __forceinline__ df df_scale2(df x, float s) { return {x.hi * s, x.lo * s}; }

// quotient: q1 = x.hi / y.hi, then one correction step with the remainder x - q1 y
__device__ __forceinline__ df df_div(df x, df y) {
    const float q1 = __fdiv_rn(x.hi, y.hi);
    const df r = df_sub(x, df_mul(df_of(q1), y));
    const float q2 = __fdiv_rn(r.hi, y.hi);
    return fast_two_sum(q1, q2);
}

// square root of x >= 0: s = sqrt(x.hi), then one Newton correction (x - s^2) / (2 s)
__device__ __forceinline__ df df_sqrt(df x) {
    if (!(x.hi > 0.0f)) return df_of(0.0f);
    const float s = __fsqrt_rn(x.hi);
    const df r = df_sub(x, two_prod(s, s));
    return fast_two_sum(s, __fdiv_rn(r.hi, 2.0f * s));
}

__device__ __forceinline__ double df_to_double(df x) { return (double)x.hi + (double)x.lo; }

// the pair nearest a double: hi its rounding to FP32, lo the rounded residual
__device__ __forceinline__ df df_from_double(double x) {
    const float hi = (float)x;
    return {hi, (float)(x - (double)hi)};
}

struct df3 {
    df x, y, z;
};

__device__ __forceinline__ df df_dot(const df3 &a, const df3 &b) {
    return df_add(df_add(df_mul(a.x, b.x), df_mul(a.y, b.y)), df_mul(a.z, b.z));
}

// a - s b, componentwise
__device__ __forceinline__ df3 df3_sub_scaled(const df3 &a, df s, const df3 &b) {
    return {df_sub(a.x, df_mul(s, b.x)), df_sub(a.y, df_mul(s, b.y)), df_sub(a.z, df_mul(s, b.z))};
}

// a + s b, componentwise
__device__ __forceinline__ df3 df3_add_scaled(const df3 &a, df s, const df3 &b) {
    return {df_add(a.x, df_mul(s, b.x)), df_add(a.y, df_mul(s, b.y)), df_add(a.z, df_mul(s, b.z))};
}

__device__ __forceinline__ df3 df3_sub(const df3 &a, const df3 &b) {
    return {df_sub(a.x, b.x), df_sub(a.y, b.y), df_sub(a.z, b.z)};
}

__device__ __forceinline__ df3 df3_of(float3 v) { return {df_of(v.x), df_of(v.y), df_of(v.z)}; }

}  // namespace sbr
