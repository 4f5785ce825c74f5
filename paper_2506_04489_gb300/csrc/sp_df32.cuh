// Double-float ("df32") arithmetic: a value is the unevaluated sum hi + lo of two
// floats with |lo| <= ulp(hi)/2, about 48 significant bits, computed on the FP32
// pipes.  GB300's FP64 rate is 1/62 of its FP32 rate, so FFT passes in double-float
// reach FP64-class accuracy several times faster than native FP64.
//
// Built from error-free transformations:
//   two_sum(a, b)        s + e = a + b exactly  (Knuth / Moller, 6 flops, no branch)
//   fast_two_sum(a, b)   s + e = a + b exactly when |a| >= |b| or a = 0 (Dekker, 3 flops)
//   two_prod(a, b)       p + e = a * b exactly  (with a fused multiply-add, 2 flops)
// Addition is the "sloppy" double-float sum: its error is bounded by a small multiple of
// 2^-48 (|a| + |b|), the form of bound an FFT's error analysis needs.  Products keep
// the hi*lo cross terms.  No operation here may be reassociated or contracted by the
// compiler: every step is an explicit round-to-nearest intrinsic.
#pragma once

#include <cuda_runtime.h>

struct __align__(8) df32 {
    float hi, lo;
};

__host__ __device__ __forceinline__ df32 df_make(float h, float l)
{
    df32 r;
    r.hi = h;
    r.lo = l;
    return r;
}

// Exact split of a double into the nearest float plus the float-rounded remainder.
__host__ __device__ __forceinline__ df32 df_from_double(double d)
{
    float h = (float)d;
    float l = (float)(d - (double)h);
    return df_make(h, l);
}

__host__ __device__ __forceinline__ double df_to_double(df32 a) { return (double)a.hi + (double)a.lo; }

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e)
{
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e)
{
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}

// Sum without a final renormalisation: hi + lo carries the sum with an error of at
// most a few 2^-48 (|a| + |b|); lo may exceed ulp(hi)/2 by a small factor, which the
// exact two-sum of the high parts and the cross terms of the product absorb.  Values
// are renormalised (df_norm) only where they leave registers.
__device__ __forceinline__ df32 operator+(df32 a, df32 b)
{
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    return df_make(s, __fadd_rn(e, __fadd_rn(a.lo, b.lo)));
}

__device__ __forceinline__ df32 operator-(df32 b) { return df_make(-b.hi, -b.lo); }

__device__ __forceinline__ df32 operator-(df32 a, df32 b)
{
    float s, e;
    two_sum(a.hi, -b.hi, s, e);
    return df_make(s, __fadd_rn(e, __fsub_rn(a.lo, b.lo)));
}

// Product with the exact high product (fused multiply-add) and both cross terms; the
// lo*lo term is below 2^-48 of the result and is dropped.
__device__ __forceinline__ df32 operator*(df32 a, df32 b)
{
    float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return df_make(p, e);
}

// a*b - c*d and a*b + c*d with one two-sum of the exact high products.
__device__ __forceinline__ df32 df_dot_sub(df32 a, df32 b, df32 c, df32 d)
{
    float p1 = __fmul_rn(a.hi, b.hi), p2 = __fmul_rn(c.hi, d.hi);
    float e1 = __fmaf_rn(a.hi, b.hi, -p1), e2 = __fmaf_rn(c.hi, d.hi, -p2);
    float s, e;
    two_sum(p1, -p2, s, e);
    e = __fadd_rn(e, __fsub_rn(e1, e2));
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    e = __fmaf_rn(-c.hi, d.lo, e);
    e = __fmaf_rn(-c.lo, d.hi, e);
    return df_make(s, e);
}

__device__ __forceinline__ df32 df_dot_add(df32 a, df32 b, df32 c, df32 d)
{
    float p1 = __fmul_rn(a.hi, b.hi), p2 = __fmul_rn(c.hi, d.hi);
    float e1 = __fmaf_rn(a.hi, b.hi, -p1), e2 = __fmaf_rn(c.hi, d.hi, -p2);
    float s, e;
    two_sum(p1, p2, s, e);
    e = __fadd_rn(e, __fadd_rn(e1, e2));
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    e = __fmaf_rn(c.hi, d.lo, e);
    e = __fmaf_rn(c.lo, d.hi, e);
    return df_make(s, e);
}

// Renormalise (fast two-sum).  Exact when |hi| >= |lo|; otherwise (hi cancelled to
// below the accumulated lo) the lost part is a rounding of lo, i.e. a small multiple of
// 2^-48 of the operands that produced the value: the same form of bound as the sum's.
__device__ __forceinline__ df32 df_norm(df32 a)
{
    df32 r;
    fast_two_sum(a.hi, a.lo, r.hi, r.lo);
    return r;
}
