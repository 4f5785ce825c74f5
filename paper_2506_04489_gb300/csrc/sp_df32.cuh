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

#include "sp_common.cuh"

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
// are renormalised (df_norm) only where they are written to global memory.
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

// ---------------------------------------------------------------------------------
// Complex double-float values, stored and computed as pairs.  A complex value keeps
// its high parts (re.hi, im.hi) and its low parts (re.lo, im.lo) side by side, so that
// the real and imaginary halves of an addition run as one packed f32x2 instruction
// (add/sub/fma.rn.f32x2: two independent IEEE round-to-nearest FP32 operations).  Each
// lane computes exactly what the scalar double-float operation above computes, so the
// results are bitwise those of the scalar form, in half the instructions.
// Memory layout (16 bytes): re.hi, im.hi, re.lo, im.lo.
// ---------------------------------------------------------------------------------
template <> struct __align__(16) cpx<df32> {
    float rh, ih, rl, il;
};

SP_HD cpx<df32> mk(df32 re, df32 im)
{
    cpx<df32> c;
    c.rh = re.hi;
    c.ih = im.hi;
    c.rl = re.lo;
    c.il = im.lo;
    return c;
}
SP_HD df32 re_of(cpx<df32> c) { return df_make(c.rh, c.rl); }
SP_HD df32 im_of(cpx<df32> c) { return df_make(c.ih, c.il); }

typedef unsigned long long f32x2;  // two floats: first in the low 32 bits

__device__ __forceinline__ f32x2 f2_pack(float a, float b)
{
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void f2_unpack(f32x2 v, float& a, float& b)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ f32x2 f2_add(f32x2 a, f32x2 b)
{
    f32x2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2 f2_sub(f32x2 a, f32x2 b)
{
    f32x2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

__device__ __forceinline__ f32x2 hi2(cpx<df32> c) { return f2_pack(c.rh, c.ih); }
__device__ __forceinline__ f32x2 lo2(cpx<df32> c) { return f2_pack(c.rl, c.il); }
__device__ __forceinline__ cpx<df32> from2(f32x2 h, f32x2 l)
{
    cpx<df32> c;
    f2_unpack(h, c.rh, c.ih);
    f2_unpack(l, c.rl, c.il);
    return c;
}

// a + b: the double-float sum of each part (two-sum of the high parts, plus the sum of
// the low parts), both parts at once.
__device__ __forceinline__ cpx<df32> operator+(cpx<df32> a, cpx<df32> b)
{
    const f32x2 ah = hi2(a), bh = hi2(b);
    const f32x2 s = f2_add(ah, bh);
    const f32x2 bb = f2_sub(s, ah);
    const f32x2 e = f2_add(f2_sub(ah, f2_sub(s, bb)), f2_sub(bh, bb));
    return from2(s, f2_add(e, f2_add(lo2(a), lo2(b))));
}

// a - b, the two-sum of a.hi and -b.hi written with subtractions (negation is exact).
__device__ __forceinline__ cpx<df32> operator-(cpx<df32> a, cpx<df32> b)
{
    const f32x2 ah = hi2(a), bh = hi2(b);
    const f32x2 s = f2_sub(ah, bh);
    const f32x2 bb = f2_sub(s, ah);
    const f32x2 e = f2_sub(f2_sub(ah, f2_sub(s, bb)), f2_add(bh, bb));
    return from2(s, f2_add(e, f2_sub(lo2(a), lo2(b))));
}

__device__ __forceinline__ cpx<df32> scale(cpx<df32> a, df32 s) { return mk(re_of(a) * s, im_of(a) * s); }
SP_HD cpx<df32> conjg(cpx<df32> a)
{
    cpx<df32> c = a;
    c.ih = -a.ih;
    c.il = -a.il;
    return c;
}
// a * (S i)
template <int S> __device__ __forceinline__ cpx<df32> mul_si(cpx<df32> a)
{
    cpx<df32> c;
    c.rh = S > 0 ? -a.ih : a.ih;
    c.rl = S > 0 ? -a.il : a.il;
    c.ih = S > 0 ? a.rh : -a.rh;
    c.il = S > 0 ? a.rl : -a.rl;
    return c;
}

// a * b and a * conj(b) (the first-generation passes' twiddle products): each part is one
// fused two-product dot, as in the register engine's twiddle products.
__device__ __forceinline__ cpx<df32> cmul(cpx<df32> a, cpx<df32> b)
{
    const df32 ar = re_of(a), ai = im_of(a), br = re_of(b), bi = im_of(b);
    return mk(df_dot_sub(ar, br, ai, bi), df_dot_add(ar, bi, ai, br));
}
__device__ __forceinline__ cpx<df32> cmulc(cpx<df32> a, cpx<df32> b)
{
    const df32 ar = re_of(a), ai = im_of(a), br = re_of(b), bi = im_of(b);
    return mk(df_dot_add(ar, br, ai, bi), df_dot_sub(ai, br, ar, bi));
}

// Renormalise both parts (fast two-sum of hi and lo).
__device__ __forceinline__ cpx<df32> df_norm_c(cpx<df32> a)
{
    const f32x2 h = hi2(a), l = lo2(a);
    const f32x2 s = f2_add(h, l);
    return from2(s, f2_sub(l, f2_sub(s, h)));
}

// Single-precision complex sums as one packed instruction: cpx<float> keeps re, im side
// by side (8 bytes), exactly an f32x2 pair; each lane rounds as the scalar sum would.
__device__ __forceinline__ f32x2 as_f2(cpx<float> a) { return f2_pack(a.re, a.im); }
__device__ __forceinline__ cpx<float> from_f2(f32x2 v)
{
    cpx<float> c;
    f2_unpack(v, c.re, c.im);
    return c;
}
__device__ __forceinline__ cpx<float> operator+(cpx<float> a, cpx<float> b) { return from_f2(f2_add(as_f2(a), as_f2(b))); }
__device__ __forceinline__ cpx<float> operator-(cpx<float> a, cpx<float> b) { return from_f2(f2_sub(as_f2(a), as_f2(b))); }
