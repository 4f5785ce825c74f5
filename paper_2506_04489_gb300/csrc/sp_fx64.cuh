// Fixed-point ("fx64") arithmetic for FP64-accuracy FFT passes: block floating point.
//
// A real value is a 64-bit two's-complement integer m standing for m * 2^s, where s is
// one exponent shared by every value of the line being transformed (the pass chooses s
// per line so that every complex value keeps |re|, |im| < 2^61 throughout the transform).
// Sums and differences are exact integer additions (one full-rate instruction on this
// GPU, where a double-float sum takes eight FP32 operations); only products round.
//
// Products are by multipliers |c| <= 1 (twiddles, butterfly constants, the convolution
// multiplier) held in Q61, q = c 2^61, split into 31-bit pieces q = q1 2^31 + q0 with
// q0 in [0, 2^31) and |q1| <= 2^30.  With the datum split the same way, m = m1 2^31 + m0
// (|m1| <= 2^30 for |m| < 2^61),
//     m q / 2^61 = 2 m1 q1 + (m1 q0 + m0 q1) / 2^30 + m0 q0 / 2^61,
// taken as 2 m1 q1 + ((m1 q0 + m0 q1) >> 30): three 32 x 32 -> 64-bit integer
// multiply(-add)s, an error below three units of m's last place (m0 q0 / 2^61 < 2 and the
// floor of the shift).  Every middle term is below 2^61 in magnitude, so the four-term
// middle sum of a complex product stays below 2^63.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "sp_common.cuh"

struct __align__(8) fx64 {
    long long m;
};

SP_HD fx64 fx_make(long long m)
{
    fx64 r;
    r.m = m;
    return r;
}

// Multipliers are kept pre-split: the 64-bit word holds q1 in its high and q0 in its low
// 32 bits (not the integer q itself), so a product reads its pieces as the two halves of
// a register pair.  Zero is 0 in both encodings.
SP_HD fx64 fx_mult_pieces(long long q)
{
    const long long q1 = q >> 31;                       // arithmetic
    const long long q0 = q & 0x7fffffffLL;              // [0, 2^31)
    return fx_make((long long)(((unsigned long long)q1 << 32) | (unsigned long long)q0));
}

// Q61 multiplier of a constant |d| <= 1, pre-split (d = +-1 is clamped to one unit
// inside, a relative error of 2^-61).
SP_HD fx64 fx_q61(double d)
{
    const long long lim = 2305843009213693951LL;  // 2^61 - 1
    const double q = d * 2305843009213693952.0;   // exact scaling by 2^61
    long long m;
    if (q >= (double)lim) m = lim;
    else if (q <= -(double)lim) m = -lim;
    else m = (long long)(q < 0 ? q - 0.5 : q + 0.5);  // |q| < 2^61: the cast is exact after rounding
    return fx_mult_pieces(m);
}
SP_D void fx_pieces(fx64 c, int& c1, int& c0)
{
    c1 = (int)(c.m >> 32);
    c0 = (int)(unsigned)(c.m & 0xffffffffLL);
}

SP_HD fx64 operator+(fx64 a, fx64 b) { return fx_make(a.m + b.m); }
SP_HD fx64 operator-(fx64 a, fx64 b) { return fx_make(a.m - b.m); }
SP_HD fx64 operator-(fx64 a) { return fx_make(-a.m); }

// Split into m1 = m >> 31 (arithmetic) and m0 = m mod 2^31 (in [0, 2^31)).
SP_D void fx_split(long long m, int& m1, int& m0)
{
    m1 = (int)(m >> 31);
    m0 = (int)((unsigned)m & 0x7fffffffu);
}

SP_D long long mul_wide(int a, int b)
{
    long long d;
    asm("mul.wide.s32 %0, %1, %2;" : "=l"(d) : "r"(a), "r"(b));
    return d;
}
SP_D long long mad_wide(int a, int b, long long c)
{
    long long d;
    asm("mad.wide.s32 %0, %1, %2, %3;" : "=l"(d) : "r"(a), "r"(b), "l"(c));
    return d;
}

// a * c with c a pre-split Q61 multiplier (error bound in the header comment).
SP_D fx64 operator*(fx64 a, fx64 c)
{
    int a1, a0, c1, c0;
    fx_split(a.m, a1, a0);
    fx_pieces(c, c1, c0);
    const long long mid = mad_wide(a0, c1, mul_wide(a1, c0));
    return fx_make(2 * mul_wide(a1, c1) + (mid >> 30));
}

// x y + u v for data x, u and Q61 multipliers y, v, all given split, rounded as one
// product (the middle terms are summed before the shift).
SP_D long long fx_dot(int x1, int x0, int y1, int y0, int u1, int u0, int v1, int v0)
{
    long long mid = mul_wide(x1, y0);
    mid = mad_wide(x0, y1, mid);
    mid = mad_wide(u1, v0, mid);
    mid = mad_wide(u0, v1, mid);
    const long long hi = mad_wide(u1, v1, mul_wide(x1, y1));
    return 2 * hi + (mid >> 30);
}
