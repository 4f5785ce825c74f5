// Common device types for the super-potential solver: complex values, the small
// DFT butterflies used by every FFT pass, and error plumbing.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#define SP_HD __host__ __device__ __forceinline__
#define SP_D __device__ __forceinline__

template <class R>
struct __align__(2 * sizeof(R)) cpx {
    R re, im;
};

template <class R> SP_HD cpx<R> mk(R a, R b) { cpx<R> c; c.re = a; c.im = b; return c; }
// Real and imaginary parts as values (a complex type may store its parts split).
template <class R> SP_HD R re_of(cpx<R> c) { return c.re; }
template <class R> SP_HD R im_of(cpx<R> c) { return c.im; }
// Constants of the arithmetic type (the double-float type specialises it).
template <class R> struct Num;
template <> struct Num<float> {
    static SP_HD float c(double d) { return (float)d; }
};
template <> struct Num<double> {
    static SP_HD double c(double d) { return d; }
};
template <class R> SP_HD cpx<R> operator+(cpx<R> a, cpx<R> b) { return mk(a.re + b.re, a.im + b.im); }
template <class R> SP_HD cpx<R> operator-(cpx<R> a, cpx<R> b) { return mk(a.re - b.re, a.im - b.im); }
template <class R> SP_HD cpx<R> scale(cpx<R> a, R s) { return mk(a.re * s, a.im * s); }
template <class R> SP_HD cpx<R> conjg(cpx<R> a) { return mk(a.re, -a.im); }
// a * b
template <class R> SP_HD cpx<R> cmul(cpx<R> a, cpx<R> b)
{
    return mk(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
// a * conj(b)
template <class R> SP_HD cpx<R> cmulc(cpx<R> a, cpx<R> b)
{
    return mk(a.re * b.re + a.im * b.im, a.im * b.re - a.re * b.im);
}
// a * (s i), s = +1 or -1
template <int S, class R> SP_HD cpx<R> mul_si(cpx<R> a)
{
    return S > 0 ? mk(-a.im, a.re) : mk(a.im, -a.re);
}

// ---------------------------------------------------------------------------------
// Small DFTs in registers: X[q] = sum_r u[r] exp(S * 2 pi i r q / R), S = -1 forward,
// +1 inverse (unnormalised).  Constants are the exact values cos/sin of multiples of
// 2 pi / R, written as sqrt expressions.  Written with re_of/im_of/mk and Num, so that the
// same butterflies serve float, double and double-float values.
// ---------------------------------------------------------------------------------
template <int S, class R> SP_D void dft2(cpx<R>* u)
{
    cpx<R> a = u[0], b = u[1];
    u[0] = a + b;
    u[1] = a - b;
}

template <int S, class R> SP_D void dft3(cpx<R>* u)
{
    const R c = Num<R>::c(-0.5);
    const R s = Num<R>::c(0.86602540378443864676372317075293618);  // sin(2 pi / 3)
    cpx<R> a = u[0], b = u[1], d = u[2];
    cpx<R> t = b + d, v = b - d;
    cpx<R> m = mk(re_of(a) + c * re_of(t), im_of(a) + c * im_of(t));
    cpx<R> w = mul_si<S>(scale(v, s));
    u[0] = a + t;
    u[1] = m + w;
    u[2] = m - w;
}

template <int S, class R> SP_D void dft4(cpx<R>* u)
{
    cpx<R> a = u[0] + u[2], b = u[0] - u[2];
    cpx<R> c = u[1] + u[3], d = mul_si<S>(u[1] - u[3]);
    u[0] = a + c;
    u[2] = a - c;
    u[1] = b + d;
    u[3] = b - d;
}

// 8 = 2 x 4: even/odd split, twiddles exp(S 2 pi i q / 8).
template <int S, class R> SP_D void dft8(cpx<R>* u)
{
    const R h = Num<R>::c(0.70710678118654752440084436210484904);  // 1/sqrt(2)
    cpx<R> e[4] = {u[0], u[2], u[4], u[6]};
    cpx<R> o[4] = {u[1], u[3], u[5], u[7]};
    dft4<S>(e);
    dft4<S>(o);
    // o[1] *= (1 + S i)/sqrt2 ; o[2] *= S i ; o[3] *= (-1 + S i)/sqrt2
    cpx<R> o1 = scale(o[1] + mul_si<S>(o[1]), h);
    cpx<R> o2 = mul_si<S>(o[2]);
    cpx<R> o3 = scale(mul_si<S>(o[3]) - o[3], h);
    u[0] = e[0] + o[0];
    u[4] = e[0] - o[0];
    u[1] = e[1] + o1;
    u[5] = e[1] - o1;
    u[2] = e[2] + o2;
    u[6] = e[2] - o2;
    u[3] = e[3] + o3;
    u[7] = e[3] - o3;
}

// Odd prime length P: with t_j = u_j + u_{P-j}, v_j = u_j - u_{P-j} (j = 1..H, H = (P-1)/2),
//   X[q]   = u_0 + sum_j t_j cos(2 pi jq/P) + S i sum_j v_j sin(2 pi jq/P)
//   X[P-q] = u_0 + sum_j t_j cos(2 pi jq/P) - S i sum_j v_j sin(2 pi jq/P),  q = 1..H.
// c[m], s[m] hold cos and sin of 2 pi m / P for m = 0..H; jq mod P is folded into that
// range by the symmetry of cos (even) and sin (odd) about P/2.
template <int S, int P, class R> SP_D void dft_odd(cpx<R>* u, const R* c, const R* s)
{
    constexpr int H = (P - 1) / 2;
    cpx<R> t[H + 1], v[H + 1];
    cpx<R> sum = u[0];
#pragma unroll
    for (int j = 1; j <= H; ++j) {
        t[j] = u[j] + u[P - j];
        v[j] = u[j] - u[P - j];
        sum = sum + t[j];
    }
    cpx<R> out[P];
    out[0] = sum;
#pragma unroll
    for (int q = 1; q <= H; ++q) {
        cpx<R> a = u[0], b = mk(Num<R>::c(0.0), Num<R>::c(0.0));
#pragma unroll
        for (int j = 1; j <= H; ++j) {
            const int m = (j * q) % P;
            const R cm = m <= H ? c[m] : c[P - m];
            const R sm = m <= H ? s[m] : -s[P - m];
            a = mk(re_of(a) + cm * re_of(t[j]), im_of(a) + cm * im_of(t[j]));
            b = mk(re_of(b) + sm * re_of(v[j]), im_of(b) + sm * im_of(v[j]));
        }
        const cpx<R> w = mul_si<S>(b);
        out[q] = a + w;
        out[P - q] = a - w;
    }
#pragma unroll
    for (int q = 0; q < P; ++q) u[q] = out[q];
}

template <int S, class R> SP_D void dft5(cpx<R>* u)
{
    // cos and sin of 2 pi m / 5, m = 0, 1, 2
    const R c[3] = {Num<R>::c(1.0), Num<R>::c(0.309016994374947424102293417182819059),
                    Num<R>::c(-0.809016994374947424102293417182819059)};
    const R s[3] = {Num<R>::c(0.0), Num<R>::c(0.951056516295153572116439333379382143),
                    Num<R>::c(0.587785252292473129168705954639072769)};
    dft_odd<S, 5>(u, c, s);
}

template <int S, class R> SP_D void dft7(cpx<R>* u)
{
    // cos and sin of 2 pi m / 7, m = 0..3
    const R c[4] = {Num<R>::c(1.0), Num<R>::c(0.623489801858733530525004884004239811),
                    Num<R>::c(-0.222520933956314404288902564496794759), Num<R>::c(-0.900968867902419126236102319507445051)};
    const R s[4] = {Num<R>::c(0.0), Num<R>::c(0.78183148246802980870844452667405775),
                    Num<R>::c(0.974927912181823607018131682993931217), Num<R>::c(0.433883739117558120475768332848358755)};
    dft_odd<S, 7>(u, c, s);
}

template <int S, class R> SP_D void dft_small(int radix, cpx<R>* u)
{
    switch (radix) {
        case 2: dft2<S>(u); break;
        case 3: dft3<S>(u); break;
        case 4: dft4<S>(u); break;
        case 5: dft5<S>(u); break;
        case 7: dft7<S>(u); break;
        case 8: dft8<S>(u); break;
        default: break;
    }
}

// Maximum number of radix stages of one transform, and the stage plan for a length.
#define SP_MAX_STAGES 16
struct RadixPlan {
    int nst;
    int r[SP_MAX_STAGES];
};

// Factor N (a product of 2s, 3s, 5s and 7s) into stages, largest power-of-two radices
// first: 8s, then a 4 or 2 for the remaining power of two, then 3s, 5s and 7s.  Returns
// false for other lengths.
static inline bool sp_radix_plan(int N, RadixPlan* p)
{
    p->nst = 0;
    int m = N, twos = 0, threes = 0, fives = 0, sevens = 0;
    while (m % 2 == 0) { m /= 2; ++twos; }
    while (m % 3 == 0) { m /= 3; ++threes; }
    while (m % 5 == 0) { m /= 5; ++fives; }
    while (m % 7 == 0) { m /= 7; ++sevens; }
    if (m != 1 || N < 2) return false;
    if (twos / 3 + (twos % 3 != 0) + threes + fives + sevens > SP_MAX_STAGES) return false;
    while (twos >= 3) { p->r[p->nst++] = 8; twos -= 3; }
    if (twos == 2) p->r[p->nst++] = 4;
    if (twos == 1) p->r[p->nst++] = 2;
    for (int i = 0; i < threes; ++i) p->r[p->nst++] = 3;
    for (int i = 0; i < fives; ++i) p->r[p->nst++] = 5;
    for (int i = 0; i < sevens; ++i) p->r[p->nst++] = 7;
    return true;
}
