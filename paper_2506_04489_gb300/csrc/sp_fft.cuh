// Register-resident mixed-radix FFT engine used by the solve passes.
//
// A length-N line is transformed by T = N/E threads that each hold E complex values in
// registers.  Stage s (radix R_s, span P_s = R_0 ... R_{s-1}) is the Stockham step
//     for i < N/R, k = i mod P:   u_r = x[i + r N/R] * w^{r k N/(P R)},  u = DFT_R(u),
//                                 y[(i - k) R + k + q P] = u_q,
// with thread t owning the butterflies i = t + T m, m < E/R.  Between stages the
// values go through shared memory once (write, barrier, read).  After the last stage
// thread t holds y[t + T m + q N/R_last]; the inverse transform runs the radices in
// reverse order, so its first stage wants exactly those values: a diagonal multiplier
// between a forward and an inverse transform is applied in registers with no exchange.
// A forward transform whose upper half of inputs is zero (zero padding) has, in its
// first radix-R stage, exactly inputs r < R/2 nonzero in every butterfly; an inverse
// whose upper half of outputs is discarded (crop) needs only outputs q < R/2 of its
// last stage.  Both are pruned at compile time.
#pragma once

#include <type_traits>

#include "sp_common.cuh"
#include "sp_df32.cuh"

// ------------------------------------------------------------------ numeric traits
// (Num<float>, Num<double>: sp_common.cuh)
template <> struct Num<df32> {
    static SP_HD df32 c(double d) { return df_from_double(d); }
};
template <class R> SP_D cpx<R> czero() { return mk(Num<R>::c(0.0), Num<R>::c(0.0)); }

// Twiddle products: the generic forms for float/double; for double-float each part is
// one fused two-product dot (df_dot_sub / df_dot_add).
template <class R> SP_D cpx<R> tw_mul(cpx<R> a, cpx<R> w) { return cmul(a, w); }
template <class R> SP_D cpx<R> tw_mulc(cpx<R> a, cpx<R> w) { return cmulc(a, w); }
template <> SP_D cpx<df32> tw_mul<df32>(cpx<df32> a, cpx<df32> w)
{
    const df32 ar = re_of(a), ai = im_of(a), wr = re_of(w), wi = im_of(w);
    return mk(df_dot_sub(ar, wr, ai, wi), df_dot_add(ar, wi, ai, wr));
}
template <> SP_D cpx<df32> tw_mulc<df32>(cpx<df32> a, cpx<df32> w)
{
    const df32 ar = re_of(a), ai = im_of(a), wr = re_of(w), wi = im_of(w);
    return mk(df_dot_add(ar, wr, ai, wi), df_dot_sub(ai, wr, ar, wi));
}
// Values written to global memory are renormalised.  Exchanges through shared memory
// between the stages of one transform keep the pair as the arithmetic left it: sums and
// products accept a low part of a few ulps of the high part (their error stays a small
// multiple of 2^-48 of the operands), so renormalising there would only cost FP32 work.
template <class R> SP_D cpx<R> norm(cpx<R> a) { return a; }
template <> SP_D cpx<df32> norm<df32>(cpx<df32> a) { return df_norm_c(a); }

// ------------------------------------------------------------------ plans
// Forward radices: powers of two first (the first stage is radix 8 or 16, so zero padding
// prunes it uniformly), then 3s.  E is a multiple of every radix.
template <int N> struct FFTPlan;
template <> struct FFTPlan<64> { static constexpr int NS = 2, E = 8; static constexpr int R[2] = {8, 8}; };
template <> struct FFTPlan<128> { static constexpr int NS = 3, E = 8; static constexpr int R[3] = {8, 8, 2}; };
template <> struct FFTPlan<192> { static constexpr int NS = 3, E = 24; static constexpr int R[3] = {8, 8, 3}; };
template <> struct FFTPlan<256> { static constexpr int NS = 3, E = 8; static constexpr int R[3] = {8, 8, 4}; };
template <> struct FFTPlan<384> { static constexpr int NS = 4, E = 24; static constexpr int R[4] = {8, 8, 2, 3}; };
template <> struct FFTPlan<512> { static constexpr int NS = 3, E = 8; static constexpr int R[3] = {8, 8, 8}; };
template <> struct FFTPlan<1024> { static constexpr int NS = 4, E = 8; static constexpr int R[4] = {8, 8, 8, 2}; };

// The plan a pass of arithmetic type R uses.  At 1024, FP32 and FP64 take a radix-16
// first stage (16 values a thread, three stages: one exchange fewer, 15 % faster at
// 512^3 in FP32); double-float keeps eight values a thread, whose 16-value form holds
// too many registers (measured 6 % slower).
struct Plan1024Radix16 {
    static constexpr int NS = 3, E = 16;
    static constexpr int R[3] = {16, 8, 8};
};
// At 384, 24 double-float values a thread hold too many registers: double-float takes
// radices 4-4-4-2-3 with 12 values a thread (7 % faster at 192^3); FP32 and FP64 keep
// 8-8-2-3 (measured faster for them).
struct Plan384Radix4 {
    static constexpr int NS = 5, E = 12;
    static constexpr int R[5] = {4, 4, 4, 2, 3};
};
// At 256, FP32 takes two radix-16 stages (16 values a thread, one exchange instead of
// two: 128^3 FP32 solve 12 % faster); the 16-byte types keep 8-8-4.
struct Plan256Radix16 {
    static constexpr int NS = 2, E = 16;
    static constexpr int R[2] = {16, 16};
};
// At 512, FP32 takes radices 32-16 (32 values a thread, one exchange instead of two:
// the x pass 19 % faster, the z passes slower, the 256^3 solve 9 % faster).
struct Plan512Radix32 {
    static constexpr int NS = 2, E = 32;
    static constexpr int R[2] = {32, 16};
};
template <class R, int N> struct PlanOf : FFTPlan<N> {};
template <> struct PlanOf<float, 512> : Plan512Radix32 {};
template <> struct PlanOf<float, 256> : Plan256Radix16 {};
// FP32 line passes at 1024: radices 32-32 (two stages; 3 % faster at 512^3 than 16-8-8,
// which its z passes keep).
struct Plan1024Radix32 {
    static constexpr int NS = 2, E = 32;
    static constexpr int R[2] = {32, 32};
};
template <> struct PlanOf<float, 1024> : Plan1024Radix32 {};
template <> struct PlanOf<double, 1024> : Plan1024Radix16 {};
template <> struct PlanOf<df32, 384> : Plan384Radix4 {};
// Plan key of the z passes (contiguous real lines, packed in pairs): the type's own plan,
// except FP32 at 512 and 1024, whose z passes run faster on 8-8-8 and 16-8-8 than on the
// radix-32 plans of its line passes.  Each axis has its own staged twiddle table, so the
// z axis can differ.
template <class R> struct ZKey {};
template <class R, int N> struct PlanOf<ZKey<R>, N> : PlanOf<R, N> {};
template <> struct PlanOf<ZKey<float>, 512> : FFTPlan<512> {};
template <> struct PlanOf<ZKey<float>, 1024> : Plan1024Radix16 {};

// Alternative radix plans of the line passes, which the autotuner times against the
// built-in plan of the same type and length (LineKey<R, 1>; LineKey<R, 0> is the built-in
// plan PlanOf<R, N>).  Each has its own staged twiddle table in global memory, after the
// built-in plan's.
template <class R, int N> struct AltPlan {
    static constexpr bool exists = false;
};
// FP32: the eight-value plans (two exchanges a transform instead of one, about a third of
// the registers, so twice the resident warps)
template <> struct AltPlan<float, 256> : FFTPlan<256> { static constexpr bool exists = true; };
template <> struct AltPlan<float, 512> : FFTPlan<512> { static constexpr bool exists = true; };
template <> struct AltPlan<float, 1024> : Plan1024Radix16 { static constexpr bool exists = true; };
// double-float: sixteen values a thread at 256 (one exchange a transform instead of two)
template <> struct AltPlan<df32, 256> : Plan256Radix16 { static constexpr bool exists = true; };
template <class R, int V> struct LineKey {};
template <class R, int N> struct PlanOf<LineKey<R, 0>, N> : PlanOf<R, N> {};
template <class R, int N> struct PlanOf<LineKey<R, 1>, N> : AltPlan<R, N> {};
template <class K> struct KeyVariant { static constexpr int v = 0; };
template <class R, int V> struct KeyVariant<LineKey<R, V>> { static constexpr int v = V; };
// radix of stage s of the forward (INV = false) or inverse (reversed) transform
template <class R, int N, bool INV> constexpr int radix_at(int s)
{
    return INV ? PlanOf<R, N>::R[PlanOf<R, N>::NS - 1 - s] : PlanOf<R, N>::R[s];
}
template <class R, int N, bool INV> constexpr int span_at(int s)
{
    int p = 1;
    for (int i = 0; i < s; ++i) p *= radix_at<R, N, INV>(i);
    return p;
}

// ------------------------------------------------------------------ butterflies
// X_q = sum_r u_r exp(S 2 pi i r q / R), in place.
template <int S, class R> SP_D void bf2(cpx<R>* u)
{
    cpx<R> a = u[0], b = u[1];
    u[0] = a + b;
    u[1] = a - b;
}

template <int S, class R> SP_D void bf3(cpx<R>* u)
{
    const R c = Num<R>::c(-0.5);
    const R s = Num<R>::c(0.86602540378443864676372317075293618);  // sin(2 pi / 3)
    cpx<R> a = u[0], t = u[1] + u[2], v = u[1] - u[2];
    cpx<R> m = a + scale(t, c);
    cpx<R> w = mul_si<S>(scale(v, s));
    u[0] = a + t;
    u[1] = m + w;
    u[2] = m - w;
}

template <int S, class R> SP_D void bf4(cpx<R>* u)
{
    cpx<R> a = u[0] + u[2], b = u[0] - u[2];
    cpx<R> c = u[1] + u[3], d = mul_si<S>(u[1] - u[3]);
    u[0] = a + c;
    u[2] = a - c;
    u[1] = b + d;
    u[3] = b - d;
}

// radix 8 as 2 x 4 (even/odd halves, then twiddles exp(S 2 pi i q / 8))
template <int S, class R> SP_D void bf8_tail(cpx<R>* u, cpx<R> e0, cpx<R> e1, cpx<R> e2, cpx<R> e3, cpx<R> o0,
                                             cpx<R> o1, cpx<R> o2, cpx<R> o3)
{
    const R h = Num<R>::c(0.70710678118654752440084436210484904);
    cpx<R> t1 = scale(o1 + mul_si<S>(o1), h);
    cpx<R> t2 = mul_si<S>(o2);
    cpx<R> t3 = scale(mul_si<S>(o3) - o3, h);
    u[0] = e0 + o0;
    u[4] = e0 - o0;
    u[1] = e1 + t1;
    u[5] = e1 - t1;
    u[2] = e2 + t2;
    u[6] = e2 - t2;
    u[3] = e3 + t3;
    u[7] = e3 - t3;
}

template <int S, class R> SP_D void bf8(cpx<R>* u)
{
    cpx<R> a0 = u[0] + u[4], a1 = u[0] - u[4], a2 = u[2] + u[6], a3 = mul_si<S>(u[2] - u[6]);
    cpx<R> b0 = u[1] + u[5], b1 = u[1] - u[5], b2 = u[3] + u[7], b3 = mul_si<S>(u[3] - u[7]);
    bf8_tail<S>(u, a0 + a2, a1 + a3, a0 - a2, a1 - a3, b0 + b2, b1 + b3, b0 - b2, b1 - b3);
}

// radix 8 with u[4..7] = 0
template <int S, class R> SP_D void bf8_half(cpx<R>* u)
{
    cpx<R> a0 = u[0], a2 = u[2], a3 = mul_si<S>(u[2]);
    cpx<R> b0 = u[1], b2 = u[3], b3 = mul_si<S>(u[3]);
    bf8_tail<S>(u, a0 + a2, a0 + a3, a0 - a2, a0 - a3, b0 + b2, b0 + b3, b0 - b2, b0 - b3);
}

// radix 16 as 2 x 8: the DFTs of the even and odd halves, then
// X_q = E_q + w^q O_q, X_{q+8} = E_q - w^q O_q with w = exp(S 2 pi i / 16).
template <int S, class R> SP_D void bf16_tail(cpx<R>* u, cpx<R>* e, cpx<R>* o)
{
    const R h = Num<R>::c(0.70710678118654752440084436210484904);   // cos(pi/4)
    const R c1 = Num<R>::c(0.92387953251128675612818318939678829);  // cos(pi/8)
    const R s1 = Num<R>::c(0.38268343236508977172845998403039887);  // sin(pi/8)
    cpx<R> t[8];
    t[0] = o[0];
    t[1] = tw_mul(o[1], mk(c1, S > 0 ? s1 : -s1));
    t[2] = scale(o[2] + mul_si<S>(o[2]), h);
    t[3] = tw_mul(o[3], mk(s1, S > 0 ? c1 : -c1));
    t[4] = mul_si<S>(o[4]);
    t[5] = tw_mul(o[5], mk(-s1, S > 0 ? c1 : -c1));
    t[6] = scale(mul_si<S>(o[6]) - o[6], h);
    t[7] = tw_mul(o[7], mk(-c1, S > 0 ? s1 : -s1));
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        u[q] = e[q] + t[q];
        u[q + 8] = e[q] - t[q];
    }
}

template <int S, class R> SP_D void bf16(cpx<R>* u)
{
    cpx<R> e[8], o[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        e[j] = u[2 * j];
        o[j] = u[2 * j + 1];
    }
    bf8<S>(e);
    bf8<S>(o);
    bf16_tail<S>(u, e, o);
}

// radix 16 with u[8..15] = 0: both halves have their upper four inputs zero
template <int S, class R> SP_D void bf16_half(cpx<R>* u)
{
    cpx<R> e[8], o[8];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        e[j] = u[2 * j];
        o[j] = u[2 * j + 1];
    }
    bf8_half<S>(e);
    bf8_half<S>(o);
    bf16_tail<S>(u, e, o);
}

// radix 32 as 2 x 16: X_q = E_q + w^q O_q, X_{q+16} = E_q - w^q O_q, w = exp(S 2 pi i / 32).
template <int S, class R> SP_D void bf32_tail(cpx<R>* u, cpx<R>* e, cpx<R>* o)
{
    // cos and sin of pi m / 16, m = 0..8
    constexpr double C[9] = {1.0, 0.980785280403230449126182236134239037, 0.923879532511286756128183189396788287,
                             0.831469612302545237078788377617905757, 0.707106781186547524400844362104849039,
                             0.555570233019602224742830813948532874, 0.382683432365089771728459984030398867,
                             0.195090322016128267848284868477022241, 0.0};
    constexpr double Sn[9] = {0.0, 0.195090322016128267848284868477022241, 0.382683432365089771728459984030398867,
                              0.555570233019602224742830813948532874, 0.707106781186547524400844362104849039,
                              0.831469612302545237078788377617905757, 0.923879532511286756128183189396788287,
                              0.980785280403230449126182236134239037, 1.0};
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        cpx<R> t;
        if (q == 0) {
            t = o[0];
        } else if (q == 8) {
            t = mul_si<S>(o[8]);
        } else {
            const double c = q < 8 ? C[q] : -C[16 - q];
            const double sn = q < 8 ? Sn[q] : Sn[16 - q];
            t = tw_mul(o[q], mk(Num<R>::c(c), Num<R>::c(S > 0 ? sn : -sn)));
        }
        u[q] = e[q] + t;
        u[q + 16] = e[q] - t;
    }
}

template <int S, class R> SP_D void bf32(cpx<R>* u)
{
    cpx<R> e[16], o[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        e[j] = u[2 * j];
        o[j] = u[2 * j + 1];
    }
    bf16<S>(e);
    bf16<S>(o);
    bf32_tail<S>(u, e, o);
}

// radix 32 with u[16..31] = 0
template <int S, class R> SP_D void bf32_half(cpx<R>* u)
{
    cpx<R> e[16], o[16];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        e[j] = u[2 * j];
        o[j] = u[2 * j + 1];
    }
    bf16_half<S>(e);
    bf16_half<S>(o);
    bf32_tail<S>(u, e, o);
}

template <int RAD, int S, bool HALF, class R> SP_D void butterfly(cpx<R>* u)
{
    if constexpr (RAD == 32) {
        if constexpr (HALF) bf32_half<S>(u);
        else bf32<S>(u);
    } else if constexpr (RAD == 16) {
        if constexpr (HALF) bf16_half<S>(u);
        else bf16<S>(u);
    } else if constexpr (RAD == 8) {
        if constexpr (HALF) bf8_half<S>(u);
        else bf8<S>(u);
    } else if constexpr (RAD == 4) {
        bf4<S>(u);
    } else if constexpr (RAD == 3) {
        bf3<S>(u);
    } else {
        bf2<S>(u);
    }
}

// ------------------------------------------------------------------ stages
// Layouts map an element index e of a line to a shared-memory slot.  They must satisfy
// lay(e + d) = lay(e) + lay.step(d) for every d that is a multiple of 8 and every e, and
// lay(8 j + q) = lay(8 j) + q * lay.unit for q < 8: the stage loops then compute one
// slot per butterfly and add compile-time offsets for the others.

// Per-stage twiddle tables (in shared memory; for double-float, one copy per plan in
// global memory): stage s (span P > 1, radix RAD) keeps w^{r k N/(P RAD)} at
// [k (RAD + 1) + r], so a butterfly reads RAD - 1 consecutive entries; the extra entry
// per row puts the rows of neighbouring k on different banks.
template <class R, int N, bool INV> constexpr int tw_stage_offset(int s)
{
    int off = 0;
    for (int i = 0; i < s; ++i)
        if (span_at<R, N, INV>(i) > 1) off += span_at<R, N, INV>(i) * (radix_at<R, N, INV>(i) + 1);
    return off;
}
template <class R, int N> constexpr int tw_stage_size()
{
    return tw_stage_offset<R, N, false>(PlanOf<R, N>::NS) + tw_stage_offset<R, N, true>(PlanOf<R, N>::NS);
}
template <class R, int N, bool INV> constexpr int tw_base() { return INV ? tw_stage_offset<R, N, false>(PlanOf<R, N>::NS) : 0; }

// Fill the staged tables of plan key K (all threads of the block; a barrier must follow).
template <class R, int N, bool INV, class K = R, int ST = 0>
SP_D void fill_stage_twiddles(cpx<R>* tws, const cpx<R>* __restrict__ tw, int tid, int nthreads)
{
    if constexpr (ST < PlanOf<K, N>::NS) {
        constexpr int P = span_at<K, N, INV>(ST), RAD = radix_at<K, N, INV>(ST);
        if constexpr (P > 1) {
            constexpr int TWS = N / (P * RAD);
            cpx<R>* dst = tws + tw_base<K, N, INV>() + tw_stage_offset<K, N, INV>(ST);
            for (int j = tid; j < P * RAD; j += nthreads) {
                const int k = j / RAD, r = j % RAD;
                dst[k * (RAD + 1) + r] = tw[r * k * TWS];
            }
        }
        fill_stage_twiddles<R, N, INV, K, ST + 1>(tws, tw, tid, nthreads);
    }
}

// A plan is usable when its radices multiply to N, every radix divides E (each thread
// runs whole butterflies) and every stage stride N / radix is a multiple of 8 (the
// layouts' step rule).
template <class K, int N> constexpr bool plan_ok()
{
    int prod = 1;
    for (int i = 0; i < PlanOf<K, N>::NS; ++i) {
        const int r = PlanOf<K, N>::R[i];
        if (PlanOf<K, N>::E % r != 0 || (N / r) % 8 != 0) return false;
        prod *= r;
    }
    return prod == N;
}

template <class R, int N, bool INV, int ST, class K = R> struct Stage {
    static_assert(plan_ok<K, N>(), "radix plan does not fit the stage rules");
    static constexpr int E = PlanOf<K, N>::E;
    static constexpr int T = N / E;
    static constexpr int RAD = radix_at<K, N, INV>(ST);
    static constexpr int P = span_at<K, N, INV>(ST);
    static constexpr int NB = E / RAD;
    static constexpr int STRIDE = N / RAD;  // a multiple of 8 for every plan

    // inputs of this stage from shared memory: v[m RAD + r] = x[t + T m + r N/RAD]
    template <class Lay> SP_D static void load(cpx<R> (&v)[E], const cpx<R>* sm, const Lay& lay, int t)
    {
#pragma unroll
        for (int m = 0; m < NB; ++m) {
            const cpx<R>* p0 = sm + lay(t + T * m);
            const int st = lay.step(STRIDE);
#pragma unroll
            for (int r = 0; r < RAD; ++r) v[m * RAD + r] = p0[r * st];
        }
    }

    // twiddles and butterflies (S = -1 forward, +1 inverse); HALF: inputs r >= RAD/2 are zero
    template <int S, bool HALF> SP_D static void compute(cpx<R> (&v)[E], const cpx<R>* tws, int t)
    {
#pragma unroll
        for (int m = 0; m < NB; ++m) {
            if constexpr (P > 1) {
                const int k = (t + T * m) % P;
                const cpx<R>* w = tws + tw_base<K, N, INV>() + tw_stage_offset<K, N, INV>(ST) + k * (RAD + 1);
                if constexpr (std::is_same<R, float>::value && RAD == 8) {
                    // FP32: w^2, w^3, w^5, w^6, w^7 from the loaded w and w^4 (two table reads
                    // instead of seven; a few ulps more twiddle error, far below FP32's bar)
                    cpx<R> ww[8];
                    ww[1] = w[1];
                    ww[4] = w[4];
                    ww[2] = cmul(ww[1], ww[1]);
                    ww[3] = cmul(ww[1], ww[2]);
                    ww[5] = cmul(ww[4], ww[1]);
                    ww[6] = cmul(ww[4], ww[2]);
                    ww[7] = cmul(ww[4], ww[3]);
#pragma unroll
                    for (int r = 1; r < RAD; ++r)
                        v[m * RAD + r] = S < 0 ? tw_mul(v[m * RAD + r], ww[r]) : tw_mulc(v[m * RAD + r], ww[r]);
                } else {
#pragma unroll
                    for (int r = 1; r < RAD; ++r)
                        v[m * RAD + r] = S < 0 ? tw_mul(v[m * RAD + r], w[r]) : tw_mulc(v[m * RAD + r], w[r]);
                }
            }
            butterfly<RAD, S, HALF>(&v[m * RAD]);
        }
    }

    // outputs of this stage to shared memory: y[(i - k) RAD + k + q P] = v[m RAD + q]
    template <class Lay> SP_D static void store(const cpx<R> (&v)[E], cpx<R>* sm, const Lay& lay, int t)
    {
#pragma unroll
        for (int m = 0; m < NB; ++m) {
            const int i = t + T * m;
            const int k = i % P;
            const int base = (i - k) * RAD + k;
            if constexpr (P % 8 == 0) {
                cpx<R>* p0 = sm + lay(base);
                const int st = lay.step(P);
#pragma unroll
                for (int q = 0; q < RAD; ++q) p0[q * st] = v[m * RAD + q];
            } else if constexpr (P == 1 && RAD == 8) {
                cpx<R>* p0 = sm + lay(base);  // base = 8 i
                const int st = lay.unit();
#pragma unroll
                for (int q = 0; q < RAD; ++q) p0[q * st] = v[m * RAD + q];
            } else {
#pragma unroll
                for (int q = 0; q < RAD; ++q) sm[lay(base + q * P)] = v[m * RAD + q];
            }
        }
    }
};

// Element index held in register slot j after the last stage of a transform (and the
// input index of slot j for the first stage of the opposite-direction transform).
template <class R, int N, bool INV> SP_D int last_element(int t, int j)
{
    constexpr int E = PlanOf<R, N>::E, T = N / E;
    constexpr int RL = radix_at<R, N, INV>(PlanOf<R, N>::NS - 1);
    return t + T * (j / RL) + (j % RL) * (N / RL);
}
// Element index of register slot j for the first stage of a transform.
template <class R, int N, bool INV> SP_D int first_element(int t, int j)
{
    constexpr int E = PlanOf<R, N>::E, T = N / E;
    constexpr int R0 = radix_at<R, N, INV>(0);
    return t + T * (j / R0) + (j % R0) * (N / R0);
}

// Run stages [0, NS) of one transform.  On entry v holds the stage-0 inputs (slot
// j = element first_element(t, j)); on return it holds the last stage's outputs (slot
// j = element last_element(t, j)).  `fresh` must be safe to write on entry (no reads of
// it pending in the block); exchanges alternate between `fresh` and `other`, one barrier
// each: a buffer is written again only after the barrier that follows every read of it.
// With other == fresh (one buffer) a second barrier follows each read.  Returns the
// buffer that is safe to write after the call.  All threads of the block must call this.
template <class R, int N, bool INV, int S, bool HALF0, class K = R, class Lay, int ST = 0>
SP_D cpx<R>* run_stages(cpx<R> (&v)[PlanOf<K, N>::E], cpx<R>* fresh, cpx<R>* other, const Lay& lay,
                        const cpx<R>* tws, int t)
{
    using St = Stage<R, N, INV, ST, K>;
    St::template compute<S, HALF0 && ST == 0>(v, tws, t);
    if constexpr (ST + 1 < PlanOf<K, N>::NS) {
        St::store(v, fresh, lay, t);
        __syncthreads();
        Stage<R, N, INV, ST + 1, K>::load(v, fresh, lay, t);
        if (other == fresh) __syncthreads();
        return run_stages<R, N, INV, S, HALF0, K, Lay, ST + 1>(v, other, fresh, lay, tws, t);
    } else {
        return fresh;
    }
}
