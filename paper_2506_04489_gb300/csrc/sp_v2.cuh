// Solve passes of Alg. 2 on the register-resident FFT engine (sp_fft.cuh), for padded
// lengths with a compile-time plan (64, 128, 192, 256, 384, 512, 1024).  The schedule
// and the workspace layout are those of the first-generation passes (sp_passes.cu):
//   z forward (packed real pairs) -> y forward -> x forward * M * x inverse
//   -> y inverse -> z inverse (packed real pairs), W[x][ky][kz] with row stride ldz.
// Included by one translation unit per arithmetic type (float, double, double-float).
#pragma once

#include "sp_fft.cuh"
#include "sp_internal.h"

namespace v2 {

// ------------------------------------------------------------------ conversions
template <class R, class Tio> SP_D R to_r(Tio x);
template <> SP_D float to_r<float, float>(float x) { return x; }
template <> SP_D double to_r<double, double>(double x) { return x; }
template <> SP_D float to_r<float, double>(double x) { return (float)x; }
template <> SP_D df32 to_r<df32, double>(double x) { return df_from_double(x); }

template <class R, class Tio> SP_D Tio from_r(R x);
template <> SP_D float from_r<float, float>(float x) { return x; }
template <> SP_D double from_r<double, double>(double x) { return x; }
template <> SP_D double from_r<float, double>(float x) { return (double)x; }
template <> SP_D double from_r<df32, double>(df32 x) { return df_to_double(x); }

template <class R> SP_D cpx<R> half_of(cpx<R> a) { return scale(a, Num<R>::c(0.5)); }

// ------------------------------------------------------------------ layouts
// Strided lines: lane b (column) is fastest.  A padding row of B entries after every 8
// rows keeps the stride-8 writes of the first stage off one bank set when a row of B
// entries is narrower than 128 bytes.
template <class R, int B> struct LayStrided {
    static constexpr int PAD = (B * (int)sizeof(cpx<R>) >= 128) ? 0 : B;
    int b;
    SP_D int operator()(int e) const { return e * B + (e >> 3) * PAD + b; }
    static constexpr int size(int N) { return N * B + (N / 8) * PAD; }
};
// Contiguous lines: lane t is fastest; one padding entry after every 8 entries.
template <int N> struct LayLine {
    static constexpr int LD = N + N / 8;
    int base;
    SP_D int operator()(int e) const { return base + e + (e >> 3); }
};

// ------------------------------------------------------------------ strided passes
enum { FWD = 0, INV = 1, XMUL = 2 };

struct LArgs {
    const void* in;
    void* out;
    long long in_os, in_es, in_bs;  // outer / element / batch strides (complex elements)
    long long out_os, out_es, out_bs;
    int ncol;                        // valid columns (kz = 0..n2)
    const void* tw;                  // exp(-2 pi i j / N), j < N
    const void* M;                   // XMUL: multiplier [|ko|][|kl|][kz], row stride ldzM
    int No, nh_line, ldzM;
};

template <int N> constexpr int lanes_b() { return N >= 1024 ? 4 : 8; }

template <class R, int N, int MODE>
__global__ void __launch_bounds__((N / FFTPlan<N>::E) * lanes_b<N>()) k2_line(LArgs a)
{
    constexpr int E = FFTPlan<N>::E, T = N / E, B = lanes_b<N>();
    constexpr int R0 = FFTPlan<N>::R[0];
    using Lay = LayStrided<R, B>;
    extern __shared__ __align__(16) unsigned char smraw[];
    cpx<R>* tw = reinterpret_cast<cpx<R>*>(smraw);
    cpx<R>* sm = tw + N;
    const int tid = threadIdx.x, b = tid % B, t = tid / B;
    for (int j = tid; j < N; j += blockDim.x) tw[j] = static_cast<const cpx<R>*>(a.tw)[j];
    const int o = blockIdx.y, c = blockIdx.x * B + b, batch = blockIdx.z;
    const bool cv = c < a.ncol;
    const cpx<R>* in = static_cast<const cpx<R>*>(a.in) + batch * a.in_bs + o * a.in_os + c;
    cpx<R>* out = static_cast<cpx<R>*>(a.out) + batch * a.out_bs + o * a.out_os + c;
    const Lay lay{b};
    cpx<R> v[E];
    if constexpr (MODE == INV) {
#pragma unroll
        for (int j = 0; j < E; ++j) {
            const int e = first_element<N, true>(t, j);
            v[j] = cv ? in[e * a.in_es] : czero<R>();
        }
    } else {
#pragma unroll
        for (int j = 0; j < E; ++j) {
            const int e = first_element<N, false>(t, j);
            v[j] = (cv && (j % R0) < R0 / 2) ? in[e * a.in_es] : czero<R>();
        }
    }
    __syncthreads();
    if constexpr (MODE == INV) {
        run_stages<R, N, true, +1, false>(v, sm, lay, tw, t);
    } else {
        run_stages<R, N, false, -1, true>(v, sm, lay, tw, t);
    }
    if constexpr (MODE == XMUL) {
        const R* M = static_cast<const R*>(a.M);
        const int ko = o <= a.No / 2 ? o : a.No - o;
        const long long mrow = (long long)ko * (a.nh_line + 1);
#pragma unroll
        for (int j = 0; j < E; ++j) {
            const int e = last_element<N, false>(t, j);
            const int ke = e <= N / 2 ? e : N - e;
            const R m = cv ? M[(mrow + ke) * a.ldzM + c] : Num<R>::c(0.0);
            v[j] = scale(v[j], m);
        }
        run_stages<R, N, true, +1, false>(v, sm, lay, tw, t);
    }
    if constexpr (MODE == FWD) {
#pragma unroll
        for (int j = 0; j < E; ++j)
            if (cv) out[last_element<N, false>(t, j) * a.out_es] = v[j];
    } else {  // the last inverse radix is R0: outputs q < R0/2 are the kept half
#pragma unroll
        for (int j = 0; j < E; ++j)
            if ((j % R0) < R0 / 2 && cv) out[last_element<N, true>(t, j) * a.out_es] = v[j];
    }
}

// ------------------------------------------------------------------ z passes
struct ZArgs2 {
    const void* rho;
    void* u;
    void* W;
    int n1, n2;
    long long lines;      // n0 n1 real lines
    long long plane;      // complex elements per x-plane of W
    int ldz;
    long long io_bs, w_bs;
    const void* tw;
};

template <int N> constexpr int pairs_per_cta() { return N >= 512 ? 4 : (N >= 256 ? 8 : 16); }

SP_D long long w_row(const ZArgs2& a, long long l) { return (l / a.n1) * a.plane + (l % a.n1) * a.ldz; }

template <class R, class Tio, int N>
__global__ void __launch_bounds__((N / FFTPlan<N>::E) * pairs_per_cta<N>()) k2_z_fwd(ZArgs2 a)
{
    constexpr int E = FFTPlan<N>::E, T = N / E, B = pairs_per_cta<N>();
    constexpr int R0 = FFTPlan<N>::R[0];
    extern __shared__ __align__(16) unsigned char smraw[];
    cpx<R>* tw = reinterpret_cast<cpx<R>*>(smraw);
    cpx<R>* sm = tw + N;
    const int tid = threadIdx.x, b = tid / T, t = tid % T;
    for (int j = tid; j < N; j += blockDim.x) tw[j] = static_cast<const cpx<R>*>(a.tw)[j];
    const int n2 = a.n2;
    const long long l0 = 2 * ((long long)blockIdx.x * B + b), l1 = l0 + 1;
    const Tio* rho = static_cast<const Tio*>(a.rho) + blockIdx.y * a.io_bs;
    cpx<R>* W = static_cast<cpx<R>*>(a.W) + blockIdx.y * a.w_bs;
    const LayLine<N> lay{b * LayLine<N>::LD};
    cpx<R> v[E];
#pragma unroll
    for (int j = 0; j < E; ++j) {
        const int z = first_element<N, false>(t, j);
        cpx<R> x = czero<R>();
        if ((j % R0) < R0 / 2) {  // z < n2: the padded half is zero
            if (l0 < a.lines) x.re = to_r<R, Tio>(rho[l0 * n2 + z]);
            if (l1 < a.lines) x.im = to_r<R, Tio>(rho[l1 * n2 + z]);
        }
        v[j] = x;
    }
    __syncthreads();
    run_stages<R, N, false, -1, true>(v, sm, lay, tw, t);
#pragma unroll
    for (int j = 0; j < E; ++j) sm[lay(last_element<N, false>(t, j))] = v[j];
    __syncthreads();
    // two real lines from one complex transform: Xa = (Z_k + conj Z_{N-k}) / 2,
    // Xb = (Z_k - conj Z_{N-k}) / (2 i), k = 0..n2
    const long long r0 = w_row(a, l0), r1 = w_row(a, l1 < a.lines ? l1 : l0);
    for (int k = t; k <= n2; k += T) {
        const cpx<R> zk = sm[lay(k)];
        const cpx<R> zm = conjg(sm[lay(k == 0 ? 0 : N - k)]);
        const cpx<R> s = zk + zm, d = zk - zm;
        if (l0 < a.lines) W[r0 + k] = half_of(s);
        if (l1 < a.lines) W[r1 + k] = half_of(mk(d.im, -d.re));
    }
}

template <class R, class Tio, int N>
__global__ void __launch_bounds__((N / FFTPlan<N>::E) * pairs_per_cta<N>()) k2_z_inv(ZArgs2 a)
{
    constexpr int E = FFTPlan<N>::E, T = N / E, B = pairs_per_cta<N>();
    constexpr int R0 = FFTPlan<N>::R[0];
    extern __shared__ __align__(16) unsigned char smraw[];
    cpx<R>* tw = reinterpret_cast<cpx<R>*>(smraw);
    cpx<R>* sm = tw + N;
    const int tid = threadIdx.x, b = tid / T, t = tid % T;
    for (int j = tid; j < N; j += blockDim.x) tw[j] = static_cast<const cpx<R>*>(a.tw)[j];
    const int n2 = a.n2;
    const long long l0 = 2 * ((long long)blockIdx.x * B + b), l1 = l0 + 1;
    Tio* u = static_cast<Tio*>(a.u) + blockIdx.y * a.io_bs;
    const cpx<R>* W = static_cast<const cpx<R>*>(a.W) + blockIdx.y * a.w_bs;
    const LayLine<N> lay{b * LayLine<N>::LD};
    // Z_k = Xa_k + i Xb_k from the Hermitian halves (DC and Nyquist take real parts)
    const long long r0 = w_row(a, l0), r1 = w_row(a, l1 < a.lines ? l1 : l0);
    for (int k = t; k <= n2; k += T) {
        cpx<R> xa = l0 < a.lines ? W[r0 + k] : czero<R>();
        cpx<R> xb = l1 < a.lines ? W[r1 + k] : czero<R>();
        if (k == 0 || k == n2) {
            xa.im = Num<R>::c(0.0);
            xb.im = Num<R>::c(0.0);
        }
        sm[lay(k)] = mk(xa.re - xb.im, xa.im + xb.re);
        if (k > 0 && k < n2) sm[lay(N - k)] = mk(xa.re + xb.im, xb.re - xa.im);
    }
    __syncthreads();
    cpx<R> v[E];
    Stage<R, N, true, 0>::load(v, sm, lay, t);
    __syncthreads();
    run_stages<R, N, true, +1, false>(v, sm, lay, tw, t);
#pragma unroll
    for (int j = 0; j < E; ++j) {
        if ((j % R0) < R0 / 2) {  // z < n2
            const int z = last_element<N, true>(t, j);
            if (l0 < a.lines) u[l0 * n2 + z] = from_r<R, Tio>(v[j].re);
            if (l1 < a.lines) u[l1 * n2 + z] = from_r<R, Tio>(v[j].im);
        }
    }
}

// ------------------------------------------------------------------ launchers
template <class K> inline sp_status smem_attr(K kernel, size_t bytes)
{
    if (bytes > 48 * 1024)
        return sp_cuda_check(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes),
                             "set shared memory size");
    return SP_OK;
}

template <class R, int N, int MODE>
sp_status launch_line(const LArgs& a, int outer, int batch, cudaStream_t st)
{
    constexpr int E = FFTPlan<N>::E, B = lanes_b<N>();
    const size_t smem = sizeof(cpx<R>) * (size_t)(N + LayStrided<R, B>::size(N));
    sp_status rc = smem_attr(k2_line<R, N, MODE>, smem);
    if (rc) return rc;
    dim3 grid((unsigned)((a.ncol + B - 1) / B), (unsigned)outer, (unsigned)batch);
    k2_line<R, N, MODE><<<grid, (N / E) * B, smem, st>>>(a);
    return sp_cuda_check(cudaGetLastError(), "v2 line pass");
}

template <class R, class Tio, int N>
sp_status launch_z(const ZArgs2& a, bool forward, int batch, cudaStream_t st)
{
    constexpr int E = FFTPlan<N>::E, B = pairs_per_cta<N>();
    const size_t smem = sizeof(cpx<R>) * (size_t)(N + B * LayLine<N>::LD);
    const long long pairs = (a.lines + 1) / 2;
    dim3 grid((unsigned)((pairs + B - 1) / B), (unsigned)batch);
    sp_status rc;
    if (forward) {
        if ((rc = smem_attr(k2_z_fwd<R, Tio, N>, smem))) return rc;
        k2_z_fwd<R, Tio, N><<<grid, (N / E) * B, smem, st>>>(a);
    } else {
        if ((rc = smem_attr(k2_z_inv<R, Tio, N>, smem))) return rc;
        k2_z_inv<R, Tio, N><<<grid, (N / E) * B, smem, st>>>(a);
    }
    return sp_cuda_check(cudaGetLastError(), forward ? "v2 z forward pass" : "v2 z inverse pass");
}

// Length dispatch: calls f.template run<N>() for a supported N.
template <class F> inline sp_status with_len(int N, F&& f)
{
    switch (N) {
        case 64: return f.template run<64>();
        case 128: return f.template run<128>();
        case 192: return f.template run<192>();
        case 256: return f.template run<256>();
        case 384: return f.template run<384>();
        case 512: return f.template run<512>();
        case 1024: return f.template run<1024>();
        default: return SP_ERR_UNSUPPORTED_SIZE;
    }
}

inline bool len_ok(int N)
{
    return N == 64 || N == 128 || N == 192 || N == 256 || N == 384 || N == 512 || N == 1024;
}

template <class R, int MODE> struct LineRun {
    const LArgs* a;
    int outer, batch;
    cudaStream_t st;
    template <int N> sp_status run() { return launch_line<R, N, MODE>(*a, outer, batch, st); }
};

template <class R, class Tio> struct ZRun {
    const ZArgs2* a;
    bool forward;
    int batch;
    cudaStream_t st;
    template <int N> sp_status run() { return launch_z<R, Tio, N>(*a, forward, batch, st); }
};

// Tables of the pass arithmetic type.
template <class R> struct Tabs {
    static const void* tw(sp_plan p, int ax);
    static const void* M(sp_plan p);
};

// The whole solve; `work` is the workspace (the plan's, or another of the same size).
template <class R, class Tio>
sp_status solve(sp_plan p, const void* rho, void* u, int batch, cudaStream_t st, bool mark)
{
    for (int ax = 0; ax < 3; ++ax)
        if (!len_ok(p->N[ax])) return SP_ERR_UNSUPPORTED_SIZE;
    sp_status rc;
    p->npass = 5;
    p->pass_name[0] = "z_forward";
    p->pass_name[1] = "y_forward";
    p->pass_name[2] = "x_multiply";
    p->pass_name[3] = "y_inverse";
    p->pass_name[4] = "z_inverse";
    ZArgs2 z;
    z.rho = rho;
    z.u = u;
    z.W = p->d_work;
    z.n1 = p->n[1];
    z.n2 = p->n[2];
    z.lines = (long long)p->n[0] * p->n[1];
    z.plane = p->plane;
    z.ldz = p->ldz;
    z.io_bs = (long long)p->n[0] * p->n[1] * p->n[2];
    z.w_bs = (long long)p->n[0] * p->plane;
    z.tw = Tabs<R>::tw(p, 2);
    LArgs y = {};
    y.in = y.out = p->d_work;
    y.in_os = y.out_os = p->plane;
    y.in_es = y.out_es = p->ldz;
    y.in_bs = y.out_bs = (long long)p->n[0] * p->plane;
    y.ncol = p->n[2] + 1;
    y.tw = Tabs<R>::tw(p, 1);
    LArgs x = y;
    x.in_os = x.out_os = p->ldz;
    x.in_es = x.out_es = p->plane;
    x.tw = Tabs<R>::tw(p, 0);
    x.M = Tabs<R>::M(p);
    x.No = p->N[1];
    x.nh_line = p->n[0];
    x.ldzM = p->ldz;
    if (mark && (rc = sp_mark(p, st))) return rc;
    if ((rc = with_len(p->N[2], ZRun<R, Tio>{&z, true, batch, st}))) return rc;
    if (mark && (rc = sp_mark(p, st))) return rc;
    if ((rc = with_len(p->N[1], LineRun<R, FWD>{&y, p->n[0], batch, st}))) return rc;
    if (mark && (rc = sp_mark(p, st))) return rc;
    if ((rc = with_len(p->N[0], LineRun<R, XMUL>{&x, p->N[1], batch, st}))) return rc;
    if (mark && (rc = sp_mark(p, st))) return rc;
    if ((rc = with_len(p->N[1], LineRun<R, INV>{&y, p->n[0], batch, st}))) return rc;
    if (mark && (rc = sp_mark(p, st))) return rc;
    if ((rc = with_len(p->N[2], ZRun<R, Tio>{&z, false, batch, st}))) return rc;
    if (mark && (rc = sp_mark(p, st))) return rc;
    return SP_OK;
}

// Forward half only (diagnostic): spectrum[kx][ky][kz], kz <= n2 dense.
template <class R, class Tio>
sp_status forward(sp_plan p, const void* rho, void* spec, cudaStream_t st)
{
    for (int ax = 0; ax < 3; ++ax)
        if (!len_ok(p->N[ax])) return SP_ERR_UNSUPPORTED_SIZE;
    ZArgs2 z = {};
    z.rho = rho;
    z.W = p->d_work;
    z.n1 = p->n[1];
    z.n2 = p->n[2];
    z.lines = (long long)p->n[0] * p->n[1];
    z.plane = p->plane;
    z.ldz = p->ldz;
    z.tw = Tabs<R>::tw(p, 2);
    LArgs y = {};
    y.in = y.out = p->d_work;
    y.in_os = y.out_os = p->plane;
    y.in_es = y.out_es = p->ldz;
    y.ncol = p->n[2] + 1;
    y.tw = Tabs<R>::tw(p, 1);
    LArgs x = y;
    x.out = spec;
    x.in_os = p->ldz;
    x.in_es = p->plane;
    x.out_os = p->n[2] + 1;
    x.out_es = (long long)p->N[1] * (p->n[2] + 1);
    x.tw = Tabs<R>::tw(p, 0);
    sp_status rc;
    if ((rc = with_len(p->N[2], ZRun<R, Tio>{&z, true, 1, st}))) return rc;
    if ((rc = with_len(p->N[1], LineRun<R, FWD>{&y, p->n[0], 1, st}))) return rc;
    return with_len(p->N[0], LineRun<R, FWD>{&x, p->N[1], 1, st});
}

}  // namespace v2
