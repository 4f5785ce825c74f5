// Solve passes of Alg. 2 (eq. convtheorem):
//   P1  pad + z real-to-complex DFT (rows z < n2 nonzero), two real lines per complex FFT
//   P2  y forward DFT (rows y < n1 nonzero)                 W[x][ky][kz], in place
//   P3  x forward DFT (x < n0 nonzero) * M * x inverse DFT, keep x < n0, in place
//   P4  y inverse DFT, keep y < n1                          in place
//   P5  z complex-to-real inverse DFT, keep z < n2 (crop)   -> u
// The padded (2n)^3 grid is never formed: zero rows are supplied on load and cropped
// rows are not stored.  Workspace W holds n0 x 2n1 x ldz complex values per right-hand
// side (row stride ldz >= n2 + 1).  The multiplier carries the 1/Ntilde of the inverse
// DFT.
//
// Each CTA transforms B lines held in shared memory as [element][line] (line fastest),
// stage by stage (mixed radix 8/4/2/3/5/7, Stockham ordering, ping-pong buffers).  Lines
// of a strided axis are taken B adjacent columns at a time so that every row access is a
// contiguous run of B complex values.  The arithmetic type is float, double or
// double-float (the latter for padded lengths the register engine has no plan for);
// double-float values written to global memory are renormalised.
#include <stdio.h>

#include <type_traits>

#include "sp_fft.cuh"
#include "sp_internal.h"

namespace {

// Density in, potential out: the I/O type to and from the arithmetic type.
template <class R, class Tio> SP_D R io_in(Tio x) { return (R)x; }
template <> SP_D df32 io_in<df32, double>(double x) { return df_from_double(x); }
template <class R, class Tio> SP_D Tio io_out(R x) { return (Tio)x; }
template <> SP_D double io_out<df32, double>(df32 x) { return df_to_double(x); }

constexpr int kThreads = 256;
constexpr int kSmemTarget = 64 * 1024;  // bytes of the two ping-pong buffers per CTA

// One Stockham stage per iteration: for i < N/R, k = i mod p:
//   u_r = x[i + r N/R] * w^{r k N/(p R)},  u = DFT_R(u),  y[(i - k) R + k + q p] = u_q.
// Returns the buffer holding the result.
template <class R>
__device__ cpx<R>* fft_lines(cpx<R>* x, cpx<R>* y, int N, int B, const RadixPlan& rp,
                             const cpx<R>* __restrict__ tw, int sign)
{
    int p = 1;
    for (int st = 0; st < rp.nst; ++st) {
        const int Rr = rp.r[st];
        const int T = N / Rr;
        const int tstep = N / (p * Rr);
        for (int t = threadIdx.x; t < T * B; t += blockDim.x) {
            const int b = t % B, i = t / B, k = i % p;
            cpx<R> u[8];
#pragma unroll
            for (int r = 0; r < 8; ++r)
                if (r < Rr) u[r] = x[(i + r * T) * B + b];
            if (k != 0) {
#pragma unroll
                for (int r = 1; r < 8; ++r) {
                    if (r < Rr) {
                        cpx<R> w = tw[r * k * tstep];
                        u[r] = sign < 0 ? cmul(u[r], w) : cmulc(u[r], w);
                    }
                }
            }
            if (sign < 0) dft_small<-1>(Rr, u);
            else dft_small<1>(Rr, u);
            const int base = (i - k) * Rr + k;
#pragma unroll
            for (int q = 0; q < 8; ++q)
                if (q < Rr) y[(base + q * p) * B + b] = u[q];
        }
        __syncthreads();
        cpx<R>* tmp = x;
        x = y;
        y = tmp;
        p *= Rr;
    }
    return x;
}

// ------------------------------------------------------------------------- strided lines
// Bluestein's algorithm on an axis without a radix plan (tab != nullptr): the table built
// by sp_bluestein_fill, [chirp N][filter fwd M][filter inv M][twiddles M], M = 2^k >= 2N - 1.
struct BlueArgs {
    const void* tab;
    int M;
    RadixPlan rp;
};

// Rows of shared memory a line transform of length N uses: N, or M for Bluestein.
__host__ __device__ inline int line_rows(int N, const BlueArgs& bl) { return bl.tab ? bl.M : N; }

// The line transform of rows 0..N-1 of x (B lines, [element][line]), as fft_lines; for a
// Bluestein axis: x_j times the chirp (conjugated for the inverse), zero rows N..M-1, the
// M-point forward transform, times the filter spectrum (1/M folded in), the M-point
// inverse, times the chirp again; rows 0..N-1 of the returned buffer hold the result.
// Both buffers hold line_rows(N, bl) rows.
template <class R>
__device__ cpx<R>* line_fft(cpx<R>* x, cpx<R>* y, int N, int B, const RadixPlan& rp, const cpx<R>* tw,
                            const BlueArgs& bl, int sign)
{
    if (!bl.tab) return fft_lines<R>(x, y, N, B, rp, tw, sign);
    const int M = bl.M;
    const cpx<R>* chirp = static_cast<const cpx<R>*>(bl.tab);
    const cpx<R>* D = chirp + N + (sign < 0 ? 0 : M);
    const cpx<R>* twM = chirp + N + 2 * M;
    for (int t = threadIdx.x; t < M * B; t += blockDim.x) {
        const int e = t / B;
        if (e < N) x[t] = sign < 0 ? cmul(x[t], chirp[e]) : cmulc(x[t], chirp[e]);
        else x[t] = czero<R>();
    }
    __syncthreads();
    cpx<R>* r = fft_lines<R>(x, y, M, B, bl.rp, twM, -1);
    for (int t = threadIdx.x; t < M * B; t += blockDim.x) r[t] = cmul(r[t], D[t / B]);
    __syncthreads();
    r = fft_lines<R>(r, r == x ? y : x, M, B, bl.rp, twM, +1);
    for (int t = threadIdx.x; t < N * B; t += blockDim.x) {
        const int e = t / B;
        r[t] = sign < 0 ? cmul(r[t], chirp[e]) : cmulc(r[t], chirp[e]);
    }
    __syncthreads();
    return r;
}

struct LineArgs {
    const void* in;
    void* out;
    int N, nin, nout, ncol, B;
    long long in_os, in_es, in_bs;    // outer, element, batch strides (complex elements)
    long long out_os, out_es, out_bs;
    RadixPlan rp;
    const void* tw;
    BlueArgs blue;
    int sign;
    // x-pass multiplier (mult != nullptr): M[(|ko| (nh_line + 1) + |kl|) ldzM + c]
    const void* mult;
    int No;       // length of the outer axis (for |ko|)
    int nh_line;  // n of the line axis
    int ldzM;
};

template <class R>
__global__ void __launch_bounds__(kThreads) k_lines(LineArgs a)
{
    extern __shared__ unsigned char smem_raw[];
    const int B = a.B, N = a.N;
    cpx<R>* b0 = reinterpret_cast<cpx<R>*>(smem_raw);
    cpx<R>* b1 = b0 + line_rows(N, a.blue) * B;
    const int o = blockIdx.y, c0 = blockIdx.x * B, batch = blockIdx.z;
    const cpx<R>* in = static_cast<const cpx<R>*>(a.in) + batch * a.in_bs + o * a.in_os;
    cpx<R>* out = static_cast<cpx<R>*>(a.out) + batch * a.out_bs + o * a.out_os;
    const cpx<R>* tw = static_cast<const cpx<R>*>(a.tw);
    for (int t = threadIdx.x; t < N * B; t += blockDim.x) {
        const int e = t / B, b = t % B, c = c0 + b;
        cpx<R> v = czero<R>();
        if (e < a.nin && c < a.ncol) v = in[e * a.in_es + c];
        b0[t] = v;
    }
    __syncthreads();
    cpx<R>* res = line_fft<R>(b0, b1, N, B, a.rp, tw, a.blue, a.sign);
    if (a.mult) {
        const R* M = static_cast<const R*>(a.mult);
        const int ko = o <= a.No / 2 ? o : a.No - o;
        for (int t = threadIdx.x; t < N * B; t += blockDim.x) {
            const int e = t / B, b = t % B, c = c0 + b;
            const int kl = e <= N / 2 ? e : N - e;
            const R m = c < a.ncol ? M[((long long)ko * (a.nh_line + 1) + kl) * a.ldzM + c] : Num<R>::c(0.0);
            res[t] = scale(res[t], m);
        }
        __syncthreads();
        cpx<R>* other = (res == b0) ? b1 : b0;
        res = line_fft<R>(res, other, N, B, a.rp, tw, a.blue, -a.sign);
    }
    for (int t = threadIdx.x; t < a.nout * B; t += blockDim.x) {
        const int e = t / B, b = t % B, c = c0 + b;
        if (c < a.ncol) out[e * a.out_es + c] = norm(res[t]);
    }
}

// ------------------------------------------------------------------------- z axis
// Real lines l = x n1 + y of rho (length n2, contiguous).  Pair c packs lines 2c and
// 2c+1 as real and imaginary parts of one complex line of length N = 2 n2.
struct ZArgs {
    const void* rho;   // P1 input (Tio)
    void* u;           // P5 output (Tio)
    void* W;           // workspace (cpx<R>)
    int n0, n1, n2, N, B;
    long long lines;   // n0 n1
    long long plane;   // complex elements per x-plane of W
    int ldz;
    long long io_bs, w_bs;  // batch strides (elements)
    RadixPlan rp;
    const void* tw;
    BlueArgs blue;
};

template <class R>
__device__ __forceinline__ long long w_index(const ZArgs& a, long long l, int k)
{
    const long long x = l / a.n1, y = l % a.n1;
    return x * a.plane + y * a.ldz + k;
}

template <class R, class Tio>
__global__ void __launch_bounds__(kThreads) k_z_forward(ZArgs a)
{
    extern __shared__ unsigned char smem_raw[];
    const int B = a.B, N = a.N, n2 = a.n2;
    cpx<R>* b0 = reinterpret_cast<cpx<R>*>(smem_raw);
    cpx<R>* b1 = b0 + line_rows(N, a.blue) * B;
    const int batch = blockIdx.y;
    const Tio* rho = static_cast<const Tio*>(a.rho) + batch * a.io_bs;
    cpx<R>* W = static_cast<cpx<R>*>(a.W) + batch * a.w_bs;
    const long long pair0 = (long long)blockIdx.x * B;
    for (int t = threadIdx.x; t < n2 * B; t += blockDim.x) {
        const int b = t / n2, z = t % n2;
        const long long l0 = 2 * (pair0 + b), l1 = l0 + 1;
        R re = l0 < a.lines ? io_in<R, Tio>(rho[l0 * n2 + z]) : Num<R>::c(0.0);
        R im = l1 < a.lines ? io_in<R, Tio>(rho[l1 * n2 + z]) : Num<R>::c(0.0);
        b0[z * B + b] = mk(re, im);
    }
    for (int t = threadIdx.x; t < (N - n2) * B; t += blockDim.x) b0[n2 * B + t] = czero<R>();
    __syncthreads();
    cpx<R>* Z = line_fft<R>(b0, b1, N, B, a.rp, static_cast<const cpx<R>*>(a.tw), a.blue, -1);
    // split: Xa = (Z_k + conj Z_{N-k}) / 2,  Xb = (Z_k - conj Z_{N-k}) / (2 i)
    for (int t = threadIdx.x; t < (n2 + 1) * B; t += blockDim.x) {
        const int b = t / (n2 + 1), k = t % (n2 + 1);
        const long long l0 = 2 * (pair0 + b), l1 = l0 + 1;
        const cpx<R> zk = Z[k * B + b];
        const cpx<R> zm = conjg(Z[((N - k) % N) * B + b]);
        const cpx<R> s = zk + zm, d = zk - zm;
        const R h = Num<R>::c(0.5), mh = Num<R>::c(-0.5);
        if (l0 < a.lines) W[w_index<R>(a, l0, k)] = norm(mk(h * re_of(s), h * im_of(s)));
        if (l1 < a.lines) W[w_index<R>(a, l1, k)] = norm(mk(h * im_of(d), mh * re_of(d)));
    }
}

template <class R, class Tio>
__global__ void __launch_bounds__(kThreads) k_z_inverse(ZArgs a)
{
    extern __shared__ unsigned char smem_raw[];
    const int B = a.B, N = a.N, n2 = a.n2;
    cpx<R>* b0 = reinterpret_cast<cpx<R>*>(smem_raw);
    cpx<R>* b1 = b0 + line_rows(N, a.blue) * B;
    const int batch = blockIdx.y;
    Tio* u = static_cast<Tio*>(a.u) + batch * a.io_bs;
    const cpx<R>* W = static_cast<const cpx<R>*>(a.W) + batch * a.w_bs;
    const long long pair0 = (long long)blockIdx.x * B;
    // Z_k = Xa_k + i Xb_k with the Hermitian halves Xa, Xb; DC and Nyquist take real parts.
    for (int t = threadIdx.x; t < N * B; t += blockDim.x) {
        const int b = t / N, k = t % N;
        const long long l0 = 2 * (pair0 + b), l1 = l0 + 1;
        const int kk = k <= n2 ? k : N - k;
        cpx<R> xa = l0 < a.lines ? W[w_index<R>(a, l0, kk)] : czero<R>();
        cpx<R> xb = l1 < a.lines ? W[w_index<R>(a, l1, kk)] : czero<R>();
        if (k == 0 || k == n2) {
            xa = mk(re_of(xa), Num<R>::c(0.0));
            xb = mk(re_of(xb), Num<R>::c(0.0));
        }
        if (k > n2) { xa = conjg(xa); xb = conjg(xb); }
        b0[k * B + b] = mk(re_of(xa) - im_of(xb), im_of(xa) + re_of(xb));
    }
    __syncthreads();
    cpx<R>* Z = line_fft<R>(b0, b1, N, B, a.rp, static_cast<const cpx<R>*>(a.tw), a.blue, +1);
    for (int t = threadIdx.x; t < n2 * B; t += blockDim.x) {
        const int b = t / n2, z = t % n2;
        const long long l0 = 2 * (pair0 + b), l1 = l0 + 1;
        const cpx<R> v = Z[z * B + b];
        if (l0 < a.lines) u[l0 * n2 + z] = io_out<R, Tio>(re_of(v));
        if (l1 < a.lines) u[l1 * n2 + z] = io_out<R, Tio>(im_of(v));
    }
}

int pick_B(int N, size_t csize)
{
    int B = 16;
    while (B > 1 && 2 * (size_t)N * B * csize > (size_t)kSmemTarget) B /= 2;
    return B;
}

template <class K>
sp_status set_smem(K kernel, size_t bytes)
{
    if (bytes > 48 * 1024)
        return sp_cuda_check(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                  (int)bytes), "set shared memory size");
    return SP_OK;
}

template <class R>
const void* tw_of(sp_plan p, int ax)
{
    if (std::is_same<R, df32>::value) return p->d_twdf[ax];  // base twiddles first
    if (std::is_same<R, double>::value) return p->d_tw64[ax];
    return p->d_tw32[ax];
}

template <class R>
const void* mult_of(sp_plan p)
{
    if (std::is_same<R, df32>::value) return p->d_Mdf;
    if (std::is_same<R, double>::value) return p->d_M64;
    return p->d_M32;
}

BlueArgs blue_of(sp_plan p, int ax)
{
    BlueArgs b = {};
    b.tab = p->d_blue[ax];
    b.M = p->blue_M[ax];
    b.rp = p->blue_rp[ax];
    return b;
}

template <class R, class Tio>
sp_status z_pass(sp_plan p, const void* rho, void* u, int batch, bool forward, cudaStream_t st)
{
    ZArgs a;
    a.rho = rho;
    a.u = u;
    a.W = p->d_work;
    a.n0 = p->n[0];
    a.n1 = p->n[1];
    a.n2 = p->n[2];
    a.N = p->N[2];
    a.lines = (long long)p->n[0] * p->n[1];
    a.plane = p->plane;
    a.ldz = p->ldz;
    a.io_bs = (long long)p->n[0] * p->n[1] * p->n[2];
    a.w_bs = (long long)p->n[0] * p->plane;
    a.rp = p->rp[2];
    a.tw = tw_of<R>(p, 2);
    a.blue = blue_of(p, 2);
    a.B = pick_B(line_rows(a.N, a.blue), sizeof(cpx<R>));
    const long long pairs = (a.lines + 1) / 2;
    dim3 grid((unsigned)((pairs + a.B - 1) / a.B), (unsigned)batch);
    size_t smem = 2 * (size_t)line_rows(a.N, a.blue) * a.B * sizeof(cpx<R>);
    sp_status rc;
    if (forward) {
        if ((rc = set_smem(k_z_forward<R, Tio>, smem))) return rc;
        k_z_forward<R, Tio><<<grid, kThreads, smem, st>>>(a);
    } else {
        if ((rc = set_smem(k_z_inverse<R, Tio>, smem))) return rc;
        k_z_inverse<R, Tio><<<grid, kThreads, smem, st>>>(a);
    }
    return sp_cuda_check(cudaGetLastError(), forward ? "z forward pass" : "z inverse pass");
}

template <class R>
sp_status line_pass(const LineArgs& a0, int outer, int batch, cudaStream_t st, const char* what)
{
    LineArgs a = a0;
    a.B = pick_B(line_rows(a.N, a.blue), sizeof(cpx<R>));
    size_t smem = 2 * (size_t)line_rows(a.N, a.blue) * a.B * sizeof(cpx<R>);
    sp_status rc;
    if ((rc = set_smem(k_lines<R>, smem))) return rc;
    dim3 grid((unsigned)((a.ncol + a.B - 1) / a.B), (unsigned)outer, (unsigned)batch);
    k_lines<R><<<grid, kThreads, smem, st>>>(a);
    return sp_cuda_check(cudaGetLastError(), what);
}

template <class R>
LineArgs y_args(sp_plan p, int sign)
{
    LineArgs a = {};
    a.in = a.out = p->d_work;
    a.N = p->N[1];
    a.nin = sign < 0 ? p->n[1] : p->N[1];
    a.nout = sign < 0 ? p->N[1] : p->n[1];
    a.ncol = p->n[2] + 1;
    a.in_os = a.out_os = p->plane;
    a.in_es = a.out_es = p->ldz;
    a.in_bs = a.out_bs = (long long)p->n[0] * p->plane;
    a.rp = p->rp[1];
    a.tw = tw_of<R>(p, 1);
    a.blue = blue_of(p, 1);
    a.sign = sign;
    return a;
}

template <class R, class Tio>
sp_status solve_t(sp_plan p, const void* rho, void* u, int batch, cudaStream_t st)
{
    sp_status rc;
    p->npass = 5;
    p->pass_name[0] = "z_forward";
    p->pass_name[1] = "y_forward";
    p->pass_name[2] = "x_multiply";
    p->pass_name[3] = "y_inverse";
    p->pass_name[4] = "z_inverse";
    if ((rc = sp_mark(p, st))) return rc;
    if ((rc = z_pass<R, Tio>(p, rho, nullptr, batch, true, st))) return rc;
    if ((rc = sp_mark(p, st))) return rc;
    if ((rc = line_pass<R>(y_args<R>(p, -1), p->n[0], batch, st, "y forward pass"))) return rc;
    if ((rc = sp_mark(p, st))) return rc;
    LineArgs x = {};
    x.in = x.out = p->d_work;
    x.N = p->N[0];
    x.nin = x.nout = p->n[0];
    x.ncol = p->n[2] + 1;
    x.in_os = x.out_os = p->ldz;
    x.in_es = x.out_es = p->plane;
    x.in_bs = x.out_bs = (long long)p->n[0] * p->plane;
    x.rp = p->rp[0];
    x.tw = tw_of<R>(p, 0);
    x.blue = blue_of(p, 0);
    x.sign = -1;
    x.mult = mult_of<R>(p);
    x.No = p->N[1];
    x.nh_line = p->n[0];
    x.ldzM = p->ldz;
    if ((rc = line_pass<R>(x, p->N[1], batch, st, "x pass"))) return rc;
    if ((rc = sp_mark(p, st))) return rc;
    if ((rc = line_pass<R>(y_args<R>(p, +1), p->n[0], batch, st, "y inverse pass"))) return rc;
    if ((rc = sp_mark(p, st))) return rc;
    if ((rc = z_pass<R, Tio>(p, nullptr, u, batch, false, st))) return rc;
    return sp_mark(p, st);
}

template <class R, class Tio>
sp_status forward_t(sp_plan p, const void* rho, void* spec, cudaStream_t st)
{
    sp_status rc;
    if ((rc = z_pass<R, Tio>(p, rho, nullptr, 1, true, st))) return rc;
    if ((rc = line_pass<R>(y_args<R>(p, -1), p->n[0], 1, st, "y forward pass"))) return rc;
    LineArgs x = {};
    x.in = p->d_work;
    x.out = spec;
    x.N = p->N[0];
    x.nin = p->n[0];
    x.nout = p->N[0];
    x.ncol = p->n[2] + 1;
    x.in_os = p->ldz;
    x.in_es = p->plane;
    x.out_os = p->n[2] + 1;
    x.out_es = (long long)p->N[1] * (p->n[2] + 1);
    x.rp = p->rp[0];
    x.tw = tw_of<R>(p, 0);
    x.blue = blue_of(p, 0);
    x.sign = -1;
    return line_pass<R>(x, p->N[1], 1, st, "x forward pass");
}

}  // namespace

bool sp_v2_supported(int N)
{
    return N == 64 || N == 128 || N == 192 || N == 256 || N == 384 || N == 512 || N == 1024;
}

sp_status sp_run_solve(sp_plan p, const void* rho, void* u, int batch, cudaStream_t st)
{
    if (p->persistent) {  // one cooperative launch for all passes (sp_plan_set_persistent)
        switch (p->prec) {
            case SP_FP64: return sp_v2_persistent_f64(p, rho, u, batch, st);
            case SP_FP32: return sp_v2_persistent_f32(p, rho, u, batch, st, false);
            case SP_MIXED: return sp_v2_persistent_f32(p, rho, u, batch, st, true);
            case SP_DF32: return sp_v2_persistent_df(p, rho, u, batch, st);
        }
    }
    // register-resident passes where every axis length has a compiled plan
    sp_status rc = SP_ERR_UNSUPPORTED_SIZE;
    switch (p->prec) {
        case SP_FP64: rc = sp_v2_solve_f64(p, rho, u, batch, st); break;
        case SP_FP32: rc = sp_v2_solve_f32(p, rho, u, batch, st, false); break;
        case SP_MIXED: rc = sp_v2_solve_f32(p, rho, u, batch, st, true); break;
        case SP_DF32: rc = sp_v2_solve_df(p, rho, u, batch, st); break;
    }
    if (rc != SP_ERR_UNSUPPORTED_SIZE) return rc;
    switch (p->prec) {
        case SP_FP64: return solve_t<double, double>(p, rho, u, batch, st);
        case SP_FP32: return solve_t<float, float>(p, rho, u, batch, st);
        case SP_MIXED: return solve_t<float, double>(p, rho, u, batch, st);
        case SP_DF32: return solve_t<df32, double>(p, rho, u, batch, st);
    }
    return sp_fail(SP_ERR_UNSUPPORTED_SIZE, "no pass plan for this grid and precision");
}

sp_status sp_run_forward(sp_plan p, const void* rho, void* spec, cudaStream_t st)
{
    sp_status rc = SP_ERR_UNSUPPORTED_SIZE;
    switch (p->prec) {
        case SP_FP64: rc = sp_v2_forward_f64(p, rho, spec, st); break;
        case SP_FP32: rc = sp_v2_forward_f32(p, rho, spec, st, false); break;
        case SP_MIXED: rc = sp_v2_forward_f32(p, rho, spec, st, true); break;
        case SP_DF32: rc = sp_v2_forward_df(p, rho, spec, st); break;
    }
    if (rc != SP_ERR_UNSUPPORTED_SIZE) return rc;
    switch (p->prec) {
        case SP_FP64: return forward_t<double, double>(p, rho, spec, st);
        case SP_FP32: return forward_t<float, float>(p, rho, spec, st);
        case SP_MIXED: return forward_t<float, double>(p, rho, spec, st);
        case SP_DF32: return forward_t<df32, double>(p, rho, spec, st);
    }
    return sp_fail(SP_ERR_UNSUPPORTED_SIZE, "no pass plan for this grid and precision");
}
