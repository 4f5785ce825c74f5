// One-time precomputation of Alg. 1 on the GPU, all in FP64:
//   K4  GS weights/exponents by sinc quadrature (eq. sin_1_x)
//   K5  1D integral tables G, H of eq. (Gten_sep) per axis
//   K6  multiplier M_k = -|kappa|^2 Vhat_k / Ntilde (eqs. Gten_sep, convtheorem)
//   K7  FFT twiddles exp(-2 pi i j / N)
// K5 and K6 are both contractions over a long index (quadrature nodes, GS terms) and
// run through one tiled FP64 GEMM kernel with problem-specific prologue/epilogue
// kernels.
#include <math.h>
#include <stdio.h>

#include <vector>

#include "sp_internal.h"

namespace {

constexpr double kPi = 3.14159265358979323846264338327950288;
constexpr int kGLQ = 16;          // Gauss-Legendre points per panel
constexpr double kFullLine = 40.0; // a L^2 at or above which the full-line forms are used

// ------------------------------------------------------------------------- K4
// tau_s = tau_lo + s h, a_s = exp(2 tau_s), w_s = (1/(8 pi)) (2/sqrt(pi)) h exp(tau_s):
// the trapezoidal rule for 1/(8 pi r) = (1/(8 pi)) (2/sqrt(pi)) int exp(tau - r^2 e^{2tau}) dtau.
__global__ void k_gs_table(double tau_lo, double h, int terms, double* w, double* a)
{
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= terms) return;
    double tau = tau_lo + s * h;
    a[s] = exp(2.0 * tau);
    w[s] = (1.0 / (4.0 * kPi * sqrt(kPi))) * h * exp(tau);
}

// ------------------------------------------------------------------------- K5
// Gauss-Legendre nodes/weights on [-1, 1] by Newton's method on P_Q (one thread per
// node).  x_i in descending order.
__global__ void k_gauss_legendre(int Q, double* x, double* w)
{
    int i = threadIdx.x;
    if (i >= Q) return;
    double z = cos(kPi * (i + 0.75) / (Q + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
        double p0 = 1.0, p1 = z;
        for (int j = 1; j < Q; ++j) {
            double p2 = ((2.0 * j + 1.0) * z * p1 - j * p0) / (j + 1.0);
            p0 = p1;
            p1 = p2;
        }
        // p1 = P_Q(z), p0 = P_{Q-1}(z)
        dp = Q * (z * p1 - p0) / (z * z - 1.0);
        double dz = p1 / dp;
        z -= dz;
        if (fabs(dz) < 1e-17) break;
    }
    // final derivative at the converged node
    {
        double p0 = 1.0, p1 = z;
        for (int j = 1; j < Q; ++j) {
            double p2 = ((2.0 * j + 1.0) * z * p1 - j * p0) / (j + 1.0);
            p0 = p1;
            p1 = p2;
        }
        dp = Q * (z * p1 - p0) / (z * z - 1.0);
    }
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
}

// Quadrature nodes of the composite rule: P panels of Q points on [0, L].
// t[j] = (panel + (1 + x_i)/2) position in units of the panel width, wq[j] = weight.
__global__ void k_nodes(int P, int Q, double L, const double* gx, const double* gw,
                        double* tpos, double* y, double* wq)
{
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= P * Q) return;
    int panel = j / Q, i = j % Q;
    double t = 0.5 * (1.0 + gx[i]);
    tpos[j] = t;
    y[j] = L * (panel + t) / P;
    wq[j] = 0.5 * (L / P) * gw[i];
}

// Quadrature weights times the integrands, per GS row s and node j:
//   E0 = wq f,  E2 = wq g,  F0 = wq f'''',  F2 = wq g''''
// with f = exp(-a y^2), g = y^2 exp(-a y^2) and their fourth derivatives
//   f'''' = (16a^4y^4 - 48a^3y^2 + 12a^2) f,  g'''' = (16a^4y^6 - 112a^3y^4 + 156a^2y^2 - 24a) f.
__global__ void k_gauss_rows(int rows, int nq, const double* a, const double* y,
                             const double* wq, double* E0, double* E2, double* F0, double* F2)
{
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)rows * nq) return;
    int s = (int)(idx / nq), j = (int)(idx % nq);
    double al = a[s], a2 = al * al, a3 = a2 * al, a4 = a3 * al;
    double yy = y[j] * y[j];
    double e = wq[j] * exp(-al * yy);
    E0[idx] = e;
    E2[idx] = e * yy;
    F0[idx] = (16.0 * a4 * yy * yy - 48.0 * a3 * yy + 12.0 * a2) * e;
    F2[idx] = (16.0 * a4 * yy * yy * yy - 112.0 * a3 * yy * yy + 156.0 * a2 * yy - 24.0 * al) * e;
}

// C[k][j] = cos(pi k y_j / L) = cos(pi ((k panel mod 2P) + k t_j) / P): the integer part
// of the phase is reduced exactly before the floating-point product.
__global__ void k_cos_rows(int nk, int P, int Q, const double* tpos, double* C)
{
    long long nq = (long long)P * Q;
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= nk * nq) return;
    int k = (int)(idx / nq);
    int j = (int)(idx % nq);
    int panel = j / Q;
    long long red = ((long long)k * panel) % (2LL * P);
    C[idx] = cospi(((double)red + (double)k * tpos[j]) / (double)P);
}

// Rows with a_s L^2 >= kFullLine: the window cut is below exp(-40) relative, and the
// full-line transforms hold:  G = sqrt(pi/a) e^{-kappa^2/4a},
// H = sqrt(pi)/(2 a^{3/2}) (1 - kappa^2/(2a)) e^{-kappa^2/4a}.
__global__ void k_full_line(int s0, int terms, int nk, double L, const double* a, double* G,
                            double* H)
{
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long rows = terms - s0;
    if (idx >= rows * nk) return;
    int s = s0 + (int)(idx / nk), k = (int)(idx % nk);
    double al = a[s];
    double kap = kPi * k / L;
    double q = kap * kap / (4.0 * al);
    double ex = exp(-q);
    G[(long long)s * nk + k] = sqrt(kPi / al) * ex;
    H[(long long)s * nk + k] = sqrt(kPi) / (2.0 * al * sqrt(al)) * (1.0 - 2.0 * q) * ex;
}

// ------------------------------------------------------------------------- GEMM
// C[m][n] = sum_k A[m][k] B[n][k] (both operands K-contiguous), FP64, 64x64 tiles,
// 256 threads with 4x4 outputs each, K staged through shared memory 16 at a time.
// The epilogue functor receives (m, n, value).
constexpr int TM = 64, TN = 64, TK = 16;

template <class Epi>
__global__ void __launch_bounds__(256) k_dgemm_nt(int M, int N, int K, const double* __restrict__ A,
                                                  long long lda, const double* __restrict__ B,
                                                  long long ldb, Epi epi)
{
    __shared__ double As[TK][TM + 1];
    __shared__ double Bs[TK][TN + 1];
    int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
    double acc[4][4] = {};
    for (int k0 = 0; k0 < K; k0 += TK) {
        for (int l = threadIdx.x; l < TM * TK; l += 256) {
            int r = l / TK, c = l % TK;
            int gm = m0 + r, gk = k0 + c;
            As[c][r] = (gm < M && gk < K) ? A[(long long)gm * lda + gk] : 0.0;
            int gn = n0 + r;
            Bs[c][r] = (gn < N && gk < K) ? B[(long long)gn * ldb + gk] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int c = 0; c < TK; ++c) {
            double av[4], bv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) av[i] = As[c][ty + 16 * i];
#pragma unroll
            for (int i = 0; i < 4; ++i) bv[i] = Bs[c][tx + 16 * i];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int gm = m0 + ty + 16 * i, gn = n0 + tx + 16 * j;
            if (gm < M && gn < N) epi(gm, gn, acc[i][j]);
        }
}

// The 1D integrals are taken in one of two exact forms per (s, k):
//  direct  (k = 0 or kappa^2 < 4 a_s):  I = int_0^L P(y) cos(kappa y) dy
//  by parts (otherwise): with kappa L = pi k and P even (P'(0) = P'''(0) = 0),
//     I = (-1)^k [P'(L)/kappa^2 - P'''(L)/kappa^4] + (1/kappa^4) int_0^L P''''(y) cos(kappa y) dy,
// which keeps the boundary terms exact where I is small next to the size of P, so that
// G and H have relative (not only absolute) accuracy at high wavenumber.
__device__ __forceinline__ bool by_parts(int k, double kap, double al) { return k > 0 && kap * kap >= 4.0 * al; }

struct EpiDirect {  // out[s][k] = 2 v where the direct form applies
    double* out;
    long long ld;
    const double* a;
    double L;
    __device__ void operator()(int m, int n, double v) const
    {
        double kap = kPi * n / L;
        if (!by_parts(n, kap, a[m])) out[(long long)m * ld + n] = 2.0 * v;
    }
};

struct EpiByParts {  // out[s][k] = 2 ((-1)^k (P'(L)/kappa^2 - P'''(L)/kappa^4) + v / kappa^4)
    double* out;
    long long ld;
    const double* a;
    double L;
    int which;  // 0: P = f = exp(-a y^2); 1: P = g = y^2 exp(-a y^2)
    __device__ void operator()(int m, int n, double v) const
    {
        double al = a[m];
        double kap = kPi * n / L;
        if (!by_parts(n, kap, al)) return;
        double e = exp(-al * L * L), a2 = al * al, a3 = a2 * al, L2 = L * L;
        double d1, d3;
        if (which == 0) {
            d1 = -2.0 * al * L * e;
            d3 = (-8.0 * a3 * L2 * L + 12.0 * a2 * L) * e;
        } else {
            d1 = (2.0 * L - 2.0 * al * L2 * L) * e;
            d3 = (-24.0 * al * L + 36.0 * a2 * L2 * L - 8.0 * a3 * L2 * L2 * L) * e;
        }
        double sgn = (n & 1) ? -1.0 : 1.0;
        double k2 = kap * kap, k4 = k2 * k2;
        out[(long long)m * ld + n] = 2.0 * (sgn * (d1 / k2 - d3 / k4) + v / k4);
    }
};

// ------------------------------------------------------------------------- K6
// A'[row][c], row = k1 (n0+1) + k0 in [row0, row0 + rows):
//   c <  S: w_c (H0[c][k0] G1[c][k1] + G0[c][k0] H1[c][k1])
//   c >= S: w_{c-S} G0[c-S][k0] G1[c-S][k1]
__global__ void k_mult_lhs(int row0, int rows, int S, int n0p, int n1p, const double* w,
                           const double* G0, const double* H0, const double* G1,
                           const double* H1, double* Ap)
{
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)rows * 2 * S) return;
    int r = (int)(idx / (2 * S)), c = (int)(idx % (2 * S));
    int row = row0 + r;
    int k1 = row / n0p, k0 = row % n0p;
    int s = c < S ? c : c - S;
    double g0 = G0[(long long)s * n0p + k0], h0 = H0[(long long)s * n0p + k0];
    double g1 = G1[(long long)s * n1p + k1], h1 = H1[(long long)s * n1p + k1];
    Ap[idx] = c < S ? w[s] * (h0 * g1 + g0 * h1) : w[s] * (g0 * g1);
}

// Original GS method without near-field correction: A'[row][s] = 2 w_s G0 G1 (the GS of
// 1/(4 pi r) is twice the 1/(8 pi r) table), B'[kz][s] = G2: V = sum_s 2 w_s G0 G1 G2.
__global__ void k_plain_lhs(int row0, int rows, int S, int n0p, int n1p, const double* w,
                            const double* G0, const double* G1, double* Ap)
{
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)rows * S) return;
    int r = (int)(idx / S), s = (int)(idx % S);
    int row = row0 + r;
    int k1 = row / n0p, k0 = row % n0p;
    Ap[idx] = 2.0 * w[s] * G0[(long long)s * n0p + k0] * G1[(long long)s * n1p + k1];
}

__global__ void k_plain_rhs(int S, int n2p, const double* G2, double* Bp)
{
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)n2p * S) return;
    int kz = (int)(idx / S), s = (int)(idx % S);
    Bp[idx] = G2[(long long)s * n2p + kz];
}

// B'[kz][c]: c < S: G2[c][kz], c >= S: H2[c-S][kz]
__global__ void k_mult_rhs(int S, int n2p, const double* G2, const double* H2, double* Bp)
{
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)n2p * 2 * S) return;
    int kz = (int)(idx / (2 * S)), c = (int)(idx % (2 * S));
    Bp[idx] = c < S ? G2[(long long)c * n2p + kz] : H2[(long long)(c - S) * n2p + kz];
}

struct EpiMultiplier {  // M[row][kz] = -(kappa0^2 + kappa1^2 + kappa2^2) V / Ntilde (or V / Ntilde)
    double* M;
    int ldz, row0, n0p;
    double c0, c1, c2;  // (pi / L_p)^2
    double invN;
    int laplacian;      // 1: super-potential (spectral Laplacian applied); 0: plain GS kernel
    __device__ void operator()(int m, int n, double v) const
    {
        int row = row0 + m;
        int k1 = row / n0p, k0 = row % n0p;
        double k2sum = c0 * (double)k0 * k0 + c1 * (double)k1 * k1 + c2 * (double)n * n;
        M[(long long)row * ldz + n] = laplacian ? -k2sum * v * invN : v * invN;
    }
};

__global__ void k_to_f32(long long count, const double* in, float* out)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) out[i] = (float)in[i];
}

__global__ void k_to_df(long long count, const double* in, df32* out)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) out[i] = df_from_double(in[i]);
}

// ------------------------------------------------------------------------- K7
__global__ void k_twiddles(int N, cpx<double>* tw64, cpx<float>* tw32, cpx<df32>* twdf)
{
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    double s, c;
    sincospi(2.0 * (double)j / (double)N, &s, &c);
    tw64[j] = mk(c, -s);
    tw32[j] = mk((float)c, (float)-s);
    twdf[j] = mk(df_from_double(c), df_from_double(-s));
}

inline unsigned nblk(long long n, int t) { return (unsigned)((n + t - 1) / t); }

struct DevBuf {  // scratch device allocation freed at scope exit (stream-ordered)
    void* p = nullptr;
    cudaStream_t st;
    explicit DevBuf(cudaStream_t s) : st(s) {}
    cudaError_t alloc(size_t bytes) { return cudaMallocAsync(&p, bytes, st); }
    ~DevBuf() { if (p) cudaFreeAsync(p, st); }
    double* d() const { return (double*)p; }
};

}  // namespace

// 1D tables of one axis: G, H [S][n+1].
static sp_status setup_axis(sp_plan p, int ax, cudaStream_t st)
{
    const int n = p->n[ax], nk = n + 1, S = p->gs_terms;
    const double L = p->L[ax];
    // split between quadrature rows and full-line rows (a_s increases with s)
    const double* a = p->h_gs_a;
    int s_split = S;
    for (int s = 0; s < S; ++s)
        if (a[s] * L * L >= kFullLine) { s_split = s; break; }
    sp_status rc;
    // full-line rows
    if (s_split < S) {
        k_full_line<<<nblk((long long)(S - s_split) * nk, 256), 256, 0, st>>>(
            s_split, S, nk, L, p->d_gs_a, p->d_G[ax], p->d_H[ax]);
    }
    if (s_split > 0) {
        const int P = n > 8 ? n : 8, Q = kGLQ;
        const long long nq = (long long)P * Q;
        DevBuf gl(st), nodes(st), E(st), C(st);
        const long long rn = (long long)s_split * nq;
        if (gl.alloc(sizeof(double) * 2 * Q) || nodes.alloc(sizeof(double) * 3 * nq) ||
            E.alloc(sizeof(double) * 4 * rn) || C.alloc(sizeof(double) * nk * nq))
            return sp_fail(SP_ERR_OOM, "setup: quadrature scratch allocation failed");
        double *gx = gl.d(), *gw = gl.d() + Q;
        double *tpos = nodes.d(), *y = nodes.d() + nq, *wq = nodes.d() + 2 * nq;
        double *E0 = E.d(), *E2 = E0 + rn, *F0 = E2 + rn, *F2 = F0 + rn;
        k_gauss_legendre<<<1, 32, 0, st>>>(Q, gx, gw);
        k_nodes<<<nblk(nq, 256), 256, 0, st>>>(P, Q, L, gx, gw, tpos, y, wq);
        k_gauss_rows<<<nblk(rn, 256), 256, 0, st>>>(s_split, (int)nq, p->d_gs_a, y, wq, E0, E2, F0, F2);
        k_cos_rows<<<nblk(nk * nq, 256), 256, 0, st>>>(nk, P, Q, tpos, C.d());
        dim3 grid(nblk(nk, TN), nblk(s_split, TM));
        k_dgemm_nt<<<grid, 256, 0, st>>>(s_split, nk, (int)nq, E0, nq, C.d(), nq,
                                         EpiDirect{p->d_G[ax], nk, p->d_gs_a, L});
        k_dgemm_nt<<<grid, 256, 0, st>>>(s_split, nk, (int)nq, E2, nq, C.d(), nq,
                                         EpiDirect{p->d_H[ax], nk, p->d_gs_a, L});
        k_dgemm_nt<<<grid, 256, 0, st>>>(s_split, nk, (int)nq, F0, nq, C.d(), nq,
                                         EpiByParts{p->d_G[ax], nk, p->d_gs_a, L, 0});
        k_dgemm_nt<<<grid, 256, 0, st>>>(s_split, nk, (int)nq, F2, nq, C.d(), nq,
                                         EpiByParts{p->d_H[ax], nk, p->d_gs_a, L, 1});
        rc = sp_cuda_check(cudaGetLastError(), "setup: 1D integral kernels");
        if (rc) return rc;
    }
    return sp_cuda_check(cudaGetLastError(), "setup: full-line kernel");
}

// GS table of eq. (sin_1_x) for the plan's (eps, delta): tau_s = tau_lo + s h_tau for
// s = 0..terms-1 (reading of the paper's sinc quadrature, see k_gs_table).
static void gs_range(const sp_plan p, double* tau_lo, int* terms)
{
    *tau_lo = log(p->eta * sqrt(kPi) / (2.0 * p->delta));
    const double tau_hi = log(sqrt(log(1.0 / p->eta)) / p->eps) + 0.5;
    *terms = (int)ceil((tau_hi - *tau_lo) / p->h_tau) + 1;
}

int sp_gs_terms(const sp_plan p)
{
    double tau_lo;
    int terms;
    gs_range(p, &tau_lo, &terms);
    return terms;
}

void sp_gs_exponents(const sp_plan p, double* a)
{
    double tau_lo;
    int terms;
    gs_range(p, &tau_lo, &terms);
    for (int s = 0; s < terms; ++s) a[s] = exp(2.0 * (tau_lo + s * p->h_tau));
}

sp_status sp_setup_run(sp_plan p, cudaStream_t st)
{
    sp_status rc;
    // K4: GS table (unless the caller supplied one at plan creation)
    if (!p->gs_user) {
        double tau_lo;
        int terms;
        gs_range(p, &tau_lo, &terms);
        if (terms != p->gs_terms) return sp_fail(SP_ERR_INVALID, "internal: GS table length changed");
        k_gs_table<<<nblk(terms, 128), 128, 0, st>>>(tau_lo, p->h_tau, terms, p->d_gs_w, p->d_gs_a);
        if ((rc = sp_cuda_check(cudaGetLastError(), "GS table kernel"))) return rc;
    }
    // per-axis tables (allocated with the plan; axes with the same (n, L) share one)
    for (int ax = 0; ax < 3; ++ax) {
        bool shared = false;
        for (int q = 0; q < ax; ++q)
            if (p->d_G[q] == p->d_G[ax]) shared = true;
        if (shared) continue;
        if ((rc = setup_axis(p, ax, st))) return rc;
    }
    const int S = p->gs_terms;
    // K6: multiplier, GEMM over the 2S GS columns, in row chunks
    {
        const int n0p = p->n[0] + 1, n1p = p->n[1] + 1, n2p = p->n[2] + 1;
        const long long rows_total = (long long)n0p * n1p;
        const int chunk = (int)(rows_total < 8192 ? rows_total : 8192);
        const bool plain = p->kernel == SP_KERNEL_GS_PLAIN;
        const int K = plain ? S : 2 * S;  // contraction length (GS columns)
        DevBuf Ap(st), Bp(st);
        if (Ap.alloc(sizeof(double) * (size_t)chunk * K) || Bp.alloc(sizeof(double) * (size_t)n2p * K))
            return sp_fail(SP_ERR_OOM, "setup: multiplier scratch allocation failed");
        if (plain)
            k_plain_rhs<<<nblk((long long)n2p * S, 256), 256, 0, st>>>(S, n2p, p->d_G[2], Bp.d());
        else
            k_mult_rhs<<<nblk((long long)n2p * 2 * S, 256), 256, 0, st>>>(S, n2p, p->d_G[2], p->d_H[2], Bp.d());
        EpiMultiplier epi;
        epi.M = p->d_M64;
        epi.ldz = p->ldz;
        epi.n0p = n0p;
        epi.c0 = (kPi / p->L[0]) * (kPi / p->L[0]);
        epi.c1 = (kPi / p->L[1]) * (kPi / p->L[1]);
        epi.c2 = (kPi / p->L[2]) * (kPi / p->L[2]);
        epi.invN = 1.0 / (8.0 * (double)p->n[0] * (double)p->n[1] * (double)p->n[2]);
        epi.laplacian = plain ? 0 : 1;
        for (long long r0 = 0; r0 < rows_total; r0 += chunk) {
            int rows = (int)((rows_total - r0) < chunk ? (rows_total - r0) : chunk);
            if (plain)
                k_plain_lhs<<<nblk((long long)rows * S, 256), 256, 0, st>>>(
                    (int)r0, rows, S, n0p, n1p, p->d_gs_w, p->d_G[0], p->d_G[1], Ap.d());
            else
                k_mult_lhs<<<nblk((long long)rows * 2 * S, 256), 256, 0, st>>>(
                    (int)r0, rows, S, n0p, n1p, p->d_gs_w, p->d_G[0], p->d_H[0], p->d_G[1], p->d_H[1], Ap.d());
            epi.row0 = (int)r0;
            dim3 grid(nblk(n2p, TN), nblk(rows, TM));
            k_dgemm_nt<<<grid, 256, 0, st>>>(rows, n2p, K, Ap.d(), K, Bp.d(), K, epi);
        }
        long long mcount = rows_total * p->ldz;
        if (p->d_M32) k_to_f32<<<nblk(mcount, 256), 256, 0, st>>>(mcount, p->d_M64, p->d_M32);
        if (p->d_Mdf) k_to_df<<<nblk(mcount, 256), 256, 0, st>>>(mcount, p->d_M64, p->d_Mdf);
        if ((rc = sp_cuda_check(cudaGetLastError(), "multiplier kernels"))) return rc;
    }
    // K7: twiddles
    for (int ax = 0; ax < 3; ++ax) {
        k_twiddles<<<nblk(p->N[ax], 256), 256, 0, st>>>(p->N[ax], p->d_tw64[ax], p->d_tw32[ax], p->d_twdf[ax]);
    }
    if ((rc = sp_cuda_check(cudaGetLastError(), "twiddle kernel"))) return rc;
    if (p->prec == SP_DF32) return sp_v2_stage_twiddles_df(p, st);
    if (p->prec == SP_FP32 || p->prec == SP_MIXED) return sp_v2_stage_twiddles_f32(p, st);
    return SP_OK;
}
