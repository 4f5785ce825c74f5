// Tables for Bluestein's algorithm (the chirp-z transform) on axes whose padded length N
// has a prime factor above 7, where no radix 2/3/4/5/7/8 plan exists.  With
// jk = (j^2 + k^2 - (k - j)^2) / 2 the length-N DFT becomes a convolution:
//   forward  X_k = c_k sum_j (x_j c_j) conj(c_{k-j}),   c_m = exp(-i pi m^2 / N),
//   inverse  X_k = conj(c_k) sum_j (x_j conj(c_j)) c_{k-j},
// which the passes evaluate as a circular convolution of length M (a power of two,
// M >= 2N - 1) through M-point FFTs.  Built here in double on the host, once per plan:
//   chirp   c_j, j < N, from the phase index j^2 mod 2N (no large angles);
//   filters D_fwd = FFT_M(e_fwd) / M and D_inv = FFT_M(e_inv) / M, where e holds the
//           filter (conj c for the forward transform, c for the inverse) at m and M - m,
//           m < N, and zeros between;
//   twiddles exp(-2 pi i q / M), q < M, for the M-point stages;
// then rounded to the plan's arithmetic type (double-float: split into hi + lo).
#include <math.h>

#include <complex>
#include <utility>
#include <vector>

#include "sp_internal.h"

namespace {

using cd = std::complex<double>;

// Unnormalised X_k = sum_j a_j exp(sign 2 pi i jk / M), M a power of two (iterative
// radix 2; each twiddle from cos/sin of its own angle).
void fft_pow2(std::vector<cd>& a, int sign)
{
    const int M = (int)a.size();
    for (int i = 1, j = 0; i < M; ++i) {
        int bit = M >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) std::swap(a[i], a[j]);
    }
    for (int len = 2; len <= M; len <<= 1) {
        const int half = len / 2, step = M / len;
        for (int i = 0; i < M; i += len)
            for (int k = 0; k < half; ++k) {
                const double ang = 2.0 * M_PI * (double)(k * step) / (double)M;
                const cd w(cos(ang), sign * sin(ang));
                const cd u = a[i + k], v = a[i + k + half] * w;
                a[i + k] = u + v;
                a[i + k + half] = u - v;
            }
    }
}

// The table of one axis in double: [chirp N][D_fwd M][D_inv M][twiddles M].
std::vector<cd> tables(int N, int M)
{
    std::vector<cd> out((size_t)N + 3 * (size_t)M);
    std::vector<cd> c(N);
    for (int j = 0; j < N; ++j) {
        const long long ph = (long long)j * j % (2LL * N);
        const double ang = M_PI * (double)ph / (double)N;
        c[j] = cd(cos(ang), -sin(ang));
        out[j] = c[j];
    }
    for (int dir = 0; dir < 2; ++dir) {  // 0: forward filter conj(c), 1: inverse filter c
        std::vector<cd> e(M, cd(0.0, 0.0));
        for (int m = 0; m < N; ++m) {
            const cd f = dir == 0 ? std::conj(c[m]) : c[m];
            e[m] = f;
            if (m > 0) e[M - m] = f;
        }
        fft_pow2(e, -1);
        for (int q = 0; q < M; ++q) out[(size_t)N + (size_t)dir * M + q] = e[q] / (double)M;
    }
    for (int q = 0; q < M; ++q) {
        const double ang = 2.0 * M_PI * (double)q / (double)M;
        out[(size_t)N + 2 * (size_t)M + q] = cd(cos(ang), -sin(ang));
    }
    return out;
}

size_t csize(sp_precision prec)
{
    return prec == SP_FP64 || prec == SP_DF32 ? 16 : 8;  // cpx<double>, cpx<df32> / cpx<float>
}

size_t table_bytes(int N, int M, sp_precision prec) { return csize(prec) * ((size_t)N + 3 * (size_t)M); }

void fill(int N, int M, sp_precision prec, void* host)
{
    const std::vector<cd> t = tables(N, M);
    for (size_t i = 0; i < t.size(); ++i) {
        const double re = t[i].real(), im = t[i].imag();
        switch (prec) {
            case SP_FP64: static_cast<cpx<double>*>(host)[i] = mk(re, im); break;
            case SP_DF32: static_cast<cpx<df32>*>(host)[i] = mk(df_from_double(re), df_from_double(im)); break;
            default: static_cast<cpx<float>*>(host)[i] = mk((float)re, (float)im); break;
        }
    }
}

}  // namespace

size_t sp_bluestein_bytes(const sp_plan_s* p, int ax) { return table_bytes(p->N[ax], p->blue_M[ax], p->prec); }

void sp_bluestein_fill(const sp_plan_s* p, int ax, void* host) { fill(p->N[ax], p->blue_M[ax], p->prec, host); }

extern "C" sp_status sp_bluestein_table(int n, sp_precision prec, int* M, void* out, size_t* bytes)
{
    sp_clear_error();
    if (!M || !bytes) return sp_fail(SP_ERR_INVALID, "M and bytes must be non-NULL");
    if (prec != SP_FP64 && prec != SP_FP32 && prec != SP_MIXED && prec != SP_DF32)
        return sp_fail(SP_ERR_INVALID, "unknown precision %d", (int)prec);
    if (n < 2 || n > 1024) return sp_fail(SP_ERR_UNSUPPORTED_SIZE, "n = %d: need 2 <= n <= 1024", n);
    const int N = 2 * n;
    RadixPlan rp;
    if (sp_radix_plan(N, &rp))
        return sp_fail(SP_ERR_UNSUPPORTED_SIZE, "2n = %d: Bluestein serves 2n <= 2048 with a prime factor above 7", N);
    int m = 1;
    while (m < 2 * N - 1) m *= 2;
    *M = m;
    const size_t need = table_bytes(N, m, prec);
    if (!out) {
        *bytes = need;
        return SP_OK;
    }
    if (*bytes < need) return sp_fail(SP_ERR_INVALID, "buffer of %zu bytes; the table needs %zu", *bytes, need);
    fill(N, m, prec, out);
    return SP_OK;
}
