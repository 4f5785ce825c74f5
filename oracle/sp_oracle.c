/*
 * Plain FP64 CPU oracle for the super-potential GS/FFT free-space Poisson solve
 * (Exl & Schaffer, "Near-field-free super-potential FFT method for the
 * three-dimensional free-space Poisson equation", arXiv:2506.04489).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct restatement
 * of the method that the CUDA library is checked against.  Only the test suite,
 * the smoke check and the CPU-baseline leg of the benchmark may load it; the
 * product library never links, calls or falls back to it.  It shares no code,
 * header, table or constant generator with the CUDA path.
 *
 * Every function follows one passage of the paper, cited beside it.  Where the
 * paper is silent the reading taken is stated in the comment:
 *   - grid: x_j = lo + j*h, h = (hi-lo)/(n-1) (both box faces are grid points);
 *   - padding factor 2 (Sec. 2, Alg. 1): period 2*n*h per axis, so the kernel
 *     window is [-L, L] with L = n*h and the wavenumbers are kappa_k = pi*k/L;
 *   - GS table: trapezoidal (sinc) quadrature of the integral representation
 *     1/r = (2/sqrt(pi)) * int_R exp(tau - r^2 e^{2 tau}) d tau  (Sec. 2, the
 *     Gamma-function identity with n = 0 and eq. (sin_1_x)).
 *
 * Parity pins for each function live in tests/ (closed forms, brute force,
 * library routines, the paper's printed tables).
 *
 * Complex arrays are interleaved (re, im) doubles.  No function allocates more
 * than its own temporaries; the caller owns every array passed in.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <float.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_PI 3.14159265358979323846264338327950288

/* ------------------------------------------------------------------------- */
/* Threads                                                                    */
/* ------------------------------------------------------------------------- */

void or_set_threads(int t)
{
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}

int or_get_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------- */
/* Gaussian-sum table, Sec. 2 eq. (sin_1_x)                                   */
/* ------------------------------------------------------------------------- */
/*
 * 1/(8 pi r) ~ sum_s w_s exp(-a_s r^2) on (eps, delta].
 * Substituting t = e^tau in (2/sqrt(pi)) int_0^inf exp(-r^2 t^2) dt = 1/r gives
 * an integrand exp(tau - r^2 e^{2 tau}) that is analytic in a strip and decays
 * doubly exponentially on both sides; the trapezoidal rule with step h_tau on
 * [tau_lo, tau_hi] is the sinc quadrature of the paper:
 *     tau_s = tau_lo + s*h_tau,  a_s = exp(2 tau_s),
 *     w_s   = (1/(8 pi)) (2/sqrt(pi)) h_tau exp(tau_s).
 * Truncation limits (reading: the paper names only S and c0):
 *     lower: the dropped part is below e^{tau_lo} (2/sqrt(pi)) r, relative eta at r = delta
 *            => tau_lo = ln(eta sqrt(pi) / (2 delta));
 *     upper: the dropped part is erfc(r e^{tau_hi}) relative; at r = eps this is
 *            below eta when e^{tau_hi} >= sqrt(ln(1/eta))/eps; half a unit of
 *            tau is added as margin.
 * Returns S+1 (the number of terms written), or -1 if max_terms is too small.
 */
int or_gs_table(double eps, double delta, double h_tau, double eta,
                int max_terms, double* w, double* a)
{
    double tau_lo = log(eta * sqrt(OR_PI) / (2.0 * delta));
    double tau_hi = log(sqrt(log(1.0 / eta)) / eps) + 0.5;
    int S = (int)ceil((tau_hi - tau_lo) / h_tau);
    if (S + 1 > max_terms) return -1;
    for (int s = 0; s <= S; ++s) {
        double tau = tau_lo + s * h_tau;
        a[s] = exp(2.0 * tau);
        w[s] = (1.0 / (8.0 * OR_PI)) * (2.0 / sqrt(OR_PI)) * h_tau * exp(tau);
    }
    return S + 1;
}

/* U_GS(r) * 8 pi r, i.e. the relative accuracy factor of eq. (sin_1_x) (Fig. 1). */
double or_gs_ratio(double r, int terms, const double* w, const double* a)
{
    long double acc = 0.0L;
    for (int s = 0; s < terms; ++s)
        acc += (long double)w[s] * expl(-(long double)a[s] * (long double)r * (long double)r);
    return (double)(acc * 8.0L * (long double)OR_PI * (long double)r);
}

/* ------------------------------------------------------------------------- */
/* One-dimensional integrals of eq. (Gten_sep), adaptive Gauss-Kronrod        */
/* ------------------------------------------------------------------------- */
/*
 * G(alpha, kappa) = 2 int_0^L exp(-alpha y^2) cos(kappa y) dy
 * H(alpha, kappa) = 2 int_0^L y^2 exp(-alpha y^2) cos(kappa y) dy
 * (the paper's factors for p != q and p == q; its window [0,1] is [0,L] in the
 * user's units).  The paper computes them by Gauss-Kronrod to machine
 * precision; this is a plain adaptive 7-point Gauss / 15-point Kronrod rule with
 * bisection, for every alpha (no closed forms are used here).
 *
 * Kronrod-15 abscissae and weights, and the embedded Gauss-7 weights (the
 * classical published values; tests check their polynomial exactness).
 */
static const double or_xk15[8] = {
    0.991455371120812639206854697526329, 0.949107912342758524526189684047851,
    0.864864423359769072789712788640926, 0.741531185599394439863864773280788,
    0.586087235467691130294144845693013, 0.405845151377397166906606412076961,
    0.207784955007898467600689403773245, 0.000000000000000000000000000000000};
static const double or_wk15[8] = {
    0.022935322010529224963732008058970, 0.063092092629978553290700663189204,
    0.104790010322250183839876322541518, 0.140653259715525918745189590510238,
    0.169004726639267902826583426598550, 0.190350578064785409913256402421014,
    0.204432940075298892414161999234649, 0.209482141084727828012999174891714};
static const double or_wg7[4] = { /* weights of the Gauss nodes xk15[1], [3], [5], [7] */
    0.129484966168869693270611432679082, 0.279705391489276667901467771423780,
    0.381830050505118944950369775488975, 0.417959183673469387755102040816327};

/*
 * Integrands on [0, L], each a polynomial in y times exp(-alpha y^2), multiplied by
 * cos(kappa y):
 *   DIRECT:  f = exp(-a y^2)  and  g = y^2 exp(-a y^2)
 *   FOURTH:  the fourth derivatives
 *            f4 = (16a^4y^4 - 48a^3y^2 + 12a^2) exp(-a y^2)
 *            g4 = (16a^4y^6 - 112a^3y^4 + 156a^2y^2 - 24a) exp(-a y^2)
 */
enum { OR_DIRECT = 0, OR_FOURTH = 1 };

static void or_integrand(int which, double alpha, double y, double* p0, double* p2)
{
    double e = exp(-alpha * y * y);
    double y2 = y * y;
    if (which == OR_DIRECT) {
        *p0 = e;
        *p2 = y2 * e;
    } else {
        double a2 = alpha * alpha, a3 = a2 * alpha, a4 = a3 * alpha;
        *p0 = (16.0 * a4 * y2 * y2 - 48.0 * a3 * y2 + 12.0 * a2) * e;
        *p2 = (16.0 * a4 * y2 * y2 * y2 - 112.0 * a3 * y2 * y2 + 156.0 * a2 * y2 - 24.0 * alpha) * e;
    }
}

/* Apply the G7/K15 pair to both integrands (times cos(kappa y)) on [lo, hi].
   abs15 receives the K15 rule applied to their absolute values. */
static void or_gk15(int which, double alpha, double kappa, double lo, double hi,
                    double k15[2], double g7[2], double abs15[2])
{
    double c = 0.5 * (lo + hi), hw = 0.5 * (hi - lo);
    k15[0] = k15[1] = g7[0] = g7[1] = abs15[0] = abs15[1] = 0.0;
    for (int i = 0; i < 8; ++i) {
        int npts = (i == 7) ? 1 : 2;
        for (int sgn = 0; sgn < npts; ++sgn) {
            double y = (sgn == 0) ? c + hw * or_xk15[i] : c - hw * or_xk15[i];
            double p0, p2;
            or_integrand(which, alpha, y, &p0, &p2);
            double cs = cos(kappa * y);
            double f0 = p0 * cs, f2 = p2 * cs;
            k15[0] += or_wk15[i] * f0;
            k15[1] += or_wk15[i] * f2;
            abs15[0] += or_wk15[i] * fabs(p0);
            abs15[1] += or_wk15[i] * fabs(p2);
            if (i & 1) {
                g7[0] += or_wg7[i >> 1] * f0;
                g7[1] += or_wg7[i >> 1] * f2;
            }
        }
    }
    k15[0] *= hw; k15[1] *= hw; g7[0] *= hw; g7[1] *= hw;
    abs15[0] *= hw; abs15[1] *= hw;
}

/*
 * Bisection until the Gauss-7 estimate agrees with Kronrod-15 to the interval's
 * share of the tolerance.  The Kronrod result is then far more accurate than
 * the difference (its degree is 22 against 13), so the tolerance on the
 * difference can sit well above the rounding level.  An interval whose
 * difference is already at the rounding level of its own sum is accepted too,
 * and bisection stops at depth 30.
 */
static void or_gk_adapt(int which, double alpha, double kappa, double lo, double hi,
                        double tol0, double tol2, int depth, double out[2])
{
    double k15[2], g7[2], ab[2];
    or_gk15(which, alpha, kappa, lo, hi, k15, g7, ab);
    double e0 = fabs(k15[0] - g7[0]), e2 = fabs(k15[1] - g7[1]);
    int ok0 = e0 <= tol0 || e0 <= 50.0 * DBL_EPSILON * ab[0];
    int ok2 = e2 <= tol2 || e2 <= 50.0 * DBL_EPSILON * ab[1];
    if (depth >= 30 || (ok0 && ok2)) {
        out[0] += k15[0];
        out[1] += k15[1];
        return;
    }
    double mid = 0.5 * (lo + hi);
    or_gk_adapt(which, alpha, kappa, lo, mid, 0.5 * tol0, 0.5 * tol2, depth + 1, out);
    or_gk_adapt(which, alpha, kappa, mid, hi, 0.5 * tol0, 0.5 * tol2, depth + 1, out);
}

/*
 * int_0^L P(y) cos(kappa y) dy for both integrands of `which`, by adaptive G7/K15
 * started from a plain initial partition, so that no first panel can miss the
 * integrand: breakpoints at 0, w, 2w, 4w, ... (w = 1/sqrt(alpha), the width of the
 * Gaussian, when it is below L/2), and each piece cut into equal parts no longer
 * than half a period of cos(kappa y).  The tolerance is relative to the integral of
 * |P| over [0, L] (estimated on that partition), because the oscillating integral
 * itself can cancel to far below it.
 */
#define OR_MAX_PIECES 8192
static void or_quad(int which, double alpha, double L, double kappa, double out[2])
{
    const double rel = 1e-14;
    double sa = sqrt(alpha);
    double bp[80];
    int nb = 0;
    bp[nb++] = 0.0;
    double wdt = (sa > 0.0) ? 1.0 / sa : L;
    for (double b = wdt; b < 0.5 * L && nb < 70; b *= 2.0) bp[nb++] = b;
    bp[nb++] = L;
    static _Thread_local double lo_[OR_MAX_PIECES], hi_[OR_MAX_PIECES];
    int np = 0;
    for (int i = 0; i + 1 < nb; ++i) {
        double len = bp[i + 1] - bp[i];
        int parts = (int)ceil(len * fabs(kappa) / OR_PI);
        if (parts < 1) parts = 1;
        for (int j = 0; j < parts && np < OR_MAX_PIECES; ++j) {
            lo_[np] = bp[i] + len * j / parts;
            hi_[np] = (j + 1 == parts) ? bp[i + 1] : bp[i] + len * (j + 1) / parts;
            ++np;
        }
    }
    double scale[2] = {0.0, 0.0};
    for (int i = 0; i < np; ++i) {
        double k15[2], g7[2], ab[2];
        or_gk15(which, alpha, kappa, lo_[i], hi_[i], k15, g7, ab);
        scale[0] += ab[0];
        scale[1] += ab[1];
    }
    out[0] = out[1] = 0.0;
    for (int i = 0; i < np; ++i) {
        double share = (hi_[i] - lo_[i]) / L;
        or_gk_adapt(which, alpha, kappa, lo_[i], hi_[i], rel * scale[0] * share, rel * scale[1] * share, 0, out);
    }
}

/*
 * G and H of eq. (Gten_sep) at wavenumber index k (kappa = pi k / L).
 *
 * For kappa^2 < 4 alpha (and k = 0) the integrals are taken directly.  Above, where G
 * and H are small next to the size of their integrands, they are taken in the form
 * that two integrations by parts give.  With kappa L = pi k, sin(kappa L) = 0 and
 * cos(kappa L) = (-1)^k, and f, g are even so their first and third derivatives
 * vanish at 0:
 *     int_0^L f cos(kappa y) dy = (-1)^k [ f1(L)/kappa^2 - f3(L)/kappa^4 ]
 *                                 + (1/kappa^4) int_0^L f4(y) cos(kappa y) dy
 * (f1, f3, f4: first, third, fourth derivative), which carries the boundary terms
 * exactly and leaves a remainder whose quadrature error is relative to the (small)
 * result.  Both forms are exact identities.
 */
void or_integrals_1d(double alpha, double L, int k, double* G, double* H)
{
    double kappa = OR_PI * (double)k / L;
    double out[2];
    if (k == 0 || kappa * kappa < 4.0 * alpha) {
        or_quad(OR_DIRECT, alpha, L, kappa, out);
        *G = 2.0 * out[0];
        *H = 2.0 * out[1];
        return;
    }
    double e = exp(-alpha * L * L);
    double a2 = alpha * alpha, a3 = a2 * alpha;
    double L2 = L * L;
    double f1 = -2.0 * alpha * L * e;                                                    /* f'(L)   */
    double f3 = (-8.0 * a3 * L2 * L + 12.0 * a2 * L) * e;                                /* f'''(L) */
    double g1 = (2.0 * L - 2.0 * alpha * L2 * L) * e;                                    /* g'(L)   */
    double g3 = (-24.0 * alpha * L + 36.0 * a2 * L2 * L - 8.0 * a3 * L2 * L2 * L) * e;   /* g'''(L) */
    double sgn = (k % 2 == 0) ? 1.0 : -1.0;
    double k2 = kappa * kappa, k4 = k2 * k2;
    or_quad(OR_FOURTH, alpha, L, kappa, out);
    *G = 2.0 * (sgn * (f1 / k2 - f3 / k4) + out[0] / k4);
    *H = 2.0 * (sgn * (g1 / k2 - g3 / k4) + out[1] / k4);
}

/* G[s*(n+1)+k], H[...] for k = 0..n, kappa_k = pi k / L  (eq. (Gten_sep)). */
void or_axis_tables(int n, double L, int terms, const double* a, double* G, double* H)
{
    int rows = terms * (n + 1);
#pragma omp parallel for schedule(dynamic, 16)
    for (int idx = 0; idx < rows; ++idx) {
        int s = idx / (n + 1), k = idx % (n + 1);
        or_integrals_1d(a[s], L, k, &G[idx], &H[idx]);
    }
}

/* ------------------------------------------------------------------------- */
/* Multiplier, eqs. (convtheorem) and (Gten_sep)                               */
/* ------------------------------------------------------------------------- */
/*
 * Vhat(k) = sum_s w_s (H1 G2 G3 + G1 H2 G3 + G1 G2 H3)       (eq. Gten_sep)
 * M(k)    = -(kappa_1^2 + kappa_2^2 + kappa_3^2) Vhat(k)       (eq. convtheorem:
 *           the spectral Laplacian of the super-potential, -pi^2 |k|^2 on the
 *           paper's period-2 scaling, kappa_p = pi k_p / L_p in the user's units).
 * Stored for |k_p| = 0..n_p (M is real and even in each k_p) as
 * M[(k0*(n1+1) + k1)*(n2+1) + k2].  No 1/N normalisation is folded in.
 * The per-axis tables are computed inside (adaptive Gauss-Kronrod); identical
 * axes are computed once.
 */
int or_multiplier(const int n[3], const double L[3], int terms,
                  const double* w, const double* a, double* M)
{
    double* G[3];
    double* H[3];
    for (int p = 0; p < 3; ++p) {
        int same = -1;
        for (int q = 0; q < p; ++q)
            if (n[q] == n[p] && L[q] == L[p]) { same = q; break; }
        if (same >= 0) { G[p] = G[same]; H[p] = H[same]; continue; }
        G[p] = (double*)malloc(sizeof(double) * (size_t)terms * (n[p] + 1));
        H[p] = (double*)malloc(sizeof(double) * (size_t)terms * (n[p] + 1));
        if (!G[p] || !H[p]) return -1;
        or_axis_tables(n[p], L[p], terms, a, G[p], H[p]);
    }
    int n1 = n[1] + 1, n2 = n[2] + 1;
#pragma omp parallel for schedule(dynamic, 1)
    for (int k0 = 0; k0 <= n[0]; ++k0) {
        double kap0 = OR_PI * k0 / L[0];
        for (int k1 = 0; k1 <= n[1]; ++k1) {
            double kap1 = OR_PI * k1 / L[1];
            for (int k2 = 0; k2 <= n[2]; ++k2) {
                double kap2 = OR_PI * k2 / L[2];
                double v = 0.0;
                for (int s = 0; s < terms; ++s) {
                    double g0 = G[0][s * (n[0] + 1) + k0], h0 = H[0][s * (n[0] + 1) + k0];
                    double g1 = G[1][s * n1 + k1], h1 = H[1][s * n1 + k1];
                    double g2 = G[2][s * n2 + k2], h2 = H[2][s * n2 + k2];
                    v += w[s] * (h0 * g1 * g2 + g0 * h1 * g2 + g0 * g1 * h2);
                }
                M[((size_t)k0 * n1 + k1) * n2 + k2] =
                    -(kap0 * kap0 + kap1 * kap1 + kap2 * kap2) * v;
            }
        }
    }
    for (int p = 0; p < 3; ++p) {
        int owner = 1;
        for (int q = 0; q < p; ++q)
            if (G[q] == G[p]) owner = 0;
        if (owner) { free(G[p]); free(H[p]); }
    }
    return 0;
}

/*
 * Multiplier of the original GS method without its near-field correction (Sec. 1
 * and the bracketed columns of Tab. 2): the convolution with the GS approximation of
 * the Newton kernel itself, U(y) = 1/(4 pi |y|) ~ sum_s 2 w_s exp(-a_s |y|^2) (twice the
 * 1/(8 pi |y|) table of eq. sin_1_x), with no Laplacian symbol:
 *     M(k) = sum_s 2 w_s G0 G1 G2.
 * Same storage as or_multiplier.
 */
int or_multiplier_gs_plain(const int n[3], const double L[3], int terms,
                           const double* w, const double* a, double* M)
{
    double* G[3];
    double* H[3];
    for (int p = 0; p < 3; ++p) {
        int same = -1;
        for (int q = 0; q < p; ++q)
            if (n[q] == n[p] && L[q] == L[p]) { same = q; break; }
        if (same >= 0) { G[p] = G[same]; H[p] = H[same]; continue; }
        G[p] = (double*)malloc(sizeof(double) * (size_t)terms * (n[p] + 1));
        H[p] = (double*)malloc(sizeof(double) * (size_t)terms * (n[p] + 1));
        if (!G[p] || !H[p]) return -1;
        or_axis_tables(n[p], L[p], terms, a, G[p], H[p]);
    }
    int n1 = n[1] + 1, n2 = n[2] + 1;
#pragma omp parallel for schedule(dynamic, 1)
    for (int k0 = 0; k0 <= n[0]; ++k0)
        for (int k1 = 0; k1 <= n[1]; ++k1)
            for (int k2 = 0; k2 <= n[2]; ++k2) {
                double v = 0.0;
                for (int s = 0; s < terms; ++s)
                    v += 2.0 * w[s] * G[0][s * (n[0] + 1) + k0] * G[1][s * n1 + k1] * G[2][s * n2 + k2];
                M[((size_t)k0 * n1 + k1) * n2 + k2] = v;
            }
    for (int p = 0; p < 3; ++p) {
        int owner = 1;
        for (int q = 0; q < p; ++q)
            if (G[q] == G[p]) owner = 0;
        if (owner) { free(G[p]); free(H[p]); }
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Own FFT: recursive mixed radix, any length (radix 2, 3, else direct DFT)   */
/* ------------------------------------------------------------------------- */
/*
 * X[k] = sum_j x[j] exp(sign * 2 pi i j k / m), unnormalised.  Decimation in
 * time: x splits into r subsequences x[j*r + t]; their DFTs of length m/r are
 * combined with twiddles exp(sign 2 pi i t k / m).  The twiddle table holds
 * exp(sign 2 pi i q / m) for q = 0..m-1, each entry from cos/sin of its own
 * angle (no recurrence), and products are indexed by (t*k) mod m exactly.
 */
static int or_smallest_factor(int m)
{
    if (m % 2 == 0) return 2;
    if (m % 3 == 0) return 3;
    for (int f = 5; f * f <= m; f += 2)
        if (m % f == 0) return f;
    return m;
}

static void or_fft_rec(int m, int top, const double* x, long stride, double* out,
                       const double* tw, double* tmp)
{
    if (m == 1) { out[0] = x[0]; out[1] = x[1]; return; }
    int r = or_smallest_factor(m), q = m / r;
    /* sub-transforms of x[t], x[t + r], ... land in out[t*q .. t*q + q) */
    for (int t = 0; t < r; ++t)
        or_fft_rec(q, top, x + 2 * t * stride, stride * r, out + 2 * t * q, tw, tmp);
    int step = top / m;  /* tw has length top: exp(sign 2 pi i q / top) */
    for (int k = 0; k < q; ++k) {
        for (int c = 0; c < r; ++c) {
            int kk = k + c * q;  /* output frequency within this length-m DFT */
            double re = 0.0, im = 0.0;
            for (int t = 0; t < r; ++t) {
                long e = ((long)t * kk) % m;
                double wr = tw[2 * (e * step)], wi = tw[2 * (e * step) + 1];
                double ar = out[2 * (t * q + k)], ai = out[2 * (t * q + k) + 1];
                re += ar * wr - ai * wi;
                im += ar * wi + ai * wr;
            }
            tmp[2 * kk] = re;
            tmp[2 * kk + 1] = im;
        }
    }
    memcpy(out, tmp, sizeof(double) * 2 * m);
}

void or_twiddles(int m, int sign, double* tw)
{
    for (int q = 0; q < m; ++q) {
        double ang = 2.0 * OR_PI * (double)q / (double)m;
        tw[2 * q] = cos(ang);
        tw[2 * q + 1] = sign * sin(ang);
    }
}

/* One line of length m, in place, with a caller-provided twiddle table and
   2*m doubles of scratch for each of the two work arrays. */
static void or_fft_line(int m, double* x, const double* tw, double* w1, double* w2)
{
    or_fft_rec(m, m, x, 1, w1, tw, w2);
    memcpy(x, w1, sizeof(double) * 2 * m);
}

int or_fft(int m, double* x, int sign)
{
    double* tw = (double*)malloc(sizeof(double) * 2 * m);
    double* w1 = (double*)malloc(sizeof(double) * 2 * m);
    double* w2 = (double*)malloc(sizeof(double) * 2 * m);
    if (!tw || !w1 || !w2) { free(tw); free(w1); free(w2); return -1; }
    or_twiddles(m, sign, tw);
    or_fft_line(m, x, tw, w1, w2);
    free(tw); free(w1); free(w2);
    return 0;
}

/* 3D transform of a C-order complex array m0 x m1 x m2, one axis at a time. */
int or_fft3(const int m[3], double* X, int sign)
{
    long s[3] = {(long)m[1] * m[2], m[2], 1};
    for (int ax = 0; ax < 3; ++ax) {
        int len = m[ax];
        int o1 = (ax == 0) ? 1 : 0, o2 = (ax == 2) ? 1 : 2;
        double* tw = (double*)malloc(sizeof(double) * 2 * len);
        if (!tw) return -1;
        or_twiddles(len, sign, tw);
        long lines = (long)m[o1] * m[o2];
        int fail = 0;
#pragma omp parallel
        {
            double* buf = (double*)malloc(sizeof(double) * 6 * len);
            if (!buf) {
#pragma omp atomic write
                fail = 1;
            } else {
#pragma omp for schedule(static)
                for (long l = 0; l < lines; ++l) {
                    long i1 = l / m[o2], i2 = l % m[o2];
                    long base = i1 * s[o1] + i2 * s[o2];
                    for (int j = 0; j < len; ++j) {
                        buf[2 * j] = X[2 * (base + j * s[ax])];
                        buf[2 * j + 1] = X[2 * (base + j * s[ax]) + 1];
                    }
                    or_fft_line(len, buf, tw, buf + 2 * len, buf + 4 * len);
                    for (int j = 0; j < len; ++j) {
                        X[2 * (base + j * s[ax])] = buf[2 * j];
                        X[2 * (base + j * s[ax]) + 1] = buf[2 * j + 1];
                    }
                }
                free(buf);
            }
        }
        free(tw);
        if (fail) return -1;
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Solve, Alg. 2 (with eq. convtheorem)                                       */
/* ------------------------------------------------------------------------- */
/*
 * u = crop( IDFT3( M .* DFT3( pad(rho) ) ) / Ntilde ).
 * pad: rho (n0 x n1 x n2, C order) is placed at the low corner of a zero
 * (2n0) x (2n1) x (2n2) grid (padding factor 2, Sec. 2 and Alg. 1).  The
 * forward DFT is unnormalised with exp(-2 pi i j k / m); frequency bin j of a
 * length-2n axis has |k| = min(j, 2n - j), and M is looked up at the three
 * |k_p|.  The inverse DFT carries the 1/Ntilde factor (Ntilde = 8 n0 n1 n2),
 * which equals the trapezoidal weight h^3 over the period volume (2 n h)^3 of
 * the Fourier coefficients in Sec. 2.  crop keeps the low n0 x n1 x n2 corner.
 * Everything is full (2n)^3 complex FP64; nothing is pruned.
 */
int or_solve(const int n[3], const double* M, const double* rho, double* u)
{
    int m[3] = {2 * n[0], 2 * n[1], 2 * n[2]};
    size_t tot = (size_t)m[0] * m[1] * m[2];
    double* X = (double*)calloc(2 * tot, sizeof(double));
    if (!X) return -1;
    for (int x = 0; x < n[0]; ++x)
        for (int y = 0; y < n[1]; ++y)
            for (int z = 0; z < n[2]; ++z)
                X[2 * (((size_t)x * m[1] + y) * m[2] + z)] =
                    rho[((size_t)x * n[1] + y) * n[2] + z];
    if (or_fft3(m, X, -1)) { free(X); return -1; }
    double inv = 1.0 / (double)tot;
#pragma omp parallel for schedule(static)
    for (int j0 = 0; j0 < m[0]; ++j0) {
        int k0 = j0 <= n[0] ? j0 : m[0] - j0;
        for (int j1 = 0; j1 < m[1]; ++j1) {
            int k1 = j1 <= n[1] ? j1 : m[1] - j1;
            for (int j2 = 0; j2 < m[2]; ++j2) {
                int k2 = j2 <= n[2] ? j2 : m[2] - j2;
                double f = M[((size_t)k0 * (n[1] + 1) + k1) * (n[2] + 1) + k2];
                size_t i = ((size_t)j0 * m[1] + j1) * m[2] + j2;
                X[2 * i] *= f;
                X[2 * i + 1] *= f;
            }
        }
    }
    if (or_fft3(m, X, +1)) { free(X); return -1; }
    for (int x = 0; x < n[0]; ++x)
        for (int y = 0; y < n[1]; ++y)
            for (int z = 0; z < n[2]; ++z)
                u[((size_t)x * n[1] + y) * n[2] + z] =
                    X[2 * (((size_t)x * m[1] + y) * m[2] + z)] * inv;
    free(X);
    return 0;
}

/* Forward spectrum of the padded density (first step of Alg. 2), returned for
   kx in [0,2n0), ky in [0,2n1), kz in [0,n2] (the non-redundant half of a real
   transform): S[((kx*(2n1) + ky)*(n2+1) + kz)] interleaved complex. */
int or_forward_spectrum(const int n[3], const double* rho, double* S)
{
    int m[3] = {2 * n[0], 2 * n[1], 2 * n[2]};
    size_t tot = (size_t)m[0] * m[1] * m[2];
    double* X = (double*)calloc(2 * tot, sizeof(double));
    if (!X) return -1;
    for (int x = 0; x < n[0]; ++x)
        for (int y = 0; y < n[1]; ++y)
            for (int z = 0; z < n[2]; ++z)
                X[2 * (((size_t)x * m[1] + y) * m[2] + z)] =
                    rho[((size_t)x * n[1] + y) * n[2] + z];
    if (or_fft3(m, X, -1)) { free(X); return -1; }
    for (int a = 0; a < m[0]; ++a)
        for (int b = 0; b < m[1]; ++b)
            for (int c = 0; c <= n[2]; ++c) {
                size_t i = ((size_t)a * m[1] + b) * m[2] + c;
                size_t o = ((size_t)a * m[1] + b) * (n[2] + 1) + c;
                S[2 * o] = X[2 * i];
                S[2 * o + 1] = X[2 * i + 1];
            }
    free(X);
    return 0;
}

/* One padded-DFT coefficient by direct summation:
   sum_{x<n0,y<n1,z<n2} rho[x,y,z] exp(-2 pi i (x k0/(2n0) + y k1/(2n1) + z k2/(2n2))).
   The phase factorises per axis; each axis phase is reduced exactly modulo its
   period before cos/sin, and the sums run in the plain nested order. */
int or_dft_coeff(const int n[3], const double* rho, const int k[3], double* re, double* im)
{
    double* ph[3];
    for (int p = 0; p < 3; ++p) {
        ph[p] = (double*)malloc(sizeof(double) * 2 * n[p]);
        if (!ph[p]) { for (int q = 0; q < p; ++q) free(ph[q]); return -1; }
        long m = 2L * n[p];
        for (long j = 0; j < n[p]; ++j) {
            long e = (j * (((long)k[p] % m + m) % m)) % m;
            double ang = 2.0 * OR_PI * (double)e / (double)m;
            ph[p][2 * j] = cos(ang);
            ph[p][2 * j + 1] = -sin(ang);
        }
    }
    double sr = 0.0, si = 0.0;
    for (long x = 0; x < n[0]; ++x) {
        double yr = 0.0, yi = 0.0;
        for (long y = 0; y < n[1]; ++y) {
            double zr = 0.0, zi = 0.0;
            const double* line = rho + (x * n[1] + y) * n[2];
            for (long z = 0; z < n[2]; ++z) {
                zr += line[z] * ph[2][2 * z];
                zi += line[z] * ph[2][2 * z + 1];
            }
            yr += zr * ph[1][2 * y] - zi * ph[1][2 * y + 1];
            yi += zr * ph[1][2 * y + 1] + zi * ph[1][2 * y];
        }
        sr += yr * ph[0][2 * x] - yi * ph[0][2 * x + 1];
        si += yr * ph[0][2 * x + 1] + yi * ph[0][2 * x];
    }
    *re = sr;
    *im = si;
    for (int p = 0; p < 3; ++p) free(ph[p]);
    return 0;
}
