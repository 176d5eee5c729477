/*
 * oracle.c -- plain FP64 CPU oracle for the interpolated EMRI mode summation.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU-baseline leg
 * of the benchmark may load this file's library.  It shares no code, header, table or
 * helper with the CUDA path; the product never calls it.
 *
 * What it computes (arXiv:2104.04582):
 *   * Sec. 3.C (Interpolated Summation): every real array on the sparse trajectory grid is
 *     fitted with a "not-a-knot" cubic spline; all arrays share one knot grid.
 *   * Sec. 4, Schwarzschild mode sum:
 *         h(t) = (mu/d_L) sum_{lmn} A_lmn(t) -2Y_lm(theta,phi) exp(-i Phi_mn(t)),
 *         Phi_mn = m Phi_phi + n Phi_r,
 *     with h = h_+ - i h_x (Sec. 2).
 *   * Eq. (amp_symmetry) with k = 0: A_{l,-m,-n} = (-1)^l conj(A_lmn); only m >= 0 modes are
 *     given, and the m < 0 partner is added for m > 0 only; the m = 0 modes of the list are
 *     taken literally, since (l,0,n) and (l,0,-n) are separate entries of the 3843-mode grid.
 *   * Sec. 6 overlap/mismatch with S_n = 1 (time-domain form via Parseval).
 *   * Sec. 3.E (RomanNet): amplitudes from reduced-basis coefficients, A = alpha . B, each
 *     knot's vector rescaled to a given norm.
 *
 * Spin-weighted spherical harmonics (named a utility in Sec. 3.D; the paper gives no
 * formula): sY_lm(theta,phi) = (-1)^s sqrt((2l+1)/(4 pi)) d^l_{m,-s}(theta) e^{i m phi},
 * with the Wigner small-d matrix written as its explicit finite factorial sum (Goldberg et
 * al. 1967 convention, Condon-Shortley phase).
 *
 * Every function here is pinned by closed forms, identities, brute force or a library
 * routine in the CPU test suite (tests/test_oracle_*.py).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_OK 0
#define OR_ERR_ARG 1
#define OR_ERR_KNOTS 2
#define OR_ERR_RANGE 4

static const double TWO_PI = 6.283185307179586476925286766559;

/* ------------------------------------------------------------------ spline (Sec. 3.C) */

/*
 * Not-a-knot cubic spline through (t_k, y_k), k = 0..K-1, K >= 4.
 * Unknowns: the knot slopes s_k.  Interior rows are the C2 conditions
 *   h_k s_{k-1} + 2(h_{k-1}+h_k) s_k + h_{k-1} s_{k+1} = 3 (h_k d_{k-1} + h_{k-1} d_k),
 * with h_k = t_{k+1}-t_k and d_k = (y_{k+1}-y_k)/h_k.  The end rows impose a continuous
 * third derivative at t_1 and at t_{K-2} (the not-a-knot condition); after eliminating
 * s_2 (resp. s_{K-3}) with the neighbouring interior row they read
 *   h_1 s_0 + (h_0+h_1) s_1 = ((2h_1+3h_0) h_1 d_0 + h_0^2 d_1) / (h_0+h_1),
 *   (h_{K-2}+h_{K-3}) s_{K-2} + h_{K-3} s_{K-1}
 *        = (h_{K-2}^2 d_{K-3} + (2h_{K-3}+3h_{K-2}) h_{K-3} d_{K-2}) / (h_{K-3}+h_{K-2}).
 * The tridiagonal system is solved by Gaussian elimination WITH partial pivoting (row
 * swaps create one extra super-diagonal), one system per call, in long double.
 * Output: coef[k*4 + p], p = 0..3, the cubic on [t_k, t_{k+1}] in x = t - t_k:
 *   c0 = y_k, c1 = s_k, c2 = (3 d_k - 2 s_k - s_{k+1})/h_k, c3 = (s_k + s_{k+1} - 2 d_k)/h_k^2.
 */
static int nak_solve(const double *t, int K, const long double *y, long double *coef)
{
    typedef long double R;
    if (K < 4) return OR_ERR_KNOTS;
    for (int k = 0; k + 1 < K; ++k)
        if (!(t[k + 1] > t[k])) return OR_ERR_KNOTS;
    int n = K;
    R *h = malloc(sizeof(R) * (n - 1));
    R *d = malloc(sizeof(R) * (n - 1));
    R *dl = calloc(n, sizeof(R));   /* sub-diagonal: dl[k] = A[k+1][k] */
    R *dg = calloc(n, sizeof(R));   /* diagonal */
    R *du = calloc(n, sizeof(R));   /* super-diagonal: du[k] = A[k][k+1] */
    R *du2 = calloc(n, sizeof(R));  /* fill-in: du2[k] = A[k][k+2] */
    R *b = calloc(n, sizeof(R));
    R *s = calloc(n, sizeof(R));
    for (int k = 0; k < n - 1; ++k) {
        h[k] = (R)t[k + 1] - (R)t[k];
        d[k] = (y[k + 1] - y[k]) / h[k];
    }
    /* row 0 */
    dg[0] = h[1];
    du[0] = h[0] + h[1];
    b[0] = ((2.0 * h[1] + 3.0 * h[0]) * h[1] * d[0] + h[0] * h[0] * d[1]) / (h[0] + h[1]);
    /* interior rows */
    for (int k = 1; k <= n - 2; ++k) {
        dl[k - 1] = h[k];
        dg[k] = 2.0 * (h[k - 1] + h[k]);
        du[k] = h[k - 1];
        b[k] = 3.0 * (h[k] * d[k - 1] + h[k - 1] * d[k]);
    }
    /* last row */
    {
        R a = h[n - 2], c = h[n - 3];
        dl[n - 2] = a + c;
        dg[n - 1] = c;
        b[n - 1] = (a * a * d[n - 3] + (2.0 * c + 3.0 * a) * c * d[n - 2]) / (c + a);
    }
    /* forward elimination with partial pivoting */
    for (int k = 0; k < n - 1; ++k) {
        if (fabsl(dg[k]) >= fabsl(dl[k])) {
            R mult = dl[k] / dg[k];
            dg[k + 1] -= mult * du[k];
            b[k + 1] -= mult * b[k];
            du2[k] = 0.0;
        } else {
            /* swap rows k and k+1; the new pivot row is the old row k+1 */
            R mult = dg[k] / dl[k];
            R old_dg1 = dg[k + 1];
            R old_du1 = (k + 1 < n - 1) ? du[k + 1] : 0.0;
            R old_duk = du[k];
            dg[k] = dl[k];
            du[k] = old_dg1;
            du2[k] = old_du1;
            dg[k + 1] = old_duk - mult * old_dg1;
            if (k + 1 < n - 1) du[k + 1] = -mult * old_du1;
            R bk = b[k];
            b[k] = b[k + 1];
            b[k + 1] = bk - mult * b[k];
        }
    }
    /* back substitution */
    s[n - 1] = b[n - 1] / dg[n - 1];
    s[n - 2] = (b[n - 2] - du[n - 2] * s[n - 1]) / dg[n - 2];
    for (int k = n - 3; k >= 0; --k)
        s[k] = (b[k] - du[k] * s[k + 1] - du2[k] * s[k + 2]) / dg[k];
    for (int k = 0; k < n - 1; ++k) {
        coef[4 * k + 0] = y[k];
        coef[4 * k + 1] = s[k];
        coef[4 * k + 2] = (3.0 * d[k] - 2.0 * s[k] - s[k + 1]) / h[k];
        coef[4 * k + 3] = (s[k] + s[k + 1] - 2.0 * d[k]) / (h[k] * h[k]);
    }
    free(h); free(d); free(dl); free(dg); free(du); free(du2); free(b); free(s);
    return OR_OK;
}

/* Double-precision interface: inputs and coefficients in double, the solve in long double. */
int oracle_spline_nak(const double *t, int K, const double *y, double *coef)
{
    if (K < 4) return OR_ERR_KNOTS;
    long double *yl = malloc(sizeof(long double) * K);
    long double *cl = malloc(sizeof(long double) * 4 * (K - 1));
    for (int k = 0; k < K; ++k) yl[k] = y[k];
    int rc = nak_solve(t, K, yl, cl);
    if (!rc)
        for (int q = 0; q < 4 * (K - 1); ++q) coef[q] = (double)cl[q];
    free(yl);
    free(cl);
    return rc;
}

/* Long-double coefficients (used for the orbital phases, which reach 1e5-1e7 rad). */
static int spline_nak_ld(const double *t, int K, const double *y, long double *coef)
{
    long double *yl = malloc(sizeof(long double) * K);
    for (int k = 0; k < K; ++k) yl[k] = y[k];
    int rc = nak_solve(t, K, yl, coef);
    free(yl);
    return rc;
}

/* Segment of t: the k with t_k <= t < t_{k+1}; a sample on the last knot uses K-2. */
static int find_segment(const double *t, int K, double x)
{
    int lo = 0, hi = K - 2;
    if (x >= t[K - 2]) return K - 2;
    while (lo < hi) {               /* largest k in [0, K-2] with t_k <= x */
        int mid = (lo + hi + 1) / 2;
        if (t[mid] <= x) lo = mid; else hi = mid - 1;
    }
    return lo;
}

/* Evaluate the spline at n points (Horner in x = t - t_k). */
void oracle_spline_eval(const double *t, int K, const double *coef, const double *x, int64_t n,
                        double *out)
{
    for (int64_t i = 0; i < n; ++i) {
        int k = find_segment(t, K, x[i]);
        double u = x[i] - t[k];
        const double *c = coef + 4 * k;
        out[i] = ((c[3] * u + c[2]) * u + c[1]) * u + c[0];
    }
}

/* ------------------------------------------------------------------ harmonics */

static long double factl(int n)
{
    long double r = 1.0L;
    for (int i = 2; i <= n; ++i) r *= (long double)i;
    return r;
}

/* Wigner small-d d^j_{mp,m}(beta), Wigner's explicit finite sum over k. */
static long double wigner_small_d(int j, int mp, int m, long double beta)
{
    long double c = cosl(0.5L * beta), s = sinl(0.5L * beta);
    long double pre = sqrtl(factl(j + mp) * factl(j - mp) * factl(j + m) * factl(j - m));
    int kmin = (m - mp > 0) ? (m - mp) : 0;
    int kmax = (j + m < j - mp) ? (j + m) : (j - mp);
    long double sum = 0.0L;
    for (int k = kmin; k <= kmax; ++k) {
        long double sign = ((mp - m + k) & 1) ? -1.0L : 1.0L;
        long double num = powl(c, (long double)(2 * j + m - mp - 2 * k)) *
                          powl(s, (long double)(mp - m + 2 * k));
        long double den = factl(j + m - k) * factl(k) * factl(mp - m + k) * factl(j - mp - k);
        sum += sign * num / den;
    }
    return pre * sum;
}

/* sY_lm(theta, phi) for integer spin s (|s| <= l, |m| <= l, else 0). */
void oracle_swsh(int s, int l, int m, double theta, double phi, double *re, double *im)
{
    if (l < abs(s) || abs(m) > l || l < 0) { *re = 0.0; *im = 0.0; return; }
    long double d = wigner_small_d(l, m, -s, (long double)theta);
    long double norm = sqrtl((2.0L * l + 1.0L) / (4.0L * 3.14159265358979323846264338327950288L));
    if (s & 1) norm = -norm;                      /* (-1)^s */
    long double v = norm * d;
    *re = (double)(v * cosl((long double)m * phi));
    *im = (double)(v * sinl((long double)m * phi));
}

/* ------------------------------------------------------------------ mode sum (Sec. 4) */

typedef struct {
    int K, N;
    const double *t;
    long double *cphi, *cr;       /* [K-1][4] phase splines (rad), long double: the phases
                                     reach 1e5-1e7 rad, where a double ulp times |m|+|n|
                                     approaches the 1e-9 rad scale of the FP64 comparison */
    double *cre, *cim;            /* [N][K-1][4] amplitude splines */
    double *yp_re, *yp_im;        /* -2Y_{l,m} per mode */
    double *ym_re, *ym_im;        /* (-1)^l -2Y_{l,-m} per mode (0 for m = 0) */
} oracle_model;

static int model_build(oracle_model *M, const double *t, int K, const double *phi_phi,
                       const double *phi_r, const int *l, const int *m, int N,
                       const double *amp_re, const double *amp_im, double theta, double phi)
{
    int S = K - 1, rc;
    M->K = K; M->N = N; M->t = t;
    M->cphi = malloc(sizeof(long double) * 4 * S);
    M->cr = malloc(sizeof(long double) * 4 * S);
    M->cre = malloc(sizeof(double) * 4 * S * (size_t)N);
    M->cim = malloc(sizeof(double) * 4 * S * (size_t)N);
    M->yp_re = malloc(sizeof(double) * N); M->yp_im = malloc(sizeof(double) * N);
    M->ym_re = malloc(sizeof(double) * N); M->ym_im = malloc(sizeof(double) * N);
    double *col = malloc(sizeof(double) * K);
    if ((rc = spline_nak_ld(t, K, phi_phi, M->cphi))) goto done;
    if ((rc = spline_nak_ld(t, K, phi_r, M->cr))) goto done;
    for (int i = 0; i < N; ++i) {
        for (int k = 0; k < K; ++k) col[k] = amp_re[(size_t)k * N + i];
        if ((rc = oracle_spline_nak(t, K, col, M->cre + (size_t)4 * S * i))) goto done;
        for (int k = 0; k < K; ++k) col[k] = amp_im[(size_t)k * N + i];
        if ((rc = oracle_spline_nak(t, K, col, M->cim + (size_t)4 * S * i))) goto done;
        oracle_swsh(-2, l[i], m[i], theta, phi, &M->yp_re[i], &M->yp_im[i]);
        if (m[i] > 0) {
            double a, b;
            oracle_swsh(-2, l[i], -m[i], theta, phi, &a, &b);
            double sg = (l[i] & 1) ? -1.0 : 1.0;
            M->ym_re[i] = sg * a; M->ym_im[i] = sg * b;
        } else {
            M->ym_re[i] = 0.0; M->ym_im[i] = 0.0;
        }
    }
done:
    free(col);
    return rc;
}

static void model_free(oracle_model *M)
{
    free(M->cphi); free(M->cr); free(M->cre); free(M->cim);
    free(M->yp_re); free(M->yp_im); free(M->ym_re); free(M->ym_im);
}

static double horner(const double *c, double x)
{
    return ((c[3] * x + c[2]) * x + c[1]) * x + c[0];
}

static long double horner_ld(const long double *c, long double x)
{
    return ((c[3] * x + c[2]) * x + c[1]) * x + c[0];
}

/* Orbital phases at t, reduced modulo one turn (each in [-1/2, 1/2] turns). */
static void reduced_phases(const oracle_model *M, int k, double ti, double *fphi, double *fr)
{
    const long double two_pi = 6.283185307179586476925286766559005768L;
    long double x = (long double)ti - (long double)M->t[k];
    long double xphi = horner_ld(M->cphi + 4 * k, x) / two_pi;
    long double xr = horner_ld(M->cr + 4 * k, x) / two_pi;
    *fphi = (double)(xphi - rintl(xphi));
    *fr = (double)(xr - rintl(xr));
}

/*
 * h(t_i) for i in [i_begin, i_begin+count), t_i = t0 + i*dt; out[2*j], out[2*j+1] = Re, Im.
 * At each sample: both phase splines are evaluated (rad) and reduced modulo 2 pi separately,
 * in turns (x - rint(x)); per mode the integer combination m*f_phi + n*f_r is reduced again
 * and passed to FP64 sin/cos; the m >= 0 term A Y+ e^{-i Phi} and, for m > 0, the partner
 * (-1)^l conj(A) -2Y_{l,-m} e^{+i Phi} are added (Eq. amp_symmetry with k = 0).
 */
int oracle_waveform(const double *t, int K, const double *phi_phi, const double *phi_r,
                    const int *l, const int *m, const int *n, int N,
                    const double *amp_re, const double *amp_im,
                    double theta, double phi, double scale, double t0, double dt,
                    int64_t i_begin, int64_t count, double *out, int nthreads)
{
    if (K < 4 || N < 1 || !(dt > 0.0) || count < 0) return OR_ERR_ARG;
    double t_last = t0 + (double)(i_begin + count - 1) * dt;
    if (count > 0 && (t0 + (double)i_begin * dt < t[0] || t_last > t[K - 1])) return OR_ERR_RANGE;
    oracle_model M;
    int rc = model_build(&M, t, K, phi_phi, phi_r, l, m, N, amp_re, amp_im, theta, phi);
    if (rc) { model_free(&M); return rc; }
    int S = K - 1;
    if (nthreads < 1) nthreads = 1;
#ifdef _OPENMP
#pragma omp parallel for num_threads(nthreads) schedule(static)
#endif
    for (int64_t j = 0; j < count; ++j) {
        double ti = t0 + (double)(i_begin + j) * dt;
        int k = find_segment(t, K, ti);
        double x = ti - t[k];
        double fphi, fr;
        reduced_phases(&M, k, ti, &fphi, &fr);
        double hr = 0.0, hi = 0.0;
        for (int i = 0; i < N; ++i) {
            const double *are = M.cre + (size_t)4 * S * i + 4 * k;
            const double *aim = M.cim + (size_t)4 * S * i + 4 * k;
            double Ar = horner(are, x), Ai = horner(aim, x);
            double ph = (double)m[i] * fphi + (double)n[i] * fr;
            ph -= rint(ph);
            double c = cos(TWO_PI * ph), s = sin(TWO_PI * ph);
            /* A Y+ (c - i s) */
            double ayr = Ar * M.yp_re[i] - Ai * M.yp_im[i];
            double ayi = Ar * M.yp_im[i] + Ai * M.yp_re[i];
            hr += ayr * c + ayi * s;
            hi += ayi * c - ayr * s;
            if (m[i] > 0) {
                /* conj(A) Y- (c + i s) */
                double byr = Ar * M.ym_re[i] + Ai * M.ym_im[i];
                double byi = Ar * M.ym_im[i] - Ai * M.ym_re[i];
                hr += byr * c - byi * s;
                hi += byi * c + byr * s;
            }
        }
        out[2 * j] = scale * hr;
        out[2 * j + 1] = scale * hi;
    }
    model_free(&M);
    return OR_OK;
}

/*
 * The orbital phases at t_i = t0 + i*dt, i in [i_begin, i_begin+count), each reduced modulo
 * 2 pi and expressed in turns: out[2j] = f_phi, out[2j+1] = f_r, in [-1/2, 1/2].
 */
int oracle_phases(const double *t, int K, const double *phi_phi, const double *phi_r,
                  double t0, double dt, int64_t i_begin, int64_t count, double *out)
{
    if (K < 4 || !(dt > 0.0) || count < 0) return OR_ERR_ARG;
    int S = K - 1;
    oracle_model M;
    memset(&M, 0, sizeof(M));
    M.K = K; M.t = t;
    M.cphi = malloc(sizeof(long double) * 4 * S);
    M.cr = malloc(sizeof(long double) * 4 * S);
    int rc = spline_nak_ld(t, K, phi_phi, M.cphi);
    if (!rc) rc = spline_nak_ld(t, K, phi_r, M.cr);
    if (!rc) {
        for (int64_t j = 0; j < count; ++j) {
            double ti = t0 + (double)(i_begin + j) * dt;
            if (ti < t[0] || ti > t[K - 1]) { rc = OR_ERR_RANGE; break; }
            reduced_phases(&M, find_segment(t, K, ti), ti, &out[2 * j], &out[2 * j + 1]);
        }
    }
    free(M.cphi);
    free(M.cr);
    return rc;
}

/*
 * Brute-force mode sum for tiny inputs: the m < 0 modes are appended explicitly to a signed
 * list with A_{l,-m,-n} = (-1)^l conj(A_lmn) (Eq. amp_symmetry, k = 0); every signed mode is
 * summed directly as A -2Y_{lm} e^{-i(m Phi_phi + n Phi_r)} in long double, with the phases
 * left unreduced and no folding of partner terms.
 */
int oracle_direct_sum(const double *t, int K, const double *phi_phi, const double *phi_r,
                      const int *l, const int *m, const int *n, int N,
                      const double *amp_re, const double *amp_im,
                      double theta, double phi, double scale, double t0, double dt,
                      int64_t count, double *out)
{
    if (K < 4 || N < 1 || !(dt > 0.0)) return OR_ERR_ARG;
    oracle_model M;
    int rc = model_build(&M, t, K, phi_phi, phi_r, l, m, N, amp_re, amp_im, theta, phi);
    if (rc) { model_free(&M); return rc; }
    int S = K - 1;
    int Ns = 0;
    for (int i = 0; i < N; ++i) Ns += (m[i] > 0) ? 2 : 1;
    int *sl = malloc(sizeof(int) * Ns), *sm = malloc(sizeof(int) * Ns), *sn = malloc(sizeof(int) * Ns);
    int *src = malloc(sizeof(int) * Ns), *cj = malloc(sizeof(int) * Ns);
    long double *yr = malloc(sizeof(long double) * Ns), *yi = malloc(sizeof(long double) * Ns);
    int q = 0;
    for (int i = 0; i < N; ++i) {
        double a, b;
        sl[q] = l[i]; sm[q] = m[i]; sn[q] = n[i]; src[q] = i; cj[q] = 0;
        oracle_swsh(-2, l[i], m[i], theta, phi, &a, &b); yr[q] = a; yi[q] = b; ++q;
        if (m[i] > 0) {
            sl[q] = l[i]; sm[q] = -m[i]; sn[q] = -n[i]; src[q] = i; cj[q] = 1;
            oracle_swsh(-2, l[i], -m[i], theta, phi, &a, &b); yr[q] = a; yi[q] = b; ++q;
        }
    }
    for (int64_t j = 0; j < count; ++j) {
        long double ti = (long double)t0 + (long double)j * (long double)dt;
        int k = find_segment(t, K, (double)ti);
        long double x = ti - (long double)t[k];
        long double Pphi = horner_ld(M.cphi + 4 * k, x);
        long double Pr = horner_ld(M.cr + 4 * k, x);
        long double hr = 0.0L, hi = 0.0L;
        for (int p = 0; p < Ns; ++p) {
            int i = src[p];
            const double *are = M.cre + (size_t)4 * S * i + 4 * k;
            const double *aim = M.cim + (size_t)4 * S * i + 4 * k;
            long double Ar = ((are[3] * x + are[2]) * x + are[1]) * x + are[0];
            long double Ai = ((aim[3] * x + aim[2]) * x + aim[1]) * x + aim[0];
            if (cj[p]) {                            /* (-1)^l conj(A) */
                long double sg = (sl[p] & 1) ? -1.0L : 1.0L;
                Ar = sg * Ar; Ai = -sg * Ai;
            }
            long double Phi = (long double)sm[p] * Pphi + (long double)sn[p] * Pr;
            long double c = cosl(Phi), s = sinl(Phi);
            long double vr = Ar * yr[p] - Ai * yi[p];
            long double vi = Ar * yi[p] + Ai * yr[p];
            hr += vr * c + vi * s;
            hi += vi * c - vr * s;
        }
        out[2 * j] = (double)(scale * hr);
        out[2 * j + 1] = (double)(scale * hi);
    }
    free(sl); free(sm); free(sn); free(src); free(cj); free(yr); free(yi);
    model_free(&M);
    return OR_OK;
}

/* ------------------------------------------------------------------ mismatch (Sec. 6) */

/*
 * overlap(a,b) = <a|b>/sqrt(<a|a><b|b>), mismatch = 1 - overlap, with S_n = 1.  For complex
 * time series h = h_+ - i h_x, Parseval turns the frequency-domain inner product into
 * sum_i Re(conj(a_i) b_i) (the sum of the + and x inner products), up to a constant factor
 * that cancels in the ratio.  Computed in long double.  Returns NaN for a zero series.
 */
double oracle_overlap(const double *a, const double *b, int64_t n)
{
    long double ab = 0.0L, aa = 0.0L, bb = 0.0L;
    for (int64_t i = 0; i < n; ++i) {
        long double ar = a[2 * i], ai = a[2 * i + 1], br = b[2 * i], bi = b[2 * i + 1];
        ab += ar * br + ai * bi;
        aa += ar * ar + ai * ai;
        bb += br * br + bi * bi;
    }
    if (aa == 0.0L || bb == 0.0L) return NAN;
    return (double)(ab / sqrtl(aa * bb));
}

/*
 * mismatch = 1 - overlap, evaluated without cancellation as 0.5*||a/|a| - b/|b|||^2, which
 * equals 1 - Re<a/|a|, b/|b|> exactly for unit vectors.
 */
double oracle_mismatch(const double *a, const double *b, int64_t n)
{
    long double aa = 0.0L, bb = 0.0L;
    for (int64_t i = 0; i < n; ++i) {
        aa += (long double)a[2 * i] * a[2 * i] + (long double)a[2 * i + 1] * a[2 * i + 1];
        bb += (long double)b[2 * i] * b[2 * i] + (long double)b[2 * i + 1] * b[2 * i + 1];
    }
    if (aa == 0.0L || bb == 0.0L) return NAN;
    long double na = 1.0L / sqrtl(aa), nb = 1.0L / sqrtl(bb), acc = 0.0L;
    for (int64_t i = 0; i < n; ++i) {
        long double dr = a[2 * i] * na - b[2 * i] * nb;
        long double di = a[2 * i + 1] * na - b[2 * i + 1] * nb;
        acc += dr * dr + di * di;
    }
    return (double)(0.5L * acc);
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------ mode selector (Sec. 3.D) */

typedef struct { double p; int i; } pw_entry;

static int pw_desc(const void *a, const void *b)
{
    const pw_entry *x = (const pw_entry *)a, *y = (const pw_entry *)b;
    if (x->p > y->p) return -1;
    if (x->p < y->p) return 1;
    return (x->i > y->i) - (x->i < y->i);   /* ties: lower mode index first */
}

/*
 * Mode Selector: at every knot the power of each mode, |A(t_k)|^2 (doubled for m > 0, which also
 * stands for its m < 0 partner of equal power), is sorted in descending order (ties by mode
 * index) and summed cumulatively; the knot keeps the shortest leading run whose cumulative power
 * reaches (1 - eps) of that knot's total.  The selection is the union over knots.  A knot with
 * zero total power keeps nothing.  mask[i] = 1 for selected modes; returns their number.
 */
int oracle_mode_select(const double *amp_re, const double *amp_im, int K, int N, const int *m,
                       double eps, unsigned char *mask)
{
    pw_entry *e = malloc(sizeof(pw_entry) * (size_t)N);
    memset(mask, 0, (size_t)N);
    for (int k = 0; k < K; ++k) {
        double total = 0.0;
        for (int i = 0; i < N; ++i) {
            double re = amp_re[(size_t)k * N + i], im = amp_im[(size_t)k * N + i];
            double p = re * re + im * im;
            if (m[i] > 0) p *= 2.0;
            e[i].p = p;
            e[i].i = i;
        }
        qsort(e, (size_t)N, sizeof(pw_entry), pw_desc);
        for (int j = 0; j < N; ++j) total += e[j].p;
        if (!(total > 0.0)) continue;
        double target = (1.0 - eps) * total, c = 0.0;
        for (int j = 0; j < N; ++j) {
            c += e[j].p;
            mask[e[j].i] = 1;
            if (c >= target) break;
        }
    }
    int count = 0;
    for (int i = 0; i < N; ++i) count += mask[i];
    free(e);
    return count;
}

/* ------------------------------------------------------------------ frame transformation (Sec. 2.A) */

static void cross3(const double *a, const double *b, double *c)
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

/*
 * Source-frame viewing angles and polarization angle from the sky position (theta_S, phi_S) and
 * the MBH spin direction (theta_K, phi_K), Sec. 2.A:
 *   R = (sin tS cos pS, sin tS sin pS, cos tS),  S = (sin tK cos pK, sin tK sin pK, cos tK),
 *   source frame x = R x S / |R x S|, y = (R - (R.S) S) / |R x S|, z = S;
 *   the wave reaches the detector along -R, whose source-frame polar angle gives
 *   cos theta_src = -R.S and whose azimuth is phi_src = -pi/2;
 *   tan psi = (cos tS sin tK cos(pS - pK) - sin tS cos tK) / (sin tK sin(pS - pK)).
 * The azimuth is computed from the projection of -R onto (x, y), not assumed.
 */
int oracle_frame_angles(double tS, double pS, double tK, double pK, double *theta_src,
                        double *phi_src, double *psi)
{
    double R[3] = {sin(tS) * cos(pS), sin(tS) * sin(pS), cos(tS)};
    double S[3] = {sin(tK) * cos(pK), sin(tK) * sin(pK), cos(tK)};
    double RxS[3];
    cross3(R, S, RxS);
    double nrm = sqrt(dot3(RxS, RxS));
    if (!(nrm > 1e-12)) return OR_ERR_ARG;   /* R parallel to S: frame undefined */
    double RS = dot3(R, S);
    double x[3] = {RxS[0] / nrm, RxS[1] / nrm, RxS[2] / nrm};
    double y[3] = {(R[0] - RS * S[0]) / nrm, (R[1] - RS * S[1]) / nrm, (R[2] - RS * S[2]) / nrm};
    double v[3] = {-R[0], -R[1], -R[2]};
    *theta_src = acos(fmax(-1.0, fmin(1.0, dot3(v, S))));
    *phi_src = atan2(dot3(v, y), dot3(v, x));
    double num = cos(tS) * sin(tK) * cos(pS - pK) - sin(tS) * cos(tK);
    double den = sin(tK) * sin(pS - pK);
    *psi = atan2(num, den);
    return OR_OK;
}

/*
 * Detector-frame (solar-system-barycentre) waveform: the source-frame sum of oracle_waveform at
 * (theta_src, phi_src), then the pi/2 rotation of the polarization basis -- a phase shift of pi --
 * and the rotation by twice the polarization angle: h -> -h e^{-2 i psi}
 * (h_+' = cos 2psi h_+ - sin 2psi h_x, h_x' = sin 2psi h_+ + cos 2psi h_x).
 */
int oracle_waveform_ssb(const double *t, int K, const double *phi_phi, const double *phi_r,
                        const int *l, const int *m, const int *n, int N,
                        const double *amp_re, const double *amp_im,
                        double tS, double pS, double tK, double pK, double scale, double t0,
                        double dt, int64_t i_begin, int64_t count, double *out, int nthreads)
{
    double th, ph, psi;
    int rc = oracle_frame_angles(tS, pS, tK, pK, &th, &ph, &psi);
    if (rc) return rc;
    rc = oracle_waveform(t, K, phi_phi, phi_r, l, m, n, N, amp_re, amp_im, th, ph, scale, t0, dt,
                         i_begin, count, out, nthreads);
    if (rc) return rc;
    double fr = -cos(2.0 * psi), fi = sin(2.0 * psi);   /* -e^{-2 i psi} */
    for (int64_t j = 0; j < count; ++j) {
        double a = out[2 * j], b = out[2 * j + 1];
        out[2 * j] = a * fr - b * fi;
        out[2 * j + 1] = a * fi + b * fr;
    }
    return OR_OK;
}

/* ------------------------------------------------------------------ direct summation (Sec. 3.C) */

/*
 * Direct (non-interpolated) summation: the trajectory and amplitudes are given at every output
 * sample (arrays of the output's density), so no spline is built:
 *   h_i = scale * sum_modes [ A_i Y+ e^{-i Phi_mn,i} + (m > 0) (-1)^l conj(A_i) -2Y_{l,-m} e^{+i Phi_mn,i} ],
 * Phi_mn,i = m phi_phi[i] + n phi_r[i]; the phases are reduced modulo 2 pi separately (in long
 * double, in turns) before the integer combination, as in oracle_waveform.
 * amp_re, amp_im: [n_samples][N] row-major; out: [n_samples][2].
 */
int oracle_direct_dense(const double *phi_phi, const double *phi_r, int64_t n_samples,
                        const int *l, const int *m, const int *n, int N, const double *amp_re,
                        const double *amp_im, double theta, double phi, double scale, double *out,
                        int nthreads)
{
    if (N < 1 || n_samples < 0) return OR_ERR_ARG;
    double *ypr = malloc(sizeof(double) * N), *ypi = malloc(sizeof(double) * N);
    double *ymr = malloc(sizeof(double) * N), *ymi = malloc(sizeof(double) * N);
    for (int i = 0; i < N; ++i) {
        oracle_swsh(-2, l[i], m[i], theta, phi, &ypr[i], &ypi[i]);
        ymr[i] = ymi[i] = 0.0;
        if (m[i] > 0) {
            double a, b;
            oracle_swsh(-2, l[i], -m[i], theta, phi, &a, &b);
            double sg = (l[i] & 1) ? -1.0 : 1.0;
            ymr[i] = sg * a;
            ymi[i] = sg * b;
        }
    }
    if (nthreads < 1) nthreads = 1;
    const long double two_pi = 6.283185307179586476925286766559005768L;
#ifdef _OPENMP
#pragma omp parallel for num_threads(nthreads) schedule(static)
#endif
    for (int64_t j = 0; j < n_samples; ++j) {
        long double xp = (long double)phi_phi[j] / two_pi, xr = (long double)phi_r[j] / two_pi;
        double fphi = (double)(xp - rintl(xp)), fr = (double)(xr - rintl(xr));
        double hr = 0.0, hi = 0.0;
        for (int i = 0; i < N; ++i) {
            double Ar = amp_re[(size_t)j * N + i], Ai = amp_im[(size_t)j * N + i];
            double ph = (double)m[i] * fphi + (double)n[i] * fr;
            ph -= rint(ph);
            double c = cos(TWO_PI * ph), s = sin(TWO_PI * ph);
            double ayr = Ar * ypr[i] - Ai * ypi[i], ayi = Ar * ypi[i] + Ai * ypr[i];
            hr += ayr * c + ayi * s;
            hi += ayi * c - ayr * s;
            if (m[i] > 0) {
                double byr = Ar * ymr[i] + Ai * ymi[i], byi = Ar * ymi[i] - Ai * ymr[i];
                hr += byr * c - byi * s;
                hi += byi * c + byr * s;
            }
        }
        out[2 * j] = scale * hr;
        out[2 * j + 1] = scale * hi;
    }
    free(ypr); free(ypi); free(ymr); free(ymi);
    return OR_OK;
}

/*
 * Reduced-basis amplitudes (Sec. 3.E, RomanNet).  Each knot k carries Nb complex reduced-basis
 * coefficients alpha_k,j; its N mode amplitudes are the coefficients times the basis,
 *     A_k,i = sum_j alpha_k,j B_j,i,
 * and, when target norms nu_k are given, the vector A_k is then rescaled to that Euclidean
 * norm: A_k <- A_k nu_k / ||A_k||, ||A_k||^2 = sum_i |A_k,i|^2 (a zero vector stays zero).
 * alpha_re/alpha_im: [M][Nb]; b_re/b_im: [Nb][N]; norms: [M] or NULL; out_re/out_im: [M][N];
 * all row-major.  Sums are accumulated in long double.
 */
int oracle_rb_amplitudes(int M, int Nb, int N, const double *alpha_re, const double *alpha_im,
                         const double *b_re, const double *b_im, const double *norms,
                         double *out_re, double *out_im, int nthreads)
{
    if (M < 0 || Nb < 1 || N < 1) return OR_ERR_ARG;
    if (nthreads < 1) nthreads = 1;
    int rc = OR_OK;
#ifdef _OPENMP
#pragma omp parallel num_threads(nthreads)
#endif
    {
        long double *rr = malloc(sizeof(long double) * N), *ri = malloc(sizeof(long double) * N);
        if (!rr || !ri) rc = OR_ERR_ARG;
#ifdef _OPENMP
#pragma omp for schedule(static)
#endif
        for (int k = 0; k < M; ++k) {
            if (!rr || !ri) continue;
            for (int i = 0; i < N; ++i) {
                long double sr = 0.0L, si = 0.0L;
                for (int j = 0; j < Nb; ++j) {
                    const long double ar = alpha_re[(size_t)k * Nb + j], ai = alpha_im[(size_t)k * Nb + j];
                    const long double br = b_re[(size_t)j * N + i], bi = b_im[(size_t)j * N + i];
                    sr += ar * br - ai * bi;
                    si += ar * bi + ai * br;
                }
                rr[i] = sr;
                ri[i] = si;
            }
            long double f = 1.0L;
            if (norms) {
                long double nn = 0.0L;
                for (int i = 0; i < N; ++i) nn += rr[i] * rr[i] + ri[i] * ri[i];
                f = nn > 0.0L ? (long double)norms[k] / sqrtl(nn) : 0.0L;
            }
            for (int i = 0; i < N; ++i) {
                out_re[(size_t)k * N + i] = (double)(rr[i] * f);
                out_im[(size_t)k * N + i] = (double)(ri[i] * f);
            }
        }
        free(rr);
        free(ri);
    }
    return rc;
}
