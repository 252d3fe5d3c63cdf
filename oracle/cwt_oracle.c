/*
 * FP64 CPU oracle for the FFT-based continuous wavelet transform (FFTCWT)
 * of Wang & He, "Comparisons between fast algorithms for the continuous
 * wavelet transform and applications in cosmology: the 1D case" (RASTI 2023,
 * arXiv:2302.03909).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * statement of what the GPU path computes.  Only the tests, the smoke check
 * and the CPU-baseline leg of the benchmark may load it.  It shares no code,
 * header, table or constant with the CUDA library.
 *
 * Everything is double precision and follows the paper's notation:
 *   - mother wavelets psi(x) and their Fourier transforms psi_hat(k), with the
 *     normalisation constants C_N (Table 2);
 *   - the discrete CWT as a direct sum (Eq. 4), periodic (with the periodic
 *     images of the dilated wavelet) or zero-boundary (true linear sum);
 *   - the FFTCWT (Sec. 3.1): f_hat(m) = (L/N) sum_n f(n) e^{+2 pi i m n/N}
 *     (Eq. 8), W_hat(w,m) = sqrt(L/(N w)) f_hat(m) psi_hat(2 pi m/(N w)) and
 *     W(w,n) = (1/L) sum_m W_hat(w,m) e^{-2 pi i m n/N} (Eqs. 9-10), where N is
 *     the (possibly zero-padded) transform length and m is taken as the signed
 *     frequency m~ in (-N/2, N/2] when psi_hat is evaluated;
 *   - the global wavelet power spectrum P(w) = <|W(w,x)|^2> over the N signal
 *     positions (Eq. 42) and the environment-split power spectrum (Eq. 41).
 *
 * Zero boundary (Sec. 4.1, Eq. 40): the signal is placed at offset 0 of a
 * length-M buffer whose remaining M-N entries are zero, and the first N
 * outputs are kept.  With M >= N + (wavelet support) this equals padding
 * zeros at both ends.
 *
 * Readings of the paper taken here (also listed in the design notes):
 *   - signed frequency: m~ = m for m <= M/2, m~ = m - M otherwise (the even-M
 *     Nyquist bin takes +M/2);
 *   - the Morlet wavelet is parameterised by omega0 (Table 2 fixes 4):
 *     psi(x) = C_N (e^{-i omega0 x} - e^{-omega0^2/2}) e^{-x^2/2},
 *     C_N = pi^{-1/4} (1 - 2 e^{-3 omega0^2/4} + e^{-omega0^2})^{-1/2};
 *   - scales are the paper's dimensionless w~ = w dx (callers convert from
 *     dilations in samples as w~ = 1/s).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846264338327950288

enum { ORC_CBSW = 0, ORC_GDW = 1, ORC_CWGDW = 2, ORC_MORLET = 3 };
enum { ORC_PERIODIC = 0, ORC_ZERO = 1 };

/* ---------------------------------------------------------------- wavelets */

/* Normalisation constant C_N of Table 2 (Morlet: general omega0). */
double orc_cn(int wavelet, double omega0)
{
    switch (wavelet) {
    case ORC_CBSW:   return sqrt(30.0 / 31.0);
    case ORC_GDW:    return pow(18.0 * ORC_PI, -0.25);
    case ORC_CWGDW:  return sqrt(8.0 / (1.0 + 5.0 * exp(1.0))) / pow(ORC_PI, 0.25);
    case ORC_MORLET: {
        double w2 = omega0 * omega0;
        return pow(ORC_PI, -0.25) / sqrt(1.0 - 2.0 * exp(-0.75 * w2) + exp(-w2));
    }
    }
    return NAN;
}

/* Cubic B-spline beta^3 (Appendix B: four-fold convolution of the unit box). */
static double beta3(double x)
{
    double a = fabs(x);
    if (a < 1.0) return 2.0 / 3.0 - a * a + 0.5 * a * a * a;
    if (a < 2.0) { double t = 2.0 - a; return t * t * t / 6.0; }
    return 0.0;
}

/* Mother wavelet psi(x) of Table 2; real wavelets return im = 0. */
void orc_psi(int wavelet, double omega0, double x, double *re, double *im)
{
    double cn = orc_cn(wavelet, omega0);
    *im = 0.0;
    switch (wavelet) {
    case ORC_CBSW:
        *re = cn * (2.0 * beta3(x) - beta3(x + 1.0) - beta3(x - 1.0));
        return;
    case ORC_GDW:
        *re = cn * (2.0 - x * x) * exp(-0.25 * x * x);
        return;
    case ORC_CWGDW:
        *re = cn * ((1.0 - x * x) * cos(x) - x * sin(x)) * exp(0.5 * (1.0 - x * x));
        return;
    case ORC_MORLET: {
        double g = cn * exp(-0.5 * x * x);
        double c = exp(-0.5 * omega0 * omega0);
        *re = g * (cos(omega0 * x) - c);
        *im = -g * sin(omega0 * x);
        return;
    }
    }
    *re = NAN;
}

/* Fourier transform psi_hat(k) = int psi(x) e^{+ikx} dx of Table 2 (real for
 * all four wavelets in the paper's convention). */
double orc_psi_hat(int wavelet, double omega0, double k)
{
    double cn = orc_cn(wavelet, omega0);
    switch (wavelet) {
    case ORC_CBSW: {
        if (k == 0.0) return 0.0;
        double s = sin(0.5 * k);
        double s2 = s * s;
        return 64.0 * cn * s2 * s2 * s2 / (k * k * k * k);
    }
    case ORC_GDW:
        return 8.0 * sqrt(ORC_PI) * cn * k * k * exp(-k * k);
    case ORC_CWGDW:
        /* k cosh k - sinh k = ((k-1) e^k + (k+1) e^-k) / 2, grouped with
         * e^{-k^2/2} so that no factor overflows */
        return sqrt(2.0 * ORC_PI) * cn * k * 0.5 *
               ((k - 1.0) * exp(k - 0.5 * k * k) + (k + 1.0) * exp(-k - 0.5 * k * k));
    case ORC_MORLET:
        return sqrt(2.0 * ORC_PI) * cn *
               (exp(-0.5 * (k - omega0) * (k - omega0)) - exp(-0.5 * (k * k + omega0 * omega0)));
    }
    return NAN;
}

/* |x| beyond which |psi(x)| < 1e-20 (CBSW: exact support [-3, 3]). */
static double psi_cut(int wavelet)
{
    switch (wavelet) {
    case ORC_CBSW:   return 3.0;
    case ORC_GDW:    return 16.0;
    case ORC_CWGDW:  return 11.0;
    case ORC_MORLET: return 10.0;
    }
    return 0.0;
}

/* --------------------------------------------------------------------- FFT */

/* e^{sign 2 pi i r / n} for 0 <= r < n, computed from the exact integer r. */
static void unit_root(int64_t r, int64_t n, int sign, double *c, double *s)
{
    double a = 2.0 * ORC_PI * (double)r / (double)n;
    *c = cos(a);
    *s = sign * sin(a);
}

static int is_pow2(int64_t n) { return n > 0 && (n & (n - 1)) == 0; }

/* In-place radix-2 decimation-in-time FFT, X(k) = sum_j x(j) e^{sign 2 pi i jk/n}. */
static void fft_pow2(int64_t n, double *re, double *im, int sign)
{
    for (int64_t i = 1, j = 0; i < n; i++) {
        int64_t bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) {
            double t = re[i]; re[i] = re[j]; re[j] = t;
            t = im[i]; im[i] = im[j]; im[j] = t;
        }
    }
    for (int64_t len = 2; len <= n; len <<= 1) {
        int64_t half = len >> 1, step = n / len;
        for (int64_t k = 0; k < half; k++) {
            double wr, wi;
            unit_root(k * step, n, sign, &wr, &wi);
            for (int64_t i = k; i < n; i += len) {
                int64_t j = i + half;
                double tr = re[j] * wr - im[j] * wi;
                double ti = re[j] * wi + im[j] * wr;
                re[j] = re[i] - tr; im[j] = im[i] - ti;
                re[i] += tr;        im[i] += ti;
            }
        }
    }
}

/* Bluestein's chirp-z evaluation of a DFT of any length n via a power-of-two
 * circular convolution: jk = (j^2 + k^2 - (k-j)^2) / 2. */
static int fft_bluestein(int64_t n, double *re, double *im, int sign)
{
    int64_t m = 1;
    while (m < 2 * n - 1) m <<= 1;
    double *ar = calloc(m, sizeof(double)), *ai = calloc(m, sizeof(double));
    double *br = calloc(m, sizeof(double)), *bi = calloc(m, sizeof(double));
    double *cr = malloc(n * sizeof(double)), *ci = malloc(n * sizeof(double));
    if (!ar || !ai || !br || !bi || !cr || !ci) {
        free(ar); free(ai); free(br); free(bi); free(cr); free(ci);
        return -1;
    }
    for (int64_t j = 0; j < n; j++) {
        /* chirp e^{sign pi i j^2 / n} = e^{sign 2 pi i (j^2 mod 2n) / (2n)} */
        int64_t r = (int64_t)(((unsigned __int128)j * (unsigned __int128)j) % (unsigned __int128)(2 * n));
        unit_root(r, 2 * n, sign, &cr[j], &ci[j]);
    }
    for (int64_t j = 0; j < n; j++) {           /* a = x * chirp */
        ar[j] = re[j] * cr[j] - im[j] * ci[j];
        ai[j] = re[j] * ci[j] + im[j] * cr[j];
    }
    br[0] = cr[0]; bi[0] = -ci[0];              /* b = conj(chirp), symmetric */
    for (int64_t j = 1; j < n; j++) {
        br[j] = br[m - j] = cr[j];
        bi[j] = bi[m - j] = -ci[j];
    }
    fft_pow2(m, ar, ai, -1);
    fft_pow2(m, br, bi, -1);
    for (int64_t j = 0; j < m; j++) {
        double tr = ar[j] * br[j] - ai[j] * bi[j];
        double ti = ar[j] * bi[j] + ai[j] * br[j];
        ar[j] = tr; ai[j] = ti;
    }
    fft_pow2(m, ar, ai, +1);
    for (int64_t k = 0; k < n; k++) {           /* X = chirp * conv / m */
        double tr = ar[k] / (double)m, ti = ai[k] / (double)m;
        re[k] = tr * cr[k] - ti * ci[k];
        im[k] = tr * ci[k] + ti * cr[k];
    }
    free(ar); free(ai); free(br); free(bi); free(cr); free(ci);
    return 0;
}

/* Unnormalised DFT of any length, X(k) = sum_j x(j) e^{sign 2 pi i jk/n}. */
int orc_fft(int64_t n, double *re, double *im, int sign)
{
    if (n <= 0 || (sign != 1 && sign != -1)) return -1;
    if (n == 1) return 0;
    if (is_pow2(n)) { fft_pow2(n, re, im, sign); return 0; }
    return fft_bluestein(n, re, im, sign);
}

/* Plain O(n^2) DFT with exact integer angle reduction (pins orc_fft). */
int orc_dft(int64_t n, const double *re, const double *im, int sign,
            double *out_re, double *out_im)
{
    if (n <= 0) return -1;
    for (int64_t k = 0; k < n; k++) {
        double sr = 0.0, si = 0.0;
        for (int64_t j = 0; j < n; j++) {
            double c, s;
            unit_root((j * k) % n, n, sign, &c, &s);
            sr += re[j] * c - im[j] * s;
            si += re[j] * s + im[j] * c;
        }
        out_re[k] = sr; out_im[k] = si;
    }
    return 0;
}

/* --------------------------------------------------- FFTCWT (Sec. 3.1) */

static int64_t signed_freq(int64_t m, int64_t M) { return (2 * m <= M) ? m : m - M; }

/* Eq. 8: f_hat(m) = (L/M) sum_n f_pad(n) e^{+2 pi i m n/M}, with f zero-extended
 * to M (zero boundary) or M = N (periodic).  naive != 0 uses the O(M^2) DFT. */
static int forward_ft(const double *f, int64_t N, int64_t M, double dx, int naive,
                      double *fr, double *fi)
{
    double L = (double)M * dx;
    double *xr = calloc(M, sizeof(double)), *xi = calloc(M, sizeof(double));
    if (!xr || !xi) { free(xr); free(xi); return -1; }
    memcpy(xr, f, N * sizeof(double));
    int rc = naive ? orc_dft(M, xr, xi, +1, fr, fi) : 0;
    if (!naive) {
        memcpy(fr, xr, M * sizeof(double));
        memcpy(fi, xi, M * sizeof(double));
        rc = orc_fft(M, fr, fi, +1);
    }
    for (int64_t m = 0; m < M; m++) { fr[m] *= L / (double)M; fi[m] *= L / (double)M; }
    free(xr); free(xi);
    return rc;
}

/* W_hat(w~, m) = sqrt(L/(M w~)) f_hat(m) psi_hat(2 pi m~ /(M w~))  (Eq. 10). */
static void spectrum_product(const double *fr, const double *fi, int64_t M, double dx,
                             double wt, int wavelet, double omega0, double *hr, double *hi)
{
    double L = (double)M * dx;
    double amp = sqrt(L / ((double)M * wt));
    for (int64_t m = 0; m < M; m++) {
        double k = 2.0 * ORC_PI * (double)signed_freq(m, M) / ((double)M * wt);
        double p = amp * orc_psi_hat(wavelet, omega0, k);
        hr[m] = fr[m] * p;
        hi[m] = fi[m] * p;
    }
}

/* FFTCWT over all scales.  W_re/W_im are [S][N] row-major; W(w~,n) =
 * (1/L) sum_m W_hat(w~,m) e^{-2 pi i m n/M} for n < N (Eq. 9).
 * naive != 0: every transform is the O(M^2) DFT (tier T1); otherwise the
 * oracle's own radix-2 / Bluestein FFT (tier T2).  nthreads <= 0: default. */
int orc_cwt_fft(const double *f, int64_t N, int64_t M, const double *wt, int32_t S,
                int wavelet, double omega0, double dx, int naive, int nthreads,
                double *W_re, double *W_im)
{
    if (N <= 0 || M < N || S < 0 || dx <= 0.0) return -1;
    double L = (double)M * dx;
    double *fr = malloc(M * sizeof(double)), *fi = malloc(M * sizeof(double));
    if (!fr || !fi) { free(fr); free(fi); return -1; }
    int rc = forward_ft(f, N, M, dx, naive, fr, fi);
    if (rc) { free(fr); free(fi); return rc; }
    int err = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1) reduction(| : err)
#endif
    for (int32_t s = 0; s < S; s++) {
        double *hr = malloc(M * sizeof(double)), *hi = malloc(M * sizeof(double));
        double *or_ = malloc(M * sizeof(double)), *oi = malloc(M * sizeof(double));
        if (!hr || !hi || !or_ || !oi) { err |= 1; free(hr); free(hi); free(or_); free(oi); continue; }
        spectrum_product(fr, fi, M, dx, wt[s], wavelet, omega0, hr, hi);
        if (naive) {
            err |= orc_dft(M, hr, hi, -1, or_, oi) != 0;
        } else {
            memcpy(or_, hr, M * sizeof(double));
            memcpy(oi, hi, M * sizeof(double));
            err |= orc_fft(M, or_, oi, -1) != 0;
        }
        for (int64_t n = 0; n < N; n++) {
            W_re[(int64_t)s * N + n] = or_[n] / L;
            W_im[(int64_t)s * N + n] = oi[n] / L;
        }
        free(hr); free(hi); free(or_); free(oi);
    }
    free(fr); free(fi);
    return err ? -1 : 0;
}

/* FFTCWT at listed points (scale index ps[p], position pn[p]): f_hat by the
 * oracle FFT, then each W(w~,n) as the O(M) sum of Eq. 9 on its own. */
int orc_cwt_fft_points(const double *f, int64_t N, int64_t M, const double *wt, int32_t S,
                       int wavelet, double omega0, double dx, const int32_t *ps,
                       const int64_t *pn, int64_t P, int nthreads,
                       double *out_re, double *out_im)
{
    if (N <= 0 || M < N || dx <= 0.0) return -1;
    for (int64_t p = 0; p < P; p++)
        if (ps[p] < 0 || ps[p] >= S || pn[p] < 0 || pn[p] >= N) return -1;
    double L = (double)M * dx;
    double *fr = malloc(M * sizeof(double)), *fi = malloc(M * sizeof(double));
    if (!fr || !fi) { free(fr); free(fi); return -1; }
    int rc = forward_ft(f, N, M, dx, 0, fr, fi);
    if (rc) { free(fr); free(fi); return rc; }
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t p = 0; p < P; p++) {
        double amp = sqrt(L / ((double)M * wt[ps[p]]));
        double sr = 0.0, si = 0.0;
        for (int64_t m = 0; m < M; m++) {
            double k = 2.0 * ORC_PI * (double)signed_freq(m, M) / ((double)M * wt[ps[p]]);
            double psi = amp * orc_psi_hat(wavelet, omega0, k);
            if (psi == 0.0) continue;
            double c, s;
            unit_root((int64_t)(((unsigned __int128)m * (unsigned __int128)pn[p]) % (unsigned __int128)M),
                      M, -1, &c, &s);
            double hr = fr[m] * psi, hi = fi[m] * psi;
            sr += hr * c - hi * s;
            si += hr * s + hi * c;
        }
        out_re[p] = sr / L;
        out_im[p] = si / L;
    }
    free(fr); free(fi);
    return 0;
}

/* ------------------------------------------------- direct sum (Eq. 4) */

/* Periodic: W(w~,n) = sqrt(w~ dx) sum_{m<N} f(m) sum_p psi(w~ (n - m + pN)).
 * Zero:     W(w~,n) = sqrt(w~ dx) sum_{m<N} f(m) psi(w~ (n - m)).
 * The periodic images are summed first into h(j) = sum_p psi(w~(j + pN)),
 * over every p with |w~ (j + pN)| inside the wavelet's numerical support. */
int orc_cwt_direct(const double *f, int64_t N, const double *wt, int32_t S,
                   int wavelet, double omega0, double dx, int boundary, int nthreads,
                   double *W_re, double *W_im)
{
    if (N <= 0 || S < 0 || dx <= 0.0) return -1;
    double cut = psi_cut(wavelet);
    int err = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1) reduction(| : err)
#endif
    for (int32_t s = 0; s < S; s++) {
        double w = wt[s], amp = sqrt(w * dx);
        int64_t span = 2 * N - 1;               /* kernel index j + N - 1, j in [-(N-1), N-1] */
        double *gr = calloc(span, sizeof(double)), *gi = calloc(span, sizeof(double));
        if (!gr || !gi) { err |= 1; free(gr); free(gi); continue; }
        if (boundary == ORC_PERIODIC) {
            /* h(j), j in [0, N): folded images, stored at j + N - 1 */
            int64_t pmax = (int64_t)ceil(cut / (w * (double)N)) + 1;
            for (int64_t j = 0; j < N; j++) {
                double sr = 0.0, si = 0.0;
                for (int64_t p = -pmax; p <= pmax; p++) {
                    double x = w * (double)(j + p * N);
                    if (fabs(x) > cut) continue;
                    double a, b;
                    orc_psi(wavelet, omega0, x, &a, &b);
                    sr += a; si += b;
                }
                gr[j + N - 1] = sr; gi[j + N - 1] = si;
            }
            for (int64_t n = 0; n < N; n++) {
                double sr = 0.0, si = 0.0;
                for (int64_t m = 0; m < N; m++) {
                    int64_t j = n - m; if (j < 0) j += N;
                    sr += f[m] * gr[j + N - 1];
                    si += f[m] * gi[j + N - 1];
                }
                W_re[(int64_t)s * N + n] = amp * sr;
                W_im[(int64_t)s * N + n] = amp * si;
            }
        } else {
            for (int64_t j = -(N - 1); j <= N - 1; j++) {
                double x = w * (double)j;
                if (fabs(x) > cut) continue;
                orc_psi(wavelet, omega0, x, &gr[j + N - 1], &gi[j + N - 1]);
            }
            for (int64_t n = 0; n < N; n++) {
                double sr = 0.0, si = 0.0;
                for (int64_t m = 0; m < N; m++) {
                    sr += f[m] * gr[n - m + N - 1];
                    si += f[m] * gi[n - m + N - 1];
                }
                W_re[(int64_t)s * N + n] = amp * sr;
                W_im[(int64_t)s * N + n] = amp * si;
            }
        }
        free(gr); free(gi);
    }
    return err ? -1 : 0;
}

/* Direct sum (Eq. 4) at listed points, each evaluated on its own. */
int orc_cwt_direct_points(const double *f, int64_t N, const double *wt, int32_t S,
                          int wavelet, double omega0, double dx, int boundary,
                          const int32_t *ps, const int64_t *pn, int64_t P, int nthreads,
                          double *out_re, double *out_im)
{
    if (N <= 0 || dx <= 0.0) return -1;
    for (int64_t p = 0; p < P; p++)
        if (ps[p] < 0 || ps[p] >= S || pn[p] < 0 || pn[p] >= N) return -1;
    double cut = psi_cut(wavelet);
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t p = 0; p < P; p++) {
        double w = wt[ps[p]];
        int64_t n = pn[p];
        double sr = 0.0, si = 0.0;
        for (int64_t m = 0; m < N; m++) {
            if (boundary == ORC_PERIODIC) {
                int64_t j = n - m;
                int64_t pmax = (int64_t)ceil(cut / (w * (double)N)) + 1;
                for (int64_t q = -pmax; q <= pmax; q++) {
                    double x = w * (double)(j + q * N);
                    if (fabs(x) > cut) continue;
                    double a, b;
                    orc_psi(wavelet, omega0, x, &a, &b);
                    sr += f[m] * a; si += f[m] * b;
                }
            } else {
                double x = w * (double)(n - m);
                if (fabs(x) > cut) continue;
                double a, b;
                orc_psi(wavelet, omega0, x, &a, &b);
                sr += f[m] * a; si += f[m] * b;
            }
        }
        out_re[p] = sqrt(w * dx) * sr;
        out_im[p] = sqrt(w * dx) * si;
    }
    return 0;
}

/* ------------------------------------------------ power spectra (Sec. 5) */

/* Global wavelet power spectrum, Eq. 42: P(w_s) = (1/N) sum_n |W(w_s, n)|^2. */
int orc_wavelet_power(const double *W_re, const double *W_im, int64_t N, int32_t S,
                      double *P)
{
    if (N <= 0 || S < 0) return -1;
    for (int32_t s = 0; s < S; s++) {
        double acc = 0.0;
        for (int64_t n = 0; n < N; n++) {
            double a = W_re[(int64_t)s * N + n], b = W_im ? W_im[(int64_t)s * N + n] : 0.0;
            acc += a * a + b * b;
        }
        P[s] = acc / (double)N;
    }
    return 0;
}

/* Environment-dependent power, Eq. 41 with the paper's two environments:
 * P_pos(w) = <|W|^2> over positions with delta(x) > 0, P_neg over delta < 0,
 * and the fractions f_pos = N_pos/N, f_neg = N_neg/N of Eq. 43. */
int orc_env_power(const double *W_re, const double *W_im, const double *delta, int64_t N,
                  int32_t S, double *P_pos, double *P_neg, double *f_pos, double *f_neg)
{
    if (N <= 0 || S < 0) return -1;
    int64_t np = 0, nn = 0;
    for (int64_t n = 0; n < N; n++) { np += delta[n] > 0.0; nn += delta[n] < 0.0; }
    *f_pos = (double)np / (double)N;
    *f_neg = (double)nn / (double)N;
    for (int32_t s = 0; s < S; s++) {
        double ap = 0.0, an = 0.0;
        for (int64_t n = 0; n < N; n++) {
            double a = W_re[(int64_t)s * N + n], b = W_im ? W_im[(int64_t)s * N + n] : 0.0;
            if (delta[n] > 0.0) ap += a * a + b * b;
            else if (delta[n] < 0.0) an += a * a + b * b;
        }
        P_pos[s] = np ? ap / (double)np : 0.0;
        P_neg[s] = nn ? an / (double)nn : 0.0;
    }
    return 0;
}
