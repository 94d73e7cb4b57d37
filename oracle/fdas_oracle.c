/*
 * FP64 CPU oracle for the FDAS hot path (arXiv:2206.12205).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or load this
 * file; only the test suite, the smoke check and the benchmark's CPU-baseline leg use it.
 * It shares no code, header, table or helper with the CUDA library.
 *
 * What it computes (paper section / equation in brackets):
 *   - the long real FFT of the series [Sec. 3, "Real FFT" of Fig. fdas_flow], here in FP64
 *     with its own iterative radix-2 FFT, DC bin zeroed [Sec. 3.2] and Nyquist dropped;
 *   - spectrum normalisation so that noise powers follow chi^2 with 2 degrees of freedom
 *     [Sec. 5.1, Fig. noise_hist];
 *   - the acceleration response templates [Sec. 2.1, Sec. 3.3]: the Fourier response of a
 *     constant-fdot sinusoid, I(q,z) = int_0^1 exp(i pi (z u^2 - 2 q u)) du, z the drift in
 *     bins over the observation [Eq. fdotz], written with Fresnel integrals;
 *   - the f-z plane as the DIRECT linear correlation of the normalised spectrum with the
 *     templates [Sec. 2.1]: the overlap-save method the paper uses reaches exactly this
 *     result, so the oracle writes the definition out instead of the blockwise FFT form;
 *   - harmonic sums of the plane at integer multiples of (f, fdot) [Sec. 2.1, Sec. 4.3]
 *     and the thresholded list of local maxima;
 *   - the Fourier-interpolated power at fractional (r, z) and its gradient (candidate
 *     refinement), by quadrature of the response and of its derivatives.
 *
 * Readings where the paper is silent (each one is listed in the design notes):
 *   r is the frequency bin at the start of the observation; templates hold m taps at
 *   q = -m/2 .. m/2-1 and are scaled to unit norm; sigma^2 is the mean |X_k|^2 over
 *   k = 1..Nb-1; the spectrum is zero outside [0, Nb); the z grid is z_i = -zmax + 2 i;
 *   harmonic j of (r, z_i) sits at (j r, j z_i); a peak is a 3x3 local maximum above the
 *   threshold of its harmonic level.
 *
 * Every loop is plain and in the order of the definitions, so that it can be read
 * against them.  Build: gcc -O2 -fopenmp -ffp-contract=off -shared -fPIC.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

static const double PI = 3.14159265358979323846264338327950288;

/* ------------------------------------------------------------------------------------ */
/* sin(pi x), cos(pi x) with exact reduction of x modulo 2 (fmod is exact in IEEE).      */
/* ------------------------------------------------------------------------------------ */
static void sincospi_exact(double x, double *s, double *c)
{
    double r = fmod(x, 2.0);            /* exact */
    if (r > 1.0) r -= 2.0;              /* exact: r in (-1, 1] */
    if (r <= -1.0) r += 2.0;
    if (r == 0.0) { *s = 0.0; *c = 1.0; return; }
    if (r == 1.0) { *s = 0.0; *c = -1.0; return; }
    if (r == 0.5) { *s = 1.0; *c = 0.0; return; }
    if (r == -0.5) { *s = -1.0; *c = 0.0; return; }
    *s = sin(PI * r);
    *c = cos(PI * r);
}

/* ------------------------------------------------------------------------------------ */
/* Complex FFT, iterative radix-2 decimation in time, in place.                          */
/*   sign = -1: A_k = sum_j a_j exp(-2 pi i j k / n)  (forward, no scaling)              */
/*   sign = +1: A_k = sum_j a_j exp(+2 pi i j k / n)  (inverse, no scaling)              */
/* n must be a power of two.  Returns 0 on success, -1 on bad n or allocation failure.   */
/* ------------------------------------------------------------------------------------ */
int orc_fft(cplx *a, int64_t n, int sign)
{
    if (n < 1 || (n & (n - 1)) != 0) return -1;
    if (n == 1) return 0;
    /* bit-reversal permutation */
    for (int64_t i = 1, j = 0; i < n; i++) {
        int64_t bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) { cplx t = a[i]; a[i] = a[j]; a[j] = t; }
    }
    /* twiddles w_k = exp(sign 2 pi i k / n), k < n/2, each from its own sin/cos */
    cplx *w = (cplx *)malloc(sizeof(cplx) * (size_t)(n / 2));
    if (!w) return -1;
    for (int64_t k = 0; k < n / 2; k++) {
        double s, c;
        sincospi_exact(2.0 * (double)k / (double)n, &s, &c);
        w[k] = c + (double)sign * s * I;
    }
    for (int64_t len = 2; len <= n; len <<= 1) {
        int64_t half = len >> 1, step = n / len;
        for (int64_t i = 0; i < n; i += len) {
            for (int64_t k = 0; k < half; k++) {
                cplx u = a[i + k];
                cplx v = a[i + k + half] * w[k * step];
                a[i + k] = u + v;
                a[i + k + half] = u - v;
            }
        }
    }
    free(w);
    return 0;
}

/* ------------------------------------------------------------------------------------ */
/* Normalised spectrum of a real series [Sec. 3 "Real FFT"; Sec. 5.1 noise law].         */
/*   X_k = sum_j x_j exp(-2 pi i j k / n), k = 0 .. nb-1, nb = n/2 (Nyquist dropped)      */
/*   X_0 := 0 (DC removed, Sec. 3.2)                                                     */
/*   sigma2 = mean_{k=1..nb-1} |X_k|^2, or the caller's fixed value if sigma2_fixed > 0    */
/*   Xhat_k = X_k * sqrt(2 / sigma2): white noise then has E|Xhat|^2 = 2 (chi^2, 2 dof)   */
/*   sigma2 = 0 (a series with no power outside DC: zero or constant): Xhat = 0, so the    */
/*   plane is zero and nothing is detected, the same choice the local variant makes for a  */
/*   block whose median power is 0.                                                        */
/* xhat receives nb complex values.  Returns 0, or -1 on bad n / allocation failure.      */
/* ------------------------------------------------------------------------------------ */
int orc_spectrum(const float *x, int64_t n, double sigma2_fixed, cplx *xhat, double *sigma2_out)
{
    if (n < 4 || (n & (n - 1)) != 0) return -1;
    int64_t nb = n / 2;
    cplx *a = (cplx *)malloc(sizeof(cplx) * (size_t)n);
    if (!a) return -1;
    for (int64_t j = 0; j < n; j++) a[j] = (double)x[j];
    if (orc_fft(a, n, -1) != 0) { free(a); return -1; }
    a[0] = 0.0;
    double sigma2 = sigma2_fixed;
    if (!(sigma2 > 0.0)) {
        double acc = 0.0;
        for (int64_t k = 1; k < nb; k++) acc += creal(a[k]) * creal(a[k]) + cimag(a[k]) * cimag(a[k]);
        sigma2 = acc / (double)(nb - 1);
    }
    double scale = sigma2 > 0.0 ? sqrt(2.0 / sigma2) : 0.0;
    for (int64_t k = 0; k < nb; k++) xhat[k] = a[k] * scale;
    if (sigma2_out) *sigma2_out = sigma2;
    free(a);
    return 0;
}

static int cmp_double(const void *pa, const void *pb)
{
    const double a = *(const double *)pa, b = *(const double *)pb;
    return (a > b) - (a < b);
}

/* ------------------------------------------------------------------------------------ */
/* Robust local normalisation (a variant of the noise normalisation above; the paper uses  */
/* one sigma2 per spectrum).  The raw spectrum X_k (X_0 = 0), then the bins of each block  */
/* b = [b B, b B + B) scaled by sqrt(2 ln 2 / med_b), med_b the lower median (the element  */
/* of rank floor((n-1)/2) in ascending order) of |X_k|^2 over the block's n bins k >= 1:   */
/* |X_k|^2 of noise is exponential, whose median is its mean times ln 2, so normalised     */
/* noise again has E|Xhat|^2 = 2, block by block; a few signal bins do not move a median.  */
/* Returns 0, or -1 on bad n / block / allocation failure.                                 */
/* ------------------------------------------------------------------------------------ */
int orc_spectrum_local(const float *x, int64_t n, int64_t block, cplx *xhat)
{
    if (n < 4 || (n & (n - 1)) != 0) return -1;
    const int64_t nb = n / 2;
    if (block < 2 || nb % block != 0) return -1;
    if (orc_spectrum(x, n, 2.0, xhat, NULL) != 0) return -1;     /* sigma2 = 2: scale 1, raw X */
    double *pw = (double *)malloc(sizeof(double) * (size_t)block);
    if (!pw) return -1;
    for (int64_t b0 = 0; b0 < nb; b0 += block) {
        int64_t cnt = 0;
        for (int64_t k = b0; k < b0 + block; k++)
            if (k >= 1) pw[cnt++] = creal(xhat[k]) * creal(xhat[k]) + cimag(xhat[k]) * cimag(xhat[k]);
        qsort(pw, (size_t)cnt, sizeof(double), cmp_double);
        const double med = pw[(cnt - 1) / 2];
        const double s = med > 0.0 ? sqrt(2.0 * log(2.0) / med) : 0.0;
        for (int64_t k = b0; k < b0 + block; k++) xhat[k] *= s;
    }
    free(pw);
    return 0;
}

/* ------------------------------------------------------------------------------------ */
/* Fresnel integrals C(x) = int_0^x cos(pi t^2/2) dt, S(x) = int_0^x sin(pi t^2/2) dt.   */
/* Written through F(x) = C + iS = ((1+i)/2) erf(w), w = (sqrt(pi)/2)(1-i) x:            */
/*   |x| <= 1.6 : power series F(x) = sum_k (i pi/2)^k x^(2k+1) / (k! (2k+1))             */
/*   |x| >  1.6 : F(x) = ((1+i)/2)(1 - erfc(w)), erfc(w) = exp(-w^2)/sqrt(pi) * K(w), with */
/*                K(w) = 1/(w + (1/2)/(w + 1/(w + (3/2)/(w + 2/(w + ...))))) the Laplace  */
/*                continued fraction (Abramowitz & Stegun 7.1.14), evaluated by the       */
/*                modified Lentz method; exp(-w^2) = exp(i pi x^2 / 2).                   */
/* Odd symmetry gives negative x.                                                        */
/* ------------------------------------------------------------------------------------ */
void orc_fresnel(double x, double *c_out, double *s_out)
{
    double ax = fabs(x);
    cplx f;
    if (ax <= 1.6) {
        cplx term = ax;                  /* k = 0: x */
        f = ax;
        double x2 = ax * ax;
        for (int k = 1; k < 200; k++) {
            /* term_k / term_{k-1} = (i pi/2) x^2 / k */
            term *= (I * (PI / 2.0) * x2) / (double)k;
            cplx add = term / (double)(2 * k + 1);
            f += add;
            if (cabs(add) < 1e-18 * cabs(f)) break;
        }
    } else {
        cplx w = (sqrt(PI) / 2.0) * (1.0 - I) * ax;
        /* modified Lentz for K = a1/(b1 + a2/(b2 + ...)), b_k = w, a1 = 1, a_k = (k-1)/2 */
        const double tiny = 1e-300;
        cplx fk = tiny, Ck = fk, Dk = 0.0;
        for (int k = 1; k < 100000; k++) {
            double ak = (k == 1) ? 1.0 : 0.5 * (double)(k - 1);
            Dk = w + ak * Dk;
            if (cabs(Dk) < tiny) Dk = tiny;
            Dk = 1.0 / Dk;
            Ck = w + ak / Ck;
            if (cabs(Ck) < tiny) Ck = tiny;
            cplx delta = Ck * Dk;
            fk *= delta;
            if (cabs(delta - 1.0) < 1e-17) break;
        }
        double s, c;
        /* exp(i pi x^2 / 2) with the argument reduced exactly from x^2 / 2 */
        sincospi_exact(0.5 * ax * ax, &s, &c);
        cplx erfc_w = (c + I * s) / sqrt(PI) * fk;
        f = 0.5 * (1.0 + I) * (1.0 - erfc_w);
    }
    if (x < 0) f = -f;
    *c_out = creal(f);
    *s_out = cimag(f);
}

/* ------------------------------------------------------------------------------------ */
/* Gauss-Legendre nodes/weights on [-1, 1] by Newton iteration on P_n.                    */
/* ------------------------------------------------------------------------------------ */
static void gauss_legendre(int n, double *xs, double *ws)
{
    for (int i = 0; i < n; i++) {
        double x = cos(PI * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; it++) {
            double p0 = 1.0, p1 = x;
            for (int k = 2; k <= n; k++) {
                double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / (double)k;
                p0 = p1; p1 = p2;
            }
            dp = n * (x * p1 - p0) / (x * x - 1.0);
            double dx = p1 / dp;
            x -= dx;
            if (fabs(dx) < 1e-16) break;
        }
        double p0 = 1.0, p1 = x;
        for (int k = 2; k <= n; k++) {
            double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / (double)k;
            p0 = p1; p1 = p2;
        }
        dp = n * (x * p1 - p0) / (x * x - 1.0);
        xs[i] = x;
        ws[i] = 2.0 / ((1.0 - x * x) * dp * dp);
    }
}

#define GL_N 20

/* ------------------------------------------------------------------------------------ */
/* Moments M_p(q, z) = int_0^1 u^p exp(i pi (z u^2 - 2 q u)) du, p = 0, 1, 2, by          */
/* composite Gauss-Legendre quadrature.  The phase changes by at most 2 pi (|z| + |q|)   */
/* over [0, 1]; panels of at most one radian-cycle each make 20 nodes exact to rounding. */
/* M_0 is the response I(q, z); M_1, M_2 give its derivatives (see orc_interp_power).    */
/* ------------------------------------------------------------------------------------ */
void orc_response_moments_quad(double q, double z, cplx *m0, cplx *m1, cplx *m2)
{
    double xs[GL_N], ws[GL_N];
    gauss_legendre(GL_N, xs, ws);
    int64_t panels = (int64_t)ceil(fabs(z) + fabs(q)) + 4;
    double h = 1.0 / (double)panels;
    cplx a0 = 0.0, a1 = 0.0, a2 = 0.0;
    for (int64_t p = 0; p < panels; p++) {
        double mid = (p + 0.5) * h;
        for (int i = 0; i < GL_N; i++) {
            double u = mid + 0.5 * h * xs[i];
            double s, c;
            /* exp(i pi (z u^2 - 2 q u)) */
            sincospi_exact(z * u * u - 2.0 * q * u, &s, &c);
            cplx e = (c + I * s) * (0.5 * h * ws[i]);
            a0 += e;
            a1 += u * e;
            a2 += u * u * e;
        }
    }
    if (m0) *m0 = a0;
    if (m1) *m1 = a1;
    if (m2) *m2 = a2;
}

/* I(q, z) by quadrature only (independent route; used to pin the Fresnel form). */
void orc_response_quad(double q, double z, cplx *out)
{
    orc_response_moments_quad(q, z, out, NULL, NULL);
}

/* ------------------------------------------------------------------------------------ */
/* Response of a constant-fdot sinusoid at offset q from its start bin, drift z bins:    */
/*   I(q, z) = int_0^1 exp(i pi (z u^2 - 2 q u)) du                                      */
/*   z = 0 : exp(-i pi q) sin(pi q)/(pi q)  (an exact delta at integer q)                 */
/*   z > 0 : exp(-i pi q^2/z)/sqrt(2z) * [F(s1) - F(s0)],                                 */
/*           s0 = -q sqrt(2/z), s1 = (z - q) sqrt(2/z), F = C + iS (completing the square) */
/*   z < 0 : conj(I(-q, -z))                                                              */
/*   0 < |z| < 1e-3 : quadrature, where the Fresnel difference loses its digits.          */
/* ------------------------------------------------------------------------------------ */
void orc_response(double q, double z, cplx *out)
{
    if (z < 0.0) {
        cplx t;
        orc_response(-q, -z, &t);
        *out = conj(t);
        return;
    }
    if (z == 0.0) {
        if (q == 0.0) { *out = 1.0; return; }
        double s, c;
        sincospi_exact(q, &s, &c);
        /* exp(-i pi q) * sin(pi q) / (pi q) */
        *out = (c - I * s) * (s / (PI * q));
        return;
    }
    if (z < 1e-3) {
        orc_response_quad(q, z, out);
        return;
    }
    double k = sqrt(2.0 / z);
    double c0, s0, c1, s1;
    orc_fresnel(-q * k, &c0, &s0);
    orc_fresnel((z - q) * k, &c1, &s1);
    double ps, pc;
    sincospi_exact(-q * q / z, &ps, &pc);
    *out = (pc + I * ps) / sqrt(2.0 * z) * ((c1 - c0) + I * (s1 - s0));
}

/* ------------------------------------------------------------------------------------ */
/* Template bank [Sec. 2.1, Sec. 3.3]: K = zmax + 1 rows, z_i = -zmax + 2 i, and m taps  */
/* at q = -m/2 .. m/2-1:  T[i][q + m/2] = I(q, z_i) / sqrt(eta_i),                        */
/* eta_i = sum_q |I(q, z_i)|^2 (unit-norm templates).  T is [K][m] row-major.             */
/* Returns 0, or -1 on a bad argument (odd or negative zmax, odd or too small m).         */
/* ------------------------------------------------------------------------------------ */
int orc_templates(int zmax, int m, cplx *T, double *eta_out)
{
    if (zmax < 0 || (zmax & 1) || m < 2 || (m & 1)) return -1;
    int K = zmax + 1;
    for (int i = 0; i < K; i++) {
        double z = -(double)zmax + 2.0 * (double)i;
        double eta = 0.0;
        for (int t = 0; t < m; t++) {
            double q = (double)(t - m / 2);
            cplx v;
            orc_response(q, z, &v);
            T[(int64_t)i * m + t] = v;
            eta += creal(v) * creal(v) + cimag(v) * cimag(v);
        }
        double inv = 1.0 / sqrt(eta);
        for (int t = 0; t < m; t++) T[(int64_t)i * m + t] *= inv;
        if (eta_out) eta_out[i] = eta;
    }
    return 0;
}

/* ------------------------------------------------------------------------------------ */
/* One cell of the f-z plane [Sec. 2.1]: the linear correlation of the normalised         */
/* spectrum with template row Ti (m taps, q = -m/2 .. m/2-1), spectrum zero outside       */
/* [0, nb):   P(r, z_i) = | sum_q Xhat_{r+q} conj(T_i(q)) |^2                             */
/* ------------------------------------------------------------------------------------ */
static double plane_cell(const cplx *xhat, int64_t nb, int m, const cplx *Ti, int64_t r)
{
    cplx acc = 0.0;
    for (int t = 0; t < m; t++) {
        int64_t k = r + (int64_t)(t - m / 2);
        if (k < 0 || k >= nb) continue;
        acc += xhat[k] * conj(Ti[t]);
    }
    return creal(acc) * creal(acc) + cimag(acc) * cimag(acc);
}

/* Whole plane, [K][nb] row-major, K = zmax + 1; rows in parallel.  Returns 0 or -1. */
int orc_plane(const cplx *xhat, int64_t nb, int zmax, int m, const cplx *T, double *plane)
{
    if (nb < 1 || zmax < 0 || (zmax & 1) || m < 2 || (m & 1)) return -1;
    int K = zmax + 1;
    #pragma omp parallel for schedule(dynamic, 1)
    for (int i = 0; i < K; i++)
        for (int64_t r = 0; r < nb; r++)
            plane[(int64_t)i * nb + r] = plane_cell(xhat, nb, m, T + (int64_t)i * m, r);
    return 0;
}

/* ------------------------------------------------------------------------------------ */
/* FP8 E4M3 (a precision ablation of the correlation): 1 sign, 4 exponent (bias 7), 3      */
/* mantissa bits; normal numbers 2^-6 .. 448 = 1.75 x 2^8, subnormals in steps of 2^-9;    */
/* round to nearest, ties to even, saturating at +-448.                                     */
/* ------------------------------------------------------------------------------------ */
double orc_e4m3(double v)
{
    double a = fabs(v);
    if (a == 0.0 || a != a) return v;
    int E;
    frexp(a, &E);                       /* a = f 2^E, f in [0.5, 1): floor(log2 a) = E - 1 */
    int e = E - 1;
    if (e < -6) e = -6;                 /* subnormal range shares the 2^-6 binade's step  */
    double step = ldexp(1.0, e - 3);
    double r = nearbyint(a / step) * step;
    if (r > 448.0) r = 448.0;
    return copysign(r, v);
}

/* Power of two s with M s <= 448 < 2 M s (the largest such scale; 1 when M = 0).          */
static double e4m3_scale(double M)
{
    if (!(M > 0.0)) return 1.0;
    int E;
    double f = frexp(M, &E);            /* M = f 2^E, 448 = 0.875 x 2^9                       */
    return ldexp(1.0, (f <= 0.875 ? 9 : 8) - E);
}

/* The direct correlation with FP8 operands (the FDAS_FP8_DIRECT ablation), emulated:        */
/*   tile t = floor(r / 1024): s_t from the largest |Re| or |Im| of Xhat over the window      */
/*   [1024 t - m/2, 1024 t + 1024 + m/2) (zero outside the spectrum); template z: sigma_z    */
/*   from the largest |Re| or |Im| of its taps;                                              */
/*   P(r, z) = |sum_q e4m3(s_t Xhat_{r+q}) conj(e4m3(sigma_z T_z(q)))|^2 / (s_t sigma_z)^2    */
/* (component-wise rounding; the sum in FP64).                                               */
#define FP8_TILE 1024

/* sigma_z and the rounded, scaled taps of every template (tq: K x m, sig: K). */
static void fp8_taps(const cplx *T, int K, int m, cplx *tq, double *sig)
{
    for (int i = 0; i < K; i++) {
        double M = 0.0;
        for (int q = 0; q < m; q++) {
            cplx t = T[(size_t)i * m + q];
            M = fmax(M, fmax(fabs(creal(t)), fabs(cimag(t))));
        }
        sig[i] = e4m3_scale(M);
        for (int q = 0; q < m; q++) {
            cplx t = T[(size_t)i * m + q];
            tq[(size_t)i * m + q] = orc_e4m3(creal(t) * sig[i]) + I * orc_e4m3(cimag(t) * sig[i]);
        }
    }
}

/* s_t of the tile starting at bin t0, and its rounded, scaled window wq[j] = e4m3(s_t Xhat_k), */
/* k = t0 - m/2 + j, j < 1024 + m.                                                              */
static double fp8_window(const cplx *xhat, int64_t nb, int m, int64_t t0, cplx *wq)
{
    double M = 0.0;
    for (int64_t k = t0 - m / 2; k < t0 + FP8_TILE + m / 2; k++)
        if (k >= 0 && k < nb) M = fmax(M, fmax(fabs(creal(xhat[k])), fabs(cimag(xhat[k]))));
    double st = e4m3_scale(M);
    for (int j = 0; j < FP8_TILE + m; j++) {
        int64_t k = t0 - m / 2 + j;
        wq[j] = (k >= 0 && k < nb) ? orc_e4m3(creal(xhat[k]) * st) + I * orc_e4m3(cimag(xhat[k]) * st) : 0.0;
    }
    return st;
}

static double fp8_cell(const cplx *wq, double st, const cplx *tq, double sig, int m, int64_t j0)
{
    cplx acc = 0.0;
    for (int q = 0; q < m; q++) acc += wq[j0 + q] * conj(tq[q]);
    double g = st * sig;
    return (creal(acc) * creal(acc) + cimag(acc) * cimag(acc)) / (g * g);
}

int orc_plane_fp8(const cplx *xhat, int64_t nb, int zmax, int m, const cplx *T, double *plane)
{
    int K = zmax + 1;
    cplx *tq = (cplx *)malloc(sizeof(cplx) * (size_t)K * m);
    double *sig = (double *)malloc(sizeof(double) * (size_t)K);
    cplx *wq = (cplx *)malloc(sizeof(cplx) * (size_t)(FP8_TILE + m));
    if (!tq || !sig || !wq) { free(tq); free(sig); free(wq); return -1; }
    fp8_taps(T, K, m, tq, sig);
    for (int64_t t0 = 0; t0 < nb; t0 += FP8_TILE) {
        double st = fp8_window(xhat, nb, m, t0, wq);
        for (int i = 0; i < K; i++)
            for (int64_t r = t0; r < t0 + FP8_TILE && r < nb; r++)
                plane[(size_t)i * nb + r] = fp8_cell(wq, st, tq + (size_t)i * m, sig[i], m, r - t0);
    }
    free(tq); free(sig); free(wq);
    return 0;
}

/* Selected cells (zi[c], r[c]) of the FP8 plane, c < n.  Returns 0, -1 on an allocation     */
/* failure, -2 on an index off the plane.                                                    */
int orc_plane_fp8_cells(const cplx *xhat, int64_t nb, int zmax, int m, const cplx *T,
                        int64_t n, const int32_t *zi, const int64_t *r, double *out)
{
    int K = zmax + 1;
    for (int64_t c = 0; c < n; c++)
        if (zi[c] < 0 || zi[c] >= K || r[c] < 0 || r[c] >= nb) return -2;
    cplx *tq = (cplx *)malloc(sizeof(cplx) * (size_t)K * m);
    double *sig = (double *)malloc(sizeof(double) * (size_t)K);
    cplx *wq = (cplx *)malloc(sizeof(cplx) * (size_t)(FP8_TILE + m));
    if (!tq || !sig || !wq) { free(tq); free(sig); free(wq); return -1; }
    fp8_taps(T, K, m, tq, sig);
    for (int64_t c = 0; c < n; c++) {
        int64_t t0 = r[c] / FP8_TILE * FP8_TILE;
        double st = fp8_window(xhat, nb, m, t0, wq);
        out[c] = fp8_cell(wq, st, tq + (size_t)zi[c] * m, sig[zi[c]], m, r[c] - t0);
    }
    free(tq); free(sig); free(wq);
    return 0;
}

/* Selected cells (zi[c], r[c]) of the plane, c < n.  Returns 0, or -1 on an index off    */
/* the plane.                                                                             */
int orc_plane_cells(const cplx *xhat, int64_t nb, int zmax, int m, const cplx *T,
                    int64_t n, const int32_t *zi, const int64_t *r, double *out)
{
    int K = zmax + 1;
    for (int64_t c = 0; c < n; c++)
        if (zi[c] < 0 || zi[c] >= K || r[c] < 0 || r[c] >= nb) return -1;
    #pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < n; c++)
        out[c] = plane_cell(xhat, nb, m, T + (int64_t)zi[c] * m, r[c]);
    return 0;
}

/* ------------------------------------------------------------------------------------ */
/* Harmonic sum and peak list [Sec. 2.1: power at integer multiples of f and fdot;        */
/* Sec. 4.3].  For a level H in {1, 2, 4, 8, 16} (H <= max_harm):                         */
/*   S_H(r, i) = sum_{h=1..H} P(h r, i_h),  z_{i_h} = h z_i, i.e. i_h = (h z_i + zmax)/2,  */
/* defined where |H z_i| <= zmax and H r < nb (every term on the plane, no rounding).      */
/* A cell is a peak of level H if S_H > thr[level] and no defined 3x3 neighbour beats it: */
/* it must be strictly above neighbours that come earlier in row-major (i, r) order and  */
/* at least equal to later ones.  Peaks come out ordered by (H, i, r).  The sums run in   */
/* the order h = 1..H in the precision of the plane (float for a float plane).           */
/* At most max_out records are written; *count receives the true number of peaks.        */
/* ------------------------------------------------------------------------------------ */
#define HS_BODY(TYPE)                                                                      \
    int K = zmax + 1;                                                                      \
    int64_t cnt = 0;                                                                       \
    for (int lev = 0; lev < 5; lev++) {                                                    \
        int H = 1 << lev;                                                                  \
        if (H > max_harm) break;                                                           \
        TYPE th = (TYPE)thr[lev];                                                          \
        int64_t rmax = (nb - 1) / H; /* last r with H r < nb */                            \
        for (int i = 0; i < K; i++) {                                                      \
            int z = -zmax + 2 * i;                                                         \
            if (abs(H * z) > zmax) continue;                                               \
            for (int64_t r = 0; r <= rmax; r++) {                                          \
                TYPE s = hsum_##TYPE(plane, nb, zmax, H, i, r);                            \
                if (!(s > th)) continue;                                                   \
                int is_peak = 1;                                                           \
                for (int di = -1; di <= 1 && is_peak; di++) {                              \
                    int ii = i + di;                                                       \
                    if (ii < 0 || ii >= K) continue;                                       \
                    if (abs(H * (-zmax + 2 * ii)) > zmax) continue;                        \
                    for (int64_t dr = -1; dr <= 1; dr++) {                                 \
                        if (di == 0 && dr == 0) continue;                                  \
                        int64_t rr = r + dr;                                               \
                        if (rr < 0 || rr > rmax) continue;                                 \
                        TYPE sn = hsum_##TYPE(plane, nb, zmax, H, ii, rr);                 \
                        int earlier = (di < 0) || (di == 0 && dr < 0);                     \
                        if (earlier ? !(s > sn) : !(s >= sn)) { is_peak = 0; break; }      \
                    }                                                                      \
                }                                                                          \
                if (!is_peak) continue;                                                    \
                if (cnt < max_out) {                                                       \
                    out_h[cnt] = H; out_zi[cnt] = i; out_r[cnt] = r; out_p[cnt] = s;       \
                }                                                                          \
                cnt++;                                                                     \
            }                                                                              \
        }                                                                                  \
    }                                                                                      \
    *count = cnt;                                                                          \
    return 0;

static float hsum_float(const float *plane, int64_t nb, int zmax, int H, int i, int64_t r)
{
    int z = -zmax + 2 * i;
    float s = 0.0f;
    for (int h = 1; h <= H; h++) {
        int ih = (h * z + zmax) / 2;
        s = s + plane[(int64_t)ih * nb + (int64_t)h * r];
    }
    return s;
}

static double hsum_double(const double *plane, int64_t nb, int zmax, int H, int i, int64_t r)
{
    int z = -zmax + 2 * i;
    double s = 0.0;
    for (int h = 1; h <= H; h++) {
        int ih = (h * z + zmax) / 2;
        s = s + plane[(int64_t)ih * nb + (int64_t)h * r];
    }
    return s;
}

/* ------------------------------------------------------------------------------------ */
/* Highest-harmonic-anchored harmonic sums with rounding (a variant of the sums above,    */
/* the form of PRESTO-style searches): the cell (r, i) is harmonic H, and harmonic j of   */
/* level L is read at r_j = round(j r / L) and at the grid z nearest j z_i / L, halves     */
/* rounded up:  r_j = floor((2 j r + L) / (2 L)),  i_j = floor((j z_i + L zmax + L)/(2 L)). */
/* Level 2L's even fractions 2j'/2L = j'/L round exactly as level L's, so the sums nest:  */
/*   S_1 = P(r, i),  S_2L = S_L + sum_{odd j < 2L, increasing} P(r_j, i_j);               */
/* every term is on the plane for every (r, i), so each level covers the whole plane.     */
/* Peaks: the same threshold and 3x3 rule on the S_L grid.                                  */
/* ------------------------------------------------------------------------------------ */
#define HSA_BODY(TYPE)                                                                     \
    int z = -zmax + 2 * i;                                                                 \
    TYPE s = plane[(int64_t)i * nb + r];                                                   \
    for (int L = 2; L <= H; L *= 2)                                                        \
        for (int j = 1; j < L; j += 2) {                                                   \
            int64_t rj = (2 * (int64_t)j * r + L) / (2 * L);                               \
            int ij = (j * z + L * zmax + L) / (2 * L);                                     \
            s = s + plane[(int64_t)ij * nb + rj];                                          \
        }                                                                                  \
    return s;

static float hsa_float(const float *plane, int64_t nb, int zmax, int H, int i, int64_t r) { HSA_BODY(float) }
static double hsa_double(const double *plane, int64_t nb, int zmax, int H, int i, int64_t r) { HSA_BODY(double) }

#define HSA_PEAKS(TYPE)                                                                    \
    int K = zmax + 1;                                                                      \
    int64_t cnt = 0;                                                                       \
    for (int lev = 0; lev < 5; lev++) {                                                    \
        int H = 1 << lev;                                                                  \
        if (H > max_harm) break;                                                           \
        TYPE th = (TYPE)thr[lev];                                                          \
        for (int i = 0; i < K; i++)                                                        \
            for (int64_t r = 0; r < nb; r++) {                                             \
                TYPE s = hsa_##TYPE(plane, nb, zmax, H, i, r);                             \
                if (!(s > th)) continue;                                                   \
                int is_peak = 1;                                                           \
                for (int di = -1; di <= 1 && is_peak; di++) {                              \
                    int ii = i + di;                                                       \
                    if (ii < 0 || ii >= K) continue;                                       \
                    for (int64_t dr = -1; dr <= 1; dr++) {                                 \
                        if (di == 0 && dr == 0) continue;                                  \
                        int64_t rr = r + dr;                                               \
                        if (rr < 0 || rr >= nb) continue;                                  \
                        TYPE sn = hsa_##TYPE(plane, nb, zmax, H, ii, rr);                  \
                        int earlier = (di < 0) || (di == 0 && dr < 0);                     \
                        if (earlier ? !(s > sn) : !(s >= sn)) { is_peak = 0; break; }      \
                    }                                                                      \
                }                                                                          \
                if (!is_peak) continue;                                                    \
                if (cnt < max_out) {                                                       \
                    out_h[cnt] = H; out_zi[cnt] = i; out_r[cnt] = r; out_p[cnt] = s;       \
                }                                                                          \
                cnt++;                                                                     \
            }                                                                              \
    }                                                                                      \
    *count = cnt;                                                                          \
    return 0;

static int hs_check(int64_t nb, int zmax, int max_harm)
{
    if (nb < 1 || zmax < 0 || (zmax & 1)) return -1;
    if (max_harm != 1 && max_harm != 2 && max_harm != 4 && max_harm != 8 && max_harm != 16) return -1;
    return 0;
}

/* Given-plane mode in float: the arithmetic a float plane admits, term order h = 1..H. */
int orc_peaks_f32(const float *plane, int64_t nb, int zmax, int max_harm, const double *thr,
                  int64_t max_out, int32_t *out_h, int32_t *out_zi, int64_t *out_r,
                  float *out_p, int64_t *count)
{
    if (hs_check(nb, zmax, max_harm)) return -1;
    HS_BODY(float)
}

/* Highest-harmonic-anchored variant, float (given-plane mode) and FP64. */
int orc_peaks_anch_f32(const float *plane, int64_t nb, int zmax, int max_harm, const double *thr,
                       int64_t max_out, int32_t *out_h, int32_t *out_zi, int64_t *out_r,
                       float *out_p, int64_t *count)
{
    if (hs_check(nb, zmax, max_harm)) return -1;
    HSA_PEAKS(float)
}

int orc_peaks_anch_f64(const double *plane, int64_t nb, int zmax, int max_harm, const double *thr,
                       int64_t max_out, int32_t *out_h, int32_t *out_zi, int64_t *out_r,
                       double *out_p, int64_t *count)
{
    if (hs_check(nb, zmax, max_harm)) return -1;
    HSA_PEAKS(double)
}

/* The same on an FP64 plane. */
int orc_peaks_f64(const double *plane, int64_t nb, int zmax, int max_harm, const double *thr,
                  int64_t max_out, int32_t *out_h, int32_t *out_zi, int64_t *out_r,
                  double *out_p, int64_t *count)
{
    if (hs_check(nb, zmax, max_harm)) return -1;
    HS_BODY(double)
}

/* ------------------------------------------------------------------------------------ */
/* Fourier-interpolated power at fractional (r, z) and its gradient (sub-bin candidate    */
/* refinement of a plane peak).  With the m-tap window anchored at bin k0 (the same      */
/* window shape as the plane):                                                            */
/*   A(r, z) = sum_{k = k0-m/2}^{k0+m/2-1} Xhat_k conj(I(k - r, z)),  P = |A|^2            */
/* (I unnormalised; taps off the spectrum are zero).  With E = exp(i pi (z u^2 - 2 q u)),  */
/* q = k - r:                                                                             */
/*   d/dr I(k - r, z) = int 2 pi i u E du = 2 pi i M_1,   d/dz I = int i pi u^2 E du = i pi M_2 */
/*   dP/dx = 2 Re(conj(A) dA/dx).                                                         */
/* The moments come from quadrature.  For a fixed k0, P is smooth in (r, z) everywhere;  */
/* the refinement keeps k0 at its seed bin so the power it climbs has no jumps.          */
/* ------------------------------------------------------------------------------------ */
void orc_interp_power_at(const cplx *xhat, int64_t nb, int m, int64_t k0, double r, double z,
                         double *P, double *dPdr, double *dPdz)
{
    cplx A = 0.0, Ar = 0.0, Az = 0.0;
    for (int t = 0; t < m; t++) {
        int64_t k = k0 + (int64_t)(t - m / 2);
        if (k < 0 || k >= nb) continue;
        cplx m0, m1, m2;
        orc_response_moments_quad((double)k - r, z, &m0, &m1, &m2);
        cplx dIr = 2.0 * PI * I * m1;
        cplx dIz = I * PI * m2;
        A += xhat[k] * conj(m0);
        Ar += xhat[k] * conj(dIr);
        Az += xhat[k] * conj(dIz);
    }
    if (P) *P = creal(A) * creal(A) + cimag(A) * cimag(A);
    if (dPdr) *dPdr = 2.0 * creal(conj(A) * Ar);
    if (dPdz) *dPdz = 2.0 * creal(conj(A) * Az);
}

/* The window centred on the nearest bin, k0 = floor(r + 1/2). */
void orc_interp_power(const cplx *xhat, int64_t nb, int m, double r, double z,
                      double *P, double *dPdr, double *dPdz)
{
    orc_interp_power_at(xhat, nb, m, (int64_t)floor(r + 0.5), r, z, P, dPdr, dPdz);
}

/* ------------------------------------------------------------------------------------ */
/* Sub-bin refinement of one candidate by preconditioned gradient ascent on P(r, z)       */
/* (every step in FP64).  The window stays anchored at k0 = floor(r_seed + 1/2).  Each    */
/* step is d = Hinv grad P / P with Hinv = (1/(2 pi^2)) [[48, -90], [-90, 180]], the       */
/* inverse of the Hessian of 1 - P/P_peak of an ideal chirp: an offset (dr, dz) leaves    */
/* the phase error 2 pi (dr u + dz u^2 / 2) over u in [0, 1], whose variance             */
/* pi^2 (dr^2/3 + dr dz/3 + 4 dz^2/45) is 1 - P/P_peak to second order.  d is scaled to    */
/* |dr| <= 1/4, |dz| <= 1 and halved at most three times until P does not decrease; the    */
/* ascent stops when no such step exists.  Returns the number of power evaluations.       */
/* ------------------------------------------------------------------------------------ */
int orc_refine(const cplx *xhat, int64_t nb, int m, double r, double z, int steps,
               double *r_out, double *z_out, double *P_out)
{
    int64_t k0 = (int64_t)floor(r + 0.5);
    double P, gr, gz;
    orc_interp_power_at(xhat, nb, m, k0, r, z, &P, &gr, &gz);
    int evals = 1;
    for (int s = 0; s < steps; s++) {
        if (!(P > 0.0)) break;
        double c = 1.0 / (2.0 * PI * PI * P);
        double dr = (48.0 * gr - 90.0 * gz) * c;
        double dz = (-90.0 * gr + 180.0 * gz) * c;
        double sc = fmax(fmax(4.0 * fabs(dr), fabs(dz)), 1.0);
        dr /= sc;
        dz /= sc;
        int ok = 0;
        double P2 = 0.0, gr2 = 0.0, gz2 = 0.0;
        for (int h = 0; h < 4; h++) {
            orc_interp_power_at(xhat, nb, m, k0, r + dr, z + dz, &P2, &gr2, &gz2);
            evals++;
            if (P2 >= P) { ok = 1; break; }
            dr *= 0.5;
            dz *= 0.5;
        }
        if (!ok) break;
        r += dr; z += dz; P = P2; gr = gr2; gz = gz2;
    }
    *r_out = r;
    *z_out = z;
    *P_out = P;
    return evals;
}

/* orc_refine over n candidates (rz: [n][2] in, out: [n][2]), threaded over candidates. */
void orc_refine_many(const cplx *xhat, int64_t nb, int m, int64_t n, const double *rz, int steps,
                     double *out, double *P_out, int32_t *evals)
{
    #pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = 0; i < n; i++) {
        int e = orc_refine(xhat, nb, m, rz[2 * i], rz[2 * i + 1], steps, &out[2 * i], &out[2 * i + 1], &P_out[i]);
        if (evals) evals[i] = e;
    }
}
