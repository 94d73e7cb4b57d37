// K5: sub-bin refinement of f-z candidates by gradient ascent on the Fourier-interpolated power
// (the plane of Sec. 2.1 evaluated between its grid points; derivatives by the adjoint sums).
//
// A plane peak sits on the integer grid (r, z_i); the signal that made it lies in between.  With
// the plane's m-tap window anchored at bin k0, the interpolated amplitude and power are
//   A(r, z) = sum_{k = k0-m/2}^{k0+m/2-1} Xhat_k conj(I(k - r, z)),   P = |A|^2,
// where I(q, z) = M_0(q, z) is the unnormalised response of a constant-fdot sinusoid (z in bins of
// drift over the observation, Eq. fdotz) and M_p(q, z) = int_0^1 u^p exp(i pi (z u^2 - 2 q u)) du.
// Differentiating under the integral, dI(k - r, z)/dr = 2 pi i M_1 and dI/dz = i pi M_2, so
//   dP/dr = 2 Re(conj(A) sum_k Xhat_k conj(2 pi i M_1)),  dP/dz = 2 Re(conj(A) sum_k Xhat_k conj(i pi M_2)).
// One warp evaluates one point: lane l takes taps l, l + 32, ... (coalesced spectrum reads, and
// neighbouring lanes take neighbouring taps, which fall in the same branch below); the three sums
// are reduced with xor shuffles, after which every lane holds the same bits, so the ascent's
// control flow is warp-uniform.
//
// Moments of one tap, for z >= 0 (z < 0 through M_p(q, z) = conj(M_p(-q, -z))), v(u) = z u - q:
//  * far tap, min_{u in [0,1]} |v| >= c max(1, sqrt z): no stationary phase near [0, 1].  Repeated
//    integration by parts (dE/du = 2 pi i v E, E = exp(i pi (z u^2 - 2 q u))) gives, at each end,
//    with w = 1/(2 pi i v) and t = z/(2 pi i v^2):
//      M_0 = [E w S0]_0^1,  M_1 = [E (u w S0 - w^2 S1)]_0^1,  M_2 = [E (u^2 w S0 - 2 u w^2 S1 + 2 w^3 S2)]_0^1,
//      S0 = sum_k (2k-1)!! t^k,  S1 = sum_k (2k+1)!! t^k,  S2 = sum_k (k+1)(2k+1)!! t^k.
//    |t| <= 1/(2 pi c^2), so 5 terms (c = 6) leave a truncation below FP32 rounding and 7 terms
//    (c = 12) below 1e-14.
//  * near tap, z >= 1: the Fresnel form.  Completing the square, with F = C + iS written at each
//    end as F(s) = c + d exp(i pi s^2/2) (its power series for |s| <= 1.5, 2.5 in FP64, where
//    d = 0; otherwise c = sgn(s)(1+i)/2 and d = -sgn(s) G(|s|),
//    G(x) = (1+i)/(2 sqrt(pi)) K((sqrt(pi)/2)(1-i) x), K the Laplace continued fraction of
//    sqrt(pi) exp(w^2) erfc(w); its depth, set per lane, bounds the warp's time, hence the wider
//    series range in FP64),
//      sqrt(2z) M_0 = (c1 - c0) exp(-i pi q^2/z) + d1 exp(i pi (z - 2q)) - d0,
//      s0 = -q sqrt(2/z),  s1 = (z - q) sqrt(2/z),
//    and one integration by parts each for the higher moments:
//      M_1 = [(E(1) - 1)/(2 pi i) + q M_0] / z,   M_2 = [(E(1) - M_0)/(2 pi i) + q M_1] / z.
//  * near tap, z < 1: 8-point Gauss-Legendre on panels spanning at most one phase cycle
//    (half a cycle in FP64).
// Phases with large arguments are reduced modulo 2 in FP64 before sincospi: E(1) =
// exp(i pi (z + 2 (r - k0))) is the same for every tap (q = j - (r - k0) with j integer), and
// q^2/z is formed in FP64 for the near taps.  Everything else runs in the evaluation type T.
//
// Refinement (k5_refine), from a seed (r, z), with k0 = floor(r + 1/2) of the seed kept for the
// whole ascent so that P is smooth along the path: up to `steps` FP32 steps, then one FP64 step, of
//   d = H^-1 grad P / P,   H^-1 = (1/(2 pi^2)) [[48, -90], [-90, 180]].
// H is the Hessian of 1 - P/P_peak of an ideal chirp at its peak: an offset (dr, dz) leaves a phase
// error 2 pi (dr u + dz u^2/2) over the observation, and 1 - P/P_peak is to second order its
// variance over u in [0, 1], pi^2 (dr^2/3 + dr dz/3 + 4 dz^2/45).  The step is scaled down to
// |dr| <= 1/4, |dz| <= 1, then halved (at most three times) until P does not decrease; when no
// such step exists the ascent stops.
#include <cmath>

#include "fdas_internal.cuh"

namespace fdas {

namespace {

constexpr double PI_D = 3.14159265358979323846;
constexpr int WARPS_PER_BLOCK = 4;

struct GL8 {
    double x[8];
    double w[8];
};

template <typename T>
struct cx {
    T re, im;
};
template <typename T>
__device__ __forceinline__ cx<T> operator+(cx<T> a, cx<T> b) {
    return {a.re + b.re, a.im + b.im};
}
template <typename T>
__device__ __forceinline__ cx<T> operator-(cx<T> a, cx<T> b) {
    return {a.re - b.re, a.im - b.im};
}
template <typename T>
__device__ __forceinline__ cx<T> operator*(cx<T> a, cx<T> b) {
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename T>
__device__ __forceinline__ cx<T> scale(T s, cx<T> a) {
    return {s * a.re, s * a.im};
}
template <typename T>
__device__ __forceinline__ cx<T> conjg(cx<T> a) {
    return {a.re, -a.im};
}
// a * conj(b)
template <typename T>
__device__ __forceinline__ cx<T> mul_conj(cx<T> a, cx<T> b) {
    return {a.re * b.re + a.im * b.im, a.im * b.re - a.re * b.im};
}
// a / (2 pi i) = -i a / (2 pi)
template <typename T>
__device__ __forceinline__ cx<T> over_2pi_i(cx<T> a) {
    const T s = T(1.0 / (2.0 * PI_D));
    return {a.im * s, -a.re * s};
}

// Per-precision choices (series lengths, far-tap threshold, continued-fraction depth, panels).
template <typename T>
struct Arith;
template <>
struct Arith<float> {
    static constexpr float cf_a = 72.f;    // continued-fraction depth floor(cf_a / x^2) + cf_b + 1
    static constexpr int cf_b = 4;
    static constexpr int series_terms = 20;
    static constexpr float far_c = 6.f;
    static constexpr int ibp_terms = 5;
    static constexpr int gl_mult = 1;
    static constexpr float series_max = 1.5f;   // power series for |s| <= series_max
    __device__ static __forceinline__ void scpi(float x, float *s, float *c) { sincospif(x, s, c); }
};
template <>
struct Arith<double> {
    static constexpr double cf_a = 260.0;
    static constexpr int cf_b = 6;
    static constexpr int series_terms = 48;
    static constexpr double far_c = 12.0;
    static constexpr int ibp_terms = 7;
    static constexpr int gl_mult = 2;
    static constexpr double series_max = 2.5;
    __device__ static __forceinline__ void scpi(double x, double *s, double *c) { sincospi(x, s, c); }
};

// exp(i pi x) for an FP64 argument of any size: exact reduction to [-1, 1], then sincospi in T.
template <typename T>
__device__ __forceinline__ cx<T> expipi(double x) {
    const double red = x - 2.0 * rint(0.5 * x);
    T s, c;
    Arith<T>::scpi((T)red, &s, &c);
    return {c, s};
}

// Power-series coefficients of F(s) / s = sum_k x^k / (k! (2k+1)), x = i pi s^2 / 2.
template <int N>
struct SeriesCoef {
    double c[N];
    constexpr SeriesCoef() : c() {
        double f = 1.0;   // k!
        for (int k = 0; k < N; k++) {
            if (k > 0) f *= k;
            c[k] = 1.0 / (f * (2 * k + 1));
        }
    }
};

// F(s) = C(s) + i S(s) as c + d exp(i pi s^2 / 2).
template <typename T>
__device__ void fresnel_end(T s, cx<T> &c, cx<T> &d) {
    const T a = fabs(s);
    if (a <= Arith<T>::series_max) {
        // Horner in the purely imaginary x = i pi s^2/2: S <- S x + c_k
        constexpr int N = Arith<T>::series_terms;
        constexpr SeriesCoef<N> sc;
        const T h = T(PI_D / 2) * s * s;
        cx<T> S = {T(sc.c[N - 1]), T(0)};
#pragma unroll
        for (int k = N - 2; k >= 0; k--) S = {T(sc.c[k]) - S.im * h, S.re * h};
        c = {s * S.re, s * S.im};
        d = {T(0), T(0)};
        return;
    }
    const T sg = s > T(0) ? T(1) : T(-1);
    // K(w) = 1/(w + (1/2)/(w + 1/(w + (3/2)/(w + ...)))), w = (sqrt(pi)/2)(1 - i)|s|, evaluated
    // from a fixed depth upwards (the depth falls as 1/s^2 for a fixed relative accuracy).  The
    // tail t_k = w + a_k / t_{k+1}, a_k = (k-1)/2, is carried as the ratio p/q
    // (p <- w p + a_k q, q <- p), so the only division is the last one.  |p| grows to at most
    // about 1e20 (FP32, |s| just above 1.5) or 1e92 (FP64), inside either format's range.
    const T hw = T(0.88622692545275801365) * a;
    const cx<T> w = {hw, -hw};
    const int depth = (int)(Arith<T>::cf_a / (a * a)) + Arith<T>::cf_b + 1;
    cx<T> p = w, q = {T(1), T(0)};
    for (int k = depth; k >= 2; k--) {
        const T ak = T(0.5) * T(k - 1);
        const cx<T> pn = {w.re * p.re - w.im * p.im + ak * q.re, w.re * p.im + w.im * p.re + ak * q.im};
        q = p;
        p = pn;
    }
    // K = 1 / t_1 = q / p, with both scaled to |p| ~ 1 first so |p|^2 cannot overflow
    const T ps = T(1) / (fabs(p.re) + fabs(p.im));
    p = scale(ps, p);
    q = scale(ps, q);
    const T inv = T(1) / (p.re * p.re + p.im * p.im);
    const cx<T> K = {(q.re * p.re + q.im * p.im) * inv, (q.im * p.re - q.re * p.im) * inv};
    const T nrm = T(0.28209479177387814347);   // 1 / (2 sqrt(pi))
    c = {T(0.5) * sg, T(0.5) * sg};
    d = {-sg * nrm * (K.re - K.im), -sg * nrm * (K.re + K.im)};
}

// What every tap of one evaluation shares (z already folded to z >= 0).
template <typename T>
struct TapCtx {
    double zz;      // |z|
    double dlt;     // q = j - dlt for tap offset j (folded)
    double inv_z;   // 1/zz (zz >= 1)
    T zf;           // zz in T
    T ks;           // sqrt(2/zz)
    T rs2z;         // 1/sqrt(2 zz)
    double dfar;    // far-tap threshold on min |v|
    cx<T> E1;       // E(1) = exp(i pi (zz + 2 dlt)), the same for every tap
};

// Integration-by-parts end term: (m0, m1, m2) at one end u of [0, 1], without the factor E(u).
template <typename T>
__device__ __forceinline__ void ibp_end(T v, T u, T zf, cx<T> &m0, cx<T> &m1, cx<T> &m2) {
    constexpr double c0[7] = {1, 1, 3, 15, 105, 945, 10395};
    constexpr double c1[7] = {1, 3, 15, 105, 945, 10395, 135135};
    constexpr double c2[7] = {1, 6, 45, 420, 4725, 62370, 945945};
    constexpr int n = Arith<T>::ibp_terms;
    const T inv2pi = T(1.0 / (2.0 * PI_D));
    // w = 1/(2 pi i v) = i wi, t = z/(2 pi i v^2) = i tau: both purely imaginary
    const T wi = -inv2pi / v;
    const T tau = -zf * inv2pi / (v * v);
    cx<T> S0 = {T(c0[n - 1]), T(0)}, S1 = {T(c1[n - 1]), T(0)}, S2 = {T(c2[n - 1]), T(0)};
#pragma unroll
    for (int k = n - 2; k >= 0; k--) {   // S = S * (i tau) + c_k
        S0 = {T(c0[k]) - S0.im * tau, S0.re * tau};
        S1 = {T(c1[k]) - S1.im * tau, S1.re * tau};
        S2 = {T(c2[k]) - S2.im * tau, S2.re * tau};
    }
    const cx<T> wS0 = {-wi * S0.im, wi * S0.re};   // w S0
    const T wi2 = wi * wi;                           // -w^2
    const T wi3 = wi2 * wi;                          // w^3 = -i wi^3
    m0 = wS0;
    // u w S0 - w^2 S1 = u w S0 + wi^2 S1
    m1 = {u * wS0.re + wi2 * S1.re, u * wS0.im + wi2 * S1.im};
    // u^2 w S0 - 2 u w^2 S1 + 2 w^3 S2 = u^2 w S0 + 2 u wi^2 S1 - 2 i wi^3 S2
    m2 = {u * u * wS0.re + T(2) * u * wi2 * S1.re + T(2) * wi3 * S2.im,
          u * u * wS0.im + T(2) * u * wi2 * S1.im - T(2) * wi3 * S2.re};
}

template <typename T>
__device__ void tap_moments(const TapCtx<T> &c, int j, const GL8 &gl, cx<T> &M0, cx<T> &M1, cx<T> &M2) {
    const double q = (double)j - c.dlt;
    const T qf = (T)q;
    const double v0 = -q, v1 = c.zz - q;
    const double D = (q >= 0.0 && q <= c.zz) ? 0.0 : fmin(fabs(v0), fabs(v1));
    if (D >= c.dfar) {
        cx<T> a0, a1, a2, b0, b1, b2;
        ibp_end<T>((T)v1, T(1), c.zf, a0, a1, a2);
        ibp_end<T>((T)v0, T(0), c.zf, b0, b1, b2);
        M0 = c.E1 * a0 - b0;
        M1 = c.E1 * a1 - b1;
        M2 = c.E1 * a2 - b2;
        return;
    }
    if (c.zz >= 1.0) {
        const T s0 = -qf * c.ks;
        const T s1 = (c.zf - qf) * c.ks;
        cx<T> c0, d0, c1, d1;
        fresnel_end<T>(s0, c0, d0);
        fresnel_end<T>(s1, c1, d1);
        const cx<T> ph = expipi<T>(-q * q * c.inv_z);
        M0 = scale(c.rs2z, (c1 - c0) * ph + d1 * c.E1 - d0);
        const T iz = (T)c.inv_z;
        const cx<T> one = {T(1), T(0)};
        M1 = scale(iz, over_2pi_i(c.E1 - one) + scale(qf, M0));
        M2 = scale(iz, over_2pi_i(c.E1 - M0) + scale(qf, M1));
        return;
    }
    // |z| < 1, |q| < dfar + 1: panels of at most one (FP64: half a) phase cycle
    const int panels = max(1, (int)ceil(fabs(q) + c.zz)) * Arith<T>::gl_mult;
    const T h = T(1) / T(panels);
    cx<T> a0 = {T(0), T(0)}, a1 = a0, a2 = a0;
    for (int p = 0; p < panels; p++) {
        const T mid = (T(p) + T(0.5)) * h;
#pragma unroll
        for (int g = 0; g < 8; g++) {
            const T u = mid + T(0.5) * h * (T)gl.x[g];
            T s, co;
            Arith<T>::scpi(u * (c.zf * u - T(2) * qf), &s, &co);
            const T wt = T(0.5) * h * (T)gl.w[g];
            const cx<T> e = {wt * co, wt * s};
            a0 = a0 + e;
            a1 = a1 + scale(u, e);
            a2 = a2 + scale(u * u, e);
        }
    }
    M0 = a0;
    M1 = a1;
    M2 = a2;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Points the evaluation accepts (anything else gives NaN): finite, |r| < 2^52, |z| < 2^20 and the
// window no further than 2^24 bins from r.
__device__ __forceinline__ bool point_ok(double r, double z, int64_t k0) {
    return isfinite(r) && isfinite(z) && fabs(r) < 4.5e15 && fabs(z) < 1048576.0 &&
           fabs(r - (double)k0) < 16777216.0;
}

// P, dP/dr, dP/dz at (r, z) with the window anchored at k0 (warp-collective; every lane returns
// the same values).
template <typename T>
__device__ void eval_point(const float2 *__restrict__ xhat, int64_t nb, int m, int64_t k0, double r, double z,
                           const GL8 &gl, T &P, T &dPdr, T &dPdz) {
    const int lane = threadIdx.x & 31;
    const bool neg = z < 0.0;
    TapCtx<T> c;
    c.zz = fabs(z);
    const double dlt = r - (double)k0;
    c.dlt = neg ? -dlt : dlt;
    c.zf = (T)c.zz;
    const bool big = c.zz >= 1.0;
    c.inv_z = big ? 1.0 / c.zz : 0.0;
    c.ks = big ? (T)sqrt(2.0 / c.zz) : T(0);
    c.rs2z = big ? (T)(1.0 / sqrt(2.0 * c.zz)) : T(0);
    c.dfar = (double)Arith<T>::far_c * fmax(1.0, sqrt(c.zz));
    c.E1 = expipi<T>(c.zz + 2.0 * c.dlt);
    cx<T> A = {T(0), T(0)}, Y1 = A, Y2 = A;
    for (int t = lane; t < m; t += 32) {
        const int j = t - m / 2;
        const int64_t k = k0 + j;
        if (k < 0 || k >= nb) continue;
        const float2 xv = __ldg(xhat + k);
        const cx<T> X = {(T)xv.x, (T)xv.y};
        cx<T> M0, M1, M2;
        tap_moments<T>(c, neg ? -j : j, gl, M0, M1, M2);
        if (neg) {
            M0 = conjg(M0);
            M1 = conjg(M1);
            M2 = conjg(M2);
        }
        A = A + mul_conj(X, M0);
        Y1 = Y1 + mul_conj(X, M1);
        Y2 = Y2 + mul_conj(X, M2);
    }
    A.re = warp_sum(A.re);
    A.im = warp_sum(A.im);
    Y1.re = warp_sum(Y1.re);
    Y1.im = warp_sum(Y1.im);
    Y2.re = warp_sum(Y2.re);
    Y2.im = warp_sum(Y2.im);
    // dA/dr = sum X conj(2 pi i M_1) = -2 pi i Y1,  dA/dz = sum X conj(i pi M_2) = -i pi Y2
    const T tp = T(2.0 * PI_D), pi = T(PI_D);
    const cx<T> Ar = {tp * Y1.im, -tp * Y1.re};
    const cx<T> Az = {pi * Y2.im, -pi * Y2.re};
    P = A.re * A.re + A.im * A.im;
    dPdr = T(2) * (A.re * Ar.re + A.im * Ar.im);
    dPdz = T(2) * (A.re * Az.re + A.im * Az.im);
}

template <typename T>
__global__ void __launch_bounds__(32 * WARPS_PER_BLOCK)
    k5_interp(const float2 *__restrict__ xhat, int64_t nb, int m, const fdas_cand *__restrict__ pts,
              const int64_t *__restrict__ k0s, int n, double *__restrict__ out, GL8 gl) {
    const int i = (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 5);
    if (i >= n) return;
    const double r = pts[i].r, z = pts[i].z;
    const int64_t k0 = k0s ? k0s[i] : (isfinite(r) && fabs(r) < 4.5e15 ? (int64_t)floor(r + 0.5) : 0);
    T P = T(NAN), gr = T(NAN), gz = T(NAN);
    if (point_ok(r, z, k0)) eval_point<T>(xhat, nb, m, k0, r, z, gl, P, gr, gz);
    if ((threadIdx.x & 31) == 0) {
        out[3 * (size_t)i + 0] = (double)P;
        out[3 * (size_t)i + 1] = (double)gr;
        out[3 * (size_t)i + 2] = (double)gz;
    }
}

// The preconditioned step (see the header comment); false when there is none.
__device__ __forceinline__ bool ascent_step(double P, double gr, double gz, double &dr, double &dz) {
    if (!(P > 0.0)) return false;
    const double s = 1.0 / (2.0 * PI_D * PI_D * P);
    dr = (48.0 * gr - 90.0 * gz) * s;
    dz = (-90.0 * gr + 180.0 * gz) * s;
    const double sc = fmax(fmax(4.0 * fabs(dr), fabs(dz)), 1.0);
    dr /= sc;
    dz /= sc;
    return isfinite(dr) && isfinite(dz);
}

constexpr int HALVINGS = 4;   // tries per step: d, d/2, d/4, d/8

__global__ void __launch_bounds__(32 * WARPS_PER_BLOCK)
    k5_refine(const float2 *__restrict__ xhat, int64_t nb, int m, const fdas_cand *__restrict__ in, int n,
              int steps, fdas_cand *__restrict__ out, double *__restrict__ pw, int32_t *__restrict__ evals_out,
              GL8 gl) {
    const int c = (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 5);
    if (c >= n) return;
    double r = in[c].r, z = in[c].z;
    const int64_t k0 = (isfinite(r) && fabs(r) < 4.5e15) ? (int64_t)floor(r + 0.5) : 0;
    int evals = 0;
    double Pd = NAN, grd = NAN, gzd = NAN;
    if (point_ok(r, z, k0)) {
        float P, gr, gz;
        eval_point<float>(xhat, nb, m, k0, r, z, gl, P, gr, gz);
        evals++;
        for (int s = 0; s < steps; s++) {
            double dr, dz;
            if (!ascent_step(P, gr, gz, dr, dz)) break;
            bool ok = false;
            float P2, gr2, gz2;
            for (int h = 0; h < HALVINGS; h++) {
                eval_point<float>(xhat, nb, m, k0, r + dr, z + dz, gl, P2, gr2, gz2);
                evals++;
                if (P2 >= P) {
                    ok = true;
                    break;
                }
                dr *= 0.5;
                dz *= 0.5;
            }
            if (!ok) break;
            r += dr;
            z += dz;
            P = P2;
            gr = gr2;
            gz = gz2;
        }
        // the final step in FP64
        eval_point<double>(xhat, nb, m, k0, r, z, gl, Pd, grd, gzd);
        evals++;
        double dr, dz;
        if (ascent_step(Pd, grd, gzd, dr, dz)) {
            for (int h = 0; h < HALVINGS; h++) {
                double P2, gr2, gz2;
                eval_point<double>(xhat, nb, m, k0, r + dr, z + dz, gl, P2, gr2, gz2);
                evals++;
                if (P2 >= Pd) {
                    r += dr;
                    z += dz;
                    Pd = P2;
                    grd = gr2;
                    gzd = gz2;
                    break;
                }
                dr *= 0.5;
                dz *= 0.5;
            }
        }
    }
    if ((threadIdx.x & 31) == 0) {
        out[c].r = r;
        out[c].z = z;
        if (pw) {
            pw[3 * (size_t)c + 0] = Pd;
            pw[3 * (size_t)c + 1] = grd;
            pw[3 * (size_t)c + 2] = gzd;
        }
        if (evals_out) evals_out[c] = evals;
    }
}

GL8 gl8() {
    static GL8 g = [] {
        GL8 t;
        gauss_legendre(8, t.x, t.w);
        return t;
    }();
    return g;
}

unsigned blocks_for(int n) { return (unsigned)((n + WARPS_PER_BLOCK - 1) / WARPS_PER_BLOCK); }

}  // namespace

cudaError_t launch_interp(Plan &p, const float2 *d_x, const fdas_cand *d_pts, const int64_t *d_k0, int n, bool fp64,
                          double *d_out, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const GL8 g = gl8();
    if (fp64)
        k5_interp<double><<<blocks_for(n), 32 * WARPS_PER_BLOCK, 0, st>>>(d_x, p.nb, p.m, d_pts, d_k0, n, d_out, g);
    else
        k5_interp<float><<<blocks_for(n), 32 * WARPS_PER_BLOCK, 0, st>>>(d_x, p.nb, p.m, d_pts, d_k0, n, d_out, g);
    p.prof.launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_refine(Plan &p, const float2 *d_x, const fdas_cand *d_in, int n, int steps, fdas_cand *d_out,
                          double *d_power, int32_t *d_evals, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k5_refine<<<blocks_for(n), 32 * WARPS_PER_BLOCK, 0, st>>>(d_x, p.nb, p.m, d_in, n, steps, d_out, d_power,
                                                              d_evals, gl8());
    p.prof.launches += 1;
    return cudaGetLastError();
}

}  // namespace fdas
