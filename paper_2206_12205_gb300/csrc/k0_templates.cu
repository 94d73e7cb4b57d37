// K0: acceleration template bank (Sec. 2.1 and Sec. 3.3 "Template conversion").
//
// The paper generates its templates once in single precision and converts them to the
// working precision with a GPU kernel.  Here the responses are integrated in FP64 on the
// GPU and rounded once, at the end, to each working precision:
//   1. taps:      I(q, z_i) = int_0^1 exp(i pi (z_i u^2 - 2 q u)) du for q = -m/2..m/2-1,
//                 z_i = -zmax + 2i, by composite 20-point Gauss-Legendre quadrature with
//                 panels no wider than one phase cycle (FP64, exact to rounding);
//   2. normalise: T_i = I(., z_i) / sqrt(eta_i), eta_i = sum_q |I(q, z_i)|^2;
//   3. transform: G_i(k) = (1/S) sum_{d<m} T_i(d - m/2) exp(-2 pi i d k / S), k < S, as a
//                 direct FP64 DFT (m terms per output), stored as FP32 and as BF16 hi/lo.
// With G in hand, the overlap-save correlation of a segment spectrum Yhat is
// conj(FFT(conj(Yhat) * G)) (see the plane kernels), so the inverse FFT becomes a forward one.
#include <cmath>
#include <vector>

#include "fdas_internal.cuh"

namespace fdas {

// Gauss-Legendre nodes and weights on [-1, 1]: Newton iteration on the Legendre polynomial
// P_n from the usual cosine start, weights 2 / ((1 - x^2) P_n'(x)^2).
void gauss_legendre(int n, double *xs, double *ws) {
    for (int i = 0; i < n; i++) {
        double x = std::cos(M_PI * (i + 0.75) / (n + 0.5));
        double dpn = 1.0;
        for (int it = 0; it < 100; it++) {
            double a = 1.0, b = x;
            for (int k = 2; k <= n; k++) {
                double c = ((2 * k - 1) * x * b - (k - 1) * a) / k;
                a = b;
                b = c;
            }
            dpn = n * (x * b - a) / (x * x - 1.0);
            double step = b / dpn;
            x -= step;
            if (std::fabs(step) < 1e-16) break;
        }
        double a = 1.0, b = x;
        for (int k = 2; k <= n; k++) {
            double c = ((2 * k - 1) * x * b - (k - 1) * a) / k;
            a = b;
            b = c;
        }
        dpn = n * (x * b - a) / (x * x - 1.0);
        xs[i] = x;
        ws[i] = 2.0 / ((1.0 - x * x) * dpn * dpn);
    }
}

namespace {

constexpr int GL_N = 20;
struct GaussLegendre {
    double x[GL_N];
    double w[GL_N];
};

GaussLegendre gauss_legendre_nodes() {
    GaussLegendre g;
    gauss_legendre(GL_N, g.x, g.w);
    return g;
}

__global__ void k0_taps(double2 *__restrict__ taps, int K, int m, int zmax, GaussLegendre gl) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= K * m) return;
    const int i = idx / m, t = idx - i * m;
    const double z = -(double)zmax + 2.0 * i;
    const double q = (double)(t - m / 2);
    const int panels = (int)ceil(fabs(z) + fabs(q)) + 4;
    const double h = 1.0 / panels;
    double re = 0.0, im = 0.0;
    for (int p = 0; p < panels; p++) {
        const double mid = (p + 0.5) * h;
#pragma unroll 4
        for (int g = 0; g < GL_N; g++) {
            const double u = fma(0.5 * h, gl.x[g], mid);
            double s, c;
            sincospi(u * (z * u - 2.0 * q), &s, &c);
            const double wt = 0.5 * h * gl.w[g];
            re = fma(wt, c, re);
            im = fma(wt, s, im);
        }
    }
    taps[idx] = make_double2(re, im);
}

// One block per template row: eta = sum |I|^2 (fixed-order tree), then scale to unit norm.
__global__ void k0_normalise(double2 *__restrict__ taps, int m, double *__restrict__ eta_out) {
    __shared__ double red[256];
    double2 *row = taps + (size_t)blockIdx.x * m;
    double acc = 0.0;
    for (int t = threadIdx.x; t < m; t += blockDim.x) acc += row[t].x * row[t].x + row[t].y * row[t].y;
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    const double eta = red[0];
    const double inv = 1.0 / sqrt(eta);
    for (int t = threadIdx.x; t < m; t += blockDim.x) {
        row[t].x *= inv;
        row[t].y *= inv;
    }
    if (threadIdx.x == 0 && eta_out) eta_out[blockIdx.x] = eta;
}

// G_i(k) = (1/S) sum_d T_i(d - m/2) W_S^{d k}: direct FP64 DFT, rounded once to each format.
// The 16-bit banks of the tensor path (S = 4096) are stored in its stage-1 operand order.
__global__ void k0_dft(const double2 *__restrict__ taps, int m, int S, const double2 *__restrict__ wS,
                       float2 *__restrict__ G, __nv_bfloat16 *__restrict__ Gbf, __half *__restrict__ Gh) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y;
    if (k >= S) return;
    const double2 *row = taps + (size_t)i * m;
    double re = 0.0, im = 0.0;
    for (int d = 0; d < m; d++) {
        const double2 tv = row[d];
        const double2 w = wS[((long long)d * k) & (S - 1)];
        re = fma(tv.x, w.x, fma(-tv.y, w.y, re));
        im = fma(tv.x, w.y, fma(tv.y, w.x, im));
    }
    re /= (double)S;
    im /= (double)S;
    const float fr = (float)re, fi = (float)im;
    G[(size_t)i * S + k] = make_float2(fr, fi);
    const size_t pos = (size_t)i * 2 * S + tc_s1_pos(k >> 6, k & 63);
    // FP16 bank of the scaled precision: S G (|S G| <= sqrt(m) for unit-norm taps), rounded once
    if (Gh) {
        Gh[pos] = __float2half_rn((float)(re * S));
        Gh[pos + 2] = __float2half_rn((float)(im * S));
    }
    // BF16 bank: the BF16 rounding of the FP32 value (the paper's conversion)
    if (Gbf) {
        Gbf[pos] = __float2bfloat16_rn(fr);
        Gbf[pos + 2] = __float2bfloat16_rn(fi);
    }
}

// Operand image of the direct path: row p * Kpad + z, K index 2 q + s (tap q, component s of the
// spectrum), entries of conj(T_z(q - m/2)) real-ified so that a row dotted with the spectrum's
// (re, im) pairs gives Re (p = 0) or Im (p = 1) of sum_q Xhat conj(T); rows z >= K are zero.
// Rounded once from FP64 to BF16, stored K-major in core matrices (8 rows x 16 bytes).
__global__ void k0_direct_image(const double2 *__restrict__ taps, int K, int m, int Kpad,
                                __nv_bfloat16 *__restrict__ img) {
    const int N = 2 * Kpad, KD = 2 * m;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)N * KD) return;
    const int row = (int)(idx / KD), k = (int)(idx % KD);
    const int p = row / Kpad, z = row % Kpad, q = k >> 1, sc = k & 1;
    double v = 0.0;
    if (z < K) {
        const double2 t = taps[(size_t)z * m + q];
        v = p == 0 ? (sc == 0 ? t.x : t.y) : (sc == 0 ? -t.y : t.x);
    }
    img[tc_kmajor_elem(N, row, k)] = __double2bfloat16(v);
}

// E4M3 code of v (1 sign, 4 exponent bits with bias 7, 3 mantissa bits; normal 2^-6 .. 448,
// subnormal steps of 2^-9), rounded once from FP64 to nearest with ties to even and saturated at
// +-448 (the FP8 operands of FDAS_FP8_DIRECT).
__device__ uint8_t e4m3_code(double v) {
    const uint8_t sgn = signbit(v) ? 0x80 : 0x00;
    const double a = fabs(v);
    if (a == 0.0) return sgn;
    int E;
    frexp(a, &E);
    int e = max(E - 1, -6);                      // binade of a; the subnormals share 2^-6's step
    double q = rint(ldexp(a, 3 - e));            // a in units of the binade's step 2^(e-3)
    if (q >= 16.0) { q = 8.0; e += 1; }          // rounded up into the next binade
    if (e > 8 || (e == 8 && q > 14.0)) return sgn | 0x7E;     // 448 = 1.75 x 2^8
    if (q < 8.0) return sgn | (uint8_t)q;                      // subnormal: exponent field 0
    return sgn | (uint8_t)(((e + 7) << 3) | ((int)q - 8));
}

// The FP8 direct path's operand image: the rows of k0_direct_image, scaled per template z by the
// power of two sigma_z that brings its largest |Re| or |Im| into [224, 448], rounded to E4M3, in
// groups of 32 templates: group g = z / 32 holds 64 rows (row p 32 + z % 32, p = 0 for the Re
// output, 1 for Im) x 2m bytes, K-major in core matrices of 8 rows x 16 bytes (element (row, k)
// at byte g 128 m + ((k / 16) 8 + row / 8) 128 + (row % 8) 16 + k % 16).  dsig[z] = 1 / sigma_z^2
// undoes the scale on the plane.  One block per padded template.
__global__ void k0_direct_image_f8(const double2 *__restrict__ taps, int K, int m, uint8_t *__restrict__ img,
                                   float *__restrict__ dsig) {
    __shared__ double red[256];
    const int z = blockIdx.x;
    double M = 0.0;
    if (z < K)
        for (int q = threadIdx.x; q < m; q += blockDim.x) {
            const double2 t = taps[(size_t)z * m + q];
            M = fmax(M, fmax(fabs(t.x), fabs(t.y)));
        }
    red[threadIdx.x] = M;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + s]);
        __syncthreads();
    }
    M = red[0];
    double sig = 1.0;
    if (M > 0.0) {
        int E;
        const double f = frexp(M, &E);           // M = f 2^E; 448 = 0.875 x 2^9
        sig = ldexp(1.0, (f <= 0.875 ? 9 : 8) - E);
    }
    if (threadIdx.x == 0) dsig[z] = z < K ? (float)(1.0 / (sig * sig)) : 0.f;
    for (int idx = threadIdx.x; idx < 2 * 2 * m; idx += blockDim.x) {
        const int p = idx / (2 * m), k = idx % (2 * m), q = k >> 1, sc = k & 1;
        double v = 0.0;
        if (z < K) {
            const double2 t = taps[(size_t)z * m + q];
            v = (p == 0 ? (sc == 0 ? t.x : t.y) : (sc == 0 ? -t.y : t.x)) * sig;
        }
        const int row = p * 32 + (z & 31);
        img[(size_t)(z >> 5) * 128 * m + ((size_t)(k >> 4) * 8 + (row >> 3)) * 128 + (row & 7) * 16 + (k & 15)] =
            e4m3_code(v);
    }
}

// exp(-2 pi i j / n) in FP64; f = 2j/n is exact for a power-of-two n and is reduced to
// (-1, 1] before the libm call, so the argument error stays below pi * 2^-53.
double2 host_unit(int64_t j, int64_t n) {
    j %= n;
    double f = 2.0 * (double)j / (double)n;
    if (f > 1.0) f -= 2.0;
    return make_double2(std::cos(M_PI * f), -std::sin(M_PI * f));
}

}  // namespace

cudaError_t launch_make_templates(Plan &p, cudaStream_t st) {
    const int K = p.K, m = p.m, S = p.S;
    cudaError_t e;
    // --- twiddle tables (host FP64 -> FP32) ---
    {
        std::vector<float2> tw(TW_MAX);
        for (int j = 0; j < TW_MAX; j++) {
            double2 w = host_unit(j, TW_MAX);
            tw[j] = make_float2((float)w.x, (float)w.y);
        }
        e = cudaMemcpyAsync(p.d_tw, tw.data(), sizeof(float2) * TW_MAX, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return e;
        const int64_t nlo = (int64_t)1 << TW_LO_BITS;
        const int64_t nhi = std::max<int64_t>(1, p.N >> TW_LO_BITS);
        std::vector<float2> lo(nlo), hi(nhi);
        for (int64_t j = 0; j < nlo; j++) {
            double2 w = host_unit(j % p.N, p.N);
            lo[j] = make_float2((float)w.x, (float)w.y);
        }
        for (int64_t j = 0; j < nhi; j++) {
            double2 w = host_unit((j << TW_LO_BITS) % p.N, p.N);
            hi[j] = make_float2((float)w.x, (float)w.y);
        }
        e = cudaMemcpyAsync(p.d_twn_lo, lo.data(), sizeof(float2) * nlo, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return e;
        e = cudaMemcpyAsync(p.d_twn_hi, hi.data(), sizeof(float2) * nhi, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return e;
        // the host vectors go out of scope: finish the copies first
        e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return e;
    }
    // --- template bank ---
    double2 *d_taps = nullptr, *d_wS = nullptr;
    double *d_eta = nullptr;
    e = cudaMalloc(&d_taps, sizeof(double2) * (size_t)K * m);
    if (e != cudaSuccess) return e;
    e = cudaMalloc(&d_wS, sizeof(double2) * (size_t)S);
    if (e != cudaSuccess) { cudaFree(d_taps); return e; }
    e = cudaMalloc(&d_eta, sizeof(double) * (size_t)K);
    if (e != cudaSuccess) { cudaFree(d_taps); cudaFree(d_wS); return e; }
    {
        std::vector<double2> wS(S);
        for (int j = 0; j < S; j++) wS[j] = host_unit(j, S);
        e = cudaMemcpyAsync(d_wS, wS.data(), sizeof(double2) * S, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    if (e == cudaSuccess) {
        const GaussLegendre gl = gauss_legendre_nodes();
        const int n = K * m;
        k0_taps<<<(n + 127) / 128, 128, 0, st>>>(d_taps, K, m, p.cfg.zmax, gl);
        k0_normalise<<<K, 256, 0, st>>>(d_taps, m, d_eta);
        dim3 grid((S + 255) / 256, K);
        if (p.d_dimg && p.cfg.precision == FDAS_FP8_DIRECT) {
            int groups = 0;
            direct_geometry_f8(p, &groups, nullptr);
            k0_direct_image_f8<<<(unsigned)(32 * groups), 256, 0, st>>>(d_taps, K, m, static_cast<uint8_t *>(p.d_dimg),
                                                                       p.d_dsig);
        } else if (p.d_dimg) {
            int Kpad = 0;
            direct_geometry(p, &Kpad, nullptr, nullptr);
            const int64_t ne = (int64_t)2 * Kpad * 2 * m;
            k0_direct_image<<<(unsigned)((ne + 255) / 256), 256, 0, st>>>(d_taps, K, m, Kpad,
                                                                            static_cast<__nv_bfloat16 *>(p.d_dimg));
        }
        const bool tc = S == TC_S_BF16;
        k0_dft<<<grid, 256, 0, st>>>(d_taps, m, S, d_wS, p.d_G,
                                     tc ? reinterpret_cast<__nv_bfloat16 *>(p.d_Gbf) : nullptr,
                                     tc ? reinterpret_cast<__half *>(p.d_Gh) : nullptr);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    cudaFree(d_taps);
    cudaFree(d_wS);
    cudaFree(d_eta);
    return e;
}

}  // namespace fdas
