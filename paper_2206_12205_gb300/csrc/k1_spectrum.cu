// K1: the long real FFT of one series, kept in FP32 (Sec. 3: it does not scale with the
// number of templates and reduced precision hurts it most), DC zeroed (Sec. 3.2), Nyquist
// dropped, and the noise normalisation sigma2 = mean_{k=1..Nb-1} |X_k|^2.
//
// A real series x[N] is read as the complex series z_n = x_{2n} + i x_{2n+1} of length
// M = N/2 = M1*M2, transformed by a four-step FFT, then split:
//   pass A (one CTA per C1 adjacent columns n2):  FFT_M1 over n1 of z[n1*M2 + n2], times
//                                    W_M^{n2 k1}, stored transposed as B[k1*M2 + n2];
//   pass B (one CTA per C2 rows k1 and their partners M1 - k1):  FFT_M2 over n2 of the row
//                                    B[k1*M2 + n2] gives Z[k1 + M1*k2]; with Z for rows k1 and
//                                    M1-k1 both in shared memory,
//                                    X_k = (Z_k + conj Z_{M-k})/2 - (i/2) W_N^k (Z_k - conj Z_{M-k}),
//                                    k < M, and a per-CTA FP64 partial of sum |X_k|^2;
//   finalize (pass B's last block):  fixed-order sum of the partials -> sigma2, scale.
// The lanes of a warp interleave over the CTA's columns (pass A) or rows (pass B), so every
// global access of a warp covers whole 32-byte sectors instead of strided single elements.
// Twiddles W_N^e come from a two-level FP32 table (W_N^e = hi[e >> 13] * lo[e & 8191]), looked
// up once per thread and once per (column, i) in pass A, once per thread and once per i in pass B
// (the factor W_N^{M1 T i} = W_64^i that steps through a thread's 32 outputs).
// sum |X_k|^2: FP32 over a thread's 32 bins, FP64 from there on (GB300's FP64 rate is low).
#include "block_fft.cuh"
#include "fdas_internal.cuh"

namespace fdas {

namespace {

__device__ __forceinline__ float2 twN(const float2 *__restrict__ lo, const float2 *__restrict__ hi, int64_t e) {
    return cmul(__ldg(hi + (e >> TW_LO_BITS)), __ldg(lo + (e & ((1 << TW_LO_BITS) - 1))));
}

// FFTs of one CTA: groups per CTA (bounded by 1024 threads and the shared memory) and the
// padding between the groups' shared-memory regions.  The G groups interleave in a warp (lane
// l serves group l mod G), so a half-warp's 8-byte accesses cover 16 / G consecutive entries of
// each group: the regions must start 32 / G banks apart, i.e. a region of E entries with
// E = 16 / G (mod 16).
#ifndef FDAS_K1A_GROUPS
#define FDAS_K1A_GROUPS 4                // pass-A columns per CTA for FFT lengths up to 2048
#endif
#ifndef FDAS_K1B_GROUPS
#define FDAS_K1B_GROUPS 2                // pass-B row pairs per CTA for FFT lengths up to 2048
#endif
constexpr int k1_groups_a(int S) { return S >= 8192 ? 1 : (S >= 4096 ? 2 : FDAS_K1A_GROUPS); }
constexpr int k1_groups_b(int S) { return S >= 8192 ? 1 : (S >= 4096 ? 2 : FDAS_K1B_GROUPS); }
constexpr int k1_gpad(int S, int G) { return (16 / G - fft_smem_entries(S) % 16 + 16) % 16; }
constexpr int k1_region(int S, int G) { return fft_smem_entries(S) + k1_gpad(S, G); }
static_assert(2 * k1_region(2048, 4) % 32 == 8 && 2 * k1_region(4096, 2) % 32 == 16 && 2 * k1_region(256, 4) % 32 == 8,
              "group regions 32 / G banks apart");
#ifndef FDAS_K1A_MIN_BLOCKS
#define FDAS_K1A_MIN_BLOCKS 1            // resident pass-A blocks per SM the registers must allow
#endif
#ifndef FDAS_K1B_MIN_BLOCKS
#define FDAS_K1B_MIN_BLOCKS 2            // resident pass-B blocks per SM the registers must allow
#endif


template <int M1>
__global__ void __launch_bounds__(k1_groups_a(M1) * (M1 / 32), FDAS_K1A_MIN_BLOCKS) k1_pass_a(const float2 *__restrict__ z,
                                                                     const float2 *__restrict__ tw,
                                                                     const float2 *__restrict__ lo,
                                                                     const float2 *__restrict__ hi,
                                                                     float2 *__restrict__ B, int M2,
                                                                     unsigned int *__restrict__ ticket,
                                                                     uint32_t *__restrict__ list_hdr) {
    constexpr int T = M1 / 32, C1 = k1_groups_a(M1);
    constexpr int E = k1_region(M1, C1);
    extern __shared__ float2 sm[];        // C1 * E entries
    __shared__ float2 wi[C1][33];         // W_N^{2 n2 T i} of each column (rows padded: the groups of a
                                          // warp read one entry each, on different banks)
    const int g = threadIdx.x % C1, t = threadIdx.x / C1;
    const int n2 = blockIdx.x * C1 + g;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *ticket = 0;                      // pass B's block count, read after this kernel
        list_hdr[0] = list_hdr[1] = 0;    // the peak search's list counters, for the same step
    }
    for (int i = t; i < 32; i += T) wi[g][i] = twN(lo, hi, 2 * (int64_t)n2 * T * i);   // T < 32 for M1 < 1024
    float2 v[32];
#pragma unroll
    for (int i = 0; i < 32; i++) v[i] = __ldg(z + (int64_t)(t + i * T) * M2 + n2);
    const float2 wt = twN(lo, hi, 2 * (int64_t)n2 * t);
    block_fft<M1>(v, sm + g * E, tw, t);
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 32; i++) {
        const int k1 = t + i * T;
        // W_M^{n2 k1} = W_N^{2 n2 k1} = W_N^{2 n2 t} W_N^{2 n2 T i}
        B[(int64_t)k1 * M2 + n2] = cmul(v[i], cmul(wt, wi[g][i]));
    }
}

// The block's sum of |X_k|^2 (acc: this thread's FP32 partial) to partial[blockIdx.x] in FP64;
// the last block to finish sums the partials in a fixed order: sigma2 = sum / (Nb - 1) unless
// fixed, scale = sqrt(2 / sigma2); a series with no power outside DC (sigma2 = 0) gets scale 0,
// a zero spectrum and plane, as the local variant does for a block of median power 0.
// NT = blockDim.x (a power of two); red: NT doubles of shared memory.
template <int NT>
__device__ __forceinline__ void k1_sum_and_finalize(float acc, double *red, double *__restrict__ partial,
                                                    unsigned int *__restrict__ ticket, int64_t nb, double sigma2_fixed,
                                                    double *__restrict__ sigma2_out, float *__restrict__ scale_out) {
    red[threadIdx.x] = (double)acc;
    __syncthreads();
    for (int s = NT / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    __shared__ bool last;
    if (threadIdx.x == 0) {
        partial[blockIdx.x] = red[0];
        __threadfence();
        last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;                    // block-uniform
    __threadfence();
    double tot = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += NT) tot += __ldcg(partial + i);
    red[threadIdx.x] = tot;
    __syncthreads();
    for (int s = NT / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double sigma2 = sigma2_fixed > 0.0 ? sigma2_fixed : red[0] / (double)(nb - 1);
        *sigma2_out = sigma2;
        *scale_out = sigma2 > 0.0 ? (float)sqrt(2.0 / sigma2) : 0.f;
    }
}

// Groups 0 .. C2-1 take rows a = p C2 + g; groups C2 .. 2 C2 - 1 their partners M1 - a (row 0,
// its own partner, lends its partner slot to row M1/2, the other self-partnered row).
template <int M2>
__global__ void __launch_bounds__(2 * k1_groups_b(M2) * (M2 / 32), FDAS_K1B_MIN_BLOCKS) k1_pass_b(const float2 *__restrict__ B,
                                                                         const float2 *__restrict__ tw,
                                                                         const float2 *__restrict__ lo,
                                                                         const float2 *__restrict__ hi,
                                                                         float2 *__restrict__ X,
                                                                         double *__restrict__ partial, int M1,
                                                                         unsigned int *__restrict__ ticket, int64_t nb,
                                                                         double sigma2_fixed, double *__restrict__ sigma2_out,
                                                                         float *__restrict__ scale_out) {
    constexpr int T = M2 / 32, C2 = k1_groups_b(M2), G = 2 * C2;
    constexpr int E = k1_region(M2, G);
    extern __shared__ float2 smb[];       // G * E entries
    __shared__ double red[G * T];
    const int g = threadIdx.x % G, t = threadIdx.x / G;
    const int a = blockIdx.x * C2 + (g % C2);
    const int row = g < C2 ? a : (a == 0 ? M1 / 2 : M1 - a);
    float2 *sm = smb + g * E;
    __shared__ float2 w64[32];            // W_N^{M1 T i} = W_64^i
    for (int i = threadIdx.x; i < 32; i += G * T) w64[i] = twN(lo, hi, (int64_t)M1 * T * i);
    float2 v[32];
#pragma unroll
    for (int i = 0; i < 32; i++) v[i] = __ldg(B + (int64_t)row * M2 + t + i * T);
    block_fft<M2>(v, sm, tw, t);
    // the last FFT stage works in registers and the previous exchange ended with a barrier
#pragma unroll
    for (int i = 0; i < 32; i++) sm[fft_pad(t + i * T)] = v[i];
    __syncthreads();
    // partner of k = row + M1 k2 is M - k = pr + M1 k2' (rows 0 and M1/2 pair with themselves)
    const bool self = (row == 0) || (row == M1 / 2);
    const int gp = self ? g : (g < C2 ? g + C2 : g - C2);
    const float2 *smp = smb + gp * E;
    const float2 wt = twN(lo, hi, row + (int64_t)M1 * t);   // W_N^k = W_N^{row + M1 t} W_64^i
    float acc = 0.f;
#pragma unroll
    for (int i = 0; i < 32; i++) {
        const int k2 = t + i * T;
        const int k2p = (row == 0) ? ((M2 - k2) & (M2 - 1)) : (M2 - 1 - k2);
        const float2 zk = v[i];
        const float2 zc = smp[fft_pad(k2p)];
        // E = (Z_k + conj Z_{M-k})/2, O = (Z_k - conj Z_{M-k})/(2i)
        const float2 ev = make_float2(0.5f * (zk.x + zc.x), 0.5f * (zk.y - zc.y));
        const float2 dv = make_float2(0.5f * (zk.x - zc.x), 0.5f * (zk.y + zc.y));
        const float2 ov = make_float2(dv.y, -dv.x);
        const int64_t k = row + (int64_t)M1 * k2;
        float2 xk = cadd(ev, cmul(cmul(wt, w64[i]), ov));
        if (k == 0) xk = make_float2(0.f, 0.f);
        X[k] = xk;
        acc = fmaf(xk.x, xk.x, fmaf(xk.y, xk.y, acc));
    }
    k1_sum_and_finalize<G * T>(acc, red, partial, ticket, nb, sigma2_fixed, sigma2_out, scale_out);
}

__global__ void k1_apply_scale(const float2 *__restrict__ X, const float *__restrict__ scale, float2 *__restrict__ out,
                               int64_t nb) {
    const float s = *scale;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nb; k += (int64_t)gridDim.x * blockDim.x) {
        const float2 v = X[k];
        out[k] = make_float2(v.x * s, v.y * s);
    }
}

// Robust local normalisation: the bins of block b = [b B, b B + B) scaled by
// sqrt(2 ln 2 / med_b), med_b = the lower median (rank floor((n - 1) / 2) in ascending order) of
// |X_k|^2 over the block's n bins with k >= 1.  For noise |X_k|^2 is exponential, whose median is
// its mean times ln 2, so the normalised noise power has mean 2 in every block; a median is not
// moved by the few bins a signal occupies.  One CTA per block: the powers are sorted in shared
// memory (bitonic, the excluded DC bin as +inf) and the rank picked exactly.
__global__ void __launch_bounds__(256) k1_local_norm(const float2 *__restrict__ X, float2 *__restrict__ out, int B) {
    extern __shared__ float pw[];
    const int64_t k0 = (int64_t)blockIdx.x * B;
    for (int i = threadIdx.x; i < B; i += 256) {
        const float2 v = X[k0 + i];
        pw[i] = (k0 + i == 0) ? INFINITY : v.x * v.x + v.y * v.y;
    }
    __syncthreads();
    for (int size = 2; size <= B; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = threadIdx.x; i < B / 2; i += 256) {
                const int lo = 2 * i - (i & (stride - 1));          // first of the pair
                const int hi = lo + stride;
                const bool up = (lo & size) == 0;
                const float a = pw[lo], b = pw[hi];
                if ((a > b) == up) {
                    pw[lo] = b;
                    pw[hi] = a;
                }
            }
            __syncthreads();
        }
    }
    const int n = (k0 == 0) ? B - 1 : B;
    const float med = pw[(n - 1) / 2];
    const float s = med > 0.f ? sqrtf(2.0f * 0.69314718f / med) : 0.f;
    for (int i = threadIdx.x; i < B; i += 256) {
        const float2 v = X[k0 + i];
        out[k0 + i] = make_float2(v.x * s, v.y * s);
    }
}

template <int M1>
cudaError_t run_pass_a(const Plan &p, const float2 *z, float2 *B, unsigned int *ticket, uint32_t *list_hdr,
                       cudaStream_t st) {
    constexpr int C1 = k1_groups_a(M1);
    const size_t smem = sizeof(float2) * C1 * k1_region(M1, C1);
    auto kern = k1_pass_a<M1>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<p.M2 / C1, C1 * (M1 / 32), smem, st>>>(z, p.d_tw, p.d_twn_lo, p.d_twn_hi, B, p.M2, ticket, list_hdr);
    return cudaGetLastError();
}

template <int M2>
cudaError_t run_pass_b(const Plan &p, const float2 *B, float2 *X, double *partial, unsigned int *ticket,
                       double *sigma2, float *scale, cudaStream_t st) {
    constexpr int C2 = k1_groups_b(M2);
    const size_t smem = 2 * C2 * sizeof(float2) * k1_region(M2, 2 * C2);
    auto kern = k1_pass_b<M2>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<p.M1 / (2 * C2), 2 * C2 * (M2 / 32), smem, st>>>(B, p.d_tw, p.d_twn_lo, p.d_twn_hi, X, partial, p.M1,
                                                              ticket, p.nb, p.cfg.sigma2, sigma2, scale);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_spectrum(const Plan &p, const float *d_series, char *ws, cudaStream_t st) {
    const float2 *z = reinterpret_cast<const float2 *>(d_series);
    float2 *B = reinterpret_cast<float2 *>(ws + p.ws_tmp);
    float2 *X = reinterpret_cast<float2 *>(ws + p.ws_x);
    double *partial = reinterpret_cast<double *>(ws + p.ws_part);
    double *sigma2 = reinterpret_cast<double *>(ws + p.ws_scale);
    float *scale = reinterpret_cast<float *>(ws + p.ws_scale + 8);
    unsigned int *ticket = reinterpret_cast<unsigned int *>(ws + p.ws_scale + 12);
    uint32_t *list_hdr = reinterpret_cast<uint32_t *>(ws + p.ws_ucount) - PEAK_LIST_WORDS;
    p.prof.begin(FDAS_STAGE_SPECTRUM, st);
    p.prof.launches += 2;
    cudaError_t e = cudaErrorInvalidValue;
    switch (p.M1) {
        case 32: e = run_pass_a<32>(p, z, B, ticket, list_hdr, st); break;
        case 64: e = run_pass_a<64>(p, z, B, ticket, list_hdr, st); break;
        case 128: e = run_pass_a<128>(p, z, B, ticket, list_hdr, st); break;
        case 256: e = run_pass_a<256>(p, z, B, ticket, list_hdr, st); break;
        case 512: e = run_pass_a<512>(p, z, B, ticket, list_hdr, st); break;
        case 1024: e = run_pass_a<1024>(p, z, B, ticket, list_hdr, st); break;
        case 2048: e = run_pass_a<2048>(p, z, B, ticket, list_hdr, st); break;
        case 4096: e = run_pass_a<4096>(p, z, B, ticket, list_hdr, st); break;
        case 8192: e = run_pass_a<8192>(p, z, B, ticket, list_hdr, st); break;
    }
    if (e != cudaSuccess) return e;
    e = cudaErrorInvalidValue;
    switch (p.M2) {
        case 32: e = run_pass_b<32>(p, B, X, partial, ticket, sigma2, scale, st); break;
        case 64: e = run_pass_b<64>(p, B, X, partial, ticket, sigma2, scale, st); break;
        case 128: e = run_pass_b<128>(p, B, X, partial, ticket, sigma2, scale, st); break;
        case 256: e = run_pass_b<256>(p, B, X, partial, ticket, sigma2, scale, st); break;
        case 512: e = run_pass_b<512>(p, B, X, partial, ticket, sigma2, scale, st); break;
        case 1024: e = run_pass_b<1024>(p, B, X, partial, ticket, sigma2, scale, st); break;
        case 2048: e = run_pass_b<2048>(p, B, X, partial, ticket, sigma2, scale, st); break;
        case 4096: e = run_pass_b<4096>(p, B, X, partial, ticket, sigma2, scale, st); break;
        case 8192: e = run_pass_b<8192>(p, B, X, partial, ticket, sigma2, scale, st); break;
    }
    if (e != cudaSuccess) return e;
    p.prof.end(FDAS_STAGE_SPECTRUM, st);
    return cudaGetLastError();
}

cudaError_t launch_local_norm(const Plan &p, const float2 *d_x, float2 *d_out, cudaStream_t st) {
    const int B = p.cfg.norm_block;
    if (B <= 0 || p.nb % B != 0) return cudaErrorInvalidValue;
    if (B * sizeof(float) > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k1_local_norm, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)(B * sizeof(float)));
        if (e != cudaSuccess) return e;
    }
    k1_local_norm<<<(unsigned)(p.nb / B), 256, B * sizeof(float), st>>>(d_x, d_out, B);
    p.prof.launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_apply_scale(const Plan &p, const char *ws, float *d_xhat, double *d_sigma2, cudaStream_t st) {
    const float2 *X = reinterpret_cast<const float2 *>(ws + p.ws_x);
    const float *scale = reinterpret_cast<const float *>(ws + p.ws_scale + 8);
    const double *sigma2 = reinterpret_cast<const double *>(ws + p.ws_scale);
    const int64_t blocks = std::min<int64_t>((p.nb + 255) / 256, 152 * 16);
    k1_apply_scale<<<(int)blocks, 256, 0, st>>>(X, scale, reinterpret_cast<float2 *>(d_xhat), p.nb);
    p.prof.launches += 1;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && d_sigma2)
        e = cudaMemcpyAsync(d_sigma2, sigma2, sizeof(double), cudaMemcpyDeviceToDevice, st);
    return e;
}

}  // namespace fdas
