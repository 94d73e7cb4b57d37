// Block-wide FP32 complex FFT in registers + shared memory (CUDA cores).
//
// One FFT of length S (32 <= S <= 8192, power of two) is carried by T = S/32 threads, each
// holding 32 points in registers.  Layout contract, for thread t of the group:
//     on entry  v[i] = x[t + i*T]        on exit  v[i] = X[t + i*T],   i < 32,
// with X_k = sum_n x_n exp(-2 pi i n k / S) (forward, unscaled).  Loads and stores at
// t + i*T are coalesced for every i, so callers fuse their own prologue (windowing,
// complex multiply) and epilogue (|.|^2, overlap discard) into the global accesses.
//
// Algorithm: Stockham autosort, decimation in time.  Stage s has radix R_s (a first
// radix-32 stage, then two stages splitting the rest), Ns = prod of earlier radices:
//   for each butterfly j < S/R:  u_r = x[j + r S/R] * W_S^{(j mod Ns) r S/(Ns R)},
//   u = DFT_R(u),  y[(j/Ns) Ns R + (j mod Ns) + r Ns] = u_r.
// Each thread runs 32/R_s butterflies per stage (j = t + b*T), which keeps the
// "x[t + i*T] in register i" pattern at every stage boundary; the exchange between
// stages goes through shared memory with one pad word per 32 entries (bank spread).
// The last stage writes its result back to registers only.
//
// Twiddles come from one table of W_8192^j (FP32 values of FP64 cosines), read through
// the read-only cache; the in-register DFT_R uses compile-time constants.
#pragma once

#include <cuda_runtime.h>
#include "fdas_internal.cuh"

namespace fdas {

// ---- compile-time trigonometry for the small-radix constants ------------------------
constexpr double kPi = 3.141592653589793238462643383279502884;

// sin / cos by Taylor series after reduction to [-pi, pi]; 40 terms leave < 1e-28.
constexpr double ct_sin(double x) {
    double term = x, sum = x;
    for (int n = 1; n < 40; n++) {
        term *= -x * x / ((2.0 * n) * (2.0 * n + 1.0));
        sum += term;
    }
    return sum;
}
constexpr double ct_cos(double x) {
    double term = 1.0, sum = 1.0;
    for (int n = 1; n < 40; n++) {
        term *= -x * x / ((2.0 * n - 1.0) * (2.0 * n));
        sum += term;
    }
    return sum;
}
// exp(-2 pi i k / R), angle reduced to [-pi, pi]
template <int k, int R>
struct Wc {
    static constexpr int kk = ((k % R) + R) % R;
    static constexpr double ang = -2.0 * kPi * (double)(2 * kk > R ? kk - R : kk) / (double)R;
    static constexpr float re = (float)ct_cos(ang);
    static constexpr float im = (float)ct_sin(ang);
};

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// conj(a) * b
__device__ __forceinline__ float2 cmul_conj_a(float2 a, float2 b) {
    return make_float2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}

// v * W_R^k with the trivial angles spelled out (no multiply by 0 or 1).
template <int k, int R>
__device__ __forceinline__ float2 tw_mul(float2 v) {
    constexpr float h = 0.70710678118654752440f;
    if constexpr (k == 0) {
        return v;
    } else if constexpr (4 * k == R) {            // -i
        return make_float2(v.y, -v.x);
    } else if constexpr (8 * k == R) {            // (1 - i)/sqrt(2)
        return make_float2((v.x + v.y) * h, (v.y - v.x) * h);
    } else if constexpr (8 * k == 3 * R) {        // (-1 - i)/sqrt(2)
        return make_float2((v.y - v.x) * h, -(v.x + v.y) * h);
    } else {
        return make_float2(v.x * Wc<k, R>::re - v.y * Wc<k, R>::im,
                           v.x * Wc<k, R>::im + v.y * Wc<k, R>::re);
    }
}

// In-register DFT of length R (natural order in and out), recursive radix-2 DIT.
template <int R>
struct Dft;

template <int R, int k>
__device__ __forceinline__ void dft_combine(float2 *u, const float2 *e, const float2 *o) {
    float2 t = tw_mul<k, R>(o[k]);
    u[k] = cadd(e[k], t);
    u[k + R / 2] = csub(e[k], t);
    if constexpr (k + 1 < R / 2) dft_combine<R, k + 1>(u, e, o);
}

template <int R>
struct Dft {
    __device__ __forceinline__ static void run(float2 *u) {
        float2 e[R / 2], o[R / 2];
#pragma unroll
        for (int k = 0; k < R / 2; k++) {
            e[k] = u[2 * k];
            o[k] = u[2 * k + 1];
        }
        Dft<R / 2>::run(e);
        Dft<R / 2>::run(o);
        dft_combine<R, 0>(u, e, o);
    }
};
template <>
struct Dft<1> {
    __device__ __forceinline__ static void run(float2 *) {}
};
template <>
struct Dft<2> {
    __device__ __forceinline__ static void run(float2 *u) {
        float2 a = u[0], b = u[1];
        u[0] = cadd(a, b);
        u[1] = csub(a, b);
    }
};

// ---- radix plan --------------------------------------------------------------------
constexpr int ct_log2(int n) { return n <= 1 ? 0 : 1 + ct_log2(n / 2); }
constexpr int fft_nstages(int S) {
    return ct_log2(S) <= 5 ? 1 : (ct_log2(S) <= 10 ? 2 : 3);
}
constexpr int fft_radix(int S, int s) {
    return s == 0 ? 32
         : (ct_log2(S) <= 10 ? (1 << (ct_log2(S) - 5))
         : (s == 1 ? (1 << ((ct_log2(S) - 4) / 2)) : (1 << ((ct_log2(S) - 5) / 2))));
}
// padded shared-memory entries for one length-S exchange buffer
constexpr int fft_smem_entries(int S) { return S + S / 32; }
__device__ __forceinline__ int fft_pad(int idx) { return idx + (idx >> 5); }

template <int S, int stage, int Ns>
__device__ __forceinline__ void fft_stage(float2 (&v)[32], float2 *sm, const float2 *__restrict__ tw,
                                          int t) {
    constexpr int P = 32, T = S / P;
    constexpr int R = fft_radix(S, stage);
    constexpr int NB = P / R;
    constexpr bool last = (stage + 1 == fft_nstages(S));
    static_assert(R >= 2 && R <= 32 && P % R == 0, "bad radix");
#pragma unroll
    for (int b = 0; b < NB; b++) {
        const int j = t + b * T;
        float2 u[R];
#pragma unroll
        for (int r = 0; r < R; r++) u[r] = v[b + r * NB];
        if constexpr (Ns > 1) {
            const int k = j & (Ns - 1);
#pragma unroll
            for (int r = 1; r < R; r++) {
                const int e = k * r * (S / (Ns * R));          // < S
                u[r] = cmul(u[r], __ldg(tw + e * (TW_MAX / S)));
            }
        }
        Dft<R>::run(u);
        if constexpr (last) {
#pragma unroll
            for (int r = 0; r < R; r++) v[b + r * NB] = u[r];
        } else {
            const int idxD = (j / Ns) * Ns * R + (j & (Ns - 1));
#pragma unroll
            for (int r = 0; r < R; r++) sm[fft_pad(idxD + r * Ns)] = u[r];
        }
    }
    if constexpr (!last) {
        __syncthreads();
#pragma unroll
        for (int i = 0; i < P; i++) v[i] = sm[fft_pad(t + i * T)];
        __syncthreads();
        fft_stage<S, stage + 1, Ns * R>(v, sm, tw, t);
    }
}

// Forward FFT of length S; every thread of the CTA must call it (it synchronises the CTA).
template <int S>
__device__ __forceinline__ void block_fft(float2 (&v)[32], float2 *sm, const float2 *__restrict__ tw,
                                          int t) {
    fft_stage<S, 0, 1>(v, sm, tw, t);
}

}  // namespace fdas
