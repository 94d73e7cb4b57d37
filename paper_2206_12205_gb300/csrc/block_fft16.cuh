// Block-wide FP32 complex FFT with 16 points per thread (CUDA cores), for the FP32 plane path.
//
// One FFT of length S (1024 .. 8192) is carried by T = S/16 threads, each holding 16 points in
// registers.  Layout contract, for thread t:
//     on entry  v[i] = x[t + i*T]        on exit  v[i] = X[t + i*T],   i < 16,
// X_k = sum_n x_n exp(-2 pi i n k / S) (forward, unscaled), so callers fuse their prologue and
// epilogue into coalesced global accesses at t + i*T.
//
// Algorithm: Stockham autosort, decimation in time, radices of at most 16 so that every stage
// fits the 16 registers of a thread (S = 1024: 16.8.8, 2048: 16.16.8, 4096: 16.16.16,
// 8192: 16.16.16.2).  Stage s has radix R and Ns = product of the earlier radices; each thread
// runs 16/R butterflies j = t + b*T:
//     u_r = x[j + r S/R] * W_{Ns R}^{(j mod Ns) r},  u = DFT_R(u),
//     y[(j / Ns) Ns R + (j mod Ns) + r Ns] = u_r.
// Between stages the points go through shared memory (one pad entry per 16, which keeps the
// stride-16 writes of the first stage and the unit-stride reads free of bank conflicts).
// The stage twiddles W_{Ns R}^{k r} are read from a per-CTA shared-memory table laid out
// [stage][r - 1][k] (consecutive lanes read consecutive k), filled once per CTA from the
// plan's FP32 table of W_8192^e (FP32 roundings of FP64 cosines).  The small DFT_R uses
// compile-time constants (block_fft.cuh).
//
// Compared with the 32-point-per-thread form of block_fft.cuh, the register footprint of a
// thread halves (radix-16 butterflies instead of radix-32, no per-butterfly global twiddle
// loads), so several CTAs share an SM and their barriers and loads overlap.
#pragma once

#include <cuda_runtime.h>
#include "block_fft.cuh"

namespace fdas {

constexpr int f16_nstages(int S) { return S == 8192 ? 4 : 3; }
constexpr int f16_radix(int S, int s) {
    return s == 0 ? 16
         : S == 1024 ? 8
         : S == 2048 ? (s == 1 ? 16 : 8)
         : S == 4096 ? 16
                     : (s < 3 ? 16 : 2);
}
constexpr int f16_ns(int S, int s) { return s == 0 ? 1 : f16_ns(S, s - 1) * f16_radix(S, s - 1); }
// offset (entries) of stage s's twiddle table; stage 0 needs none
constexpr int f16_tw_off(int S, int s) {
    return s <= 1 ? 0 : f16_tw_off(S, s - 1) + (f16_radix(S, s - 1) - 1) * f16_ns(S, s - 1);
}
constexpr int f16_tw_entries(int S) { return f16_tw_off(S, f16_nstages(S)); }
constexpr int f16_xchg_entries(int S) { return S + S / 16; }
__device__ __forceinline__ int f16_pad(int i) { return i + (i >> 4); }

// Fill the shared twiddle table (every thread of the CTA calls it; the first exchange barrier of
// the FFT orders these writes before the first table read).
template <int S, int s = 1>
__device__ __forceinline__ void f16_load_twiddles(float2 *tws, const float2 *__restrict__ tw8192, int t) {
    if constexpr (s < f16_nstages(S)) {
        constexpr int T = S / 16, R = f16_radix(S, s), Ns = f16_ns(S, s);
        constexpr int n = (R - 1) * Ns, step = TW_MAX / (Ns * R);
        for (int e = t; e < n; e += T) {
            const int r = e / Ns + 1, k = e - (r - 1) * Ns;
            tws[f16_tw_off(S, s) + e] = __ldg(tw8192 + ((k * r * step) & (TW_MAX - 1)));
        }
        f16_load_twiddles<S, s + 1>(tws, tw8192, t);
    }
}

// One Stockham stage and the rest of the transform.  xa / xb: exchange buffers used by even /
// odd exchanges (the same buffer when DB is false, then each exchange is fenced on both sides).
template <int S, int s, bool DB>
__device__ __forceinline__ void f16_stage(float2 (&v)[16], float2 *xa, float2 *xb, const float2 *tws, int t) {
    constexpr int T = S / 16;
    constexpr int R = f16_radix(S, s);
    constexpr int NB = 16 / R;
    constexpr int Ns = f16_ns(S, s);
    constexpr bool last = (s + 1 == f16_nstages(S));
    float2 *xs = (s & 1) ? xb : xa;
#pragma unroll
    for (int b = 0; b < NB; b++) {
        const int j = t + b * T;
        float2 u[R];
#pragma unroll
        for (int r = 0; r < R; r++) u[r] = v[b + r * NB];
        if constexpr (Ns > 1) {
            const int k = j & (Ns - 1);
#pragma unroll
            for (int r = 1; r < R; r++) u[r] = cmul(u[r], tws[f16_tw_off(S, s) + (r - 1) * Ns + k]);
        }
        Dft<R>::run(u);
        if constexpr (last) {
#pragma unroll
            for (int r = 0; r < R; r++) v[b + r * NB] = u[r];
        } else {
            const int d = (j / Ns) * Ns * R + (j & (Ns - 1));
#pragma unroll
            for (int r = 0; r < R; r++) xs[f16_pad(d + r * Ns)] = u[r];
        }
    }
    if constexpr (!last) {
        __syncthreads();
#pragma unroll
        for (int i = 0; i < 16; i++) v[i] = xs[f16_pad(t + i * T)];
        if constexpr (!DB) __syncthreads();
        f16_stage<S, s + 1, DB>(v, xa, xb, tws, t);
    }
}

// Forward FFT of length S on T = S/16 threads; every thread of the CTA calls it.  With DB the
// two exchange buffers alternate, which needs an even number of exchanges per transform so that
// the next transform's first exchange writes the buffer every thread has finished reading.
template <int S, bool DB>
__device__ __forceinline__ void block_fft16(float2 (&v)[16], float2 *xa, float2 *xb, const float2 *tws, int t) {
    static_assert(!DB || (f16_nstages(S) - 1) % 2 == 0, "alternating buffers need an even exchange count");
    f16_stage<S, 0, DB>(v, xa, xb, tws, t);
}

}  // namespace fdas
