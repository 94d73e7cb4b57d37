// K2 + K3, FP32 path: the overlap-save correlation that produces the f-z plane
// (Sec. 2.1 and Fig. fdas_flow, the "blue box" the paper times).
//
// Segment j covers spectrum bins [jL - m/2, jL - m/2 + S), L <= S - m + 1 (here S - m + 1 rounded
// down to a multiple of 32), zero outside [0, Nb).  With Yhat_j its length-S DFT and G_z the
// template DFT (K0), the circular correlation of the window with template z at offset t < L is
//     W_{j,z}(t) = sum_{d<m} Y_j(t + d) conj(T_z(d - m/2)) = conj( FFT_S(conj(Yhat_j) * G_z) )(t),
// free of wrap-around for t < L, so P[z][jL + t] = |FFT_S(conj(Yhat_j) * G_z)(t)|^2.
//
//   K2 (CTAs striding over the segments): window load (scaled by sqrt(2/sigma2) when the spectrum
//       is unnormalised), forward FFT, Yhat stored [n_seg][S].
//   K3 (one CTA per segment and run of templates): complex multiply fused into the FFT's
//       coalesced loads, forward FFT, |.|^2 and overlap discard fused into its coalesced
//       stores: the plane is written exactly once and nothing else touches HBM in bulk.  Inside
//       a search it also marks the 512-bin units holding a power above the level-1 threshold
//       (the level-1 pass of the peak search then visits only those).
// Both run the 16-point-per-thread block FFT of block_fft16.cuh (T = S/16 threads per transform).
#include "block_fft16.cuh"
#include "fdas_internal.cuh"

#include <algorithm>

namespace fdas {

namespace {

// Shared memory of one CTA: the stage twiddle table, then one or two exchange buffers.
template <int S>
constexpr size_t f16_smem(bool db) {
    return sizeof(float2) * (size_t)(f16_tw_entries(S) + (db ? 2 : 1) * f16_xchg_entries(S));
}

// K2: the segment spectra.  Each CTA transforms segments j = blockIdx.x, blockIdx.x + gridDim.x, ...
// (the shared twiddle table is filled once per CTA).
template <int S>
__global__ void __launch_bounds__(S / 16) k2_segments(const float2 *__restrict__ X, const float *__restrict__ scale_ptr,
                                                      const float2 *__restrict__ tw, float2 *__restrict__ Y,
                                                      int64_t n_seg, int64_t nb, int L, int half_m) {
    constexpr int T = S / 16;
    extern __shared__ float2 sm[];
    float2 *tws = sm;
    float2 *xs = sm + f16_tw_entries(S);
    const int t = threadIdx.x;
    f16_load_twiddles<S>(tws, tw, t);
    const float scale = scale_ptr ? __ldg(scale_ptr) : 1.0f;
    for (int64_t j = blockIdx.x; j < n_seg; j += gridDim.x) {
        const int64_t base = j * L - half_m;
        float2 v[16];
#pragma unroll
        for (int i = 0; i < 16; i++) {
            const int64_t k = base + t + i * T;
            float2 x = make_float2(0.f, 0.f);
            if (k >= 0 && k < nb) x = __ldg(X + k);
            v[i] = make_float2(x.x * scale, x.y * scale);
        }
        block_fft16<S, false>(v, xs, xs, tws, t);
        float2 *out = Y + j * S;
#pragma unroll
        for (int i = 0; i < 16; i++) out[t + i * T] = v[i];
    }
}

// K3: CTA (j, g) correlates segment j with templates [g K / G, (g + 1) K / G), G = groups.
// PRE: the segment spectrum stays in registers and the next template's spectrum is loaded while
// the current transform runs (its L2 latency is then hidden behind the FFT).
template <int S, bool DB, int MINB, bool PRE>
__global__ void __launch_bounds__(S / 16, MINB) k3_plane_fp32(const float2 *__restrict__ Y, const float2 *__restrict__ G,
                                                             const float2 *__restrict__ tw, float *__restrict__ plane,
                                                             int K, int groups, int64_t nb, int L,
                                                             uint8_t *__restrict__ l1flag, int64_t chunks1, float thr1) {
    constexpr int T = S / 16;
    extern __shared__ float2 sm[];
    float2 *tws = sm;
    float2 *xa = sm + f16_tw_entries(S);
    float2 *xb = DB ? xa + f16_xchg_entries(S) : xa;
    const int t = threadIdx.x;
    f16_load_twiddles<S>(tws, tw, t);
    // segment-major block order: consecutive blocks write consecutive stretches of the same rows
    // (with the groups of a segment adjacent instead, its spectrum came from DRAM once, 40 MB
    // instead of 232 MB read at N = 2^23, but the kernel took 0.943 ms instead of 0.926 ms)
    const int64_t n_seg = gridDim.x / groups;
    const int grp = (int)(blockIdx.x / n_seg);
    const int64_t j = blockIdx.x - (int64_t)grp * n_seg;
    const int z0 = (int)((int64_t)grp * K / groups);
    const int z1 = (int)((int64_t)(grp + 1) * K / groups);
    const float2 *Yj = Y + j * S;
    const int64_t r0 = j * L;
    const int lim = (int)min((int64_t)L, nb - r0);   // ragged last segment
    float2 y[PRE ? 16 : 1], g[PRE ? 16 : 1];
    if constexpr (PRE) {
        if (z0 < z1) {
            const float2 *Gz = G + (int64_t)z0 * S;
#pragma unroll
            for (int i = 0; i < 16; i++) {
                y[i] = __ldg(Yj + t + i * T);
                g[i] = __ldg(Gz + t + i * T);
            }
        }
    }
    for (int z = z0; z < z1; z++) {
        float2 v[16];
        if constexpr (PRE) {
#pragma unroll
            for (int i = 0; i < 16; i++) v[i] = cmul_conj_a(y[i], g[i]);
            if (z + 1 < z1) {
                const float2 *Gn = G + (int64_t)(z + 1) * S;
#pragma unroll
                for (int i = 0; i < 16; i++) g[i] = __ldg(Gn + t + i * T);
            }
        } else {
            const float2 *Gz = G + (int64_t)z * S;
#pragma unroll
            for (int i = 0; i < 16; i++) {
                const int k = t + i * T;
                v[i] = cmul_conj_a(__ldg(Yj + k), __ldg(Gz + k));
            }
        }
        block_fft16<S, DB>(v, xa, xb, tws, t);
        float *row = plane + (int64_t)z * nb + r0;
        float vm[4] = {0.f, 0.f, 0.f, 0.f};          // four short max chains (latency)
#pragma unroll
        for (int i = 0; i < 16; i++) {
            const int o = t + i * T;
            const float pw = v[i].x * v[i].x + v[i].y * v[i].y;
            vm[i & 3] = fmaxf(vm[i & 3], pw);
            if (o < lim) row[o] = pw;
        }
        const float vmax = fmaxf(fmaxf(vm[0], vm[1]), fmaxf(vm[2], vm[3]));
        if (l1flag != nullptr && vmax > thr1) {      // rare: recompute the same powers
            uint8_t *frow = l1flag + (int64_t)z * chunks1;
#pragma unroll
            for (int i = 0; i < 16; i++) {
                const int o = t + i * T;
                if (o < lim && v[i].x * v[i].x + v[i].y * v[i].y > thr1) frow[(r0 + o) >> 9] = 1;
            }
        }
    }
}

int sm_count(const Plan &p) {
    int sms = 152;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p.device >= 0 ? p.device : 0);
    return sms;
}

template <int S>
cudaError_t run_segments(const Plan &p, const float2 *d_x, const float *d_scale, float2 *Y, cudaStream_t st) {
    const size_t smem = f16_smem<S>(false);
    cudaError_t e = cudaFuncSetAttribute(k2_segments<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    // enough CTAs to fill every SM a few times; each fills its twiddle table once
    const int64_t grid = std::min<int64_t>(p.n_seg, (int64_t)sm_count(p) * std::max(1, 4096 / S) * 2);
    p.prof.begin(FDAS_STAGE_SEGMENTS, st);
    k2_segments<S><<<(unsigned)grid, S / 16, smem, st>>>(d_x, d_scale, p.d_tw, Y, p.n_seg, p.nb, p.L, p.m / 2);
    p.prof.end(FDAS_STAGE_SEGMENTS, st);
    p.prof.launches += 1;
    return cudaGetLastError();
}

template <int S, bool DB, int MINB, bool PRE>
cudaError_t run_correlate(const Plan &p, const float2 *Y, float *plane, cudaStream_t st, uint8_t *l1flag) {
    const size_t smem = f16_smem<S>(DB);
    cudaError_t e = cudaFuncSetAttribute(k3_plane_fp32<S, DB, MINB, PRE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    // templates per CTA: about zb (at most 16 by default), the K rows split evenly over the groups
    int zb = (int)std::max<int64_t>(1, std::min<int64_t>(16, (p.n_seg * p.K) / ((int64_t)sm_count(p) * 8)));
    if (p.tune_zb > 0) zb = std::min(p.tune_zb, p.K);
    const int groups = (p.K + zb - 1) / zb;
    const int64_t grid = p.n_seg * groups;
    if (l1flag) {
        e = cudaMemsetAsync(l1flag, 0, (size_t)p.K * (size_t)(p.nb / PEAK_CHUNK), st);
        if (e != cudaSuccess) return e;
    }
    p.prof.begin(FDAS_STAGE_CORRELATE, st);
    k3_plane_fp32<S, DB, MINB, PRE><<<(unsigned)grid, S / 16, smem, st>>>(Y, p.d_G, p.d_tw, plane, p.K, groups, p.nb,
                                                                        p.L, l1flag, p.nb / PEAK_CHUNK, mark_threshold(p));
    p.prof.end(FDAS_STAGE_CORRELATE, st);
    p.prof.launches += 1;
    return cudaGetLastError();
}

// Launch shapes, measured at N = 2^23, 85 templates, 256 taps (correlation kernel, ms):
//   S = 1024: both exchange buffers, 8 CTAs of 2 warps per SM                         0.925
//   S = 2048: segment spectrum held in registers and the next template's spectrum
//             loaded during the transform, one exchange buffer, 3 CTAs of 4 warps   0.922
//   S = 4096: both exchange buffers, 2 CTAs of 8 warps per SM                         1.086
//   S = 8192: one exchange buffer (three exchanges), one CTA of 16 warps per SM        1.309
// Neither more CTAs per SM at fewer registers (spills) nor the other buffer / prefetch choices
// measured faster at any S.
template <int S>
cudaError_t run_plane(const Plan &p, const float2 *d_x, const float *d_scale, float2 *Y, float *plane,
                      cudaStream_t st, uint8_t *l1flag) {
    cudaError_t e = run_segments<S>(p, d_x, d_scale, Y, st);
    if (e != cudaSuccess) return e;
    if constexpr (S == 8192) return run_correlate<S, false, 1, false>(p, Y, plane, st, l1flag);
    else if constexpr (S == 4096) return run_correlate<S, true, 2, false>(p, Y, plane, st, l1flag);
    else if constexpr (S == 2048) return run_correlate<S, false, 3, true>(p, Y, plane, st, l1flag);
    else return run_correlate<S, true, 8, false>(p, Y, plane, st, l1flag);
}

}  // namespace

static_assert(PEAK_CHUNK == 512, "the level-1 marks index units as bin >> 9");

cudaError_t launch_plane_fp32(const Plan &p, const float2 *d_x, const float *d_scale, char *ws, float *d_plane,
                              cudaStream_t st, uint8_t *l1flag) {
    float2 *Y = reinterpret_cast<float2 *>(ws + p.ws_y);
    switch (p.S) {
        case 1024: return run_plane<1024>(p, d_x, d_scale, Y, d_plane, st, l1flag);
        case 2048: return run_plane<2048>(p, d_x, d_scale, Y, d_plane, st, l1flag);
        case 4096: return run_plane<4096>(p, d_x, d_scale, Y, d_plane, st, l1flag);
        case 8192: return run_plane<8192>(p, d_x, d_scale, Y, d_plane, st, l1flag);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_segments_fp32(const Plan &p, const float2 *d_x, const float *d_scale, float2 *d_yhat,
                                 cudaStream_t st) {
    if (p.S != 4096) return cudaErrorInvalidValue;
    return run_segments<4096>(p, d_x, d_scale, d_yhat, st);
}

cudaError_t launch_plane_fp32_scratch(const Plan &p, const float2 *d_x, const float *d_scale, float2 *d_yhat,
                                      float *d_plane, cudaStream_t st) {
    switch (p.S) {
        case 1024: return run_plane<1024>(p, d_x, d_scale, d_yhat, d_plane, st, nullptr);
        case 2048: return run_plane<2048>(p, d_x, d_scale, d_yhat, d_plane, st, nullptr);
        case 4096: return run_plane<4096>(p, d_x, d_scale, d_yhat, d_plane, st, nullptr);
        case 8192: return run_plane<8192>(p, d_x, d_scale, d_yhat, d_plane, st, nullptr);
    }
    return cudaErrorInvalidValue;
}

}  // namespace fdas
