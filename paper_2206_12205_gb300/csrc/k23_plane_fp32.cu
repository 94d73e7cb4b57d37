// K2 + K3, FP32 path: the overlap-save correlation that produces the f-z plane
// (Sec. 2.1 and Fig. fdas_flow, the "blue box" the paper times).
//
// Segment j covers spectrum bins [jL - m/2, jL - m/2 + S), L = S - m + 1, zero outside
// [0, Nb).  With Yhat_j its length-S DFT and G_z the template DFT (K0), the circular
// correlation of the window with template z at offset t < L is
//     W_{j,z}(t) = sum_{d<m} Y_j(t + d) conj(T_z(d - m/2)) = conj( FFT_S(conj(Yhat_j) * G_z) )(t),
// free of wrap-around for t < L, so P[z][jL + t] = |FFT_S(conj(Yhat_j) * G_z)(t)|^2.
//
//   K2 (one CTA per segment): window load (scaled by sqrt(2/sigma2) when the spectrum is
//       unnormalised), forward FFT, Yhat stored [n_seg][S].
//   K3 (one CTA per segment and run of templates): complex multiply fused into the FFT's
//       coalesced loads, forward FFT, |.|^2 and overlap discard fused into its coalesced
//       stores: the plane is written exactly once and nothing else touches HBM in bulk.  Inside
//       a search it also marks the 512-bin units holding a power above the level-1 threshold
//       (the level-1 pass of the peak search then visits only those).
#include "block_fft.cuh"
#include "fdas_internal.cuh"

namespace fdas {

namespace {

template <int S>
__global__ void __launch_bounds__(S / 32) k2_segments(const float2 *__restrict__ X, const float *__restrict__ scale_ptr,
                                                      const float2 *__restrict__ tw, float2 *__restrict__ Y,
                                                      int64_t nb, int L, int half_m) {
    constexpr int T = S / 32;
    extern __shared__ float2 sm[];
    const int t = threadIdx.x;
    const int64_t j = blockIdx.x;
    const float scale = scale_ptr ? __ldg(scale_ptr) : 1.0f;
    const int64_t base = j * L - half_m;
    float2 v[32];
#pragma unroll
    for (int i = 0; i < 32; i++) {
        const int64_t k = base + t + i * T;
        float2 x = make_float2(0.f, 0.f);
        if (k >= 0 && k < nb) x = __ldg(X + k);
        v[i] = make_float2(x.x * scale, x.y * scale);
    }
    block_fft<S>(v, sm, tw, t);
    float2 *out = Y + j * S;
#pragma unroll
    for (int i = 0; i < 32; i++) out[t + i * T] = v[i];
}

template <int S>
__global__ void __launch_bounds__(S / 32) k3_plane_fp32(const float2 *__restrict__ Y, const float2 *__restrict__ G,
                                                        const float2 *__restrict__ tw, float *__restrict__ plane,
                                                        int K, int zb, int64_t nb, int L, uint8_t *__restrict__ l1flag,
                                                        int64_t chunks1, float thr1) {
    constexpr int T = S / 32;
    extern __shared__ float2 sm[];
    const int t = threadIdx.x;
    const int64_t j = blockIdx.x;
    const int z0 = blockIdx.y * zb;
    const int z1 = min(K, z0 + zb);
    const float2 *Yj = Y + j * S;
    const int64_t r0 = j * L;
    const int lim = (int)min((int64_t)L, nb - r0);   // ragged last segment
    for (int z = z0; z < z1; z++) {
        const float2 *Gz = G + (int64_t)z * S;
        float2 v[32];
#pragma unroll
        for (int i = 0; i < 32; i++) {
            const int k = t + i * T;
            v[i] = cmul_conj_a(__ldg(Yj + k), __ldg(Gz + k));
        }
        block_fft<S>(v, sm, tw, t);
        float *row = plane + (int64_t)z * nb + r0;
        float vm[4] = {0.f, 0.f, 0.f, 0.f};          // four short max chains (latency)
#pragma unroll
        for (int i = 0; i < 32; i++) {
            const int o = t + i * T;
            const float pw = v[i].x * v[i].x + v[i].y * v[i].y;
            vm[i & 3] = fmaxf(vm[i & 3], pw);
            if (o < lim) row[o] = pw;
        }
        const float vmax = fmaxf(fmaxf(vm[0], vm[1]), fmaxf(vm[2], vm[3]));
        if (l1flag != nullptr && vmax > thr1) {      // rare: recompute the same powers
            uint8_t *frow = l1flag + (int64_t)z * chunks1;
#pragma unroll
            for (int i = 0; i < 32; i++) {
                const int o = t + i * T;
                if (o < lim && v[i].x * v[i].x + v[i].y * v[i].y > thr1) frow[(r0 + o) >> 9] = 1;
            }
        }
    }
}

template <int S>
cudaError_t run_plane(const Plan &p, const float2 *d_x, const float *d_scale, float2 *Y, float *plane,
                      cudaStream_t st, uint8_t *l1flag) {
    const size_t smem = sizeof(float2) * fft_smem_entries(S);
    cudaError_t e = cudaFuncSetAttribute(k2_segments<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k3_plane_fp32<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    p.prof.begin(FDAS_STAGE_SEGMENTS, st);
    k2_segments<S><<<(unsigned)p.n_seg, S / 32, smem, st>>>(d_x, d_scale, p.d_tw, Y, p.nb, p.L, p.m / 2);
    p.prof.end(FDAS_STAGE_SEGMENTS, st);
    p.prof.launches += 1;
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // templates per CTA: enough CTAs to fill the GPU several times over
    int zb = (int)std::max<int64_t>(1, std::min<int64_t>(16, (p.n_seg * p.K) / (152 * 8)));
    if (p.tune_zb > 0) zb = std::min(p.tune_zb, p.K);
    dim3 grid((unsigned)p.n_seg, (unsigned)((p.K + zb - 1) / zb));
    if (l1flag) {
        e = cudaMemsetAsync(l1flag, 0, (size_t)p.K * (size_t)(p.nb / PEAK_CHUNK), st);
        if (e != cudaSuccess) return e;
    }
    p.prof.begin(FDAS_STAGE_CORRELATE, st);
    k3_plane_fp32<S><<<grid, S / 32, smem, st>>>(Y, p.d_G, p.d_tw, plane, p.K, zb, p.nb, p.L, l1flag,
                                                 p.nb / PEAK_CHUNK, p.cfg.thr[0]);
    p.prof.end(FDAS_STAGE_CORRELATE, st);
    p.prof.launches += 1;
    return cudaGetLastError();
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
    const size_t smem = sizeof(float2) * fft_smem_entries(4096);
    cudaError_t e = cudaFuncSetAttribute(k2_segments<4096>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    p.prof.begin(FDAS_STAGE_SEGMENTS, st);
    k2_segments<4096><<<(unsigned)p.n_seg, 4096 / 32, smem, st>>>(d_x, d_scale, p.d_tw, d_yhat, p.nb, p.L, p.m / 2);
    p.prof.end(FDAS_STAGE_SEGMENTS, st);
    p.prof.launches += 1;
    return cudaGetLastError();
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
