// K2 + K3, BF16 path (Sec. 3: the convolution section in bfloat16, the long FFT kept in FP32):
// the overlap-save correlation with the segment FFT's DFT stages run on the tensor cores
// (tcgen05, BF16 operands, FP32 accumulation in TMEM) and a BF16 plane.
//
// Segments are S = 4096 bins long with stride L = 64 * floor((S - m + 1) / 64) (any
// L <= S - m + 1 gives the same plane; a multiple of 64 keeps the stores aligned).
// With x = conj(Yhat_j) * G_z (length S, n = 64 n1 + n2) the plane row segment is
// |X|^2 with the four-step DFT
//     X[k1 + 64 k2] = sum_{n2} W_64^{n2 k2} W_S^{n2 k1} sum_{n1} W_64^{n1 k1} x[64 n1 + n2],
// computed for two templates at a time as two real GEMMs of 128 x 128 x 128:
//   stage 1  D1[(k1,p), (z,n2)] = F'[(k1,p), (n1,s)] . B1[(n1,s), (z,n2)],  B1 = x (BF16)
//   twiddle  B2[(n2,s), (z,k1)] = W_S^{n2 k1} D1[k1, (z, n2)]               (CUDA cores, BF16)
//   stage 2  D2[(k2,p), (z,k1)] = F'[(k2,p), (n2,s)] . B2[(n2,s), (z,k1)]
//   output   P[z][jL + k1 + 64 k2] = |D2[k2, (z, k1)]|^2 for k1 + 64 k2 < L   (BF16, 16-byte stores)
// where F' is the radix-64 DFT real-ified with re/im interleaved (row 2k+p, column 2n+s), so
// the real and imaginary parts of one value sit in adjacent TMEM lanes (adjacent threads).
//
// B1 and B2 share one shared-memory tile and D1 and D2 one set of TMEM columns: each is
// rewritten only after the MMA that reads it (or the loads that drain it) has completed.  One
// persistent CTA per slot (3 per SM: 64 KB shared memory, 128 of 512 TMEM columns each) walks a
// contiguous range of (segment, template pair) items, so a segment's spectrum stays in L1.  Every mbarrier wait is bounded; a timeout sets FDAS_DEV_TIMEOUT and the CTA stops
// after its MMAs have drained, freeing its TMEM.
#include <cmath>
#include <cstring>
#include <vector>

#include "block_fft.cuh"
#include "fdas_internal.cuh"
#include "tc_sm100.cuh"

namespace fdas {

namespace {

constexpr int TC_R = 64;
constexpr int TC_G = 2;                          // templates per item
constexpr int TC_N = TC_G * TC_R;                // GEMM N (columns)
constexpr int TC_M = 2 * TC_R;                   // GEMM M (real-ified rows)
constexpr int TC_K = 2 * TC_R;                   // GEMM K
constexpr int TC_THREADS = 256;
constexpr uint32_t TILE_BYTES = TC_M * TC_K * 2;  // 32 KB: F' and B are 128 x 128 BF16
constexpr uint32_t SMEM_BYTES = 2 * TILE_BYTES + 64;
constexpr uint32_t TMEM_COLS = TC_N;              // D1 and D2 share the columns
constexpr int CTAS_PER_SM = 3;                    // 64 KB shared memory, 128 TMEM columns each
constexpr long long WAIT_CYCLES = 4000000000LL;   // about 2 s at 2 GHz

static_assert(TC_S_BF16 == TC_R * TC_R, "segment length must be 64 x 64");

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&h);
}

__device__ __forceinline__ float2 unpack_bf16x2(__nv_bfloat162 v) { return __bfloat1622float2(v); }

// Segment FFTs (FP32 CUDA-core block FFT), stored as BF16 pairs for the tensor stages.
__global__ void __launch_bounds__(TC_S_BF16 / 32) k2_segments_bf16(const float2 *__restrict__ X,
                                                                   const float *__restrict__ scale_ptr,
                                                                   const float2 *__restrict__ tw,
                                                                   __nv_bfloat162 *__restrict__ Y, int64_t nb, int L,
                                                                   int half_m) {
    constexpr int S = TC_S_BF16, T = S / 32;
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
    __nv_bfloat162 *out = Y + j * S;
#pragma unroll
    for (int i = 0; i < 32; i++) out[t + i * T] = __floats2bfloat162_rn(v[i].x, v[i].y);
}

// Split the re (even lane) / im (odd lane) halves of a 16-column TMEM chunk so that each
// thread of the pair ends up with 8 complex values: the even lane keeps columns 0..7, the
// odd lane columns 8..15.
__device__ __forceinline__ void pair_exchange(const uint32_t (&r)[16], int rho, float (&re)[8], float (&im)[8]) {
#pragma unroll
    for (int q = 0; q < 8; q++) {
        const float send = rho == 0 ? __uint_as_float(r[8 + q]) : __uint_as_float(r[q]);
        const float recv = __shfl_xor_sync(0xffffffffu, send, 1);
        if (rho == 0) {
            re[q] = __uint_as_float(r[q]);
            im[q] = recv;
        } else {
            re[q] = recv;
            im[q] = __uint_as_float(r[8 + q]);
        }
    }
}

__global__ void __launch_bounds__(TC_THREADS) k3_plane_tc(const __nv_bfloat162 *__restrict__ Y,
                                                          const __nv_bfloat162 *__restrict__ G,
                                                          const uint4 *__restrict__ Fimg,
                                                          const float2 *__restrict__ tw,
                                                          __nv_bfloat16 *__restrict__ plane, int K, int64_t nb,
                                                          int L, int64_t n_items, int n_groups,
                                                          int64_t items_per_cta, int32_t *__restrict__ status) {
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char *sF = smem;
    unsigned char *sB1 = smem + TILE_BYTES;
    unsigned char *sB2 = sB1;                      // B2 overwrites B1 once stage 1 has read it
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + 2 * TILE_BYTES);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(smem + 2 * TILE_BYTES + 16);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (warp == 0) {
        tc::tmem_alloc(tslot, TMEM_COLS);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        tc::mbar_init(&bar[0], 1);
        tc::mbar_init(&bar[1], 1);
    }
    for (int i = tid; i < (int)(TILE_BYTES / 16); i += TC_THREADS) reinterpret_cast<uint4 *>(sF)[i] = __ldg(Fimg + i);
    tc::fence_proxy_async_smem();
    tc::fence_before_thread_sync();
    __syncthreads();
    tc::fence_after_thread_sync();

    const uint32_t tbase = *tslot;
    const uint32_t tD1 = tbase, tD2 = tbase;       // D2 overwrites D1 once it has been read
    const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
    const uint32_t idesc = tc::idesc_bf16_f32(TC_M, TC_N);
    const uint32_t aF = tc::smem_u32(sF), aB1 = tc::smem_u32(sB1), aB2 = tc::smem_u32(sB2);
    const int row = 32 * (warp & 3) + lane;      // TMEM lane = GEMM row (k, p)
    const int kk = row >> 1, rho = row & 1;
    const int zl_epi = warp >> 2;                 // warps 0-3: first template, 4-7: second

    uint32_t phase = 0;
    int pending = 0;                               // MMA groups committed but not yet waited for
    bool ok = true;
    const int64_t it0 = (int64_t)blockIdx.x * items_per_cta;
    const int64_t it1 = min(n_items, it0 + items_per_cta);
    for (int64_t it = it0; it < it1; it++) {
        const int64_t j = it / n_groups;
        const int z0 = (int)(it % n_groups) * TC_G;

        // ---- B1[(n1, s), (zl, n2)] = conj(Yhat_j[64 n1 + n2]) * G_{z0+zl}[64 n1 + n2]
        {
            const int c = tid & (TC_N - 1);
            const int zl = c >> 6, n2 = c & 63;
            const int z = z0 + zl;
            const bool zvalid = z < K;
            const __nv_bfloat162 *Yj = Y + j * TC_S_BF16;
            const __nv_bfloat162 *Gz = G + (int64_t)(zvalid ? z : 0) * TC_S_BF16;
#pragma unroll 8
            for (int b = tid >> 7; b < 16; b += 2) {
                uint32_t w[4];
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    const int n = 64 * (4 * b + q) + n2;
                    const float2 y = unpack_bf16x2(Yj[n]);
                    const float2 g = zvalid ? unpack_bf16x2(__ldg(Gz + n)) : make_float2(0.f, 0.f);
                    w[q] = pack_bf16x2(y.x * g.x + y.y * g.y, y.x * g.y - y.y * g.x);
                }
                *reinterpret_cast<uint4 *>(sB1 + tc::kmajor_offset(TC_N, c, 8 * b)) = make_uint4(w[0], w[1], w[2], w[3]);
            }
        }
        tc::fence_proxy_async_smem();
        tc::fence_before_thread_sync();
        __syncthreads();
        tc::fence_after_thread_sync();

        // ---- stage 1: D1 = F' B1
        if (tid == 0) {
#pragma unroll
            for (int s = 0; s < TC_K / 16; s++)
                tc::mma_bf16(tD1, tc::smem_desc(aF + s * TC_M * 32, TC_M * 16, 128),
                             tc::smem_desc(aB1 + s * TC_N * 32, TC_N * 16, 128), idesc, s > 0 ? 1u : 0u);
            tc::mma_commit(&bar[0]);
        }
        pending = 1;
        ok = __syncthreads_and(tc::mbar_wait_bounded(&bar[0], phase, WAIT_CYCLES));
        if (!ok) break;
        pending = 0;
        tc::fence_after_thread_sync();

        // ---- twiddle: B2[(n2, s), (zl, k1)] = W_S^{n2 k1} D1[(k1, .), (zl, n2)]
#pragma unroll 1
        for (int ch = 0; ch < 4; ch++) {
            uint32_t r[16];
            tc::tmem_ld16(tD1 + lane_base + zl_epi * TC_R + 16 * ch, r);
            tc::tmem_ld_wait();
            float re[8], im[8];
            pair_exchange(r, rho, re, im);
            const int n2_0 = 16 * ch + 8 * rho;
            const float4 *twp = reinterpret_cast<const float4 *>(tw + kk * TC_R + n2_0);
            uint32_t w[8];
#pragma unroll
            for (int q2 = 0; q2 < 4; q2++) {
                const float4 t2 = __ldg(twp + q2);
                const int q = 2 * q2;
                w[q] = pack_bf16x2(re[q] * t2.x - im[q] * t2.y, re[q] * t2.y + im[q] * t2.x);
                w[q + 1] = pack_bf16x2(re[q + 1] * t2.z - im[q + 1] * t2.w, re[q + 1] * t2.w + im[q + 1] * t2.z);
            }
            const int c2 = zl_epi * TC_R + kk;
            *reinterpret_cast<uint4 *>(sB2 + tc::kmajor_offset(TC_N, c2, 2 * n2_0)) = make_uint4(w[0], w[1], w[2], w[3]);
            *reinterpret_cast<uint4 *>(sB2 + tc::kmajor_offset(TC_N, c2, 2 * n2_0 + 8)) =
                make_uint4(w[4], w[5], w[6], w[7]);
        }
        tc::fence_proxy_async_smem();
        tc::fence_before_thread_sync();
        __syncthreads();
        tc::fence_after_thread_sync();

        // ---- stage 2: D2 = F' B2
        if (tid == 0) {
#pragma unroll
            for (int s = 0; s < TC_K / 16; s++)
                tc::mma_bf16(tD2, tc::smem_desc(aF + s * TC_M * 32, TC_M * 16, 128),
                             tc::smem_desc(aB2 + s * TC_N * 32, TC_N * 16, 128), idesc, s > 0 ? 1u : 0u);
            tc::mma_commit(&bar[1]);
        }
        pending = 2;
        ok = __syncthreads_and(tc::mbar_wait_bounded(&bar[1], phase, WAIT_CYCLES));
        if (!ok) break;
        pending = 0;
        tc::fence_after_thread_sync();

        // ---- |X|^2 for X[k1 + 64 k2], k1 = 16 ch + 8 p + q: eight consecutive bins per thread
        {
            const int z = z0 + zl_epi;
            const int64_t r0 = j * L;
#pragma unroll 1
            for (int ch = 0; ch < 4; ch++) {
                uint32_t r[16];
                tc::tmem_ld16(tD2 + lane_base + zl_epi * TC_R + 16 * ch, r);
                tc::tmem_ld_wait();
                float re[8], im[8];
                pair_exchange(r, rho, re, im);
                const int t = 64 * kk + 16 * ch + 8 * rho;
                const int64_t rr = r0 + t;
                if (z < K && t < L && rr < nb) {
                    uint4 o;
                    o.x = pack_bf16x2(re[0] * re[0] + im[0] * im[0], re[1] * re[1] + im[1] * im[1]);
                    o.y = pack_bf16x2(re[2] * re[2] + im[2] * im[2], re[3] * re[3] + im[3] * im[3]);
                    o.z = pack_bf16x2(re[4] * re[4] + im[4] * im[4], re[5] * re[5] + im[5] * im[5]);
                    o.w = pack_bf16x2(re[6] * re[6] + im[6] * im[6], re[7] * re[7] + im[7] * im[7]);
                    *reinterpret_cast<uint4 *>(plane + (int64_t)z * nb + rr) = o;
                }
            }
        }
        tc::fence_before_thread_sync();
        __syncthreads();
        phase ^= 1;
    }
    if (!ok) {
        if (tid == 0) atomicOr(status, FDAS_DEV_TIMEOUT);
        // let the outstanding MMAs drain (bounded) before the TMEM is released
        tc::mbar_wait_bounded(&bar[pending == 2 ? 1 : 0], phase, WAIT_CYCLES);
    }
    tc::fence_before_thread_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tbase, TMEM_COLS);
}

}  // namespace

namespace {
uint16_t host_bf16(float f) {
    uint32_t u;
    std::memcpy(&u, &f, 4);
    u += 0x7FFFu + ((u >> 16) & 1u);           // round to nearest even
    return (uint16_t)(u >> 16);
}
}  // namespace

// Host tables of the tensor path: F'[(k,p),(n,s)] (W_64^{kn} real-ified, re/im interleaved) as a
// K-major BF16 operand image, and the four-step twiddles W_4096^{n2 k1}; FP64 then rounded.
cudaError_t launch_prepare_bf16(Plan &p, cudaStream_t st) {
    std::vector<uint16_t> img(TC_M * TC_K, 0);
    for (int k = 0; k < TC_R; k++)
        for (int n = 0; n < TC_R; n++) {
            const int e = (k * n) % TC_R;
            double f = 2.0 * e / TC_R;
            if (f > 1.0) f -= 2.0;
            const double wr = std::cos(M_PI * f), wi = -std::sin(M_PI * f);
            const float v[2][2] = {{(float)wr, (float)-wi}, {(float)wi, (float)wr}};
            for (int pr = 0; pr < 2; pr++)
                for (int sg = 0; sg < 2; sg++)
                    img[tc::kmajor_offset(TC_M, 2 * k + pr, 2 * n + sg) / 2] = host_bf16(v[pr][sg]);
        }
    std::vector<float2> tw(TC_R * TC_R);
    for (int k1 = 0; k1 < TC_R; k1++)
        for (int n2 = 0; n2 < TC_R; n2++) {
            const int e = (n2 * k1) % TC_S_BF16;
            double f = 2.0 * e / TC_S_BF16;
            if (f > 1.0) f -= 2.0;
            tw[k1 * TC_R + n2] = make_float2((float)std::cos(M_PI * f), (float)-std::sin(M_PI * f));
        }
    cudaError_t e = cudaMemcpyAsync(p.d_tcF, img.data(), img.size() * 2, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(p.d_tcTw, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e;
}

cudaError_t launch_plane_bf16(const Plan &p, const float2 *d_x, const float *d_scale, char *ws,
                              __nv_bfloat16 *d_plane, cudaStream_t st) {
    if (p.S != TC_S_BF16) return cudaErrorInvalidValue;
    __nv_bfloat162 *Y = reinterpret_cast<__nv_bfloat162 *>(ws + p.ws_y);
    const size_t smem2 = sizeof(float2) * fft_smem_entries(TC_S_BF16);
    cudaError_t e = cudaFuncSetAttribute(k2_segments_bf16, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k3_plane_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES);
    if (e != cudaSuccess) return e;
    p.prof.begin(FDAS_STAGE_SEGMENTS, st);
    k2_segments_bf16<<<(unsigned)p.n_seg, TC_S_BF16 / 32, smem2, st>>>(d_x, d_scale, p.d_tw, Y, p.nb, p.L, p.m / 2);
    p.prof.end(FDAS_STAGE_SEGMENTS, st);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int n_groups = (p.K + TC_G - 1) / TC_G;
    const int64_t n_items = p.n_seg * n_groups;
    int sms = 152;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p.device >= 0 ? p.device : 0);
    const int64_t ctas = std::min<int64_t>(n_items, CTAS_PER_SM * (int64_t)sms);
    const int64_t per = (n_items + ctas - 1) / ctas;
    const int64_t grid = (n_items + per - 1) / per;
    p.prof.begin(FDAS_STAGE_CORRELATE, st);
    k3_plane_tc<<<(unsigned)grid, TC_THREADS, SMEM_BYTES, st>>>(Y, p.d_Gbf, reinterpret_cast<const uint4 *>(p.d_tcF),
                                                               p.d_tcTw, d_plane, p.K, p.nb, p.L, n_items, n_groups,
                                                               per, p.d_status);
    p.prof.end(FDAS_STAGE_CORRELATE, st);
    p.prof.launches += 2;
    return cudaGetLastError();
}

}  // namespace fdas
