// K2 + K3, BF16 path (Sec. 3: the convolution section in bfloat16, the long FFT kept in FP32):
// the overlap-save correlation with the segment FFT's DFT stages run on the tensor cores
// (tcgen05, BF16 operands, FP32 accumulation in TMEM) and a BF16 plane.
//
// Segments are S = 4096 bins long with stride L = 64 * floor((S - m + 1) / 64) (any
// L <= S - m + 1 gives the same plane; a multiple of 64 keeps the stores aligned).
// With x = conj(Yhat_j) * G_z (length S, n = 64 n1 + n2) the plane row segment is
// |X|^2 with the four-step DFT
//     X[k1 + 64 k2] = sum_{n2} W_64^{n2 k2} W_S^{n2 k1} sum_{n1} W_64^{n1 k1} x[64 n1 + n2],
// computed for two templates at a time as two real GEMMs of 128 x 128 x 128 (below), where F'
// is the radix-64 DFT real-ified with re/im interleaved (row 2k+p, column 2n+s).
//
// One persistent, warp-specialised CTA per SM walks a contiguous range of (segment, template
// pair) items with producer, MMA and two epilogue roles overlapped through double-buffered
// shared-memory tiles and TMEM accumulators (layout below the helpers).  Every mbarrier wait
// is bounded; a timeout sets FDAS_DEV_TIMEOUT, all roles stop, the issued MMAs drain and the
// TMEM is released.
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
constexpr uint32_t TILE_BYTES = TC_M * TC_K * 2;  // 32 KB: F' and every B tile are 128 x 128 BF16
constexpr long long WAIT_CYCLES = 4000000000LL;   // about 2 s at 2 GHz

static_assert(TC_S_BF16 == TC_R * TC_R, "segment length must be 64 x 64");

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&h);
}

// Operand formats of the tensor stages: BF16 (the paper's Sec. 3 variant, BF16 plane) or FP16 with
// per-segment scaling (the Sec. 3.2 ablation, FP32 plane times the segment's unscale factor).
struct OpsBF16 {
    using V = __nv_bfloat162;
    using Out = __nv_bfloat16;
    static constexpr uint32_t idesc = tc::idesc_bf16_f32(TC_M, TC_N);
    __device__ __forceinline__ static V high2(V a) { return __high2bfloat162(a); }
    __device__ __forceinline__ static V low2(V a) { return __low2bfloat162(a); }
    __device__ __forceinline__ static uint32_t pack(float lo, float hi) { return pack_bf16x2(lo, hi); }
    __device__ __forceinline__ static Out out(float pw, float) { return __float2bfloat16_rn(pw); }
};
struct OpsF16 {
    using V = __half2;
    using Out = float;
    static constexpr uint32_t idesc = tc::idesc_f16_f32(TC_M, TC_N);
    __device__ __forceinline__ static V high2(V a) { return __high2half2(a); }
    __device__ __forceinline__ static V low2(V a) { return __low2half2(a); }
    __device__ __forceinline__ static uint32_t pack(float lo, float hi) {
        const __half2 h = __floats2half2_rn(lo, hi);
        return *reinterpret_cast<const uint32_t *>(&h);
    }
    __device__ __forceinline__ static Out out(float pw, float unscale) { return pw * unscale; }
};

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

// Segment FFTs for the FP16 stages: the segment's largest component |re| or |im| is brought into
// [0.5, 1) by a power of two s_j (exact), the values stored as FP16 pairs, and the plane's factor
// 1 / (s_j gscale)^2 (gscale: the template bank's scale) kept per segment.
__global__ void __launch_bounds__(TC_S_BF16 / 32) k2_segments_f16(const float2 *__restrict__ X,
                                                                  const float *__restrict__ scale_ptr,
                                                                  const float2 *__restrict__ tw,
                                                                  __half2 *__restrict__ Y, float *__restrict__ unscale,
                                                                  float gscale, int64_t nb, int L, int half_m) {
    constexpr int S = TC_S_BF16, T = S / 32;
    extern __shared__ float2 sm[];
    __shared__ float wmax[T / 32];
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
    float mx = 0.f;
#pragma unroll
    for (int i = 0; i < 32; i++) mx = fmaxf(mx, fmaxf(fabsf(v[i].x), fabsf(v[i].y)));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((t & 31) == 0) wmax[t >> 5] = mx;
    __syncthreads();
    mx = wmax[0];
#pragma unroll
    for (int w = 1; w < T / 32; w++) mx = fmaxf(mx, wmax[w]);
    int ex = 0;
    if (mx > 0.f) frexpf(mx, &ex);                  // mx = f 2^ex, f in [0.5, 1)
    const float sj = ldexpf(1.0f, -ex);
    __half2 *out = Y + j * S;
#pragma unroll
    for (int i = 0; i < 32; i++) out[t + i * T] = __floats2half2_rn(v[i].x * sj, v[i].y * sj);
    if (t == 0) {
        const float g = sj * gscale;
        unscale[j] = 1.0f / (g * g);
    }
}

// ---------------------------------------------------------------------------------------
// Warp-specialised persistent kernel, one CTA per SM, 25 warps.  Both GEMMs run transposed,
// data as the A operand (M = 128 rows = two templates x 64) and F' as the B operand:
//   stage 1  D1t[(z,n2), (k1,p)] = B1[(z,n2), (n1,s)] . F'^T        (B1 = x, from the producer)
//   stage 2  D2t[(z,k1), (k2,p)] = A2[(z,k1), (n2,s)] . F'^T        (A2 = twiddled D1t, transposed)
// so a thread's TMEM row holds the real and imaginary parts of its values side by side.
//   warp 0       TMEM allocation; lane 0 issues the MMAs (stage 1 of item i+1 before stage 2 of i)
//   warps 1-8    producer:   B1[slot] = conj(Yhat_j) * G_z, one 4 x 4 (n1, n2) block per thread
//                with all of its 16-byte loads in flight at once
//   warps 9-16   epilogue 1: D1t[slot] -> W_S^{n2 k1} -> A2[slot] (warps 9-12 and 13-16 take the
//                two halves of k1)
//   warps 17-24  epilogue 2: D2t[slot] -> |.|^2 -> BF16 plane (halves of k2)
// Two slots of B1, A2 (shared memory) and D1t, D2t (TMEM, 4 x 128 of the 512 columns).
// Hand-offs are mbarriers, one per slot:
//   b1_full  (256 producer arrivals)   s1_done (MMA commit: D1t ready, B1 free)
//   b2_full  (256 epilogue-1 arrivals: A2 ready, D1t drained)
//   s2_done  (MMA commit: D2t ready, A2 free)   d2_free (256 epilogue-2 arrivals: D2t drained)
// The k-th use of a slot waits for phase parity k & 1; every wait is bounded and also gives
// up when another role has aborted.
constexpr int WS_PRODUCERS = 256;                            // warps 1-8
constexpr int WS_E1 = 1 + WS_PRODUCERS / 32;                 // first epilogue-1 warp (9)
constexpr int WS_E2 = WS_E1 + 8;                             // first epilogue-2 warp (17)
constexpr int WS_THREADS = (WS_E2 + 8) * 32;                 // 25 warps
// B1 tiles (stage-1 A operand): core matrices 144 B apart along M, 16 x 144 B along K
constexpr uint32_t B_SBO = 144, B_LBO = 16 * B_SBO;
constexpr uint32_t B_TILE = 16 * B_LBO;                      // 36 KB
// A2 tiles (stage-2 A operand): 128 B along M, 2064 B (16 mod 128) along K
constexpr uint32_t A2_SBO = 128, A2_LBO = 16 * 128 + 16;
constexpr uint32_t A2_TILE = 16 * A2_LBO;                    // 32.25 KB
constexpr uint32_t F_LBO = TC_M * 16, F_SBO = 128;           // F': dense
constexpr uint32_t OFF_F = 0;
constexpr uint32_t OFF_B1 = OFF_F + TILE_BYTES;              // 2 slots
constexpr uint32_t OFF_A2 = OFF_B1 + 2 * B_TILE;             // 2 slots
// twiddles W_S^{n2 k1}, one row per n2 padded to 66 entries (528 B = 16 mod 128) so that the
// 16-byte row reads of a warp's 32 different rows spread over all banks
constexpr int TW_LD = TC_R + 2;
constexpr uint32_t OFF_TW = OFF_A2 + 2 * A2_TILE;
constexpr uint32_t OFF_BAR = OFF_TW + TC_R * TW_LD * 8;
constexpr uint32_t WS_SMEM = OFF_BAR + 16 * 8 + 32;
constexpr uint32_t WS_TMEM_COLS = 512;

struct WsBars {
    uint64_t b1_full[2], s1_done[2], b2_full[2], s2_done[2], d2_free[2], drain;
};

__device__ __forceinline__ bool ws_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag) {
    const long long t0 = clock64();
    while (!tc::mbar_try_wait(bar, parity)) {
        if (*abort_flag) return false;
        if (clock64() - t0 > WAIT_CYCLES) {
            *abort_flag = 1;
            return false;
        }
    }
    return true;
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(bar)) : "memory");
}

template <class Ops>
__global__ void __launch_bounds__(WS_THREADS, 1) k3_plane_tc(const typename Ops::V *__restrict__ Y,
                                                             const typename Ops::V *__restrict__ G,
                                                             const uint4 *__restrict__ Fimg,
                                                             const float2 *__restrict__ tw,
                                                             typename Ops::Out *__restrict__ plane, int K, int64_t nb,
                                                             int L, int64_t n_items, int n_groups,
                                                             int64_t items_per_cta, const float *__restrict__ unscale,
                                                             int32_t *__restrict__ status) {
    extern __shared__ __align__(1024) unsigned char smem[];
    WsBars *bars = reinterpret_cast<WsBars *>(smem + OFF_BAR);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(smem + OFF_BAR + sizeof(WsBars));
    volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + OFF_BAR + sizeof(WsBars) + 8);
    float2 *sTw = reinterpret_cast<float2 *>(smem + OFF_TW);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (warp == 0) {
        tc::tmem_alloc(tslot, WS_TMEM_COLS);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        for (int s = 0; s < 2; s++) {
            tc::mbar_init(&bars->b1_full[s], WS_PRODUCERS);
            tc::mbar_init(&bars->s1_done[s], 1);
            tc::mbar_init(&bars->b2_full[s], 256);
            tc::mbar_init(&bars->s2_done[s], 1);
            tc::mbar_init(&bars->d2_free[s], 256);
        }
        tc::mbar_init(&bars->drain, 1);
        *abort_flag = 0;
    }
    for (int i = tid; i < (int)(TILE_BYTES / 16); i += WS_THREADS)
        reinterpret_cast<uint4 *>(smem + OFF_F)[i] = __ldg(Fimg + i);
    for (int i = tid; i < TC_S_BF16; i += WS_THREADS) sTw[(i / TC_R) * TW_LD + (i % TC_R)] = __ldg(tw + i);
    tc::fence_proxy_async_smem();
    tc::fence_before_thread_sync();
    __syncthreads();
    tc::fence_after_thread_sync();

    const uint32_t tbase = *tslot;
    const int64_t it0 = (int64_t)blockIdx.x * items_per_cta;
    const int64_t it1 = min(n_items, it0 + items_per_cta);
    const int64_t n_my = it1 - it0;

    if (warp == 0) {
        // ---------------------------------------------------------------- MMA issuer
        if (lane == 0 && n_my > 0) {
            const uint32_t idesc = Ops::idesc;
            const uint32_t bF = tc::smem_u32(smem + OFF_F);
            auto issue = [&](uint32_t dcol, uint32_t asm_, uint32_t albo, uint32_t asbo) {
#pragma unroll
                for (int s = 0; s < TC_K / 16; s++)
                    tc::mma_bf16(tbase + dcol, tc::smem_desc(asm_ + s * 2 * albo, albo, asbo),
                                 tc::smem_desc(bF + s * 2 * F_LBO, F_LBO, F_SBO), idesc, s > 0 ? 1u : 0u);
            };
            bool ok = ws_wait(&bars->b1_full[0], 0, abort_flag);
            if (ok) {
                tc::fence_after_thread_sync();
                issue(0, tc::smem_u32(smem + OFF_B1), B_LBO, B_SBO);
                tc::mma_commit(&bars->s1_done[0]);
            }
            for (int64_t k = 0; k < n_my && ok; k++) {
                const int sl = (int)(k & 1);
                const uint32_t par = (uint32_t)((k >> 1) & 1);
                if (k + 1 < n_my) {                                    // stage 1 of the next item
                    const int sn = (int)((k + 1) & 1);
                    ok = ws_wait(&bars->b1_full[sn], (uint32_t)(((k + 1) >> 1) & 1), abort_flag);
                    if (!ok) break;
                    tc::fence_after_thread_sync();
                    issue(sn * TC_N, tc::smem_u32(smem + OFF_B1 + sn * B_TILE), B_LBO, B_SBO);
                    tc::mma_commit(&bars->s1_done[sn]);
                }
                ok = ws_wait(&bars->b2_full[sl], par, abort_flag);     // A2 ready, D1t drained
                if (ok && k >= 2) ok = ws_wait(&bars->d2_free[sl], par ^ 1u, abort_flag);
                if (!ok) break;
                tc::fence_after_thread_sync();
                issue((2 + sl) * TC_N, tc::smem_u32(smem + OFF_A2 + sl * A2_TILE), A2_LBO, A2_SBO);
                tc::mma_commit(&bars->s2_done[sl]);
            }
            // drain: every MMA issued above has completed before TMEM can be released
            tc::mma_commit(&bars->drain);
            tc::mbar_wait_bounded(&bars->drain, 0, WAIT_CYCLES);
        }
        __syncwarp();
    } else if (warp < WS_E1) {
        // ---------------------------------------------------------------- producer
        // thread -> block (n1 = 4 n1q .. 4 n1q + 3, n2 = 4 n2q .. 4 n2q + 3) of both templates
        const int pt = tid - 32;
        const int n2q = pt & 15, n1q = pt >> 4;
        for (int64_t k = 0; k < n_my; k++) {
            const int64_t it = it0 + k;
            const int64_t j = it / n_groups;
            const int z0 = (int)(it % n_groups) * TC_G;
            const int sl = (int)(k & 1);
            const uint4 *Yj = reinterpret_cast<const uint4 *>(Y + j * TC_S_BF16);
            uint4 yv[4], gv[TC_G][4];
#pragma unroll
            for (int q = 0; q < 4; q++) yv[q] = __ldg(Yj + (64 * (4 * n1q + q) + 4 * n2q) / 4);
#pragma unroll
            for (int zl = 0; zl < TC_G; zl++) {
                const int z = z0 + zl;
                const uint4 *Gz = reinterpret_cast<const uint4 *>(G + (int64_t)(z < K ? z : 0) * TC_S_BF16);
#pragma unroll
                for (int q = 0; q < 4; q++)
                    gv[zl][q] = z < K ? __ldg(Gz + (64 * (4 * n1q + q) + 4 * n2q) / 4) : make_uint4(0, 0, 0, 0);
            }
            if (k >= 2 && !ws_wait(&bars->s1_done[sl], (uint32_t)(((k - 2) >> 1) & 1), abort_flag)) break;
            unsigned char *b1 = smem + OFF_B1 + sl * B_TILE;
#pragma unroll
            for (int zl = 0; zl < TC_G; zl++) {
                uint32_t w[4][4];                                  // [n2 offset e][n1 offset q]
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    const uint32_t ys[4] = {yv[q].x, yv[q].y, yv[q].z, yv[q].w};
                    const uint32_t gs[4] = {gv[zl][q].x, gv[zl][q].y, gv[zl][q].z, gv[zl][q].w};
#pragma unroll
                    for (int e = 0; e < 4; e++) {
                        // conj(y) g = (yr, yr) (gr, gi) + (yi, yi) (gi, -gr), in packed BF16 arithmetic
                        using V = typename Ops::V;
                        const V y = *reinterpret_cast<const V *>(&ys[e]);
                        const V g = *reinterpret_cast<const V *>(&gs[e]);
                        V gb = __lowhigh2highlow(g);
                        *reinterpret_cast<uint32_t *>(&gb) ^= 0x80000000u;
                        const V x = __hfma2(Ops::high2(y), gb, __hmul2(Ops::low2(y), g));
                        w[e][q] = *reinterpret_cast<const uint32_t *>(&x);
                    }
                }
#pragma unroll
                for (int e = 0; e < 4; e++) {
                    const int c = zl * TC_R + 4 * n2q + e;
                    *reinterpret_cast<uint4 *>(b1 + tc::kmajor_offset_strided(B_SBO, B_LBO, c, 8 * n1q)) =
                        make_uint4(w[e][0], w[e][1], w[e][2], w[e][3]);
                }
            }
            tc::fence_proxy_async_smem();
            mbar_arrive(&bars->b1_full[sl]);
        }
    } else {
        // ---------------------------------------------------------------- epilogues
        const bool epi1 = warp < WS_E2;
        const int quad = warp & 3;                      // TMEM lane quadrant this warp may access
        const int half = ((warp - (epi1 ? WS_E1 : WS_E2)) >> 2) & 1;   // which 64 of the 128 columns
        const int lrow = 32 * quad + lane;              // TMEM lane = GEMM row = (zl, n2) or (zl, k1)
        const int zl = lrow >> 6, idx = lrow & 63;
        const uint32_t lane_base = (uint32_t)(32 * quad) << 16;
        for (int64_t k = 0; k < n_my; k++) {
            const int64_t it = it0 + k;
            const int sl = (int)(k & 1);
            const uint32_t par = (uint32_t)((k >> 1) & 1);
            if (epi1) {
                // idx = n2; columns (k1, p) for k1 in [32 half, 32 half + 32)
                if (!ws_wait(&bars->s1_done[sl], par, abort_flag)) break;
                if (k >= 2 && !ws_wait(&bars->s2_done[sl], par ^ 1u, abort_flag)) break;   // A2[sl] free
                tc::fence_after_thread_sync();
                unsigned char *a2 = smem + OFF_A2 + sl * A2_TILE;
                const float2 *twr = sTw + idx * TW_LD;                      // W_S^{n2 k1}, row n2
#pragma unroll 1
                for (int ch2 = 0; ch2 < 4; ch2 += 2) {
                    uint32_t rr[2][16];
                    tc::tmem_ld16(tbase + lane_base + sl * TC_N + 64 * half + 16 * ch2, rr[0]);
                    tc::tmem_ld16(tbase + lane_base + sl * TC_N + 64 * half + 16 * ch2 + 16, rr[1]);
                    tc::tmem_ld_wait();
#pragma unroll
                    for (int hh = 0; hh < 2; hh++) {
                        const int k1_0 = 32 * half + 8 * (ch2 + hh);
                        const float4 *tp = reinterpret_cast<const float4 *>(twr + k1_0);
#pragma unroll
                        for (int q2 = 0; q2 < 4; q2++) {
                            const float4 t2 = tp[q2];
#pragma unroll
                            for (int u = 0; u < 2; u++) {
                                const int q = 2 * q2 + u;
                                const float re = __uint_as_float(rr[hh][2 * q]), im = __uint_as_float(rr[hh][2 * q + 1]);
                                const float tx = u ? t2.z : t2.x, ty = u ? t2.w : t2.y;
                                const uint32_t wv = Ops::pack(re * tx - im * ty, re * ty + im * tx);
                                const int row = zl * TC_R + k1_0 + q;
                                *reinterpret_cast<uint32_t *>(a2 + tc::kmajor_offset_strided(A2_SBO, A2_LBO, row, 2 * idx)) = wv;
                            }
                        }
                    }
                }
                tc::fence_before_thread_sync();
                tc::fence_proxy_async_smem();
                mbar_arrive(&bars->b2_full[sl]);
            } else {
                // idx = k1; columns (k2, p) for k2 in [32 half, 32 half + 32)
                if (!ws_wait(&bars->s2_done[sl], par, abort_flag)) break;
                tc::fence_after_thread_sync();
                const int64_t j = it / n_groups;
                const int z = (int)(it % n_groups) * TC_G + zl;
                const int64_t r0 = j * L;
                const float us = unscale ? __ldg(unscale + j) : 1.0f;
                typename Ops::Out *prow = plane + (int64_t)(z < K ? z : 0) * nb + r0 + idx;
#pragma unroll 1
                for (int ch2 = 0; ch2 < 4; ch2 += 2) {
                    uint32_t rr[2][16];
                    tc::tmem_ld16(tbase + lane_base + (2 + sl) * TC_N + 64 * half + 16 * ch2, rr[0]);
                    tc::tmem_ld16(tbase + lane_base + (2 + sl) * TC_N + 64 * half + 16 * ch2 + 16, rr[1]);
                    tc::tmem_ld_wait();
#pragma unroll
                    for (int hh = 0; hh < 2; hh++) {
                        const int k2_0 = 32 * half + 8 * (ch2 + hh);
#pragma unroll
                        for (int q = 0; q < 8; q++) {
                            const int t = idx + 64 * (k2_0 + q);
                            if (z < K && t < L && r0 + t < nb) {
                                const float re = __uint_as_float(rr[hh][2 * q]), im = __uint_as_float(rr[hh][2 * q + 1]);
                                prow[64 * (k2_0 + q)] = Ops::out(re * re + im * im, us);
                            }
                        }
                    }
                }
                tc::fence_before_thread_sync();
                mbar_arrive(&bars->d2_free[sl]);
            }
        }
    }
    tc::fence_before_thread_sync();
    __syncthreads();
    if (tid == 0 && *abort_flag) atomicOr(status, FDAS_DEV_TIMEOUT);
    if (warp == 0) {
        tc::fence_after_thread_sync();
        tc::tmem_dealloc(tbase, WS_TMEM_COLS);
    }
}

// ---------------------------------------------------------------------------------------
// Compensated split-BF16 variant (accuracy recovery): every operand v is carried as
// v_hi + v_lo with v_hi = bf16(v), v_lo = bf16(v - v_hi) (about 16 significant bits), and each
// product as a_hi b_hi + a_lo b_hi + a_hi b_lo (the a_lo b_lo term, ~2^-18 relative, is
// dropped): three MMAs per K step, FP32 accumulation in TMEM.  Inputs are the FP32 segment
// spectra and the FP32 templates; the plane is stored in FP32.  Same transposed two-stage
// DFT as above, one item at a time per CTA (synchronous), 8 warps.
constexpr int SP_THREADS = 256;
constexpr uint32_t SP_OFF_FHI = 0;
constexpr uint32_t SP_OFF_FLO = TILE_BYTES;
constexpr uint32_t SP_OFF_AHI = 2 * TILE_BYTES;                      // A tiles (B1 layout / A2 layout)
constexpr uint32_t SP_TILE = B_TILE > A2_TILE ? B_TILE : A2_TILE;
constexpr uint32_t SP_OFF_ALO = SP_OFF_AHI + SP_TILE;
constexpr uint32_t SP_OFF_BAR = SP_OFF_ALO + SP_TILE;
constexpr uint32_t SP_SMEM = SP_OFF_BAR + 64;

__device__ __forceinline__ void split_bf16x2(float re, float im, uint32_t &hi, uint32_t &lo) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(re, im);
    const float2 hf = __bfloat1622float2(h);
    const __nv_bfloat162 l = __floats2bfloat162_rn(re - hf.x, im - hf.y);
    hi = *reinterpret_cast<const uint32_t *>(&h);
    lo = *reinterpret_cast<const uint32_t *>(&l);
}

__global__ void __launch_bounds__(SP_THREADS, 1) k3_plane_tc_split(const float2 *__restrict__ Y,
                                                                   const float2 *__restrict__ G,
                                                                   const uint4 *__restrict__ Fhi_img,
                                                                   const uint4 *__restrict__ Flo_img,
                                                                   const float2 *__restrict__ tw,
                                                                   float *__restrict__ plane, int K, int64_t nb, int L,
                                                                   int64_t n_items, int n_groups, int64_t items_per_cta,
                                                                   int32_t *__restrict__ status) {
    extern __shared__ __align__(1024) unsigned char smem[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + SP_OFF_BAR);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(smem + SP_OFF_BAR + 16);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 0) {
        tc::tmem_alloc(tslot, TC_N);
        tc::tmem_relinquish();
    }
    if (tid == 0) tc::mbar_init(bar, 1);
    for (int i = tid; i < (int)(TILE_BYTES / 16); i += SP_THREADS) {
        reinterpret_cast<uint4 *>(smem + SP_OFF_FHI)[i] = __ldg(Fhi_img + i);
        reinterpret_cast<uint4 *>(smem + SP_OFF_FLO)[i] = __ldg(Flo_img + i);
    }
    tc::fence_proxy_async_smem();
    tc::fence_before_thread_sync();
    __syncthreads();
    tc::fence_after_thread_sync();
    const uint32_t tD = *tslot;
    const uint32_t idesc = tc::idesc_bf16_f32(TC_M, TC_N);
    const uint32_t fhi = tc::smem_u32(smem + SP_OFF_FHI), flo = tc::smem_u32(smem + SP_OFF_FLO);
    const uint32_t ahi = tc::smem_u32(smem + SP_OFF_AHI), alo = tc::smem_u32(smem + SP_OFF_ALO);
    unsigned char *sAhi = smem + SP_OFF_AHI, *sAlo = smem + SP_OFF_ALO;
    const int quad = warp & 3, half = warp >> 2;
    const int lrow = 32 * quad + lane, zl_e = lrow >> 6, idx = lrow & 63;
    const uint32_t lane_base = (uint32_t)(32 * quad) << 16;
    uint32_t phase = 0;
    bool ok = true;

    auto mma3 = [&](uint32_t a_hi, uint32_t a_lo, uint32_t albo, uint32_t asbo) {
#pragma unroll 1
        for (int s = 0; s < TC_K / 16; s++) {
            const uint64_t dh = tc::smem_desc(a_hi + s * 2 * albo, albo, asbo);
            const uint64_t dl = tc::smem_desc(a_lo + s * 2 * albo, albo, asbo);
            const uint64_t bh = tc::smem_desc(fhi + s * 2 * F_LBO, F_LBO, F_SBO);
            const uint64_t bl = tc::smem_desc(flo + s * 2 * F_LBO, F_LBO, F_SBO);
            tc::mma_bf16(tD, dh, bh, idesc, s > 0 ? 1u : 0u);
            tc::mma_bf16(tD, dl, bh, idesc, 1u);
            tc::mma_bf16(tD, dh, bl, idesc, 1u);
        }
        tc::mma_commit(bar);
    };

    const int64_t it0 = (int64_t)blockIdx.x * items_per_cta;
    const int64_t it1 = min(n_items, it0 + items_per_cta);
    for (int64_t it = it0; it < it1 && ok; it++) {
        const int64_t j = it / n_groups;
        const int z0 = (int)(it % n_groups) * TC_G;
        // ---- x = conj(Yhat_j) G_z in FP32, split, as the stage-1 A tile (B1 layout)
        {
            const int n2q = tid & 15, n1q = tid >> 4;
            const float2 *Yj = Y + j * TC_S_BF16;
#pragma unroll
            for (int zl = 0; zl < TC_G; zl++) {
                const int z = z0 + zl;
                const float2 *Gz = G + (int64_t)(z < K ? z : 0) * TC_S_BF16;
                uint32_t wh[4][4], wl[4][4];
#pragma unroll
                for (int q = 0; q < 4; q++) {
#pragma unroll
                    for (int e = 0; e < 4; e++) {
                        const int n = 64 * (4 * n1q + q) + 4 * n2q + e;
                        const float2 y = __ldg(Yj + n);
                        const float2 g = z < K ? __ldg(Gz + n) : make_float2(0.f, 0.f);
                        split_bf16x2(y.x * g.x + y.y * g.y, y.x * g.y - y.y * g.x, wh[e][q], wl[e][q]);
                    }
                }
#pragma unroll
                for (int e = 0; e < 4; e++) {
                    const int c = zl * TC_R + 4 * n2q + e;
                    const uint32_t off = tc::kmajor_offset_strided(B_SBO, B_LBO, c, 8 * n1q);
                    *reinterpret_cast<uint4 *>(sAhi + off) = make_uint4(wh[e][0], wh[e][1], wh[e][2], wh[e][3]);
                    *reinterpret_cast<uint4 *>(sAlo + off) = make_uint4(wl[e][0], wl[e][1], wl[e][2], wl[e][3]);
                }
            }
        }
        tc::fence_proxy_async_smem();
        tc::fence_before_thread_sync();
        __syncthreads();
        tc::fence_after_thread_sync();
        if (tid == 0) mma3(ahi, alo, B_LBO, B_SBO);
        ok = __syncthreads_and(tc::mbar_wait_bounded(bar, phase, WAIT_CYCLES));
        phase ^= 1;
        if (!ok) break;
        tc::fence_after_thread_sync();
        // ---- twiddle, split, as the stage-2 A tile (A2 layout); row (z, k1), K (n2, s)
#pragma unroll 1
        for (int ch = 0; ch < 4; ch++) {
            uint32_t rr[16];
            tc::tmem_ld16(tD + lane_base + 64 * half + 16 * ch, rr);
            tc::tmem_ld_wait();
#pragma unroll
            for (int q = 0; q < 8; q++) {
                const int k1 = 32 * half + 8 * ch + q;
                const float2 t = __ldg(tw + idx * TC_R + k1);
                const float re = __uint_as_float(rr[2 * q]), im = __uint_as_float(rr[2 * q + 1]);
                uint32_t h, l;
                split_bf16x2(re * t.x - im * t.y, re * t.y + im * t.x, h, l);
                const uint32_t off = tc::kmajor_offset_strided(A2_SBO, A2_LBO, zl_e * TC_R + k1, 2 * idx);
                *reinterpret_cast<uint32_t *>(sAhi + off) = h;
                *reinterpret_cast<uint32_t *>(sAlo + off) = l;
            }
        }
        tc::fence_proxy_async_smem();
        tc::fence_before_thread_sync();
        __syncthreads();
        tc::fence_after_thread_sync();
        if (tid == 0) mma3(ahi, alo, A2_LBO, A2_SBO);
        ok = __syncthreads_and(tc::mbar_wait_bounded(bar, phase, WAIT_CYCLES));
        phase ^= 1;
        if (!ok) break;
        tc::fence_after_thread_sync();
        // ---- |X|^2 -> FP32 plane; thread row (z, k1), columns (k2, p)
        {
            const int z = z0 + zl_e;
            const int64_t r0 = j * L;
#pragma unroll 1
            for (int ch = 0; ch < 4; ch++) {
                uint32_t rr[16];
                tc::tmem_ld16(tD + lane_base + 64 * half + 16 * ch, rr);
                tc::tmem_ld_wait();
#pragma unroll
                for (int q = 0; q < 8; q++) {
                    const int k2 = 32 * half + 8 * ch + q;
                    const int t = idx + 64 * k2;
                    if (z < K && t < L && r0 + t < nb) {
                        const float re = __uint_as_float(rr[2 * q]), im = __uint_as_float(rr[2 * q + 1]);
                        plane[(int64_t)z * nb + r0 + t] = re * re + im * im;
                    }
                }
            }
        }
        tc::fence_before_thread_sync();
        __syncthreads();
    }
    if (!ok) {
        if (tid == 0) atomicOr(status, FDAS_DEV_TIMEOUT);
        tc::mbar_wait_bounded(bar, phase ^ 1, WAIT_CYCLES);   // the MMAs still in flight
    }
    tc::fence_before_thread_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tD, TC_N);
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
    std::vector<uint16_t> img(TC_M * TC_K, 0), img_lo(TC_M * TC_K, 0), img_h(TC_M * TC_K, 0);
    for (int k = 0; k < TC_R; k++)
        for (int n = 0; n < TC_R; n++) {
            const int e = (k * n) % TC_R;
            double f = 2.0 * e / TC_R;
            if (f > 1.0) f -= 2.0;
            const double wr = std::cos(M_PI * f), wi = -std::sin(M_PI * f);
            const float v[2][2] = {{(float)wr, (float)-wi}, {(float)wi, (float)wr}};
            const double vd[2][2] = {{wr, -wi}, {wi, wr}};
            for (int pr = 0; pr < 2; pr++)
                for (int sg = 0; sg < 2; sg++) {
                    const uint32_t o = tc::kmajor_offset(TC_M, 2 * k + pr, 2 * n + sg) / 2;
                    img[o] = host_bf16(v[pr][sg]);
                    uint32_t hb = (uint32_t)img[o] << 16;
                    float hf;
                    std::memcpy(&hf, &hb, 4);
                    img_lo[o] = host_bf16((float)(vd[pr][sg] - (double)hf));
                    const __half h = __float2half_rn(v[pr][sg]);
                    std::memcpy(&img_h[o], &h, 2);
                }
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
        e = cudaMemcpyAsync(static_cast<char *>(p.d_tcF) + img.size() * 2, img_lo.data(), img_lo.size() * 2,
                            cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(p.d_tcTw, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && p.d_tcFh)
        e = cudaMemcpyAsync(p.d_tcFh, img_h.data(), img_h.size() * 2, cudaMemcpyHostToDevice, st);
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
    e = cudaFuncSetAttribute(k3_plane_tc<OpsBF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)WS_SMEM);
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
    const int64_t ctas = std::min<int64_t>(n_items, (int64_t)sms);     // one persistent CTA per SM
    const int64_t per = (n_items + ctas - 1) / ctas;
    const int64_t grid = (n_items + per - 1) / per;
    p.prof.begin(FDAS_STAGE_CORRELATE, st);
    k3_plane_tc<OpsBF16><<<(unsigned)grid, WS_THREADS, WS_SMEM, st>>>(
        Y, p.d_Gbf, reinterpret_cast<const uint4 *>(p.d_tcF), p.d_tcTw, d_plane, p.K, p.nb, p.L, n_items, n_groups,
        per, nullptr, p.d_status);
    p.prof.end(FDAS_STAGE_CORRELATE, st);
    p.prof.launches += 2;
    return cudaGetLastError();
}

// FP16-scaled ablation: scaled FP16 segment spectra, the FP16 bank (S G) and DFT image, FP32 plane.
cudaError_t launch_plane_f16(const Plan &p, const float2 *d_x, const float *d_scale, char *ws, float *d_plane,
                             cudaStream_t st) {
    if (p.S != TC_S_BF16 || !p.d_Gh || !p.d_tcFh) return cudaErrorInvalidValue;
    __half2 *Y = reinterpret_cast<__half2 *>(ws + p.ws_y);
    float *unscale = reinterpret_cast<float *>(ws + p.ws_segscale);
    const size_t smem2 = sizeof(float2) * fft_smem_entries(TC_S_BF16);
    cudaError_t e = cudaFuncSetAttribute(k2_segments_f16, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k3_plane_tc<OpsF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)WS_SMEM);
    if (e != cudaSuccess) return e;
    p.prof.begin(FDAS_STAGE_SEGMENTS, st);
    k2_segments_f16<<<(unsigned)p.n_seg, TC_S_BF16 / 32, smem2, st>>>(d_x, d_scale, p.d_tw, Y, unscale,
                                                                     (float)TC_S_BF16, p.nb, p.L, p.m / 2);
    p.prof.end(FDAS_STAGE_SEGMENTS, st);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int n_groups = (p.K + TC_G - 1) / TC_G;
    const int64_t n_items = p.n_seg * n_groups;
    int sms = 152;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p.device >= 0 ? p.device : 0);
    const int64_t ctas = std::min<int64_t>(n_items, (int64_t)sms);
    const int64_t per = (n_items + ctas - 1) / ctas;
    const int64_t grid = (n_items + per - 1) / per;
    p.prof.begin(FDAS_STAGE_CORRELATE, st);
    k3_plane_tc<OpsF16><<<(unsigned)grid, WS_THREADS, WS_SMEM, st>>>(
        Y, p.d_Gh, reinterpret_cast<const uint4 *>(p.d_tcFh), p.d_tcTw, d_plane, p.K, p.nb, p.L, n_items, n_groups,
        per, unscale, p.d_status);
    p.prof.end(FDAS_STAGE_CORRELATE, st);
    p.prof.launches += 2;
    return cudaGetLastError();
}

}  // namespace fdas

namespace fdas {
cudaError_t launch_plane_fp32_scratch(const Plan &p, const float2 *d_x, const float *d_scale, float2 *d_yhat,
                                      float *d_plane, cudaStream_t st);
cudaError_t launch_plane_split(const Plan &p, const float2 *d_x, const float *d_scale, char *ws, float *d_plane,
                               cudaStream_t st) {
    if (p.S != TC_S_BF16) return cudaErrorInvalidValue;
    float2 *Y = reinterpret_cast<float2 *>(ws + p.ws_y);
    // FP32 segment spectra (4096-bin CUDA-core block FFT), then the compensated tensor stages
    cudaError_t e = launch_segments_fp32(p, d_x, d_scale, Y, st);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k3_plane_tc_split, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SP_SMEM);
    if (e != cudaSuccess) return e;
    const int n_groups = (p.K + TC_G - 1) / TC_G;
    const int64_t n_items = p.n_seg * n_groups;
    int sms = 152;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p.device >= 0 ? p.device : 0);
    const int64_t ctas = std::min<int64_t>(n_items, (int64_t)sms * (p.tune_cta_per_sm > 0 ? p.tune_cta_per_sm : 1));
    const int64_t per = (n_items + ctas - 1) / ctas;
    const int64_t grid = (n_items + per - 1) / per;
    const uint4 *F = reinterpret_cast<const uint4 *>(p.d_tcF);
    p.prof.begin(FDAS_STAGE_CORRELATE, st);
    k3_plane_tc_split<<<(unsigned)grid, SP_THREADS, SP_SMEM, st>>>(Y, p.d_G, F, F + TILE_BYTES / 16, p.d_tcTw,
                                                                   d_plane, p.K, p.nb, p.L, n_items, n_groups, per,
                                                                   p.d_status);
    p.prof.end(FDAS_STAGE_CORRELATE, st);
    p.prof.launches += 1;
    return cudaGetLastError();
}
}  // namespace fdas
