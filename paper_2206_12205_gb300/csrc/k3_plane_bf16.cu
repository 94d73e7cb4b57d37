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

// ---------------------------------------------------------------------------------------
// Warp-specialised persistent kernel (one CTA per SM, 13 warps):
//   warp 0      TMEM allocation; lane 0 issues the MMAs (stage 1 of item i+1 before stage 2 of i)
//   warps 1-8   producer:   B1[slot] = conj(Yhat_j) * G_z, one 4 x 4 (n1, n2) block per thread
//               with all of its 16-byte loads in flight at once
//   warps 9-12  epilogue 1: D1[slot] (TMEM) -> twiddle -> B2[slot]
//   warps 13-16 epilogue 2: D2[slot] (TMEM) -> |.|^2 -> BF16 plane
// Two slots of B1, B2 (shared memory) and D1, D2 (TMEM, 4 x 128 of the 512 columns).
// Hand-offs are mbarriers, one per slot:
//   b1_full  (256 producer arrivals)   s1_done (MMA commit: D1 ready, B1 free)
//   b2_full  (128 epilogue-1 arrivals: B2 ready, D1 drained)
//   s2_done  (MMA commit: D2 ready, B2 free)   d2_free (128 epilogue-2 arrivals: D2 drained)
// The k-th use of a slot waits for phase parity k & 1; every wait is bounded and also gives
// up when another role has aborted.
constexpr int WS_PRODUCERS = 256;                            // warps 1-8
constexpr int WS_E1 = 1 + WS_PRODUCERS / 32;                 // first epilogue-1 warp (9)
constexpr int WS_E2 = WS_E1 + 4;                             // first epilogue-2 warp (13)
constexpr int WS_THREADS = (WS_E2 + 4) * 32;                 // 17 warps
// B tiles: K-major, core matrices 144 B apart along N and 16 x 144 B apart along K
constexpr uint32_t B_SBO = 144, B_LBO = 16 * B_SBO;
constexpr uint32_t B_TILE = 16 * B_LBO;                      // 36 KB (K = 128 = 16 core matrices)
constexpr uint32_t OFF_F = 0;                                // F': dense, 32 KB
constexpr uint32_t OFF_B1 = OFF_F + TILE_BYTES;              // 2 slots
constexpr uint32_t OFF_B2 = OFF_B1 + 2 * B_TILE;             // 2 slots
constexpr uint32_t OFF_TW = OFF_B2 + 2 * B_TILE;             // twiddles, 4096 x float2 = 32 KB
constexpr uint32_t OFF_BAR = OFF_TW + TC_S_BF16 * 8;
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

__global__ void __launch_bounds__(WS_THREADS, 1) k3_plane_tc(const __nv_bfloat162 *__restrict__ Y,
                                                             const __nv_bfloat162 *__restrict__ G,
                                                             const uint4 *__restrict__ Fimg,
                                                             const float2 *__restrict__ tw,
                                                             __nv_bfloat16 *__restrict__ plane, int K, int64_t nb,
                                                             int L, int64_t n_items, int n_groups,
                                                             int64_t items_per_cta, int32_t *__restrict__ status) {
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
            tc::mbar_init(&bars->b2_full[s], 128);
            tc::mbar_init(&bars->s2_done[s], 1);
            tc::mbar_init(&bars->d2_free[s], 128);
        }
        tc::mbar_init(&bars->drain, 1);
        *abort_flag = 0;
    }
    for (int i = tid; i < (int)(TILE_BYTES / 16); i += WS_THREADS)
        reinterpret_cast<uint4 *>(smem + OFF_F)[i] = __ldg(Fimg + i);
    for (int i = tid; i < TC_S_BF16; i += WS_THREADS) sTw[i] = __ldg(tw + i);
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
            const uint32_t idesc = tc::idesc_bf16_f32(TC_M, TC_N);
            const uint32_t aF = tc::smem_u32(smem + OFF_F);
            auto issue = [&](uint32_t dcol, uint32_t bsm) {
#pragma unroll
                for (int s = 0; s < TC_K / 16; s++)
                    tc::mma_bf16(tbase + dcol, tc::smem_desc(aF + s * TC_M * 32, TC_M * 16, 128),
                                 tc::smem_desc(bsm + s * 2 * B_LBO, B_LBO, B_SBO), idesc, s > 0 ? 1u : 0u);
            };
            bool ok = ws_wait(&bars->b1_full[0], 0, abort_flag);
            if (ok) {
                tc::fence_after_thread_sync();
                issue(0 * TC_N, tc::smem_u32(smem + OFF_B1));
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
                    issue(sn * TC_N, tc::smem_u32(smem + OFF_B1 + sn * B_TILE));
                    tc::mma_commit(&bars->s1_done[sn]);
                }
                ok = ws_wait(&bars->b2_full[sl], par, abort_flag);     // B2 ready, D1 drained
                if (ok && k >= 2) ok = ws_wait(&bars->d2_free[sl], par ^ 1u, abort_flag);
                if (!ok) break;
                tc::fence_after_thread_sync();
                issue((2 + sl) * TC_N, tc::smem_u32(smem + OFF_B2 + sl * B_TILE));
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
                        const float2 y = unpack_bf16x2(*reinterpret_cast<const __nv_bfloat162 *>(&ys[e]));
                        const float2 g = unpack_bf16x2(*reinterpret_cast<const __nv_bfloat162 *>(&gs[e]));
                        w[e][q] = pack_bf16x2(y.x * g.x + y.y * g.y, y.x * g.y - y.y * g.x);
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
        const int row = 32 * quad + lane;               // GEMM row (k, p)
        const int kk = row >> 1, rho = row & 1;
        const uint32_t lane_base = (uint32_t)(32 * quad) << 16;
        for (int64_t k = 0; k < n_my; k++) {
            const int64_t it = it0 + k;
            const int sl = (int)(k & 1);
            const uint32_t par = (uint32_t)((k >> 1) & 1);
            if (epi1) {
                if (!ws_wait(&bars->s1_done[sl], par, abort_flag)) break;
                if (k >= 2 && !ws_wait(&bars->s2_done[sl], par ^ 1u, abort_flag)) break;   // B2[sl] free
                tc::fence_after_thread_sync();
                unsigned char *b2 = smem + OFF_B2 + sl * B_TILE;
#pragma unroll 1
                for (int ch2 = 0; ch2 < 8; ch2 += 2) {
                  uint32_t rr2[2][16];
                  tc::tmem_ld16(tbase + lane_base + sl * TC_N + 16 * ch2, rr2[0]);
                  tc::tmem_ld16(tbase + lane_base + sl * TC_N + 16 * ch2 + 16, rr2[1]);
                  tc::tmem_ld_wait();
#pragma unroll
                  for (int hh = 0; hh < 2; hh++) {
                    const int ch = ch2 + hh;
                    const int zl = ch >> 2;
                    float re[8], im[8];
                    pair_exchange(rr2[hh], rho, re, im);
                    const int n2_0 = 16 * (ch & 3) + 8 * rho;
                    const float4 *twp = reinterpret_cast<const float4 *>(sTw + kk * TC_R + n2_0);
                    uint32_t w[8];
#pragma unroll
                    for (int q2 = 0; q2 < 4; q2++) {
                        const float4 t2 = twp[q2];
                        const int q = 2 * q2;
                        w[q] = pack_bf16x2(re[q] * t2.x - im[q] * t2.y, re[q] * t2.y + im[q] * t2.x);
                        w[q + 1] = pack_bf16x2(re[q + 1] * t2.z - im[q + 1] * t2.w, re[q + 1] * t2.w + im[q + 1] * t2.z);
                    }
                    const int c2 = zl * TC_R + kk;
                    *reinterpret_cast<uint4 *>(b2 + tc::kmajor_offset_strided(B_SBO, B_LBO, c2, 2 * n2_0)) =
                        make_uint4(w[0], w[1], w[2], w[3]);
                    *reinterpret_cast<uint4 *>(b2 + tc::kmajor_offset_strided(B_SBO, B_LBO, c2, 2 * n2_0 + 8)) =
                        make_uint4(w[4], w[5], w[6], w[7]);
                  }
                }
                tc::fence_before_thread_sync();
                tc::fence_proxy_async_smem();
                mbar_arrive(&bars->b2_full[sl]);
            } else {
                if (!ws_wait(&bars->s2_done[sl], par, abort_flag)) break;
                tc::fence_after_thread_sync();
                const int64_t j = it / n_groups;
                const int z0 = (int)(it % n_groups) * TC_G;
                const int64_t r0 = j * L;
#pragma unroll 1
                for (int ch2 = 0; ch2 < 8; ch2 += 2) {
                  uint32_t rr2[2][16];
                  tc::tmem_ld16(tbase + lane_base + (2 + sl) * TC_N + 16 * ch2, rr2[0]);
                  tc::tmem_ld16(tbase + lane_base + (2 + sl) * TC_N + 16 * ch2 + 16, rr2[1]);
                  tc::tmem_ld_wait();
#pragma unroll
                  for (int hh = 0; hh < 2; hh++) {
                    const int ch = ch2 + hh;
                    const int zl = ch >> 2;
                    const int z = z0 + zl;
                    float re[8], im[8];
                    pair_exchange(rr2[hh], rho, re, im);
                    const int t = 64 * kk + 16 * (ch & 3) + 8 * rho;
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
    e = cudaFuncSetAttribute(k3_plane_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)WS_SMEM);
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
    k3_plane_tc<<<(unsigned)grid, WS_THREADS, WS_SMEM, st>>>(Y, p.d_Gbf, reinterpret_cast<const uint4 *>(p.d_tcF),
                                                               p.d_tcTw, d_plane, p.K, p.nb, p.L, n_items, n_groups,
                                                               per, p.d_status);
    p.prof.end(FDAS_STAGE_CORRELATE, st);
    p.prof.launches += 2;
    return cudaGetLastError();
}

}  // namespace fdas
