// K3, direct form (FDAS_BF16_DIRECT): the correlation of the spectrum with the templates computed
// straight from its definition, P(r, z) = |sum_{q=-m/2}^{m/2-1} Xhat_{r+q} conj(T_z(q))|^2 (the
// linear correlation that overlap-save reaches, Sec. 2.1), as one real GEMM per block of bins on
// the tensor cores: no segment FFTs, no twiddles.  8 m flops per cell against the DFT path's
// ~1100, so it pays for short templates and is a cross-check of the DFT path.
//
// GEMM: D[r, (p, z)] = sum_{(q, s)} A[r, (q, s)] B[(p, z), (q, s)] with
//   A[r, (q, s)] = component s of Xhat_{r+q-m/2} (BF16; the Hankel matrix of the spectrum),
//   B[(0, z), (q, 0)] = Re T,  B[(0, z), (q, 1)] = Im T,  B[(1, z), (q, 0)] = -Im T,  B[(1, z), (q, 1)] = Re T,
// so D[r, (0, z)] + i D[r, (1, z)] = sum_q Xhat_{r+q-m/2} conj(T_z(q)).  B holds the unit-norm taps
// of all K templates (rows p * Kpad + z, zero beyond K), rounded once to BF16, in shared memory.
//
// The Hankel operand needs no copy per row: rows r = r0 + 4 a + b (b = 0..3 fixed per MMA) are
// 16 bytes apart in the packed spectrum, which is exactly the K-major no-swizzle layout with
// 16-byte rows (core matrices 128 B apart along M, 16 B along K).  Each 512-bin tile keeps four
// copies of its spectrum window in shared memory, shifted by b words so every descriptor starts
// on a 16-byte boundary; the four MMA sets of a tile cover its 512 bins.
//
// One persistent CTA per SM (10 warps): warp 0 issues the MMAs (converged, elect.sync), warp 1
// copies the windows, warps 2-9 read the accumulators (TMEM lanes = a, columns = (p, z)), form
// |.|^2 and store the BF16 plane.  Two accumulator slots in TMEM, two window slots in shared
// memory, every mbarrier wait bounded (timeout -> FDAS_DEV_TIMEOUT, MMAs drained, TMEM freed).
#include <cuda_fp8.h>

#include "fdas_internal.cuh"
#include "tc_sm100.cuh"

namespace fdas {

namespace {

constexpr int DT = 512;                          // bins per tile (4 sets x 128 rows)
constexpr int D_WARPS = 10;
constexpr int D_EPI0 = 2;                        // first epilogue warp
constexpr long long D_WAIT = 4000000000LL;       // about 2 s at 2 GHz
constexpr uint32_t D_MIN_SMEM = 120 * 1024;      // keeps one CTA (and one TMEM allocation) per SM

struct DBars {
    uint64_t w_full[2], w_free[2], d_full[2], d_free[2], drain;
};

__device__ __forceinline__ bool d_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag) {
    if (tc::mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!tc::mbar_try_wait(bar, parity)) {
        if (*abort_flag) return false;
        if (clock64() - t0 > D_WAIT) {
            *abort_flag = 1;
            return false;
        }
    }
    return true;
}

__device__ __forceinline__ void d_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void tmem_ld4(uint32_t taddr, uint32_t (&r)[4]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(taddr));
}

// Xb[k] = Xhat[k - m/2] as a BF16 pair (zero outside the spectrum), k < n_out.
__global__ void k3d_pack(const float2 *__restrict__ X, const float *__restrict__ scale_ptr, uint32_t *__restrict__ Xb,
                         int64_t nb, int half_m, int64_t n_out) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_out) return;
    const float sc = scale_ptr ? __ldg(scale_ptr) : 1.0f;
    const int64_t s = k - half_m;
    float2 v = make_float2(0.f, 0.f);
    if (s >= 0 && s < nb) v = __ldg(X + s);
    const __nv_bfloat162 h = __floats2bfloat162_rn(v.x * sc, v.y * sc);
    Xb[k] = *reinterpret_cast<const uint32_t *>(&h);
}

__global__ void __launch_bounds__(D_WARPS * 32, 1) k3_plane_direct(const uint32_t *__restrict__ Xb,
                                                                   const uint4 *__restrict__ Bimg,
                                                                   __nv_bfloat16 *__restrict__ plane, int K, int Kpad,
                                                                   int m, int64_t nb, int64_t n_tiles,
                                                                   int64_t tiles_per_cta, uint32_t tmem_cols,
                                                                   uint8_t *__restrict__ l1flag, int64_t chunks1,
                                                                   float thr1, int32_t *__restrict__ status) {
    extern __shared__ __align__(1024) unsigned char smem[];
    const int N = 2 * Kpad, KD = 2 * m, WW = DT + m;
    const uint32_t b_bytes = (uint32_t)N * KD * 2;
    unsigned char *sB = smem;
    uint32_t *sW = reinterpret_cast<uint32_t *>(smem + b_bytes);                  // [2 slots][4 copies][WW]
    DBars *bars = reinterpret_cast<DBars *>(smem + b_bytes + 2u * 4u * WW * 4u);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tslot + 2);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (warp == 0) {
        tc::tmem_alloc(tslot, tmem_cols);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        for (int s = 0; s < 2; s++) {
            tc::mbar_init(&bars->w_full[s], 32);
            tc::mbar_init(&bars->w_free[s], 1);
            tc::mbar_init(&bars->d_full[s], 1);
            tc::mbar_init(&bars->d_free[s], 256);
        }
        tc::mbar_init(&bars->drain, 1);
        *abort_flag = 0;
    }
    for (uint32_t i = tid; i < b_bytes / 16; i += D_WARPS * 32) reinterpret_cast<uint4 *>(sB)[i] = __ldg(Bimg + i);
    tc::fence_proxy_async_smem();
    tc::fence_before_thread_sync();
    __syncthreads();
    tc::fence_after_thread_sync();

    const uint32_t tbase = *tslot;
    const int64_t t0 = (int64_t)blockIdx.x * tiles_per_cta;
    const int64_t t1 = min(n_tiles, t0 + tiles_per_cta);
    const int64_t n_my = t1 - t0;

    if (warp == 0) {
        // ---------------------------------------------------------------- MMA issuer
        if (n_my > 0) {
            auto wait = [&](uint64_t *bar, uint32_t parity) {
                return __shfl_sync(0xffffffffu, (int)d_wait(bar, parity, abort_flag), 0) != 0;
            };
            const uint32_t id = tc::idesc_bf16_f32(128, (uint32_t)N);
            const uint64_t bdesc = tc::smem_desc(tc::smem_u32(sB), (uint32_t)N * 16, 128);
            const uint64_t wdesc = tc::smem_desc(tc::smem_u32(sW), 16, 128);   // Hankel rows 16 B apart
            bool ok = true;
            for (int64_t k = 0; k < n_my && ok; k++) {
                ok = wait(&bars->w_full[k & 1], (uint32_t)((k >> 1) & 1));
                if (!ok) break;
                tc::fence_after_thread_sync();
                for (int b = 0; b < 4 && ok; b++) {
                    const int64_t u = 4 * k + b;                                   // set counter
                    const int sl = (int)(u & 1);
                    if (u >= 2) ok = wait(&bars->d_free[sl], (uint32_t)(((u - 2) >> 1) & 1));
                    if (!ok) break;
                    tc::fence_after_thread_sync();
                    const uint64_t a = wdesc + (uint64_t)((((k & 1) * 4 + b) * WW * 4) >> 4);
                    for (int s = 0; s < KD / 16; s++)                              // 16-byte units
                        tc::mma_bf16_warp(tbase + (uint32_t)sl * N, a + (uint64_t)(2 * s),
                                          bdesc + (uint64_t)(s * 2 * N), id, s > 0 ? 1u : 0u);
                    tc::mma_commit_warp(&bars->d_full[sl]);
                }
                tc::mma_commit_warp(&bars->w_free[k & 1]);
            }
            tc::mma_commit_warp(&bars->drain);
            tc::mbar_wait_bounded(&bars->drain, 0, D_WAIT);
        }
        __syncwarp();
    } else if (warp == 1) {
        // ---------------------------------------------------------------- window copies
        // copy b of slot s holds Xb[r0 + b + j], j < WW (the rows r0 + 4 a + b, a < 128, read
        // Xb[r0 + 4 a + b + q], q < m)
        for (int64_t k = 0; k < n_my; k++) {
            if (k >= 2 && !d_wait(&bars->w_free[k & 1], (uint32_t)(((k - 2) >> 1) & 1), abort_flag)) break;
            const int64_t r0 = (t0 + k) * DT;
            uint32_t *dst = sW + (size_t)(k & 1) * 4 * WW;
#pragma unroll 1
            for (int b = 0; b < 4; b++)
                for (int j = lane; j < WW; j += 32) dst[b * WW + j] = __ldg(Xb + r0 + b + j);
            tc::fence_proxy_async_smem();
            d_arrive(&bars->w_full[k & 1]);
        }
    } else {
        // ---------------------------------------------------------------- epilogue
        // thread -> TMEM lane a (row r = r0 + 4 a + b), templates z in [h Kh, h Kh + Kh)
        const int quad = warp & 3, h = (warp - D_EPI0) >> 2;
        const int a = 32 * quad + lane, Kh = Kpad / 2;
        const uint32_t lane_base = (uint32_t)(32 * quad) << 16;
        for (int64_t k = 0; k < n_my; k++) {
            const int64_t r0 = (t0 + k) * DT;
            bool ok = true;
            for (int b = 0; b < 4; b++) {
                const int64_t u = 4 * k + b;
                const int sl = (int)(u & 1);
                if (!d_wait(&bars->d_full[sl], (uint32_t)((u >> 1) & 1), abort_flag)) {
                    ok = false;
                    break;
                }
                tc::fence_after_thread_sync();
                const int64_t r = r0 + 4 * a + b;
                const bool in = r < nb;
                const uint32_t col = tbase + lane_base + (uint32_t)sl * N;
                for (int z0 = h * Kh; z0 < h * Kh + Kh; z0 += 4) {
                    uint32_t re[4], im[4];
                    tmem_ld4(col + z0, re);
                    tmem_ld4(col + Kpad + z0, im);
                    tc::tmem_ld_wait();
                    if (z0 + 4 >= h * Kh + Kh) {                 // the slot's last read: release it
                        tc::fence_before_thread_sync();
                        d_arrive(&bars->d_free[sl]);
                    }
                    if (in) {
                        float vs[4];
#pragma unroll
                        for (int e = 0; e < 4; e++) {
                            const int z = z0 + e;
                            vs[e] = -INFINITY;
                            if (z < K) {
                                const float xr = __uint_as_float(re[e]), xi = __uint_as_float(im[e]);
                                const __nv_bfloat16 v = __float2bfloat16_rn(xr * xr + xi * xi);
                                plane[(int64_t)z * nb + r] = v;
                                vs[e] = __bfloat162float(v);
                            }
                        }
                        // level-1 marks of the units (z, r / 512) whose stored value is above thr1 (rare)
                        if (l1flag != nullptr && fmaxf(fmaxf(vs[0], vs[1]), fmaxf(vs[2], vs[3])) > thr1) {
#pragma unroll
                            for (int e = 0; e < 4; e++)
                                if (vs[e] > thr1) l1flag[(int64_t)(z0 + e) * chunks1 + (r >> 9)] = 1;
                        }
                    }
                }
            }
            if (!ok) break;
        }
    }
    tc::fence_before_thread_sync();
    __syncthreads();
    if (tid == 0 && *abort_flag) atomicOr(status, FDAS_DEV_TIMEOUT);
    if (warp == 0) {
        tc::fence_after_thread_sync();
        tc::tmem_dealloc(tbase, tmem_cols);
    }
}

// ---------------------------------------------------------------------------------------
// FP8 ablation of the direct form (FDAS_FP8_DIRECT): the paper argues BF16 suffices for the
// correlation (Sec. 3, judged by Eq. perc_diff); this path takes one step further down, to E4M3
// operands (3 mantissa bits) with power-of-two scales -- per 1024-bin tile for the spectrum
// (largest |Re| or |Im| of the tile's window brought into [224, 448]) and per template for the
// taps -- kind::f8f6f4 MMAs with FP32 accumulation, and an FP32 plane times 1 / (s_t sigma_z)^2.
// Inside a search the epilogue also marks the 512-bin units holding a power above thr[0].
//
// A complex E4M3 pair is 2 bytes, so the Hankel rows 16 bytes apart are r = r0 + 8 a + b: a tile
// is 1024 bins in 8 sets b of 128 rows, and keeps 8 shifted copies of its window.  A lane of the
// accumulator thus holds bins 8 apart; an FP32 plane written set by set would touch every 32-byte
// sector eight times.  Instead the templates go in groups of 32 (N = 64: Re and Im rows), and the
// eight sets of one group sit in eight TMEM slots of 64 columns (all 512): the epilogue drains
// slot b into registers and frees it at once, and after the eighth set every thread holds eight
// consecutive bins per template -- one whole sector, written with two 16-byte stores.
//
// Warp 0 issues the MMAs, warp 1 stages the FP32 spectrum window of the next tile in shared
// memory with one bulk copy (cp.async.bulk, completion on an mbarrier), takes its maximum and
// writes the 8 rounded copies, warps 2-9 drain the slots (two warps per TMEM lane quarter, 16
// templates each) and store the plane.  Every wait is bounded (FDAS_DEV_TIMEOUT), copies in
// flight are awaited and TMEM is freed before exit.
constexpr int DT8 = 1024;
constexpr int F8_TPG = 32;                       // templates per group (N = 64)
constexpr int F8_N = 2 * F8_TPG;

struct DBars8 {
    uint64_t w_full[2], w_free[2], raw_full[2], s_full[4], d_full[8], d_free[8], drain;
};

__device__ __forceinline__ float e4m3_scale(float M) {       // largest 2^k with M 2^k <= 448
    if (!(M > 0.f)) return 1.f;
    int E;
    const float f = frexpf(M, &E);
    return ldexpf(1.f, (f <= 0.875f ? 9 : 8) - E);
}

__device__ __forceinline__ uint16_t e4m3x2(float re, float im) {
    return (uint16_t)__nv_cvt_float2_to_fp8x2(make_float2(re, im), __NV_SATFINITE, __NV_E4M3);
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tc::smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// Untiled bulk copy global -> shared; both addresses 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     tc::smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(tc::smem_u32(bar))
                 : "memory");
}

__global__ void __launch_bounds__(D_WARPS * 32, 1) k3_plane_direct_f8(const float2 *__restrict__ X,
                                                                      const float *__restrict__ scale_ptr,
                                                                      const uint4 *__restrict__ Bimg,
                                                                      const float *__restrict__ tsig,
                                                                      float *__restrict__ plane, int K, int n_groups, int m,
                                                                      int64_t nb, int64_t n_tiles, int64_t tiles_per_cta,
                                                                      uint8_t *__restrict__ l1flag, int64_t chunks1,
                                                                      float thr1, int32_t *__restrict__ status) {
    extern __shared__ __align__(1024) unsigned char smem[];
    const int WW = DT8 + m, WL = WW + 8;                           // window copy / raw window (bins)
    const uint32_t b_bytes = (uint32_t)n_groups * F8_N * 2 * m;
    unsigned char *sB = smem;
    uint16_t *sW = reinterpret_cast<uint16_t *>(smem + b_bytes);               // [2 slots][8 copies][WW]
    float2 *sRaw = reinterpret_cast<float2 *>(smem + b_bytes + 32u * WW);      // [2 slots][WL]
    // 1 / s_t^2 of tile k at [k % 4], published by s_full[k % 4]: entry k % 4 is rewritten for tile
    // k + 4 only after the MMAs of tile k + 2 are done, which needs the epilogue past tile k + 1
    float *s_inv2 = reinterpret_cast<float *>(sRaw + 2 * WL);
    DBars8 *bars = reinterpret_cast<DBars8 *>(s_inv2 + 4);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tslot + 2);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (warp == 0) {
        tc::tmem_alloc(tslot, 512);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        for (int s = 0; s < 2; s++) {
            tc::mbar_init(&bars->w_full[s], 32);
            tc::mbar_init(&bars->w_free[s], 1);
            tc::mbar_init(&bars->raw_full[s], 1);
        }
        for (int s = 0; s < 4; s++) tc::mbar_init(&bars->s_full[s], 1);
        for (int s = 0; s < 8; s++) {
            tc::mbar_init(&bars->d_full[s], 1);
            tc::mbar_init(&bars->d_free[s], 256);
        }
        tc::mbar_init(&bars->drain, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (uint32_t i = tid; i < b_bytes / 16; i += D_WARPS * 32) reinterpret_cast<uint4 *>(sB)[i] = __ldg(Bimg + i);
    tc::fence_proxy_async_smem();
    tc::fence_before_thread_sync();
    __syncthreads();
    tc::fence_after_thread_sync();

    const uint32_t tbase = *tslot;
    const int64_t t0 = (int64_t)blockIdx.x * tiles_per_cta;
    const int64_t t1 = min(n_tiles, t0 + tiles_per_cta);
    const int64_t n_my = t1 - t0;
    const int KD = 2 * m;                                          // bytes of K per row

    if (warp == 0) {
        // ------------------------------------------------------------------ MMA issuer
        if (n_my > 0) {
            auto wait = [&](uint64_t *bar, uint32_t parity) {
                return __shfl_sync(0xffffffffu, (int)d_wait(bar, parity, abort_flag), 0) != 0;
            };
            const uint32_t id = (1u << 4) | ((uint32_t)(F8_N >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);  // F32 D, E4M3
            // B: group g's 64 rows x KD bytes, core matrices 8 rows x 16 bytes, K-direction stride 1 KB
            const uint64_t bdesc = tc::smem_desc(tc::smem_u32(sB), F8_N * 16, 128);
            const uint64_t wdesc = tc::smem_desc(tc::smem_u32(sW), 16, 128);   // Hankel rows 16 B apart
            bool ok = true;
            for (int64_t k = 0; k < n_my && ok; k++) {
                ok = wait(&bars->w_full[k & 1], (uint32_t)((k >> 1) & 1));
                if (!ok) break;
                tc::fence_after_thread_sync();
                for (int g = 0; g < n_groups && ok; g++) {
                    const int64_t use = k * n_groups + g;                  // use count of every slot
                    const uint64_t bg = bdesc + (uint64_t)((g * F8_N * KD) >> 4);
                    for (int b = 0; b < 8 && ok; b++) {
                        if (use >= 1) ok = wait(&bars->d_free[b], (uint32_t)((use - 1) & 1));
                        if (!ok) break;
                        tc::fence_after_thread_sync();
                        const uint64_t a = wdesc + (uint64_t)((((k & 1) * 8 + b) * WW * 2) >> 4);
                        for (int s = 0; s < KD / 32; s++)                  // 32 bytes of K per MMA
                            tc::mma_f8_warp(tbase + (uint32_t)(b * F8_N), a + (uint64_t)(2 * s),
                                            bg + (uint64_t)(s * 2 * F8_N), id, s > 0 ? 1u : 0u);
                        tc::mma_commit_warp(&bars->d_full[b]);
                    }
                }
                tc::mma_commit_warp(&bars->w_free[k & 1]);
            }
            tc::mma_commit_warp(&bars->drain);
            tc::mbar_wait_bounded(&bars->drain, 0, D_WAIT);
        }
        __syncwarp();
    } else if (warp == 1) {
        // ------------------------------------------------------------------ window producer
        // raw window of tile k: Xhat[w0 + w], w < WL, w0 = 1024 (t0 + k) - m/2; the part inside the
        // spectrum arrives by one bulk copy, the rest reads as zero
        const float gsc = scale_ptr ? __ldg(scale_ptr) : 1.0f;
        auto span = [&](int64_t k, int64_t &lo, int64_t &hi) {
            const int64_t w0 = (t0 + k) * DT8 - m / 2;
            lo = w0 < 0 ? 0 : w0;
            hi = w0 + WL > nb ? nb : w0 + WL;
        };
        auto issue = [&](int64_t k) {
            tc::fence_proxy_async_smem();                             // the slot's earlier reads, then
            __syncwarp();                                             // the bulk copy that overwrites it
            if (lane == 0) {
                int64_t lo, hi;
                span(k, lo, hi);
                const int64_t w0 = (t0 + k) * DT8 - m / 2;
                mbar_expect_tx(&bars->raw_full[k & 1], (uint32_t)((hi - lo) * 8));
                bulk_g2s(sRaw + (k & 1) * WL + (lo - w0), X + lo, (uint32_t)((hi - lo) * 8), &bars->raw_full[k & 1]);
            }
        };
        int64_t issued = 0, landed = 0;
        if (n_my > 0) issue(issued++);
        for (int64_t k = 0; k < n_my; k++) {
            if (issued < n_my) issue(issued++);
            if (!d_wait(&bars->raw_full[k & 1], (uint32_t)((k >> 1) & 1), abort_flag)) break;
            landed = k + 1;
            if (k >= 2 && !d_wait(&bars->w_free[k & 1], (uint32_t)(((k - 2) >> 1) & 1), abort_flag)) break;
            int64_t lo, hi;
            span(k, lo, hi);
            const int64_t w0 = (t0 + k) * DT8 - m / 2;
            const int wlo = (int)(lo - w0), whi = (int)(hi - w0);
            const float2 *raw = sRaw + (k & 1) * WL;
            float M = 0.f;                                             // over the window's WW bins
            for (int w = wlo + lane; w < min(whi, WW); w += 32) {
                const float2 v = raw[w];
                M = fmaxf(M, fmaxf(fabsf(v.x * gsc), fabsf(v.y * gsc)));
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) M = fmaxf(M, __shfl_xor_sync(0xffffffffu, M, o));
            const float st = e4m3_scale(M);
            uint16_t *dst = sW + (size_t)(k & 1) * 8 * WW;
            for (int w = lane; w < WL; w += 32) {
                float2 v = make_float2(0.f, 0.f);
                if (w >= wlo && w < whi) {
                    v = raw[w];
                    v = make_float2(v.x * gsc * st, v.y * gsc * st);
                }
                const uint16_t q = e4m3x2(v.x, v.y);
#pragma unroll
                for (int b = 0; b < 8; b++) {
                    const int j = w - b;
                    if (j >= 0 && j < WW) dst[b * WW + j] = q;
                }
            }
            if (lane == 0) {
                s_inv2[k & 3] = 1.0f / (st * st);
                d_arrive(&bars->s_full[k & 3]);
            }
            tc::fence_proxy_async_smem();
            d_arrive(&bars->w_full[k & 1]);
        }
        // copies still in flight land before the CTA exits
        for (int64_t k = landed; k < issued; k++)
            tc::mbar_wait_bounded(&bars->raw_full[k & 1], (uint32_t)((k >> 1) & 1), D_WAIT);
    } else {
        // ------------------------------------------------------------------ epilogue
        const int quad = warp & 3, h = (warp - D_EPI0) >> 2;
        const int a = 32 * quad + lane;
        const uint32_t lane_base = (uint32_t)(32 * quad) << 16;
        bool ok = true;
        for (int64_t k = 0; k < n_my && ok; k++) {
            if (!d_wait(&bars->s_full[k & 3], (uint32_t)((k >> 2) & 1), abort_flag)) break;
            const float si = s_inv2[k & 3];
            const int64_t r = (t0 + k) * DT8 + 8 * a;                  // this thread's 8 bins r .. r + 7
            for (int g = 0; g < n_groups && ok; g++) {
                const int64_t use = k * n_groups + g;
                float pw[8][16];
#pragma unroll
                for (int b = 0; b < 8; b++) {
                    if (!d_wait(&bars->d_full[b], (uint32_t)(use & 1), abort_flag)) {
                        ok = false;
                        break;
                    }
                    tc::fence_after_thread_sync();
                    uint32_t re[16], im[16];
                    const uint32_t col = tbase + lane_base + (uint32_t)(b * F8_N + 16 * h);
                    tc::tmem_ld16(col, re);
                    tc::tmem_ld16(col + F8_TPG, im);
                    tc::tmem_ld_wait();
                    tc::fence_before_thread_sync();
                    d_arrive(&bars->d_free[b]);
#pragma unroll
                    for (int e = 0; e < 16; e++) {
                        const float xr = __uint_as_float(re[e]), xi = __uint_as_float(im[e]);
                        pw[b][e] = (xr * xr + xi * xi) * si;
                    }
                }
                if (!ok) break;
                if (r + 8 <= nb) {
#pragma unroll
                    for (int e = 0; e < 16; e++) {
                        const int z = g * F8_TPG + 16 * h + e;
                        if (z < K) {
                            const float ts = __ldg(tsig + z);
                            float4 *o = reinterpret_cast<float4 *>(plane + (int64_t)z * nb + r);
                            const float4 lo = make_float4(pw[0][e] * ts, pw[1][e] * ts, pw[2][e] * ts, pw[3][e] * ts);
                            const float4 hi = make_float4(pw[4][e] * ts, pw[5][e] * ts, pw[6][e] * ts, pw[7][e] * ts);
                            o[0] = lo;
                            o[1] = hi;
                            // level-1 mark: the 8 bins lie in one 512-bin unit
                            if (l1flag != nullptr &&
                                fmaxf(fmaxf(fmaxf(lo.x, lo.y), fmaxf(lo.z, lo.w)), fmaxf(fmaxf(hi.x, hi.y), fmaxf(hi.z, hi.w))) > thr1)
                                l1flag[(int64_t)z * chunks1 + (r >> 9)] = 1;
                        }
                    }
                }
            }
        }
    }
    tc::fence_before_thread_sync();
    __syncthreads();
    if (tid == 0 && *abort_flag) atomicOr(status, FDAS_DEV_TIMEOUT);
    if (warp == 0) {
        tc::fence_after_thread_sync();
        tc::tmem_dealloc(tbase, 512);
    }
}

}  // namespace

// FP8 direct path geometry: template groups of 32 and the shared memory (the groups' taps image,
// two slots of 8 window copies, two raw FP32 windows, scales and barriers).
bool direct_geometry_f8(const Plan &p, int *n_groups, uint32_t *smem_bytes) {
    if (p.m % 16 != 0) return false;
    const int G = (p.K + F8_TPG - 1) / F8_TPG;
    const uint64_t WW = DT8 + (uint64_t)p.m, WL = WW + 8;
    const uint64_t need = (uint64_t)G * F8_N * 2 * p.m + 32 * WW + 16 * WL + 16 + sizeof(DBars8) + 16;
    if (need > 227 * 1024) return false;
    if (n_groups) *n_groups = G;
    if (smem_bytes) *smem_bytes = (uint32_t)std::max<uint64_t>(need, D_MIN_SMEM);
    return true;
}

cudaError_t launch_plane_direct_f8(const Plan &p, const float2 *d_x, const float *d_scale, char *ws, float *d_plane,
                                   cudaStream_t st, uint8_t *l1flag) {
    int G = 0;
    uint32_t smem = 0;
    if (!p.d_dimg || !p.d_dsig || !direct_geometry_f8(p, &G, &smem)) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(k3_plane_direct_f8, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    // the bulk copies read the spectrum from 16-byte boundaries: a spectrum on an 8-byte one is
    // first copied to the (256-byte aligned) scratch area
    if ((reinterpret_cast<uintptr_t>(d_x) & 15) != 0) {
        float2 *tmp = reinterpret_cast<float2 *>(ws + p.ws_tmp);
        e = cudaMemcpyAsync(tmp, d_x, sizeof(float2) * (size_t)p.nb, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return e;
        d_x = tmp;
    }
    if (l1flag) {
        e = cudaMemsetAsync(l1flag, 0, (size_t)p.K * (size_t)(p.nb / PEAK_CHUNK), st);
        if (e != cudaSuccess) return e;
    }
    const int64_t n_tiles = (p.nb + DT8 - 1) / DT8;
    int sms = 152;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p.device >= 0 ? p.device : 0);
    const int64_t ctas = std::min<int64_t>(n_tiles, (int64_t)sms);
    const int64_t per = (n_tiles + ctas - 1) / ctas;
    const int64_t grid = (n_tiles + per - 1) / per;
    p.prof.begin(FDAS_STAGE_CORRELATE, st);
    k3_plane_direct_f8<<<(unsigned)grid, D_WARPS * 32, smem, st>>>(d_x, d_scale, reinterpret_cast<const uint4 *>(p.d_dimg),
                                                                   p.d_dsig, d_plane, p.K, G, p.m, p.nb, n_tiles, per,
                                                                   l1flag, p.nb / PEAK_CHUNK, mark_threshold(p), p.d_status);
    p.prof.end(FDAS_STAGE_CORRELATE, st);
    p.prof.launches += 1;
    return cudaGetLastError();
}

// Geometry of the direct path for a plan: padded template count, shared memory, TMEM columns.
bool direct_geometry(const Plan &p, int *Kpad, uint32_t *smem_bytes, uint32_t *tmem_cols) {
    const int kp = (p.K + 7) / 8 * 8;                  // N = 2 Kpad, a multiple of 16
    const int N = 2 * kp;
    if (N > 256 || p.m % 8 != 0) return false;
    const uint64_t need = (uint64_t)N * 2 * p.m * 2 + 2ull * 4 * (DT + p.m) * 4 + sizeof(DBars) + 16;
    if (need > 227 * 1024) return false;
    uint32_t cols = 32;
    while (cols < (uint32_t)(2 * N)) cols <<= 1;
    if (Kpad) *Kpad = kp;
    if (smem_bytes) *smem_bytes = (uint32_t)std::max<uint64_t>(need, D_MIN_SMEM);
    if (tmem_cols) *tmem_cols = cols;
    return true;
}

size_t direct_pack_words(const Plan &p) {
    const int64_t n_tiles = (p.nb + DT - 1) / DT;
    return (size_t)(n_tiles * DT + p.m + 4);
}

cudaError_t launch_plane_direct(const Plan &p, const float2 *d_x, const float *d_scale, char *ws,
                                __nv_bfloat16 *d_plane, cudaStream_t st, uint8_t *l1flag) {
    int Kpad = 0;
    uint32_t smem = 0, cols = 0;
    if (!p.d_dimg || !direct_geometry(p, &Kpad, &smem, &cols)) return cudaErrorInvalidValue;
    uint32_t *Xb = reinterpret_cast<uint32_t *>(ws + p.ws_y);
    const int64_t n_out = (int64_t)direct_pack_words(p);
    p.prof.begin(FDAS_STAGE_SEGMENTS, st);
    k3d_pack<<<(unsigned)((n_out + 255) / 256), 256, 0, st>>>(d_x, d_scale, Xb, p.nb, p.m / 2, n_out);
    p.prof.end(FDAS_STAGE_SEGMENTS, st);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k3_plane_direct, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (l1flag) {
        e = cudaMemsetAsync(l1flag, 0, (size_t)p.K * (size_t)(p.nb / PEAK_CHUNK), st);
        if (e != cudaSuccess) return e;
    }
    const int64_t n_tiles = (p.nb + DT - 1) / DT;
    int sms = 152;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p.device >= 0 ? p.device : 0);
    const int64_t ctas = std::min<int64_t>(n_tiles, (int64_t)sms);
    const int64_t per = (n_tiles + ctas - 1) / ctas;
    const int64_t grid = (n_tiles + per - 1) / per;
    p.prof.begin(FDAS_STAGE_CORRELATE, st);
    k3_plane_direct<<<(unsigned)grid, D_WARPS * 32, smem, st>>>(Xb, reinterpret_cast<const uint4 *>(p.d_dimg), d_plane,
                                                                p.K, Kpad, p.m, p.nb, n_tiles, per, cols, l1flag,
                                                                p.nb / PEAK_CHUNK, mark_threshold(p), p.d_status);
    p.prof.end(FDAS_STAGE_CORRELATE, st);
    p.prof.launches += 2;
    return cudaGetLastError();
}

}  // namespace fdas
