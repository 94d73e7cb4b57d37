// K2 + K3, BF16 path (Sec. 3: the convolution section in bfloat16, the long FFT kept in FP32):
// the overlap-save correlation with the segment FFT's DFT stages run on the tensor cores
// (tcgen05, BF16 operands, FP32 accumulation in TMEM) and a BF16 plane.
//
// Segments are S = 4096 bins long with stride L = 64 * floor((S - m + 1) / 64) (any
// L <= S - m + 1 gives the same plane; a multiple of 64 keeps the stores aligned).
// With x = conj(Yhat_j) * G_z (length S, n = 64 n1 + n2) the plane row segment is
// |X|^2 with the four-step DFT
//     X[k1 + 64 k2] = sum_{n2} W_64^{n2 k2} W_S^{n2 k1} sum_{n1} W_64^{n1 k1} x[64 n1 + n2],
// computed for two templates at a time as two real GEMMs of 128 x 128 x 128 (below) against
// real-ified radix-64 DFT matrices F1 and F2 (each complex entry w as the 2 x 2 block
// [[Re w, -Im w], [Im w, Re w]], rows and columns permuted as described below).
//
// One persistent, warp-specialised CTA per SM walks a contiguous range of (segment, template
// pair) items, segments fastest (item = pair * n_seg + segment, so a CTA keeps one pair's template
// spectra in registers across its items), with producer, MMA and two epilogue roles overlapped
// through TMEM and shared-memory buffers (layout below the helpers).  Every mbarrier wait is bounded; a timeout sets
// FDAS_DEV_TIMEOUT, all roles stop, the issued MMAs drain and the TMEM is released.
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
constexpr uint32_t TILE_BYTES = TC_M * TC_K * 2;  // 32 KB: every 128 x 128 16-bit operand tile
constexpr long long WAIT_CYCLES = 4000000000LL;   // about 2 s at 2 GHz

static_assert(TC_S_BF16 == TC_R * TC_R, "segment length must be 64 x 64");

// Stage-1 operand order (tc_s1_pos): products of its 16-bit pairs are again such pairs, so the
// producer forms conj(Yhat) G with packed arithmetic and no rearrangement and stores the 64 pairs
// of a row as the row's 64 TMEM columns (stage-1 K index 2 c + h = half h of column c).  It is
// also the order in which the segment FFT holds its outputs (thread t: n2 = t mod 64,
// n1 = t / 64 + 2 i).
// The inverse on the K axis: stage-1 K index kk -> (n1, s), s = 0 real part, 1 imaginary part.
__host__ __device__ constexpr int s1_n1(int kk) {
    return ((kk >> 3) & 1) + 8 * (kk >> 4) + 4 * ((kk >> 2) & 1) + 2 * (kk & 1);
}
__host__ __device__ constexpr int s1_s(int kk) { return (kk >> 1) & 1; }

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&h);
}
__device__ __forceinline__ uint32_t pack_f16x2(float lo, float hi) {
    const __half2 h = __floats2half2_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&h);
}

// Operand formats of the tensor stages: BF16 (the paper's Sec. 3 variant, BF16 plane) or FP16 with
// per-segment scaling (the Sec. 3.2 ablation, FP32 plane times the segment's unscale factor).
struct OpsBF16 {
    using V = __nv_bfloat162;
    using Out = __nv_bfloat16;
    static constexpr uint32_t idesc = tc::idesc_bf16_f32(TC_M, TC_N);
    __device__ __forceinline__ static uint32_t pack(float lo, float hi) { return pack_bf16x2(lo, hi); }
    __device__ __forceinline__ static Out out(float pw, float) { return __float2bfloat16_rn(pw); }
    // the stored value as the peak search reads it (BF16 widened exactly)
    __device__ __forceinline__ static float stored(float pw, float) { return __bfloat162float(__float2bfloat16_rn(pw)); }
};
struct OpsF16 {
    using V = __half2;
    using Out = float;
    static constexpr uint32_t idesc = tc::idesc_f16_f32(TC_M, TC_N);
    __device__ __forceinline__ static uint32_t pack(float lo, float hi) { return pack_f16x2(lo, hi); }
    __device__ __forceinline__ static Out out(float pw, float unscale) { return pw * unscale; }
    __device__ __forceinline__ static float stored(float pw, float unscale) { return pw * unscale; }
};

// Segment FFTs (FP32 CUDA-core block FFT), stored as BF16 pairs in the stage-1 order.
// It also clears the plane kernel's unit marks (zero16: n_zero16 16-byte words, or none), which
// saves the plane kernel a separate clearing launch.
__global__ void __launch_bounds__(TC_S_BF16 / 32) k2_segments_bf16(const float2 *__restrict__ X,
                                                                   const float *__restrict__ scale_ptr,
                                                                   const float2 *__restrict__ tw,
                                                                   uint4 *__restrict__ Y, int64_t nb, int L,
                                                                   int half_m, uint4 *__restrict__ zero16,
                                                                   int64_t n_zero16) {
    constexpr int S = TC_S_BF16, T = S / 32;
    extern __shared__ float2 sm[];
    const int t = threadIdx.x;
    const int64_t j = blockIdx.x;
    for (int64_t w = j * T + t; w < n_zero16; w += (int64_t)gridDim.x * T) zero16[w] = make_uint4(0u, 0u, 0u, 0u);
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
    // v[i] = X[t + 128 i]: n2 = t mod 64, n1 = t / 64 + 2 i; chunk 2 c + t / 64 takes v[4c .. 4c+3]
    uint4 *out = Y + j * (S / 4) + (t & 63);
#pragma unroll
    for (int c = 0; c < 8; c++)
        out[(2 * c + (t >> 6)) * 64] =
            make_uint4(pack_bf16x2(v[4 * c].x, v[4 * c + 1].x), pack_bf16x2(v[4 * c].y, v[4 * c + 1].y),
                       pack_bf16x2(v[4 * c + 2].x, v[4 * c + 3].x), pack_bf16x2(v[4 * c + 2].y, v[4 * c + 3].y));
}

// Segment FFTs for the FP16 stages: the segment's largest component |re| or |im| is brought into
// [0.5, 1) by a power of two s_j (exact), the values stored as FP16 pairs in the stage-1 order,
// and the plane's factor 1 / (s_j gscale)^2 (gscale: the template bank's scale) kept per segment.
__global__ void __launch_bounds__(TC_S_BF16 / 32) k2_segments_f16(const float2 *__restrict__ X,
                                                                  const float *__restrict__ scale_ptr,
                                                                  const float2 *__restrict__ tw,
                                                                  uint4 *__restrict__ Y, float *__restrict__ unscale,
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
    uint4 *out = Y + j * (S / 4) + (t & 63);
#pragma unroll
    for (int c = 0; c < 8; c++)
        out[(2 * c + (t >> 6)) * 64] = make_uint4(
            pack_f16x2(v[4 * c].x * sj, v[4 * c + 1].x * sj), pack_f16x2(v[4 * c].y * sj, v[4 * c + 1].y * sj),
            pack_f16x2(v[4 * c + 2].x * sj, v[4 * c + 3].x * sj), pack_f16x2(v[4 * c + 2].y * sj, v[4 * c + 3].y * sj));
    if (t == 0) {
        const float g = sj * gscale;
        unscale[j] = 1.0f / (g * g);
    }
}

// ---------------------------------------------------------------------------------------
// Warp-specialised persistent kernel, one CTA per SM, 28 warps.  Both GEMMs run transposed,
// data as the A operand (M = 128 rows = two templates x 64) and a DFT matrix as B:
//   stage 1  D1[(z,n2), (p,k1)] = A1[(z,n2), K1] . F1^T          A1 = x, in TMEM (K1: stage-1 order)
//   stage 2  D2[(z,k1), (p,k2)] = A2[(z,k1), (s,n2)] . F2^T      A2 = W_S^{n2 k1} D1, shared memory
// Stage-1 rows interleave the two templates within each 32-row TMEM quadrant q: row
// 32 q + 16 z + (n2 mod 16) holds n2 = 16 q + (n2 mod 16), so the two threads of a warp that form
// rows (0, n2) and (1, n2) load the same Yhat words and the warp's loads coalesce.  Stage-2 rows
// are 64 z + k1 (the order epilogue 1 writes A2 in).
// Accumulator columns are ordered (p, k): the 64 real parts, then the 64 imaginary parts, so a
// thread's TMEM row yields 8 consecutive real (or imaginary) parts per 8 columns.  A2 is stored
// MN-major: the 8 consecutive k1 of one (z, n2, s) are one 16-byte row of a core matrix, which is
// what an epilogue-1 thread (one n2, consecutive k1) writes in one store; the tensor core reads the
// transposed operand from it.
//   warp 0       TMEM allocation; issues the stage-1 MMAs
//   warp 1       issues the stage-2 MMAs (warps 2-3 idle: they complete warpgroup 0 for the
//                register hand-over)
//   warps 4-11   producer:   A1[slot] row (z, n2), half of its 64 columns, = conj(Yhat_j) G_z in packed
//                16-bit arithmetic, written with tcgen05.st
//   warps 12-19  epilogue 1: D1[slot] -> W_S^{n2 k1} (FP32, packed pairs) -> A2[slot]; warps 12-15 and
//                16-19 take the two halves of k1
//   warps 20-27  epilogue 2: D2 -> |.|^2 -> plane (halves of k2)
// TMEM (512 columns): three accumulator slots of 128 columns (item k uses slot k mod 3 for D1 and,
// once epilogue 1 has drained it, for D2) and two A1 slots of 64 columns (item k: k mod 2).
// Shared memory: F1, F2 (32 KB each), two A2 slots (32 KB each, item k: k mod 2) and the W_S^{n2 k1} table.
// Hand-offs are mbarriers, each with one signalling and one waiting role:
//   a1_full[2]  producer -> MMA (256 arrivals)        a1_free[2]  MMA commit after stage 1 -> producer
//   d1_full[3]  MMA commit after stage 1 -> epi 1      b2_full[2]  epi 1 -> MMA (256: A2 ready, D1 read)
//   a2_free[2]  MMA commit after stage 2 -> epi 1      d2_full[3]  MMA commit after stage 2 -> epi 2
//   d_free[3]   epi 2 -> MMA (256 arrivals: accumulator slot drained)
// The u-th use of a barrier waits for phase parity u & 1; a role can never be two phases behind
// (the next phase of every barrier depends on the waiting role's own progress).  Every wait is
// bounded and also gives up when another role has aborted.  Epilogue 1 reads the twiddle W_S^{n2 k1}
// from a shared-memory copy of the plan's table, one 16-byte word per pair of consecutive k1.
constexpr int WS_P0 = 4;                                     // first producer warp
constexpr int WS_PRODUCERS = 256;                            // warps 4-11
constexpr int WS_E1 = WS_P0 + WS_PRODUCERS / 32;             // first epilogue-1 warp (12)
constexpr int WS_E2 = WS_E1 + 8;                             // first epilogue-2 warp (20)
constexpr int WS_THREADS = (WS_E2 + 8) * 32;                 // 28 warps = 7 warpgroups
// Registers: 72 a thread at launch (7 warps on each SM sub-partition).  Warpgroup 0 (the MMA
// warps and two idle warps) gives 16 back and epilogue 1 gives 8; the producers (the pair's
// template spectrum held across items) and epilogue 2 (a whole accumulator row half loaded at
// once) take 8 more: 128 x 56 + 256 x 80 + 256 x 64 + 256 x 80 = 896 x 72.
constexpr int REG_LAUNCH = 72, REG_MMA = 56, REG_PROD = 80, REG_E1 = 64, REG_E2 = 80;
static_assert(128 * REG_MMA + 256 * (REG_PROD + REG_E1 + REG_E2) == WS_THREADS * REG_LAUNCH,
              "register split must add up to the launch allocation");
constexpr uint32_t A2_CM = 128, A2_CK = (TC_M / 8) * 128;    // A2 MN-major: core matrices along M, K
constexpr uint32_t F_LBO = TC_M * 16, F_SBO = 128;           // F1, F2: dense K-major
constexpr uint32_t OFF_F1 = 0, OFF_F2 = TILE_BYTES;
constexpr uint32_t OFF_A2 = 2 * TILE_BYTES;                  // 2 slots
constexpr uint32_t OFF_BAR = OFF_A2 + 2 * TILE_BYTES;
// W_S^{n2 k1} for the k1 pairs (2 kp, 2 kp + 1) as float4 {Re, Re, Im, Im} at [kp][n2] (32 KB)
constexpr uint32_t OFF_TWS = OFF_BAR + 256;
constexpr uint32_t WS_SMEM = OFF_TWS + (TC_R / 2) * TC_R * 16;
constexpr uint32_t WS_TMEM_COLS = 512;
constexpr uint32_t COL_A1 = 3 * TC_N;                        // accumulator slots at 0, 128, 256

struct WsBars {
    uint64_t a1_full[2], a1_free[2], d1_full[3], b2_full[2], a2_free[2], d2_full[3], d_free[3], drain[2];
};

__device__ __forceinline__ bool ws_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag) {
    if (tc::mbar_try_wait(bar, parity)) return true;
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

// max(a, b, c) in one instruction (three-input max.f32, sm_100 and later)
__device__ __forceinline__ float fmax3(float a, float b, float c) {
    float d;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

__device__ __forceinline__ float2 u2f2(uint32_t a, uint32_t b) {
    return make_float2(__uint_as_float(a), __uint_as_float(b));
}

template <class Ops>
__global__ void __launch_bounds__(WS_THREADS, 1) k3_plane_tc(const uint4 *__restrict__ Y, const uint4 *__restrict__ G,
                                                             const uint4 *__restrict__ Fimg,
                                                             const float2 *__restrict__ tw,
                                                             typename Ops::Out *__restrict__ plane, int K, int64_t nb,
                                                             int L, int64_t n_items, int n_groups,
                                                             int64_t items_per_cta, const float *__restrict__ unscale,
                                                             uint8_t *__restrict__ l1flag, int64_t chunks1, float thr1,
                                                             int32_t *__restrict__ status) {
    using V = typename Ops::V;
    extern __shared__ __align__(1024) unsigned char smem[];
    WsBars *bars = reinterpret_cast<WsBars *>(smem + OFF_BAR);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(smem + OFF_BAR + sizeof(WsBars));
    volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + OFF_BAR + sizeof(WsBars) + 8);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (warp == 0) {
        tc::tmem_alloc(tslot, WS_TMEM_COLS);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        for (int s = 0; s < 2; s++) {
            tc::mbar_init(&bars->a1_full[s], WS_PRODUCERS);
            tc::mbar_init(&bars->a1_free[s], 1);
            tc::mbar_init(&bars->b2_full[s], 256);
            tc::mbar_init(&bars->a2_free[s], 1);
        }
        for (int s = 0; s < 3; s++) {
            tc::mbar_init(&bars->d1_full[s], 1);
            tc::mbar_init(&bars->d2_full[s], 1);
            tc::mbar_init(&bars->d_free[s], 256);
        }
        tc::mbar_init(&bars->drain[0], 1);
        tc::mbar_init(&bars->drain[1], 1);
        *abort_flag = 0;
    }
    for (int i = tid; i < (int)(2 * TILE_BYTES / 16); i += WS_THREADS)
        reinterpret_cast<uint4 *>(smem + OFF_F1)[i] = __ldg(Fimg + i);
    for (int e = tid; e < (TC_R / 2) * TC_R; e += WS_THREADS) {
        const int kp = e / TC_R, n2 = e % TC_R;
        const float2 a = __ldg(tw + (2 * kp) * TC_R + n2), b = __ldg(tw + (2 * kp + 1) * TC_R + n2);
        reinterpret_cast<float4 *>(smem + OFF_TWS)[e] = make_float4(a.x, b.x, a.y, b.y);
    }
    tc::fence_proxy_async_smem();
    tc::fence_before_thread_sync();
    __syncthreads();
    tc::fence_after_thread_sync();

    const uint32_t tbase = *tslot;
    const int64_t it0 = (int64_t)blockIdx.x * items_per_cta;
    const int64_t it1 = min(n_items, it0 + items_per_cta);
    const int64_t n_my = it1 - it0;
    const int64_t n_seg = n_items / n_groups;           // items are pair * n_seg + segment
    const int quad = warp & 3;                          // TMEM lane quadrant this warp may access
    const int lrow = 32 * quad + lane;                  // TMEM lane = GEMM row
    const int zl = lrow >> 6, idx = lrow & 63;          // stage-2 row: (template in the pair, k1)
    const uint32_t lane_base = (uint32_t)(32 * quad) << 16;

    if (warp < WS_P0) {
        // ---------------------------------------------------------------- MMA issuers
        // Warp 0 issues stage 1, warp 1 stage 2: the tensor pipe queues only a few MMAs, so
        // while one issuer waits on its barriers the other keeps it fed.  Each warp runs its loop
        // (waits included) in converged control flow and one elected lane issues each MMA and
        // commit; a commit covers the MMAs of its own warp.
        asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(REG_MMA));
        if (warp < 2 && n_my > 0) {
            auto wait = [&](uint64_t *bar, uint32_t parity) {
                return __shfl_sync(0xffffffffu, (int)ws_wait(bar, parity, abort_flag), 0) != 0;
            };
            int s3 = 0, u3 = 0;                         // accumulator slot k mod 3 and its use count k / 3
            if (warp == 0) {
                const uint32_t id1 = Ops::idesc;
                const uint64_t f1 = tc::smem_desc(tc::smem_u32(smem + OFF_F1), F_LBO, F_SBO);
                for (int64_t k = 0; k < n_my; k++) {
                    if (!wait(&bars->a1_full[k & 1], (uint32_t)((k >> 1) & 1))) break;
                    if (u3 >= 1 && !wait(&bars->d_free[s3], (uint32_t)((u3 - 1) & 1))) break;
                    tc::fence_after_thread_sync();
                    const uint32_t d = tbase + (uint32_t)s3 * TC_N, a = tbase + COL_A1 + (uint32_t)(k & 1) * (TC_K / 2);
#pragma unroll
                    for (int s = 0; s < TC_K / 16; s++)       // descriptor start addresses: 16-byte units
                        tc::mma_tmem_a_warp(d, a + 8 * s, f1 + (uint64_t)(s * 2 * F_LBO / 16), id1, s > 0 ? 1u : 0u);
                    tc::mma_commit_warp(&bars->a1_free[k & 1]);
                    tc::mma_commit_warp(&bars->d1_full[s3]);
                    if (++s3 == 3) {
                        s3 = 0;
                        u3++;
                    }
                }
            } else {
                const uint32_t id2 = Ops::idesc | (1u << 15);                  // A MN-major
                const uint64_t f2 = tc::smem_desc(tc::smem_u32(smem + OFF_F2), F_LBO, F_SBO);
                const uint64_t a2 = tc::smem_desc(tc::smem_u32(smem + OFF_A2), A2_CK, A2_CM);
                for (int64_t k = 0; k < n_my; k++) {
                    if (!wait(&bars->b2_full[k & 1], (uint32_t)((k >> 1) & 1))) break;   // A2 ready, D1 read
                    tc::fence_after_thread_sync();
                    const uint32_t d = tbase + (uint32_t)s3 * TC_N;
                    const uint64_t a = a2 + (uint64_t)((k & 1) * (TILE_BYTES / 16));
#pragma unroll
                    for (int s = 0; s < TC_K / 16; s++)
                        tc::mma_bf16_warp(d, a + (uint64_t)(s * 2 * A2_CK / 16), f2 + (uint64_t)(s * 2 * F_LBO / 16),
                                          id2, s > 0 ? 1u : 0u);
                    tc::mma_commit_warp(&bars->a2_free[k & 1]);
                    tc::mma_commit_warp(&bars->d2_full[s3]);
                    if (++s3 == 3) {
                        s3 = 0;
                        u3++;
                    }
                }
            }
            // drain: every MMA this warp issued has completed before TMEM can be released
            tc::mma_commit_warp(&bars->drain[warp]);
            tc::mbar_wait_bounded(&bars->drain[warp], 0, WAIT_CYCLES);
        }
        __syncwarp();
    } else if (warp < WS_E1) {
        // ---------------------------------------------------------------- producer
        // thread -> A1 row (z1, n2) (interleaved order), columns 32 hp .. 32 hp + 31 (chunks 8 hp .. 8 hp + 7)
        asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(REG_PROD));
        const int hp = (warp - WS_P0) >> 2;
        const int z1 = (lane >> 4) & 1, n2 = 16 * quad + (lane & 15);      // interleaved stage-1 row
        const uint4 *Yb = Y + 8 * hp * TC_R + n2;
        int64_t j = it0 % n_seg;                        // segment of the current item
        int grp = (int)(it0 / n_seg);                   // its template pair
        int gcur = -1;                                  // the pair whose spectrum gv holds
        uint4 gv[8];
        for (int64_t k = 0; k < n_my; k++) {
            const int z = grp * TC_G + z1;
            const int sl = (int)(k & 1);
            if (grp != gcur) {
                const uint4 *Gz = G + (z < K ? z : 0) * (TC_S_BF16 / 4) + 8 * hp * TC_R + n2;
#pragma unroll
                for (int c = 0; c < 8; c++) gv[c] = z < K ? __ldg(Gz + c * TC_R) : make_uint4(0, 0, 0, 0);
                gcur = grp;
            }
            uint4 yv[8];
            const uint4 *Yj = Yb + j * (TC_S_BF16 / 4);
#pragma unroll
            for (int c = 0; c < 8; c++) yv[c] = __ldg(Yj + c * TC_R);
            if (k >= 2 && !ws_wait(&bars->a1_free[sl], (uint32_t)(((k - 2) >> 1) & 1), abort_flag)) break;
            tc::fence_after_thread_sync();
            // conj(y) g: Re = yr gr + yi gi, Im = yr gi - yi gr, two n1 per packed pair; written in
            // place over the spectrum words and stored as two 16-column halves
#pragma unroll
            for (int hh = 0; hh < 2; hh++) {
                uint32_t w[16];
#pragma unroll
                for (int c = 0; c < 4; c++) {
                    const uint4 yq = yv[4 * hh + c], gq = gv[4 * hh + c];
                    const uint32_t ys[4] = {yq.x, yq.y, yq.z, yq.w};
                    const uint32_t gs[4] = {gq.x, gq.y, gq.z, gq.w};
#pragma unroll
                    for (int e = 0; e < 4; e += 2) {
                        const V yr = *reinterpret_cast<const V *>(&ys[e]), yi = *reinterpret_cast<const V *>(&ys[e + 1]);
                        const V gr = *reinterpret_cast<const V *>(&gs[e]), gi = *reinterpret_cast<const V *>(&gs[e + 1]);
                        const V re = __hfma2(yi, gi, __hmul2(yr, gr));
                        const V im = __hfma2(__hneg2(yi), gr, __hmul2(yr, gi));
                        w[4 * c + e] = *reinterpret_cast<const uint32_t *>(&re);
                        w[4 * c + e + 1] = *reinterpret_cast<const uint32_t *>(&im);
                    }
                }
                tc::tmem_st16(tbase + lane_base + COL_A1 + sl * (TC_K / 2) + 32 * hp + 16 * hh, w);
            }
            tc::tmem_st_wait();
            tc::fence_before_thread_sync();
            mbar_arrive(&bars->a1_full[sl]);
            if (++j == n_seg) {
                j = 0;
                grp++;
            }
        }
    } else if (warp < WS_E2) {
        // ---------------------------------------------------------------- epilogue 1
        // thread -> D1 row (z1, n2) (interleaved order), k1 in [32 h, 32 h + 32)
        asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(REG_E1));
        const int h = (warp - WS_E1) >> 2;
        const int z1 = (lane >> 4) & 1, n2 = 16 * quad + (lane & 15);
        // W_S^{n2 k1} for k1 = 32 h + 8 g + 2 i + {0, 1}: word (16 h + 4 g + i) * 64 + n2
        const float4 *tws = reinterpret_cast<const float4 *>(smem + OFF_TWS) + 16 * h * TC_R + n2;
        // A2 byte offset of (m = 64 z1 + 32 h, k = n2); k = 64 + n2 (imaginary part) is 8 A2_CK further
        const uint32_t a2_row = (uint32_t)(8 * z1 + 4 * h) * A2_CM + (uint32_t)(n2 >> 3) * A2_CK + (n2 & 7) * 16;
        int s3 = 0, u3 = 0;                             // slot k mod 3 and its use count k / 3
        for (int64_t k = 0; k < n_my; k++) {
            const int sl = (int)(k & 1);
            const uint32_t dcol = (uint32_t)s3 * TC_N;
            if (!ws_wait(&bars->d1_full[s3], (uint32_t)(u3 & 1), abort_flag)) break;
            if (k >= 2 && !ws_wait(&bars->a2_free[sl], (uint32_t)(((k - 2) >> 1) & 1), abort_flag)) break;
            tc::fence_after_thread_sync();
            unsigned char *a2 = smem + OFF_A2 + sl * TILE_BYTES + a2_row;
#pragma unroll
            for (int gg = 0; gg < 2; gg++) {
                uint32_t rr[16], ri[16];
                tc::tmem_ld16(tbase + lane_base + dcol + 32 * h + 16 * gg, rr);
                tc::tmem_ld16(tbase + lane_base + dcol + TC_R + 32 * h + 16 * gg, ri);
                tc::tmem_ld_wait();
#pragma unroll
                for (int g2 = 0; g2 < 2; g2++) {
                    const int g = 2 * gg + g2;
                    uint32_t ore[4], oim[4];
#pragma unroll
                    for (int i = 0; i < 4; i++) {
                        const float4 t = tws[(4 * g + i) * TC_R];
                        const float2 wx = make_float2(t.x, t.y), wy = make_float2(t.z, t.w);
                        const float2 dr = u2f2(rr[8 * g2 + 2 * i], rr[8 * g2 + 2 * i + 1]);
                        const float2 di = u2f2(ri[8 * g2 + 2 * i], ri[8 * g2 + 2 * i + 1]);
                        const float2 q = __fmul2_rn(di, wy);
                        const float2 yr = __ffma2_rn(dr, wx, make_float2(-q.x, -q.y));
                        const float2 yi = __ffma2_rn(dr, wy, __fmul2_rn(di, wx));
                        ore[i] = Ops::pack(yr.x, yr.y);
                        oim[i] = Ops::pack(yi.x, yi.y);
                    }
                    *reinterpret_cast<uint4 *>(a2 + g * A2_CM) = make_uint4(ore[0], ore[1], ore[2], ore[3]);
                    *reinterpret_cast<uint4 *>(a2 + g * A2_CM + 8 * A2_CK) = make_uint4(oim[0], oim[1], oim[2], oim[3]);
                }
            }
            tc::fence_before_thread_sync();
            tc::fence_proxy_async_smem();
            mbar_arrive(&bars->b2_full[sl]);
            if (++s3 == 3) {
                s3 = 0;
                u3++;
            }
        }
    } else {
        // ---------------------------------------------------------------- epilogue 2
        // thread -> D2 row (zl, k1 = idx), k2 in [32 h, 32 h + 32)
        asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(REG_E2));
        const int h = (warp - WS_E2) >> 2;
        const int kl = L / TC_R;                        // k2 < L / 64  <=>  bin t = k1 + 64 k2 < L
        int64_t j = it0 % n_seg;
        int grp = (int)(it0 / n_seg);
        int slot = 0, u3 = 0;                           // slot k mod 3 and its use count k / 3
        for (int64_t k = 0; k < n_my; k++) {
            const uint32_t dcol = (uint32_t)slot * TC_N;
            if (!ws_wait(&bars->d2_full[slot], (uint32_t)(u3 & 1), abort_flag)) break;
            tc::fence_after_thread_sync();
            const int z = grp * TC_G + zl;
            const int64_t r0 = j * L;
            const float us = unscale ? __ldg(unscale + j) : 1.0f;
            if (++j == n_seg) {                         // the next item
                j = 0;
                grp++;
            }
            // stored k2 (this thread): k2 < kmax, from t < L, r0 + t < nb and z < K (a segment wholly
            // inside the row stores all L / 64)
            int kmax = kl;
            if (z >= K) {
                kmax = 0;
            } else if (r0 + L > nb) {
                const int64_t rest = nb - r0 - idx;
                const int64_t kr = (rest + TC_R - 1) / TC_R;
                kmax = rest <= 0 ? 0 : (kr < (int64_t)kl ? (int)kr : kl);
            }
            kmax -= 32 * h;
            float pw[32];
            {
                // the row half's 32 real and 32 imaginary parts in one round trip
                uint32_t rr[2][16], ri[2][16];
#pragma unroll
                for (int gg = 0; gg < 2; gg++) {
                    tc::tmem_ld16(tbase + lane_base + dcol + 32 * h + 16 * gg, rr[gg]);
                    tc::tmem_ld16(tbase + lane_base + dcol + TC_R + 32 * h + 16 * gg, ri[gg]);
                }
                tc::tmem_ld_wait();
                tc::fence_before_thread_sync();
                mbar_arrive(&bars->d_free[slot]);                        // accumulator slot drained
#pragma unroll
                for (int gg = 0; gg < 2; gg++)
#pragma unroll
                    for (int i = 0; i < 8; i++) {
                        const float2 re = u2f2(rr[gg][2 * i], rr[gg][2 * i + 1]);
                        const float2 im = u2f2(ri[gg][2 * i], ri[gg][2 * i + 1]);
                        const float2 p = __ffma2_rn(re, re, __fmul2_rn(im, im));
                        pw[16 * gg + 2 * i] = p.x;
                        pw[16 * gg + 2 * i + 1] = p.y;
                    }
            }
            if (++slot == 3) {
                slot = 0;
                u3++;
            }
            typename Ops::Out *prow = plane + (int64_t)(z < K ? z : 0) * nb + r0 + idx + 64 * 32 * h;
            // level-1 marks: the 512-bin units of row z holding a stored value above thr1 (rounding
            // is monotone, so the largest value decides whether any does; four interleaved chains
            // of three-input maxima keep the maximum's dependency chain short)
            if (l1flag != nullptr && kmax > 0) {
                float m[4];
#pragma unroll
                for (int c = 0; c < 4; c++)          // chain c: pw[c + 4 i], i < 8
                    m[c] = fmaxf(fmax3(fmax3(pw[c], pw[c + 4], pw[c + 8]), pw[c + 12], pw[c + 16]),
                                 fmax3(pw[c + 20], pw[c + 24], pw[c + 28]));
                if (Ops::stored(fmax3(fmaxf(m[0], m[1]), m[2], m[3]), us) > thr1) {
                    uint8_t *frow = l1flag + (int64_t)z * chunks1;
                    const int64_t b0 = r0 + idx + 64 * 32 * h;
#pragma unroll
                    for (int i = 0; i < 32; i++)
                        if (i < kmax && Ops::stored(pw[i], us) > thr1) frow[(b0 + 64 * i) >> 9] = 1;
                }
            }
            if (kmax >= 32) {
#pragma unroll
                for (int i = 0; i < 32; i++) prow[64 * i] = Ops::out(pw[i], us);
            } else {
#pragma unroll
                for (int i = 0; i < 32; i++)
                    if (i < kmax) prow[64 * i] = Ops::out(pw[i], us);
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
// B1 tiles (stage-1 A operand, K-major): core matrices 144 B apart along M, 16 x 144 B along K
constexpr uint32_t B_SBO = 144, B_LBO = 16 * B_SBO;
constexpr uint32_t B_TILE = 16 * B_LBO;                      // 36 KB
// A2 tiles (stage-2 A operand, K-major): 128 B along M, 2064 B (16 mod 128) along K
constexpr uint32_t A2_SBO = 128, A2_LBO = 16 * 128 + 16;
constexpr uint32_t A2_TILE = 16 * A2_LBO;                    // 32.25 KB
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

// Host tables of the tensor path, FP64 then rounded once:
//  - the split variant's F'[(k,p),(n,s)] (real-ified W_64^{kn}, re/im interleaved), K-major BF16
//    images hi and lo;
//  - F1 (stage 1: rows (p, k1), K in the stage-1 order) and F2 (stage 2: rows (p, k2), K = (s, n2)),
//    K-major, in BF16 and in FP16;
//  - the four-step twiddles W_4096^{n2 k1}, [k1][n2].
// Entry (p, s) of the real-ified W_64^{kn}: [[Re w, -Im w], [Im w, Re w]].
static double dft64_real(int k, int n, int p, int s) {
    const int e = (k * n) % TC_R;
    double f = 2.0 * e / TC_R;
    if (f > 1.0) f -= 2.0;
    const double wr = std::cos(M_PI * f), wi = -std::sin(M_PI * f);
    return p == 0 ? (s == 0 ? wr : -wi) : (s == 0 ? wi : wr);
}

cudaError_t launch_prepare_bf16(Plan &p, cudaStream_t st) {
    const size_t T = (size_t)TC_M * TC_K;
    std::vector<uint16_t> img(4 * T, 0), img_h(2 * T, 0);
    auto put = [&](size_t tile, int row, int k, double v) {
        const uint32_t o = tc::kmajor_offset(TC_M, row, k) / 2;
        img[tile * T + o] = host_bf16((float)v);
        if (tile >= 2) {
            const __half h = __float2half_rn((float)v);
            std::memcpy(&img_h[(tile - 2) * T + o], &h, 2);
        }
    };
    for (int k = 0; k < TC_R; k++)
        for (int n = 0; n < TC_R; n++)
            for (int pr = 0; pr < 2; pr++)
                for (int sg = 0; sg < 2; sg++) {
                    const double v = dft64_real(k, n, pr, sg);
                    const uint32_t o = tc::kmajor_offset(TC_M, 2 * k + pr, 2 * n + sg) / 2;
                    img[o] = host_bf16((float)v);
                    uint32_t hb = (uint32_t)img[o] << 16;
                    float hf;
                    std::memcpy(&hf, &hb, 4);
                    img[T + o] = host_bf16((float)(v - (double)hf));
                }
    for (int pr = 0; pr < 2; pr++)
        for (int k = 0; k < TC_R; k++)
            for (int kk = 0; kk < TC_K; kk++) {
                put(2, TC_R * pr + k, kk, dft64_real(k, s1_n1(kk), pr, s1_s(kk)));     // F1
                put(3, TC_R * pr + k, kk, dft64_real(k, kk & 63, pr, kk >> 6));         // F2
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
    if (e == cudaSuccess && p.d_tcFh)
        e = cudaMemcpyAsync(p.d_tcFh, img_h.data(), img_h.size() * 2, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e;
}

// The register hand-over inside k3_plane_tc (setmaxnreg) assumes the launch allocation the kernel
// was compiled for; a different one could leave the increasing warps waiting, so it is checked
// before every launch.
template <class Ops>
static cudaError_t prepare_plane_tc() {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, k3_plane_tc<Ops>);
    if (e != cudaSuccess) return e;
    if (fa.numRegs != REG_LAUNCH) return cudaErrorInvalidDeviceFunction;
    return cudaFuncSetAttribute(k3_plane_tc<Ops>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)WS_SMEM);
}

static_assert(PEAK_CHUNK == 512, "the level-1 marks index units as bin >> 9");

bool level1_fusable(const Plan &p) {
    return p.cfg.precision == FDAS_FP32 || p.cfg.precision == FDAS_BF16 || p.cfg.precision == FDAS_FP16_SCALED ||
           p.cfg.precision == FDAS_BF16_DIRECT || p.cfg.precision == FDAS_FP8_DIRECT;
}

// Clear the level-1 unit marks before the plane kernel sets them.
static cudaError_t clear_marks(const Plan &p, uint8_t *l1flag, cudaStream_t st) {
    if (!l1flag) return cudaSuccess;
    return cudaMemsetAsync(l1flag, 0, (size_t)p.K * (size_t)(p.nb / PEAK_CHUNK), st);
}

cudaError_t launch_plane_bf16(const Plan &p, const float2 *d_x, const float *d_scale, char *ws,
                              __nv_bfloat16 *d_plane, cudaStream_t st, uint8_t *l1flag) {
    if (p.S != TC_S_BF16) return cudaErrorInvalidValue;
    uint4 *Y = reinterpret_cast<uint4 *>(ws + p.ws_y);
    const size_t smem2 = sizeof(float2) * fft_smem_entries(TC_S_BF16);
    cudaError_t e = cudaFuncSetAttribute(k2_segments_bf16, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2);
    if (e != cudaSuccess) return e;
    e = prepare_plane_tc<OpsBF16>();
    if (e != cudaSuccess) return e;
    // the unit marks are cleared by the segment kernel: their workspace slot is 256-byte aligned
    // and padded to 256 bytes, so whole 16-byte words cover it
    const int64_t n_zero16 = l1flag ? ((int64_t)p.K * (p.nb / PEAK_CHUNK) + 15) / 16 : 0;
    p.prof.begin(FDAS_STAGE_SEGMENTS, st);
    k2_segments_bf16<<<(unsigned)p.n_seg, TC_S_BF16 / 32, smem2, st>>>(d_x, d_scale, p.d_tw, Y, p.nb, p.L, p.m / 2,
                                                                      reinterpret_cast<uint4 *>(l1flag), n_zero16);
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
        Y, reinterpret_cast<const uint4 *>(p.d_Gbf), reinterpret_cast<const uint4 *>(p.d_tcF) + 2 * TILE_BYTES / 16,
        p.d_tcTw, d_plane, p.K, p.nb, p.L, n_items, n_groups, per, nullptr, l1flag, p.nb / PEAK_CHUNK, mark_threshold(p),
        p.d_status);
    p.prof.end(FDAS_STAGE_CORRELATE, st);
    p.prof.launches += 2;
    return cudaGetLastError();
}

// FP16-scaled ablation: scaled FP16 segment spectra, the FP16 bank (S G) and DFT image, FP32 plane.
cudaError_t launch_plane_f16(const Plan &p, const float2 *d_x, const float *d_scale, char *ws, float *d_plane,
                             cudaStream_t st, uint8_t *l1flag) {
    if (p.S != TC_S_BF16 || !p.d_Gh || !p.d_tcFh) return cudaErrorInvalidValue;
    uint4 *Y = reinterpret_cast<uint4 *>(ws + p.ws_y);
    float *unscale = reinterpret_cast<float *>(ws + p.ws_segscale);
    const size_t smem2 = sizeof(float2) * fft_smem_entries(TC_S_BF16);
    cudaError_t e = cudaFuncSetAttribute(k2_segments_f16, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2);
    if (e != cudaSuccess) return e;
    e = prepare_plane_tc<OpsF16>();
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
    e = clear_marks(p, l1flag, st);
    if (e != cudaSuccess) return e;
    p.prof.begin(FDAS_STAGE_CORRELATE, st);
    k3_plane_tc<OpsF16><<<(unsigned)grid, WS_THREADS, WS_SMEM, st>>>(
        Y, reinterpret_cast<const uint4 *>(p.d_Gh), reinterpret_cast<const uint4 *>(p.d_tcFh), p.d_tcTw, d_plane,
        p.K, p.nb, p.L, n_items, n_groups, per, unscale, l1flag, p.nb / PEAK_CHUNK, mark_threshold(p), p.d_status);
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
