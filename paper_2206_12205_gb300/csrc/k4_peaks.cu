// K4: harmonic sums and the thresholded peak list (Sec. 2.1: a pulsar shows as peaks at
// integer multiples of f and fdot, and the summed power of the harmonics is the detection
// statistic).
//
// For level H (1, 2, 4, 8, 16): S_H(r, i) = sum_{h=1..H} P(h r, i_h), z_{i_h} = h z_i,
// summed in FP32 in the order h = 1..H (BF16 planes are widened by placing the 16 stored
// bits in the top half of a float, the paper's quick cast of Sec. 3.1), defined where
// |H z_i| <= zmax and H r < Nb.  Peak: S_H > thr and a 3x3 local maximum (strictly above
// earlier neighbours in row-major (i, r) order, >= later ones, undefined neighbours ignored).
//
// The defined regions nest (level 2H's lies inside level H's), so one pass builds every level
// in place: a tile of RB rows x CB bins (plus a one-cell halo) is loaded once into shared
// memory as S_1 = P, peaks of level 1 are detected, then S_2 = S_1 + P(2r, i_2) is formed in
// place (cells outside level 2's region become -inf), and so on up to max_harm.  The running
// sum adds the terms in the order h = 1..H, so every S_H is bit-identical to the direct sum.
//
// Output order (H, i, r) without a sort: a "unit" is (level, row, chunk of CB bins), units
// are numbered in that order, and
//   pass A (k4_detect) writes each unit's peak count and, when non-zero, its CB-bit mask;
//   pass B (k4_scan_blocks, k4_scan_top) turns the counts into exclusive offsets + total;
//   pass C (k4_emit, one warp per unit, empty units skipped) recomputes S_H at the few
//   marked cells and writes the records at offset + rank.
#include <cmath>

#include "fdas_internal.cuh"

namespace fdas {

namespace {

constexpr int RB = PEAK_ROWS;            // rows per tile (one warp each)
constexpr int CB = PEAK_CHUNK;           // bins per tile / unit
constexpr int SW = CB + 2;               // staged cells per row: bins r0-1 .. r0+CB
constexpr int SOFF = 3;                  // staged cell c sits at S[row][c + SOFF]: the interior
constexpr int SWP = CB + 8;              // (c = 1 .. CB) starts on a 16-byte boundary; row pitch
constexpr int WORDS = CB / 32;           // mask words per unit
constexpr int SCAN_BLOCK = PEAK_SCAN_BLOCK;

__device__ __forceinline__ float ld_plane(const float *p, int64_t i) { return __ldg(p + i); }
__device__ __forceinline__ float ld_plane(const __nv_bfloat16 *p, int64_t i) {
    const unsigned short bits = __ldg(reinterpret_cast<const unsigned short *>(p) + i);
    return __uint_as_float(((unsigned)bits) << 16);
}

// 16-byte vector of plane values widened to float: 4 FP32 or 8 BF16 elements.
template <typename E>
struct Vec;
template <>
struct Vec<float> {
    static constexpr int N = 4;
    __device__ __forceinline__ static void load(const float *p, float (&o)[4]) {
        const float4 v = __ldg(reinterpret_cast<const float4 *>(p));
        o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
    }
};
template <>
struct Vec<__nv_bfloat16> {
    static constexpr int N = 8;
    __device__ __forceinline__ static void load(const __nv_bfloat16 *p, float (&o)[8]) {
        const uint4 v = __ldg(reinterpret_cast<const uint4 *>(p));
        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int k = 0; k < 4; k++) {
            o[2 * k] = __uint_as_float(w[k] << 16);
            o[2 * k + 1] = __uint_as_float(w[k] & 0xFFFF0000u);
        }
    }
};

template <typename E>
__device__ __forceinline__ float harm_sum(const E *plane, int64_t nb, int zmax, int H, int i, int64_t r) {
    const int z = -zmax + 2 * i;
    float s = 0.0f;
    for (int h = 1; h <= H; h++) {
        const int ih = (h * z + zmax) >> 1;
        s = __fadd_rn(s, ld_plane(plane, (int64_t)ih * nb + (int64_t)h * r));
    }
    return s;
}

__device__ __forceinline__ bool row_in_level(int i, int K, int zmax, int H) {
    const int z = -zmax + 2 * i;
    return i >= 0 && i < K && abs(H * z) <= zmax;
}

// S_H = S_{H/2} + sum_{h = H/2+1 .. H} P(h r, i_h) for every staged cell inside level H's region
// (-inf outside).  A thread owns columns tid, tid + 256, tid + 512 of every staged row; the row
// pointers of each harmonic are formed once per row, and a batch of rows issues all of its
// loads before the ordered sums, so that about 16 independent loads are in flight per thread.
template <typename E, int H>
__device__ __forceinline__ void level_update(float (*S)[SWP], const E *__restrict__ plane, int64_t nb, int zmax,
                                             int K, int i0, int64_t r0, int64_t rmax) {
    constexpr int NH = H / 2;
    constexpr int NC = (SW + RB * 32 - 1) / (RB * 32);            // columns per thread (3)
    constexpr int RBAT = (16 / (NH * NC)) > 0 ? 16 / (NH * NC) : 1;
    for (int ri0 = 0; ri0 < RB + 2; ri0 += RBAT) {
        float v[RBAT][NC][NH];
        bool ok[RBAT][NC];
#pragma unroll
        for (int rb = 0; rb < RBAT; rb++) {
            const int ri = ri0 + rb;
            const int i = i0 - 1 + ri;
            const bool row_ok = ri < RB + 2 && row_in_level(i, K, zmax, H);
            const int z = -zmax + 2 * i;
            const E *base[NH];
#pragma unroll
            for (int q = 0; q < NH; q++)
                base[q] = plane + (row_ok ? (int64_t)(((NH + 1 + q) * z + zmax) >> 1) * nb : 0);
#pragma unroll
            for (int cc = 0; cc < NC; cc++) {
                const int c = threadIdx.x + cc * RB * 32;
                const int64_t r = r0 - 1 + c;
                ok[rb][cc] = row_ok && c < SW && r >= 0 && r <= rmax;
#pragma unroll
                for (int q = 0; q < NH; q++)
                    v[rb][cc][q] = ok[rb][cc] ? ld_plane(base[q], (int64_t)(NH + 1 + q) * r) : 0.0f;
            }
        }
#pragma unroll
        for (int rb = 0; rb < RBAT; rb++) {
            const int ri = ri0 + rb;
            if (ri >= RB + 2) break;
#pragma unroll
            for (int cc = 0; cc < NC; cc++) {
                const int c = threadIdx.x + cc * RB * 32;
                if (c >= SW) break;
                float sum = -INFINITY;
                if (ok[rb][cc]) {
                    sum = S[ri][c + SOFF];
#pragma unroll
                    for (int q = 0; q < NH; q++) sum = __fadd_rn(sum, v[rb][cc][q]);
                }
                S[ri][c + SOFF] = sum;
            }
        }
    }
}

template <typename E>
__global__ void __launch_bounds__(RB * 32, 4) k4_detect(const E *__restrict__ plane, int64_t nb, int zmax, int K,
                                                     LevelTable lt, int n_rb, int32_t *__restrict__ unit_count,
                                                     uint32_t *__restrict__ unit_mask) {
    __shared__ __align__(16) float S[RB + 2][SWP];
    const int tile = blockIdx.x;
    const int rb = tile % n_rb;                    // row blocks of one chunk run side by side (halo rows hit L2)
    const int64_t chunk = tile / n_rb;
    const int i0 = rb * RB;
    const int64_t r0 = chunk * CB;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row = i0 + warp;

    // level 1: S_1 = P on rows i0-1 .. i0+RB, bins r0-1 .. r0+CB.  The chunk interior
    // [r0, r0 + CB) is 16-byte aligned (r0 is a multiple of CB, Nb a power of two): vector loads,
    // all issued before the shared-memory stores; the two halo columns are loaded singly.
    {
        constexpr int EPV = Vec<E>::N;
        constexpr int VPR = CB / EPV;                       // vectors per row
        constexpr int NV = ((RB + 2) * VPR + RB * 32 - 1) / (RB * 32);
        float vals[NV][EPV];
#pragma unroll
        for (int k = 0; k < NV; k++) {
            const int v = threadIdx.x + k * RB * 32;
            const int ri = v / VPR, q = v % VPR;
            const int i = i0 - 1 + ri;
            const int64_t r = r0 + (int64_t)q * EPV;
            if (ri < RB + 2 && i >= 0 && i < K && r < nb) {
                Vec<E>::load(plane + (int64_t)i * nb + r, vals[k]);
            } else {
#pragma unroll
                for (int e = 0; e < EPV; e++) vals[k][e] = -INFINITY;
            }
        }
#pragma unroll
        for (int k = 0; k < NV; k++) {
            const int v = threadIdx.x + k * RB * 32;
            const int ri = v / VPR, q = v % VPR;
            if (ri < RB + 2) {
#pragma unroll
                for (int e = 0; e < EPV; e += 4)
                    *reinterpret_cast<float4 *>(&S[ri][1 + SOFF + q * EPV + e]) =
                        make_float4(vals[k][e], vals[k][e + 1], vals[k][e + 2], vals[k][e + 3]);
            }
        }
        if (threadIdx.x < 2 * (RB + 2)) {
            const int ri = threadIdx.x >> 1;
            const int c = (threadIdx.x & 1) ? SW - 1 : 0;
            const int i = i0 - 1 + ri;
            const int64_t r = r0 - 1 + c;
            S[ri][c + SOFF] = (i >= 0 && i < K && r >= 0 && r < nb) ? ld_plane(plane + (int64_t)i * nb, r) : -INFINITY;
        }
    }
    __syncthreads();

    for (int l = 0; l < lt.n_levels; l++) {
        const LevelDesc &d = lt.lev[l];
        const int H = d.H;
        if (r0 > d.rmax) break;                                     // regions nest: nothing further
        const int rlo = max(i0 - 1, d.i_lo), rhi = min(i0 + RB, d.i_lo + d.rows - 1);
        if (rlo > rhi) break;
        if (l > 0) {
            // S_H = S_{H/2} + sum_{h = H/2+1 .. H} P(h r, i_h) inside level H's region, -inf outside
            __syncthreads();
            switch (H) {
                case 2: level_update<E, 2>(S, plane, nb, zmax, K, i0, r0, d.rmax); break;
                case 4: level_update<E, 4>(S, plane, nb, zmax, K, i0, r0, d.rmax); break;
                case 8: level_update<E, 8>(S, plane, nb, zmax, K, i0, r0, d.rmax); break;
                default: level_update<E, 16>(S, plane, nb, zmax, K, i0, r0, d.rmax); break;
            }
            __syncthreads();
        }
        // detection: warp `warp` owns row i0 + warp; lane handles bins r0 + lane + 32 e
        if (row_in_level(row, K, zmax, H)) {
            int cnt = 0;
            uint32_t words[WORDS];
            const int cmax = (int)min((int64_t)CB, d.rmax - r0 + 1);   // valid bins in this chunk
            // fast path: nothing in the row segment above the threshold -> an empty unit
            float vmax = -INFINITY;
#pragma unroll
            for (int e = 0; e < WORDS; e++)
                if (lane + 32 * e < cmax) vmax = fmaxf(vmax, S[warp + 1][1 + SOFF + lane + 32 * e]);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
            if (!(vmax > d.thr)) {
                if (lane == 0) unit_count[d.unit0 + (int64_t)(row - d.i_lo) * d.chunks + chunk] = 0;
            } else {
#pragma unroll
            for (int e = 0; e < WORDS; e++) {
                const int c = 1 + SOFF + lane + 32 * e;
                bool pk = false;
                if (lane + 32 * e < cmax) {
                    const float v = S[warp + 1][c];
                    if (v > d.thr) {
                        pk = v > S[warp][c - 1] && v > S[warp][c] && v > S[warp][c + 1] && v > S[warp + 1][c - 1] &&
                             v >= S[warp + 1][c + 1] && v >= S[warp + 2][c - 1] && v >= S[warp + 2][c] &&
                             v >= S[warp + 2][c + 1];
                    }
                }
                words[e] = __ballot_sync(0xffffffffu, pk);
                cnt += __popc(words[e]);
            }
            const int64_t u = d.unit0 + (int64_t)(row - d.i_lo) * d.chunks + chunk;
            if (lane == 0) unit_count[u] = cnt;
            if (cnt > 0 && lane < WORDS) {
                uint32_t w = 0;
#pragma unroll
                for (int e = 0; e < WORDS; e++)
                    if (e == lane) w = words[e];
                unit_mask[u * WORDS + lane] = w;
            }
            }
        }
    }
}

// First-level scan: exclusive prefix of the counts inside each block of SCAN_BLOCK units.
__global__ void __launch_bounds__(1024) k4_scan_blocks(const int32_t *__restrict__ cnt, int64_t n,
                                                       int32_t *__restrict__ off, int64_t *__restrict__ block_sum) {
    __shared__ int32_t warp_tot[32];
    const int64_t base = (int64_t)blockIdx.x * SCAN_BLOCK + threadIdx.x * 4;
    int32_t v[4];
#pragma unroll
    for (int k = 0; k < 4; k++) v[k] = (base + k < n) ? cnt[base + k] : 0;
    const int32_t sum = v[0] + v[1] + v[2] + v[3];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int32_t incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int32_t t = warp_tot[lane], ti = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t y = __shfl_up_sync(0xffffffffu, ti, o);
            if (lane >= o) ti += y;
        }
        warp_tot[lane] = ti - t;                 // exclusive warp offsets
        if (lane == 31) block_sum[blockIdx.x] = ti;
    }
    __syncthreads();
    int32_t run = warp_tot[warp] + incl - sum;
#pragma unroll
    for (int k = 0; k < 4; k++) {
        if (base + k < n) off[base + k] = run;
        run += v[k];
    }
}

// Second level (one CTA, fixed order): block offsets in place, total count, overflow flag.
__global__ void __launch_bounds__(1024) k4_scan_top(int64_t *__restrict__ block_sum, int64_t nblocks,
                                                    int32_t *__restrict__ npeaks, int max_peaks,
                                                    int32_t *__restrict__ status) {
    __shared__ int64_t warp_tot[32];
    __shared__ int64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t b0 = 0; b0 < nblocks; b0 += 1024) {
        const int64_t b = b0 + threadIdx.x;
        const int64_t v = (b < nblocks) ? block_sum[b] : 0;
        int64_t incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) warp_tot[warp] = incl;
        __syncthreads();
        int64_t before = carry;
        for (int w = 0; w < warp; w++) before += warp_tot[w];
        if (b < nblocks) block_sum[b] = before + incl - v;
        __syncthreads();
        if (threadIdx.x == 1023) carry = before + incl;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const int64_t total = carry;
        *npeaks = (int32_t)(total < 0x7fffffff ? total : 0x7fffffff);
        if (total > max_peaks) atomicOr(status, FDAS_DEV_PEAK_OVERFLOW);
    }
}

struct UnitRef {
    int l, row;
    int64_t chunk;
};

__device__ __forceinline__ UnitRef unit_of(const LevelTable &lt, int64_t u) {
    int l = 0;
#pragma unroll
    for (int k = 1; k < 5; k++)
        if (k < lt.n_levels && u >= lt.lev[k].unit0) l = k;
    const LevelDesc &d = lt.lev[l];
    const int64_t local = u - d.unit0;
    UnitRef ref;
    ref.l = l;
    ref.row = d.i_lo + (int)(local / d.chunks);
    ref.chunk = local % d.chunks;
    return ref;
}

// One warp per non-empty unit: records at (block offset + in-block offset + rank).
template <typename E>
__global__ void __launch_bounds__(256) k4_emit(const E *__restrict__ plane, int64_t nb, int zmax, LevelTable lt,
                                               int64_t n_units, const int32_t *__restrict__ unit_count,
                                               const int32_t *__restrict__ unit_off,
                                               const int64_t *__restrict__ block_off,
                                               const uint32_t *__restrict__ unit_mask, fdas_peak *__restrict__ out,
                                               int max_peaks, uint32_t series) {
    const int lane = threadIdx.x & 31;
    const int64_t warp_id = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t n_warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t u = warp_id; u < n_units; u += n_warps) {
        const int32_t cnt = unit_count[u];
        if (cnt == 0) continue;                                  // warp-uniform
        const int64_t base = block_off[u / SCAN_BLOCK] + unit_off[u];
        const UnitRef ref = unit_of(lt, u);
        const int H = lt.lev[ref.l].H;
        const uint32_t w = lane < WORDS ? unit_mask[u * WORDS + lane] : 0u;
        int incl = __popc(w);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        int64_t pos = base + incl - __popc(w);
        uint32_t bits = w;
        while (bits) {
            const int b = __ffs(bits) - 1;
            bits &= bits - 1;
            if (pos < max_peaks) {
                const int64_t r = ref.chunk * CB + lane * 32 + b;
                fdas_peak pk;
                pk.series = series;
                pk.r = (uint32_t)r;
                pk.zi = (int16_t)ref.row;
                pk.harm = (uint8_t)H;
                pk.pad = 0;
                pk.power = harm_sum(plane, nb, zmax, H, ref.row, r);
                out[pos] = pk;
            }
            pos++;
        }
    }
}

template <typename E>
cudaError_t run_peaks(const Plan &p, const E *plane, char *ws, fdas_peak *peaks, int32_t *npeaks, uint32_t series,
                      cudaStream_t st) {
    const LevelTable lt = make_levels(p);
    int32_t *unit_count = reinterpret_cast<int32_t *>(ws + p.ws_ucount);
    int32_t *unit_off = reinterpret_cast<int32_t *>(ws + p.ws_uoff);
    uint32_t *unit_mask = reinterpret_cast<uint32_t *>(ws + p.ws_umask);
    int64_t *block_off = reinterpret_cast<int64_t *>(ws + p.ws_ublock);
    const int n_rb = (p.K + RB - 1) / RB;
    const int64_t chunks1 = lt.lev[0].chunks;
    const int64_t n_units = p.n_units;
    const int64_t n_blocks = (n_units + SCAN_BLOCK - 1) / SCAN_BLOCK;
    p.prof.begin(FDAS_STAGE_PEAKS, st);
    p.prof.launches += 4;
    k4_detect<E><<<(unsigned)(n_rb * chunks1), RB * 32, 0, st>>>(plane, p.nb, p.cfg.zmax, p.K, lt, n_rb, unit_count,
                                                                  unit_mask);
    k4_scan_blocks<<<(unsigned)n_blocks, 1024, 0, st>>>(unit_count, n_units, unit_off, block_off);
    k4_scan_top<<<1, 1024, 0, st>>>(block_off, n_blocks, npeaks, p.cfg.max_peaks, p.d_status);
    const int64_t emit_blocks = std::min<int64_t>((n_units + 7) / 8, 152 * 16);
    k4_emit<E><<<(unsigned)emit_blocks, 256, 0, st>>>(plane, p.nb, p.cfg.zmax, lt, n_units, unit_count, unit_off,
                                                       block_off, unit_mask, peaks, p.cfg.max_peaks, series);
    p.prof.end(FDAS_STAGE_PEAKS, st);
    return cudaGetLastError();
}

}  // namespace

LevelTable make_levels(const Plan &p) {
    LevelTable lt{};
    int64_t unit0 = 0;
    int n = 0;
    for (int l = 0; l < 5; l++) {
        const int H = 1 << l;
        if (H > p.cfg.max_harm) break;
        int zl = p.cfg.zmax / H;
        zl -= zl & 1;                               // largest even z with |H z| <= zmax
        LevelDesc &d = lt.lev[n];
        d.H = H;
        d.i_lo = (p.cfg.zmax - zl) / 2;
        d.rows = zl + 1;
        d.rmax = (p.nb - 1) / H;
        d.chunks = (d.rmax + 1 + PEAK_CHUNK - 1) / PEAK_CHUNK;
        d.unit0 = unit0;
        d.thr = p.cfg.thr[l];
        unit0 += (int64_t)d.rows * d.chunks;
        n++;
    }
    lt.n_levels = n;
    return lt;
}

cudaError_t launch_peaks(const Plan &p, const void *d_plane, bool bf16, char *ws, fdas_peak *d_peaks,
                         int32_t *d_npeaks, uint32_t series, cudaStream_t st) {
    if (bf16)
        return run_peaks<__nv_bfloat16>(p, reinterpret_cast<const __nv_bfloat16 *>(d_plane), ws, d_peaks, d_npeaks,
                                        series, st);
    return run_peaks<float>(p, reinterpret_cast<const float *>(d_plane), ws, d_peaks, d_npeaks, series, st);
}

}  // namespace fdas
