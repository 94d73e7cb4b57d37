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
// The defined regions nest (level 2H's lies inside level H's), so one pass builds every level:
// a warp owns one (row i, chunk of CB = 512 bins) of the plane and the running sums S_H of its
// bins stay in registers; S_2H = S_H + sum_{h = H+1 .. 2H} P(h r, i_h) adds the new harmonics in
// order, so every S_H is bit-identical to the direct sum.  Level 1 (a stream over the whole plane,
// or over the units the plane kernel marked) gives lane l the 16 consecutive bins r0 + 16 l ..
// r0 + 16 l + 15, read as 16-byte vectors.  Levels 2 .. 16 interleave instead -- lane l holds
// r0 + l + 32 e, e < 16 -- so that one warp-wide load of harmonic h reads 32 elements h apart,
// a span of whole sectors, where consecutive bins per lane would touch 32 sectors per load.  A
// lane tests its 16 values against the threshold through their maximum; only cells above it (a
// handful per plane) recompute their 3x3 neighbourhood's sums to decide the peak.
//
// Output order (H, i, r): a "unit" is (level, row, chunk of CB bins), units are numbered in
// that order, and
//   pass A (k4_level1 over the plane, k4_levels over level 2's region) writes each unit's peak
//     count and, when non-zero, its CB-bit mask, and lists the non-empty units (in no order);
//   pass B (k4_emit_listed, one block): when the list holds every non-empty unit (PEAK_LIST_CAP;
//     the usual case) it sorts the list's unit numbers, scans their counts into offsets and
//     writes the records; otherwise it scans every unit's count in order.  Either way a
//     record's power is S_H recomputed at its cell, at offset + rank.
#include <algorithm>
#include <cmath>
#include <vector>

#include "fdas_internal.cuh"

namespace fdas {

namespace {

constexpr int CB = PEAK_CHUNK;           // bins per unit (a warp's chunk)
constexpr int LB = CB / 32;              // bins per lane (16)
constexpr int WORDS = CB / 32;           // mask words per unit
constexpr int DETECT_WARPS = 4;          // warps per k4_level1 / k4_levels block
#ifndef FDAS_K4_CPW
#define FDAS_K4_CPW 1                    // chunks per k4_levels warp
#endif
constexpr int CPW = FDAS_K4_CPW;
static_assert((CPW & (CPW - 1)) == 0 && CPW <= 2, "chunks per warp: 1 or 2 (chunks1 >= 2 is a power of two)");
#ifndef FDAS_K4_L1_MIN_BLOCKS
#define FDAS_K4_L1_MIN_BLOCKS 2          // resident k4_level1 blocks per SM the registers must allow
#endif
#ifndef FDAS_K4_RAY_BF16
#define FDAS_K4_RAY_BF16 1               // 1: the BF16 plane's levels in ray order too (the FP32 plane's always are)
#endif
#ifndef FDAS_K4_MIN_BLOCKS
#define FDAS_K4_MIN_BLOCKS 4             // resident k4_levels blocks per SM the registers must allow
#endif

static_assert(LB == 16, "a lane owns 16 bins: two BF16 or four FP32 16-byte vectors");

__device__ __forceinline__ float ld_plane(const float *p, int64_t i) { return __ldg(p + i); }
__device__ __forceinline__ float ld_plane(const __nv_bfloat16 *p, int64_t i) {
    const unsigned short bits = __ldg(reinterpret_cast<const unsigned short *>(p) + i);
    return __uint_as_float(((unsigned)bits) << 16);
}

// Plane element formats: elements per 16-byte vector, widening of one vector, and the maximum of
// a lane's 16 values (BF16 compares packed pairs; widening is exact, so the order is the same).
template <typename E>
struct Fmt;
template <>
struct Fmt<float> {
    static constexpr int EPV = 4;
    struct Raw {
        float4 v[LB / 4];
    };
    __device__ __forceinline__ static void load_raw(const float *p, Raw &r) {
#pragma unroll
        for (int k = 0; k < LB / 4; k++) r.v[k] = __ldg(reinterpret_cast<const float4 *>(p) + k);
    }
    __device__ __forceinline__ static void widen(const Raw &r, float (&s)[LB]) {
#pragma unroll
        for (int k = 0; k < LB / 4; k++) {
            s[4 * k] = r.v[k].x; s[4 * k + 1] = r.v[k].y; s[4 * k + 2] = r.v[k].z; s[4 * k + 3] = r.v[k].w;
        }
    }
    __device__ __forceinline__ static float max16(const Raw &r) {
        float m = -INFINITY;
#pragma unroll
        for (int k = 0; k < LB / 4; k++) m = fmaxf(fmaxf(m, fmaxf(r.v[k].x, r.v[k].y)), fmaxf(r.v[k].z, r.v[k].w));
        return m;
    }
    __device__ __forceinline__ static void load(const float *p, float (&o)[4]) {
        const float4 v = __ldg(reinterpret_cast<const float4 *>(p));
        o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
    }
    __device__ __forceinline__ static float load16(const float *p, float (&s)[LB]) {
        float m = -INFINITY;
#pragma unroll
        for (int k = 0; k < LB / 4; k++) {
            float v[4];
            load(p + 4 * k, v);
#pragma unroll
            for (int e = 0; e < 4; e++) {
                s[4 * k + e] = v[e];
                m = fmaxf(m, v[e]);
            }
        }
        return m;
    }
};
template <>
struct Fmt<__nv_bfloat16> {
    static constexpr int EPV = 8;
    struct Raw {
        uint4 v[LB / 8];
    };
    __device__ __forceinline__ static void load_raw(const __nv_bfloat16 *p, Raw &r) {
#pragma unroll
        for (int k = 0; k < LB / 8; k++) r.v[k] = __ldg(reinterpret_cast<const uint4 *>(p) + k);
    }
    __device__ __forceinline__ static void widen(const Raw &r, float (&s)[LB]) {
        const uint32_t w[8] = {r.v[0].x, r.v[0].y, r.v[0].z, r.v[0].w, r.v[1].x, r.v[1].y, r.v[1].z, r.v[1].w};
#pragma unroll
        for (int k = 0; k < 8; k++) {
            s[2 * k] = __uint_as_float(w[k] << 16);
            s[2 * k + 1] = __uint_as_float(w[k] & 0xFFFF0000u);
        }
    }
    // packed BF16 maximum (exact: widening preserves the order)
    __device__ __forceinline__ static float max16(const Raw &r) {
        const uint32_t w[8] = {r.v[0].x, r.v[0].y, r.v[0].z, r.v[0].w, r.v[1].x, r.v[1].y, r.v[1].z, r.v[1].w};
        __nv_bfloat162 m = *reinterpret_cast<const __nv_bfloat162 *>(&w[0]);
#pragma unroll
        for (int k = 1; k < 8; k++) m = __hmax2(m, *reinterpret_cast<const __nv_bfloat162 *>(&w[k]));
        return fmaxf(__low2float(m), __high2float(m));
    }
    __device__ __forceinline__ static void load(const __nv_bfloat16 *p, float (&o)[8]) {
        const uint4 v = __ldg(reinterpret_cast<const uint4 *>(p));
        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int k = 0; k < 4; k++) {
            o[2 * k] = __uint_as_float(w[k] << 16);
            o[2 * k + 1] = __uint_as_float(w[k] & 0xFFFF0000u);
        }
    }
    __device__ __forceinline__ static float load16(const __nv_bfloat16 *p, float (&s)[LB]) {
        const uint4 a = __ldg(reinterpret_cast<const uint4 *>(p));
        const uint4 b = __ldg(reinterpret_cast<const uint4 *>(p + 8));
        const uint32_t w[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
        __nv_bfloat162 m = *reinterpret_cast<const __nv_bfloat162 *>(&w[0]);
#pragma unroll
        for (int k = 0; k < 8; k++) {
            m = __hmax2(m, *reinterpret_cast<const __nv_bfloat162 *>(&w[k]));
            s[2 * k] = __uint_as_float(w[k] << 16);
            s[2 * k + 1] = __uint_as_float(w[k] & 0xFFFF0000u);
        }
        return fmaxf(__low2float(m), __high2float(m));
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

// Highest-harmonic-anchored sum with rounding (harm_mode 1): the cell (r, i) is harmonic H; the
// harmonic j of level L sits at r_j = floor((2 j r + L) / (2 L)) (j r / L rounded, halves up) and
// row floor((j z + L zmax + L) / (2 L)) (the grid row nearest j z / L, halves up).  Level 2L's
// even fractions are level L's with the same rounding, so S_2L = S_L + the odd j < 2L in
// increasing j, S_1 = P; FP32 adds in that order.
template <typename E>
__device__ float harm_sum_anch(const E *plane, int64_t nb, int zmax, int H, int i, int64_t r) {
    const int z = -zmax + 2 * i;
    float s = ld_plane(plane, (int64_t)i * nb + r);
    for (int l = 1; (1 << l) <= H; l++) {
        const int L = 1 << l;
        for (int j = 1; j < L; j += 2) {
            const int ij = (j * z + L * zmax + L) >> (l + 1);
            const int64_t rj = (2 * (int64_t)j * r + L) >> (l + 1);
            s = __fadd_rn(s, ld_plane(plane, (int64_t)ij * nb + rj));
        }
    }
    return s;
}

__device__ __forceinline__ bool row_in_level(int i, int K, int zmax, int H) {
    const int z = -zmax + 2 * i;
    return i >= 0 && i < K && abs(H * z) <= zmax;
}

// Levels 2 .. 16 interleave the bins: lane l of a warp owns bins r0 + l + 32 e (e < 16) of its
// 512-bin chunk, so one load of harmonic h for the whole warp reads the 32 elements h (r0 + l +
// 32 e), l < 32 -- a span of 32 h elements, whole sectors -- instead of 32 lanes each touching
// their own sectors.  s[e] += P(h r, i_h) for the lane's bins r = rb + 32 e with r <= rmax (then
// h r <= H rmax < Nb); the sums keep the order h = 1..H.
// S_H from S_{H/2}: the new harmonics h = H/2 + 1 .. H in order, the loads of FDAS_K4_HBATCH
// harmonics in flight together (16 per harmonic and lane; the adds keep the order h = 1..H).
#ifndef FDAS_K4_HBATCH
#define FDAS_K4_HBATCH 1                 // 2 measured 0.210 ms against 0.180 ms for 1 (BF16, N = 2^23)
#endif
template <typename E, int H>
__device__ __forceinline__ void add_level(const E *__restrict__ plane, int64_t nb, int zmax, int z, int64_t rb,
                                          int64_t rmax, float (&s)[LB]) {
    constexpr int NB = FDAS_K4_HBATCH < H / 2 ? FDAS_K4_HBATCH : H / 2;
#pragma unroll
    for (int q0 = 0; q0 < H / 2; q0 += NB) {
        float v[NB][LB];
#pragma unroll
        for (int q = 0; q < NB; q++) {
            const int h = H / 2 + 1 + q0 + q;
            const E *row = plane + (int64_t)((h * z + zmax) >> 1) * nb;
#pragma unroll
            for (int e = 0; e < LB; e++) {
                const int64_t r = rb + 32 * e;
                v[q][e] = r <= rmax ? ld_plane(row, (int64_t)h * r) : 0.0f;
            }
        }
#pragma unroll
        for (int q = 0; q < NB; q++)
#pragma unroll
            for (int e = 0; e < LB; e++) s[e] = __fadd_rn(s[e], v[q][e]);
        // bound the loads in flight (the registers of levels 8, 16)
        asm volatile("" ::: "memory");
    }
}

// The 3x3 rule for a cell of level H holding S_H = v: strictly above the defined neighbours that
// come earlier in row-major (i, r) order, at least equal to the later ones.
template <typename E>
__device__ __noinline__ bool local_max(const E *plane, int64_t nb, int zmax, int K, int H, int64_t rmax, int i, int64_t r, float v,
                                       bool anchored = false) {
    for (int di = -1; di <= 1; di++) {
        const int ii = i + di;
        if (anchored ? (ii < 0 || ii >= K) : !row_in_level(ii, K, zmax, H)) continue;
        for (int dr = -1; dr <= 1; dr++) {
            if (di == 0 && dr == 0) continue;
            const int64_t rr = r + dr;
            if (rr < 0 || rr > rmax) continue;
            const float w = anchored ? harm_sum_anch(plane, nb, zmax, H, ii, rr) : harm_sum(plane, nb, zmax, H, ii, rr);
            const bool earlier = di < 0 || (di == 0 && dr < 0);
            if (earlier ? !(v > w) : !(v >= w)) return false;
        }
    }
    return true;
}

// The non-empty unit list of the step: PEAK_LIST_WORDS words directly before the counts (word 0
// the number of non-empty units, words 4 .. the first PEAK_LIST_CAP unit numbers, in no order).
__device__ __forceinline__ unsigned int *unit_list(int32_t *unit_count) {
    return reinterpret_cast<unsigned int *>(unit_count) - PEAK_LIST_WORDS;
}
__device__ __forceinline__ const unsigned int *unit_list(const int32_t *unit_count) {
    return reinterpret_cast<const unsigned int *>(unit_count) - PEAK_LIST_WORDS;
}
// A unit's count, and the unit on the list when it holds peaks (one thread per unit; the list
// append, a handful of times per plane, out of line so that it costs the callers no registers).
__device__ __noinline__ void list_unit(int32_t *unit_count, int64_t u) {
    unsigned int *list = unit_list(unit_count);
    const unsigned int slot = atomicAdd(list, 1u);
    if (slot < (unsigned int)PEAK_LIST_CAP) list[4 + slot] = (unsigned int)u;
}
__device__ __forceinline__ void count_unit(int32_t *__restrict__ unit_count, int64_t u, int cnt) {
    unit_count[u] = cnt;
    if (cnt > 0) list_unit(unit_count, u);
}

// One level H > 1 of one (row, chunk), lane bins rb + 32 e: S_H from S_{H/2}, then the unit's count
// and mask (word e of the mask, bins 32 e .. 32 e + 31 of the chunk, is the warp's ballot of bit e).
// Returns false when the chunk lies outside level H's region (the regions nest: stop there).
template <typename E, int H, bool ADD = true>
__device__ __forceinline__ bool level_step(const E *__restrict__ plane, int64_t nb, int zmax, int K,
                                           const LevelDesc &d, int i, int z, int chunk, int64_t rb, float (&s)[LB],
                                           int32_t *__restrict__ unit_count, uint32_t *__restrict__ unit_mask) {
    const int lane = threadIdx.x & 31;
    if (!row_in_level(i, K, zmax, H) || (int64_t)chunk * CB > d.rmax) return false;   // warp-uniform
    if (ADD) add_level<E, H>(plane, nb, zmax, z, rb, d.rmax, s);
    float vmax = -INFINITY;
#pragma unroll
    for (int e = 0; e < LB; e++)
        if (rb + 32 * e <= d.rmax) vmax = fmaxf(vmax, s[e]);
    // unit indices fit 32 bits (at most 1023 rows x 2^17 chunks per level, five levels)
    const int u = (int)d.unit0 + (i - d.i_lo) * (int)d.chunks + chunk;
    if (__any_sync(0xffffffffu, vmax > d.thr)) {
        uint32_t pk = 0;
        if (vmax > d.thr) {
#pragma unroll
            for (int e = 0; e < LB; e++) {
                const int64_t r = rb + 32 * e;
                if (r <= d.rmax && s[e] > d.thr && local_max(plane, nb, zmax, K, H, d.rmax, i, r, s[e])) pk |= 1u << e;
            }
        }
        int cnt = __popc(pk);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
        if (lane == 0) count_unit(unit_count, u, cnt);
        if (cnt > 0) {
            uint32_t word = 0;
#pragma unroll
            for (int e = 0; e < LB; e++) {
                const uint32_t b = __ballot_sync(0xffffffffu, (pk >> e) & 1u);
                if (lane == e) word = b;
            }
            if (lane < WORDS) unit_mask[(int64_t)u * WORDS + lane] = word;
        }
    } else if (lane == 0) {
        unit_count[u] = 0;
    }
    return true;
}

// Levels 4, 8 and 16 (under 10 % of the cells): out of line, so that their gathers do not set
// the register budget of the common path (level 2).
template <typename E>
__device__ __noinline__ void high_levels(const E *__restrict__ plane, int64_t nb, int zmax, int K,
                                         const LevelTable *lt, int i, int z, int chunk, int64_t rb,
                                         const float *s_in, int32_t *__restrict__ unit_count,
                                         uint32_t *__restrict__ unit_mask) {
    float s[LB];
#pragma unroll
    for (int e = 0; e < LB; e++) s[e] = s_in[e];
    const int n = lt->n_levels;
    if (!level_step<E, 4>(plane, nb, zmax, K, lt->lev[2], i, z, chunk, rb, s, unit_count, unit_mask)) return;
    if (n < 4 || !level_step<E, 8>(plane, nb, zmax, K, lt->lev[3], i, z, chunk, rb, s, unit_count, unit_mask))
        return;
    if (n > 4) level_step<E, 16>(plane, nb, zmax, K, lt->lev[4], i, z, chunk, rb, s, unit_count, unit_mask);
}

// Levels 2 .. of one (row, chunk) inside level 2's region; s holds S_2 of the lane's bins on entry
// (the caller reads S_1 and the second harmonic together).
template <typename E>
__device__ __forceinline__ void detect_chunk(const E *__restrict__ plane, int64_t nb, int zmax, int K,
                                             const LevelTable &lt, int i, int z, int chunk, int64_t rb,
                                             float (&s)[LB], int32_t *__restrict__ unit_count,
                                             uint32_t *__restrict__ unit_mask) {
    if (!level_step<E, 2, false>(plane, nb, zmax, K, lt.lev[1], i, z, chunk, rb, s, unit_count, unit_mask)) return;
    if (lt.n_levels > 2 && row_in_level(i, K, zmax, 4) && (int64_t)chunk * CB <= lt.lev[2].rmax) {
        float t[LB];                                 // the out-of-line call's copy (S_2 stays in registers)
#pragma unroll
        for (int e = 0; e < LB; e++) t[e] = s[e];
        high_levels<E>(plane, nb, zmax, K, &lt, i, z, chunk, rb, t, unit_count, unit_mask);
    }
}

// The level-1 peaks among a lane's 16 bins rl .. rl + 15 of row i (a lane holding a value above
// the threshold, a handful per plane): re-read, test each against the 3x3 rule, return the mask.
template <typename E>
__device__ __noinline__ uint32_t level1_peaks(const E *__restrict__ plane, int64_t nb, int zmax, int K,
                                              const LevelDesc d, int i, int64_t rl) {
    uint32_t pk = 0;
    for (int e = 0; e < LB; e++) {
        const float v = ld_plane(plane, (int64_t)i * nb + rl + e);
        if (v > d.thr && local_max(plane, nb, zmax, K, 1, d.rmax, i, rl + e, v)) pk |= 1u << e;
    }
    return pk;
}

// Level 1 over the whole plane: a pure stream.  Grid (ceil(chunks1 / (DETECT_WARPS * CPW1)), K);
// each warp takes CPW1 consecutive chunks of row blockIdx.y, all loads issued first; a lane tests
// its 16 values through their maximum (BF16: packed) and widens them only when it holds a
// candidate.  Few registers, so many warps keep the loads in flight.
template <typename E>
__global__ void __launch_bounds__(DETECT_WARPS * 32, FDAS_K4_L1_MIN_BLOCKS) k4_level1(const E *__restrict__ plane, int64_t nb, int zmax,
                                                              int K, LevelDesc d, int chunks1,
                                                              int32_t *__restrict__ unit_count,
                                                              uint32_t *__restrict__ unit_mask) {
    constexpr int CPW1 = Fmt<E>::EPV == 8 ? 4 : 2;
    const int lane = threadIdx.x & 31;
    const int i = blockIdx.y;
    const int c0 = (blockIdx.x * DETECT_WARPS + (threadIdx.x >> 5)) * CPW1;
    if (c0 >= chunks1) return;                       // warp-uniform
    const E *row = plane + (int64_t)i * nb;
    typename Fmt<E>::Raw raw[CPW1];
#pragma unroll
    for (int c = 0; c < CPW1; c++)
        if (c0 + c < chunks1) Fmt<E>::load_raw(row + (int64_t)(c0 + c) * CB + LB * lane, raw[c]);
#pragma unroll
    for (int c = 0; c < CPW1; c++) {
        if (c0 + c >= chunks1) break;
        const float vmax = Fmt<E>::max16(raw[c]);
        const int u = (int)d.unit0 + i * (int)d.chunks + c0 + c;
        if (__any_sync(0xffffffffu, vmax > d.thr)) {
            const uint32_t pk =
                vmax > d.thr ? level1_peaks(plane, nb, zmax, K, d, i, (int64_t)(c0 + c) * CB + LB * lane) : 0u;
            int cnt = __popc(pk);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
            const uint32_t hi = __shfl_down_sync(0xffffffffu, pk, 1);
            if (lane == 0) count_unit(unit_count, u, cnt);
            if (cnt > 0 && !(lane & 1)) unit_mask[(int64_t)u * WORDS + (lane >> 1)] = pk | (hi << 16);
        } else if (lane == 0) {
            unit_count[u] = 0;
        }
    }
}

// Whether chunk c of row i (in level 2's region) can hold a level-2 .. peak given the plane
// kernel's unit marks: always inside level 4's region; outside it only when its unit or one of the
// two units of its second harmonic is marked (see levels_group).
__device__ __forceinline__ bool chunk_needs_search(const uint8_t *__restrict__ marks, int64_t chunks1, int zmax, int K,
                                                   const LevelTable &lt, int i, int c) {
    if (lt.n_levels >= 3 && row_in_level(i, K, zmax, 4) && (int64_t)c * CB <= lt.lev[2].rmax) return true;
    const int i2 = (2 * (-zmax + 2 * i) + zmax) >> 1;
    return __ldg(marks + (int64_t)i * chunks1 + c) | __ldg(marks + (int64_t)i2 * chunks1 + 2 * c) |
           __ldg(marks + (int64_t)i2 * chunks1 + 2 * c + 1);
}

// The level search's work list: one thread per entry k of the block order (row << 16 | 4-chunk
// group); an entry is kept when any of its chunks needs the search (chunk_needs_search), else its
// chunks' level-2 units count zero here.  Kept entries are appended per warp in the order's order
// (ballot prefix, one atomic per warp), so the list keeps the ray order's locality; *count
// (word 1 of the unit list's header) was cleared before the peak search.  Whole warps call it.
__device__ __noinline__ void select_entry(int64_t k, const uint32_t *__restrict__ order, int64_t n_order,
                                             const uint8_t *__restrict__ marks, int zmax, int K, const LevelTable &lt,
                                             int chunks2, uint32_t *__restrict__ work, unsigned int *__restrict__ count,
                                             int32_t *__restrict__ unit_count) {
    const int lane = threadIdx.x & 31;
    bool keep = false;
    uint32_t o = 0;
    if (k < n_order) {
        o = __ldg(order + k);
        const int a = (int)(o >> 16);
        if (a < lt.lev[1].rows) {
            const int i = lt.lev[1].i_lo + a;
            const int64_t chunks1 = lt.lev[0].chunks;
            const int c0 = (int)(o & 0xffffu) * DETECT_WARPS * CPW;
            for (int w = 0; w < DETECT_WARPS * CPW && c0 + w < chunks2; w++)
                keep |= chunk_needs_search(marks, chunks1, zmax, K, lt, i, c0 + w);
            if (!keep)
                for (int w = 0; w < DETECT_WARPS * CPW && c0 + w < chunks2; w++)
                    unit_count[(int)lt.lev[1].unit0 + a * (int)lt.lev[1].chunks + c0 + w] = 0;
        }
    }
    const uint32_t b = __ballot_sync(0xffffffffu, keep);
    unsigned int base = 0;
    if (lane == 0 && b) base = atomicAdd(count, (unsigned int)__popc(b));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (keep) work[base + __popc(b & ((1u << lane) - 1u))] = o;
}

// Level 1 after a plane kernel that marked its units (flags[u] != 0: the unit u = i chunks + c holds
// a stored value above the threshold): a warp takes 32 units, writes a zero count for the unmarked
// ones and runs the level-1 test of k4_level1 on each marked one (a handful per plane).  The
// plane is not streamed; the result is the same as k4_level1's.
// The blocks from l1_blocks on build the level search's work list instead (select_entry, one
// thread per entry of the block order; n_order = 0: none): the list depends only on the marks.
template <typename E>
__global__ void __launch_bounds__(DETECT_WARPS * 32) k4_level1_marked(const E *__restrict__ plane, int64_t nb, int zmax,
                                                                    int K, LevelDesc d, int64_t n_units1,
                                                                    const uint8_t *__restrict__ flags,
                                                                    int32_t *__restrict__ unit_count,
                                                                    uint32_t *__restrict__ unit_mask,
                                                                    int64_t l1_blocks,
                                                                    const uint32_t *__restrict__ order, int64_t n_order,
                                                                    LevelTable lt, int chunks2, uint32_t *__restrict__ work) {
    const int lane = threadIdx.x & 31;
    if (blockIdx.x >= l1_blocks) {                   // block-uniform
        select_entry((int64_t)(blockIdx.x - l1_blocks) * blockDim.x + threadIdx.x, order, n_order, flags, zmax, K, lt,
                     chunks2, work, unit_list(unit_count) + 1, unit_count);
        return;
    }
    const int64_t u0 = ((int64_t)blockIdx.x * DETECT_WARPS + (threadIdx.x >> 5)) * 32;
    if (u0 >= n_units1) return;                      // warp-uniform
    const int64_t u = u0 + lane;
    const bool marked = u < n_units1 && flags[u] != 0;
    if (u < n_units1 && !marked) unit_count[d.unit0 + u] = 0;
    uint32_t todo = __ballot_sync(0xffffffffu, marked);
    while (todo) {
        const int64_t uu = u0 + (__ffs(todo) - 1);
        todo &= todo - 1;
        const int i = (int)(uu / d.chunks);
        const int64_t rl = (uu - (int64_t)i * d.chunks) * CB + LB * lane;
        typename Fmt<E>::Raw raw;
        Fmt<E>::load_raw(plane + (int64_t)i * nb + rl, raw);
        const uint32_t pk = Fmt<E>::max16(raw) > d.thr ? level1_peaks(plane, nb, zmax, K, d, i, rl) : 0u;
        int cnt = __popc(pk);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
        const uint32_t hi = __shfl_down_sync(0xffffffffu, pk, 1);
        if (lane == 0) count_unit(unit_count, d.unit0 + uu, cnt);
        if (cnt > 0 && !(lane & 1)) unit_mask[(d.unit0 + uu) * WORDS + (lane >> 1)] = pk | (hi << 16);
    }
}

// Levels 2 .. 16 of one (row i, CPW chunks from c0) of level 2's region: each warp re-reads S_1
// of its chunks (interleaved bins, see add_level) and carries the running sums through the
// levels in registers.
//   With the plane kernel's unit marks (l2mark: the units holding a stored value above
// mark_threshold <= thr[1] / 2), a chunk outside level 4's region whose unit and the two units of
// its second harmonic are all unmarked is skipped: every P(r) and P(2 r) there is at most
// thr[1] / 2, so S_2 = P(r) + P(2 r) rounds to at most thr[1] (rounded addition is monotone and
// 2 (thr[1] / 2) is exact) and no cell can be a level-2 peak; its unit counts zero without reading
// the plane.  On a noise plane (mean 2) about one 512-bin unit in a hundred holds a value above
// thr[1] / 2 for the thresholds of the searches here, so most of these chunks are skipped.
template <typename E>
__device__ __forceinline__ void levels_group(const E *__restrict__ plane, int64_t nb, int zmax, int K,
                                             const LevelTable &lt, int chunks2, int i, int c0,
                                             int32_t *__restrict__ unit_count, uint32_t *__restrict__ unit_mask,
                                             const uint8_t *__restrict__ l2mark) {
    const int lane = threadIdx.x & 31;
    const int z = -zmax + 2 * i;
    if (l2mark != nullptr && CPW == 1 &&
        (lt.n_levels < 3 || !row_in_level(i, K, zmax, 4) || (int64_t)c0 * CB > lt.lev[2].rmax)) {
        const int64_t chunks1 = lt.lev[0].chunks;
        const int i2 = (2 * z + zmax) >> 1;
        const int64_t mu = lane == 0 ? (int64_t)i * chunks1 + c0 : (int64_t)i2 * chunks1 + 2 * c0 + (lane - 1);
        const bool marked = lane < 3 && __ldg(l2mark + mu) != 0;
        if (!__any_sync(0xffffffffu, marked)) {
            if (lane == 0) unit_count[(int)lt.lev[1].unit0 + (i - lt.lev[1].i_lo) * (int)lt.lev[1].chunks + c0] = 0;
            return;
        }
    }
    const E *row = plane + (int64_t)i * nb;
    const E *row2 = plane + (int64_t)((2 * z + zmax) >> 1) * nb;      // harmonic 2
    const int64_t rmax2 = lt.lev[1].rmax;
    float s2[CPW][LB];                               // S_2 of the lane's bins r0 + lane + 32 e
#pragma unroll
    for (int c = 0; c < CPW; c++)
        if (c0 + c < chunks2) {
            float v[LB];
#pragma unroll
            for (int e = 0; e < LB; e++) {           // S_1 and the second harmonic, all loads at once
                const int64_t r = (int64_t)(c0 + c) * CB + lane + 32 * e;
                s2[c][e] = ld_plane(row, r);
                v[e] = r <= rmax2 ? ld_plane(row2, 2 * r) : 0.0f;
            }
#pragma unroll
            for (int e = 0; e < LB; e++) s2[c][e] = __fadd_rn(s2[c][e], v[e]);
        }
#pragma unroll
    for (int c = 0; c < CPW; c++) {
        if (c0 + c >= chunks2) break;
        detect_chunk<E>(plane, nb, zmax, K, lt, i, z, c0 + c, (int64_t)(c0 + c) * CB + lane, s2[c], unit_count,
                        unit_mask);
    }
}

// Level 2's region row by row: grid (ceil(chunks2 / (DETECT_WARPS * CPW)), rows2), blocks of
// DETECT_WARPS warps on consecutive chunks of one row.
template <typename E>
__global__ void __launch_bounds__(DETECT_WARPS * 32, FDAS_K4_MIN_BLOCKS) k4_levels(const E *__restrict__ plane, int64_t nb, int zmax, int K,
                                                              LevelTable lt, int chunks2,
                                                              int32_t *__restrict__ unit_count,
                                                              uint32_t *__restrict__ unit_mask,
                                                              const uint8_t *__restrict__ l2mark) {
    const int c0 = (blockIdx.x * DETECT_WARPS + (threadIdx.x >> 5)) * CPW;
    if (c0 >= chunks2) return;                       // warp-uniform
    levels_group<E>(plane, nb, zmax, K, lt, chunks2, lt.lev[1].i_lo + blockIdx.y, c0, unit_count, unit_mask, l2mark);
}

// Level 2's region in the ray order of upload_levels_order, each entry a (row << 16 | chunk
// group): block b takes the entries b, b + gridDim.x, ... (so the blocks in flight keep to a short
// stretch of the order); with a persistent grid the next entry's code is loaded while the current
// one runs, which keeps the table's latency (about 1 us under load) off the critical path.  Any
// grid size covers every entry once; a grid of one block per entry runs the loop once.
template <typename E>
__global__ void __launch_bounds__(DETECT_WARPS * 32, FDAS_K4_MIN_BLOCKS) k4_levels_ordered(const E *__restrict__ plane, int64_t nb, int zmax, int K,
                                                                      LevelTable lt, int chunks2,
                                                                      const uint32_t *__restrict__ order, int64_t n_order,
                                                                      const unsigned int *__restrict__ d_count,
                                                                      int32_t *__restrict__ unit_count,
                                                                      uint32_t *__restrict__ unit_mask,
                                                                      const uint8_t *__restrict__ l2mark) {
    if (d_count != nullptr) n_order = *d_count;   // a work list (the level-1 pass's selection blocks), written before this launch
    int64_t idx = blockIdx.x;
    uint32_t next = idx < n_order ? __ldg(order + idx) : 0u;
    for (; idx < n_order; idx += gridDim.x) {
        const uint32_t o = next;
        if (idx + gridDim.x < n_order) next = __ldg(order + idx + gridDim.x);
        if ((int)(o >> 16) >= lt.lev[1].rows) continue;                       // block-uniform
        const int c0 = ((int)(o & 0xffffu) * DETECT_WARPS + (threadIdx.x >> 5)) * CPW;
        if (c0 >= chunks2) continue;                                          // warp-uniform
        levels_group<E>(plane, nb, zmax, K, lt, chunks2, lt.lev[1].i_lo + (int)(o >> 16), c0, unit_count, unit_mask,
                        l2mark);
    }
}

// Levels 2 .. 16 of the highest-harmonic-anchored sums (harm_mode 1) over the whole plane: grid
// (K rows, ceil(chunks / DETECT_WARPS)), so the blocks in flight share chunk positions across rows
// and the rows they gather from stay in L2.  A warp owns one (row, 512-bin chunk) with the lane
// bins interleaved (lane l holds r0 + l + 32 e) and carries the running sums through the levels.
// For each new harmonic j of level L, the terms r_j = floor((2 j r + L) / (2 L)) of 32
// consecutive r are at most 32 consecutive elements of row i_j, so each warp-wide load reads one
// or two sectors; a harmonic's 16 loads per lane are issued together.
#ifndef FDAS_K4A_BATCH
#define FDAS_K4A_BATCH 2                 // anchored harmonics whose loads are issued together
#endif
// S_L from S_{L/2} for the anchored sums: the odd harmonics j < L in increasing order, the loads
// of FDAS_K4A_BATCH harmonics in flight together (16 per harmonic and lane).  2 j r + L < 2^31 (r < Nb <= 2^26, j < 16),
// so the index arithmetic is 32-bit.  Lane bin r = rb + 32 e gathers at (2 j r + L) >> (LOG + 1) =
// ((2 j rb + L) >> (LOG + 1)) + 32 j e / L exactly (64 j e is a multiple of 2 L for L <= 32), so one
// index per harmonic and lane serves all 16 loads, which then differ by compile-time offsets.
template <typename E, int LOG>
__device__ __forceinline__ void anch_add_level(const E *__restrict__ plane, int64_t nb, int zmax, int z, uint32_t rb,
                                               float (&s)[LB]) {
    constexpr int L = 1 << LOG;
    constexpr int NB = FDAS_K4A_BATCH;
#pragma unroll
    for (int j0 = 1; j0 < L; j0 += 2 * NB) {
        float v[NB][LB];
#pragma unroll
        for (int q = 0; q < NB; q++) {
            const int j = j0 + 2 * q;
            if (j < L) {
                const int ij = (j * z + L * zmax + L) >> (LOG + 1);
                const uint32_t b = (2u * (uint32_t)j * rb + (uint32_t)L) >> (LOG + 1);
                const E *rowj = plane + (int64_t)ij * nb + b;
                static_assert(LOG + 1 <= 6, "the e-offsets are exact while 2 L divides 64");
#pragma unroll
                for (int e = 0; e < LB; e++) v[q][e] = ld_plane(rowj, (int64_t)((64 * j * e) >> (LOG + 1)));
            }
        }
#pragma unroll
        for (int q = 0; q < NB; q++)
            if (j0 + 2 * q < L) {
#pragma unroll
                for (int e = 0; e < LB; e++) s[e] = __fadd_rn(s[e], v[q][e]);
            }
        asm volatile("" ::: "memory");
    }
}

// The count and mask of one anchored unit (row i, chunk c) of level L, lane bins rb + 32 e.
template <typename E>
__device__ __forceinline__ void anch_unit(const E *__restrict__ plane, int64_t nb, int zmax, int K, const LevelDesc &d,
                                          int L, int i, int c, int64_t rb, const float (&s)[LB],
                                          int32_t *__restrict__ unit_count, uint32_t *__restrict__ unit_mask) {
    const int lane = threadIdx.x & 31;
    float vmax = s[0];
#pragma unroll
    for (int e = 1; e < LB; e++) vmax = fmaxf(vmax, s[e]);
    const int u = (int)d.unit0 + i * (int)d.chunks + c;
    if (__any_sync(0xffffffffu, vmax > d.thr)) {
        uint32_t pk = 0;
        if (vmax > d.thr) {
            for (int e = 0; e < LB; e++)
                if (s[e] > d.thr && local_max(plane, nb, zmax, K, L, d.rmax, i, rb + 32 * e, s[e], true)) pk |= 1u << e;
        }
        int cnt = __popc(pk);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
        if (lane == 0) count_unit(unit_count, u, cnt);
        if (cnt > 0) {
            uint32_t word = 0;
#pragma unroll
            for (int e = 0; e < LB; e++) {
                const uint32_t bal = __ballot_sync(0xffffffffu, (pk >> e) & 1u);
                if (lane == e) word = bal;
            }
            if (lane < WORDS) unit_mask[(int64_t)u * WORDS + lane] = word;
        }
    } else if (lane == 0) {
        unit_count[u] = 0;
    }
}

// Levels 2 .. 16 of the anchored sums for one (row i, chunk c), lane bins rb + 32 e.
template <typename E>
__device__ __forceinline__ void anch_chunk(const E *__restrict__ plane, int64_t nb, int zmax, int K, const LevelTable &lt,
                                           int i, int c, int32_t *__restrict__ unit_count,
                                           uint32_t *__restrict__ unit_mask) {
    const int lane = threadIdx.x & 31;
    const int z = -zmax + 2 * i;
    const int64_t rb = (int64_t)c * CB + lane;
    float s[LB];
    {
        const E *row = plane + (int64_t)i * nb;
#pragma unroll
        for (int e = 0; e < LB; e++) s[e] = ld_plane(row, rb + 32 * e);
    }
    anch_add_level<E, 1>(plane, nb, zmax, z, (uint32_t)rb, s);
    anch_unit<E>(plane, nb, zmax, K, lt.lev[1], 2, i, c, rb, s, unit_count, unit_mask);
    if (lt.n_levels < 3) return;
    anch_add_level<E, 2>(plane, nb, zmax, z, (uint32_t)rb, s);
    anch_unit<E>(plane, nb, zmax, K, lt.lev[2], 4, i, c, rb, s, unit_count, unit_mask);
    if (lt.n_levels < 4) return;
    anch_add_level<E, 3>(plane, nb, zmax, z, (uint32_t)rb, s);
    anch_unit<E>(plane, nb, zmax, K, lt.lev[3], 8, i, c, rb, s, unit_count, unit_mask);
    if (lt.n_levels < 5) return;
    anch_add_level<E, 4>(plane, nb, zmax, z, (uint32_t)rb, s);
    anch_unit<E>(plane, nb, zmax, K, lt.lev[4], 16, i, c, rb, s, unit_count, unit_mask);
}

template <typename E>
__global__ void __launch_bounds__(DETECT_WARPS * 32, FDAS_K4_MIN_BLOCKS) k4a_levels(const E *__restrict__ plane, int64_t nb,
                                                                               int zmax, int K, LevelTable lt,
                                                                               int chunks,
                                                                               int32_t *__restrict__ unit_count,
                                                                               uint32_t *__restrict__ unit_mask) {
    const int c = blockIdx.y * DETECT_WARPS + (threadIdx.x >> 5);
    if (c >= chunks) return;                         // warp-uniform
    anch_chunk<E>(plane, nb, zmax, K, lt, blockIdx.x, c, unit_count, unit_mask);
}

// The anchored levels in the ray order of upload_levels_order (whole plane, entries
// row << 16 | chunk group): the gathers of cell (r, z) lie on the segment from the origin to
// (r, z), so blocks taken by increasing z / r read each plane sector within a short stretch of
// the kernel's progress (from DRAM about once, where the row-major grid re-fetches the sectors of
// each fraction j / L of the chunk positions).  One block per entry.
template <typename E>
__global__ void __launch_bounds__(DETECT_WARPS * 32, FDAS_K4_MIN_BLOCKS) k4a_levels_ordered(
    const E *__restrict__ plane, int64_t nb, int zmax, int K, LevelTable lt, int chunks,
    const uint32_t *__restrict__ order, int32_t *__restrict__ unit_count, uint32_t *__restrict__ unit_mask) {
    const uint32_t o = __ldg(order + blockIdx.x);
    const int c = (int)(o & 0xffffu) * DETECT_WARPS + (threadIdx.x >> 5);
    if (c >= chunks) return;                         // warp-uniform
    anch_chunk<E>(plane, nb, zmax, K, lt, (int)(o >> 16), c, unit_count, unit_mask);
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

// The records of one non-empty unit u, the first at out[base]: one warp, the unit's mask words
// one per lane, the peaks in bin order (the order of the output within a unit).
template <typename E>
__device__ __forceinline__ void emit_unit(const E *__restrict__ plane, int64_t nb, int zmax, const LevelTable &lt,
                                          int64_t u, int64_t base, const uint32_t *__restrict__ unit_mask,
                                          fdas_peak *__restrict__ out, int max_peaks, uint32_t series) {
    const int lane = threadIdx.x & 31;
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
            pk.power = lt.anchored ? harm_sum_anch(plane, nb, zmax, H, ref.row, r)
                                   : harm_sum(plane, nb, zmax, H, ref.row, r);
            out[pos] = pk;
        }
        pos++;
    }
}

// Exclusive scan of one value per thread over a block of 1024 threads; *total = the block's sum.
// warp_tot: 32 ints of shared memory.  Every thread calls it (two barriers).
__device__ __forceinline__ int32_t block_excl_scan(int32_t c, int32_t *warp_tot, int32_t *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int32_t incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const int32_t wt = warp_tot[lane];
        int32_t wi = wt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        warp_tot[lane] = wi - wt;                        // exclusive warp offsets
        if (lane == 31) warp_tot[32] = wi;
    }
    __syncthreads();
    *total = warp_tot[32];
    return warp_tot[warp] + incl - c;
}

// The step's peaks, blocks of 1024 threads.  Usually the non-empty unit list holds every
// non-empty unit (a handful to a few hundred of ~10^6): block 0 alone sorts its unit numbers by
// rank (they are distinct: rank = how many are smaller), scans their counts in that order into
// output offsets and emits each unit's records with one warp; the other blocks return at once.
// Units are numbered in (level, row, chunk) order, so the records come out in (H, i, r) order.
// When more than PEAK_LIST_CAP units hold peaks (low thresholds, up to millions of peaks), every
// block takes a contiguous range of units: it sums the counts before its range (its first output
// offset; a few MB read from L2 per block, no communication between blocks), then scans its
// range 4096 units a round and emits the non-empty units as it goes.  The last block (or block 0
// on the listed path) writes the total and the overflow flag.
template <typename E>
__global__ void __launch_bounds__(1024) k4_emit_listed(const E *__restrict__ plane, int64_t nb, int zmax, LevelTable lt,
                                                       int64_t n_units, const int32_t *__restrict__ unit_count,
                                                       const uint32_t *__restrict__ unit_mask,
                                                       fdas_peak *__restrict__ out, int max_peaks, uint32_t series,
                                                       int32_t *__restrict__ npeaks, int32_t *__restrict__ status) {
    __shared__ uint32_t key[PEAK_LIST_CAP], sorted[PEAK_LIST_CAP];
    __shared__ int32_t offs[PEAK_LIST_CAP];
    __shared__ int32_t warp_tot[33];
    const int t = threadIdx.x, warp = t >> 5;
    const unsigned int *list = unit_list(unit_count);
    const int n = (int)*list;
    int64_t total = 0;
    bool writer = false;                                 // the block that writes the total
    if (n <= PEAK_LIST_CAP) {                            // grid-uniform
        if (blockIdx.x != 0) return;
        writer = true;
        if (t < n) key[t] = list[4 + t];
        __syncthreads();
        if (t < n) {
            const uint32_t k = key[t];
            int rank = 0;
            for (int j = 0; j < n; j++) rank += key[j] < k;
            sorted[rank] = k;
        }
        __syncthreads();
        // at most 1024 units x 512 peaks: 32-bit offsets
        const int32_t c = t < n ? unit_count[sorted[t]] : 0;
        int32_t tot;
        const int32_t ex = block_excl_scan(c, warp_tot, &tot);
        if (t < n) offs[t] = ex;
        total = tot;
        __syncthreads();
        for (int k = warp; k < n; k += 32)
            emit_unit<E>(plane, nb, zmax, lt, (int64_t)sorted[k], offs[k], unit_mask, out, max_peaks, series);
    } else {
        // this block's units [ub, ue) (whole rounds of 4096) and the count before them
        const int64_t rounds = (n_units + 4095) / 4096;
        const int64_t per = (rounds + gridDim.x - 1) / gridDim.x;
        const int64_t ub = min(n_units, (int64_t)blockIdx.x * per * 4096);
        const int64_t ue = min(n_units, ub + per * 4096);
        writer = blockIdx.x == gridDim.x - 1;
        {
            __shared__ unsigned long long pre_tot;       // counts are non-negative
            if (t == 0) pre_tot = 0ull;
            __syncthreads();
            unsigned long long acc = 0ull;
            for (int64_t u = t; u < ub; u += 1024) acc += (unsigned long long)unit_count[u];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if ((t & 31) == 0) atomicAdd(&pre_tot, acc);
            __syncthreads();
            total = (int64_t)pre_tot;
        }
        for (int64_t u0 = ub; u0 < ue; u0 += 4 * 1024) {
            const int64_t b0 = u0 + 4 * t;               // this thread's 4 units
            int32_t v[4];
#pragma unroll
            for (int k = 0; k < 4; k++) v[k] = b0 + k < ue ? unit_count[b0 + k] : 0;
            int32_t tot;
            int32_t run = block_excl_scan(v[0] + v[1] + v[2] + v[3], warp_tot, &tot);
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const int32_t mine = run;                // offset (in the round) of unit b0 + k
                run += v[k];
                uint32_t busy = __ballot_sync(0xffffffffu, v[k] != 0);
                while (busy) {                           // warp-uniform
                    const int j = __ffs(busy) - 1;
                    busy &= busy - 1;
                    const int32_t off_j = __shfl_sync(0xffffffffu, mine, j);
                    emit_unit<E>(plane, nb, zmax, lt, u0 + 4 * (32 * warp + j) + k, total + off_j, unit_mask, out,
                                 max_peaks, series);
                }
            }
            total += tot;
            __syncthreads();                             // warp_tot is reused by the next round
        }
    }
    if (writer && t == 0) {
        *npeaks = (int32_t)(total < 0x7fffffff ? total : 0x7fffffff);
        if (total > max_peaks) atomicOr(status, FDAS_DEV_PEAK_OVERFLOW);
    }
}

template <typename E>
cudaError_t run_peaks(const Plan &p, const E *plane, char *ws, fdas_peak *peaks, int32_t *npeaks, uint32_t series,
                      cudaStream_t st, const uint8_t *l1flag, bool list_cleared) {
    const LevelTable lt = make_levels(p);
    int32_t *unit_count = reinterpret_cast<int32_t *>(ws + p.ws_ucount);
    uint32_t *unit_mask = reinterpret_cast<uint32_t *>(ws + p.ws_umask);
    const int64_t chunks1 = lt.lev[0].chunks;
    constexpr int CPW1 = Fmt<E>::EPV == 8 ? 4 : 2;
    const dim3 level1_grid((unsigned)((chunks1 + DETECT_WARPS * CPW1 - 1) / (DETECT_WARPS * CPW1)), (unsigned)p.K);
    const int64_t chunks2 = lt.n_levels > 1 ? lt.lev[1].chunks : 0;
    const dim3 levels_grid((unsigned)((chunks2 + DETECT_WARPS * CPW - 1) / (DETECT_WARPS * CPW)),
                           (unsigned)(lt.n_levels > 1 ? lt.lev[1].rows : 0));
    if (lt.n_levels > 1 && !lt.anchored &&
        (!p.d_k4order || p.k4order_n != (int64_t)lt.lev[1].rows * ((chunks2 + DETECT_WARPS * CPW - 1) / (DETECT_WARPS * CPW))))
        return cudaErrorInvalidValue;                // the block order was not built for this region
    const int64_t n_units = p.n_units;
    // the plane kernel's unit marks (mark_threshold) bound the level-2 sums too
    const uint8_t *l2mark = l1flag && lt.n_levels > 1 ? l1flag : nullptr;
    p.prof.begin(FDAS_STAGE_PEAKS, st);
    // the non-empty unit list starts empty (its counter: the word PEAK_LIST_WORDS before the counts)
    // and so does the level search's work count (the next word); a search's long FFT has cleared
    // both already (list_cleared)
    uint32_t *list_hdr = reinterpret_cast<uint32_t *>(unit_count) - PEAK_LIST_WORDS;
    if (!list_cleared) {
        cudaError_t e0 = cudaMemsetAsync(list_hdr, 0, 2 * sizeof(uint32_t), st);
        if (e0 != cudaSuccess) return e0;
    }
    p.prof.launches += lt.n_levels > 1 ? 3 : 2;
    // with the marks, the level search's work list is built by extra blocks of the level-1 pass
    const bool select_list = l2mark != nullptr && lt.n_levels > 1 && !lt.anchored && (sizeof(E) == 4 || FDAS_K4_RAY_BF16);
    uint32_t *work = reinterpret_cast<uint32_t *>(ws + p.ws_k4work);
    unsigned int *wcount = select_list ? list_hdr + 1 : nullptr;
    p.prof.begin(PROF_PEAKS_LEVEL1, st);
    if (l1flag) {
        const int64_t n1 = (int64_t)p.K * chunks1;
        const int64_t blocks = (n1 + DETECT_WARPS * 32 - 1) / (DETECT_WARPS * 32);
        const int64_t n_sel = select_list ? p.k4order_n : 0;
        const int64_t sel_blocks = (n_sel + DETECT_WARPS * 32 - 1) / (DETECT_WARPS * 32);
        k4_level1_marked<E><<<(unsigned)(blocks + sel_blocks), DETECT_WARPS * 32, 0, st>>>(
            plane, p.nb, p.cfg.zmax, p.K, lt.lev[0], n1, l1flag, unit_count, unit_mask, blocks, p.d_k4order, n_sel,
            lt, (int)chunks2, work);
        p.prof.level1_fused++;
    } else {
        k4_level1<E><<<level1_grid, DETECT_WARPS * 32, 0, st>>>(plane, p.nb, p.cfg.zmax, p.K, lt.lev[0], (int)chunks1,
                                                                 unit_count, unit_mask);
    }
    p.prof.end(PROF_PEAKS_LEVEL1, st);
    if (lt.n_levels > 1 && lt.anchored) {
        p.prof.begin(PROF_PEAKS_LEVELS, st);
        const int64_t agroups = (chunks1 + DETECT_WARPS - 1) / DETECT_WARPS;
        if (p.d_k4order_a && p.k4order_a_n == (int64_t)p.K * agroups) {
            k4a_levels_ordered<E><<<(unsigned)p.k4order_a_n, DETECT_WARPS * 32, 0, st>>>(
                plane, p.nb, p.cfg.zmax, p.K, lt, (int)chunks1, p.d_k4order_a, unit_count, unit_mask);
        } else {
            const dim3 agrid((unsigned)p.K, (unsigned)agroups);
            k4a_levels<E><<<agrid, DETECT_WARPS * 32, 0, st>>>(plane, p.nb, p.cfg.zmax, p.K, lt, (int)chunks1,
                                                               unit_count, unit_mask);
        }
        p.prof.end(PROF_PEAKS_LEVELS, st);
    } else if (lt.n_levels > 1) {
        p.prof.begin(PROF_PEAKS_LEVELS, st);
        if (sizeof(E) == 4 || FDAS_K4_RAY_BF16) {
            // BF16 plane: a persistent grid (0.182 ms against 0.238 ms for one block per entry at
            // N = 2^23, 85 templates); FP32 plane: one block per entry (0.219 ms against 0.322 ms
            // persistent, its entries carry twice the bytes and the static stride balances worse)
            int sms = 0;
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p.device >= 0 ? p.device : 0);
            const int64_t blocks = sizeof(E) == 4 ? p.k4order_n
                                                  : std::min<int64_t>(p.k4order_n, (int64_t)std::max(sms, 1) * FDAS_K4_MIN_BLOCKS);
            // with the marks: select the entries to search first (a list in the workspace), so that the
            // skipped chunks cost one thread each instead of a warp's round trip in the search
            // (the work list from the level-1 pass's extra blocks, when the marks exist)
            const uint32_t *order = select_list ? work : p.d_k4order;
            k4_levels_ordered<E><<<(unsigned)blocks, DETECT_WARPS * 32, 0, st>>>(
                plane, p.nb, p.cfg.zmax, p.K, lt, (int)chunks2, order, p.k4order_n, wcount, unit_count,
                unit_mask, l2mark);
        } else {
            k4_levels<E><<<levels_grid, DETECT_WARPS * 32, 0, st>>>(plane, p.nb, p.cfg.zmax, p.K, lt, (int)chunks2,
                                                                     unit_count, unit_mask, l2mark);
        }
        p.prof.end(PROF_PEAKS_LEVELS, st);
    }
    // one block per SM: block 0 serves the usual (listed) case, all of them the overflowing one
    int sms_out = 152;
    cudaDeviceGetAttribute(&sms_out, cudaDevAttrMultiProcessorCount, p.device >= 0 ? p.device : 0);
    k4_emit_listed<E><<<(unsigned)std::max(1, sms_out), 1024, 0, st>>>(
        plane, p.nb, p.cfg.zmax, lt, n_units, unit_count, unit_mask, peaks, p.cfg.max_peaks, series, npeaks, p.d_status);
    p.prof.end(FDAS_STAGE_PEAKS, st);
    return cudaGetLastError();
}

}  // namespace

// Level H's region: rows [i_lo, i_lo + rows) and bins r <= rmax.  Plain sums: the rows with
// |H z| <= zmax and H r < Nb; anchored sums: the whole plane.
static void level_region(const Plan &p, int H, bool anchored, LevelDesc &d) {
    int zl = p.cfg.zmax / H;
    zl -= zl & 1;                                   // largest even z with |H z| <= zmax
    if (anchored) zl = p.cfg.zmax;
    d.H = H;
    d.i_lo = (p.cfg.zmax - zl) / 2;
    d.rows = zl + 1;
    d.rmax = anchored ? p.nb - 1 : (p.nb - 1) / H;
    d.chunks = (d.rmax + 1 + PEAK_CHUNK - 1) / PEAK_CHUNK;
}

LevelTable make_levels(const Plan &p) {
    LevelTable lt{};
    int64_t unit0 = 0;
    int n = 0;
    for (int l = 0; l < 5; l++) {
        const int H = 1 << l;
        if (H > p.cfg.max_harm) break;
        LevelDesc &d = lt.lev[n];
        level_region(p, H, p.cfg.harm_mode == 1, d);
        d.unit0 = unit0;
        d.thr = p.cfg.thr[l];
        unit0 += (int64_t)d.rows * d.chunks;
        n++;
    }
    lt.n_levels = n;
    lt.anchored = p.cfg.harm_mode == 1;
    return lt;
}

// The order in which k4_levels_ordered takes the (row, chunk group) blocks of level 2's region.
// Cell (r, z) gathers its harmonics at (h r, h z), on the ray from the origin through (r, z),
// where every other cell of that ray gathers too, and the rest of each gathered sector belongs
// to neighbouring rays.  Taking the blocks by increasing z / r (of the group's middle bin; ties
// by row, then group) brings all reads of a plane sector into a short stretch of the kernel's
// progress, so it comes from DRAM about once; row by row (k4_levels) the harmonic rows of rows
// far apart are fetched again, about twice the bytes.  Built for level 2's region whatever
// max_harm and harm_mode say, so that plans of one shape can share it.
bool levels_order(const Plan &p, std::vector<uint32_t> &order, bool anchored) {
    LevelDesc d{};
    level_region(p, 2, anchored, d);                  // anchored: the whole plane
    const int64_t per = DETECT_WARPS * (anchored ? 1 : CPW);   // chunks per block
    const int64_t groups = (d.chunks + per - 1) / per;
    if (d.rows >= (1 << 16) || groups >= (1 << 16)) return false;
    struct Item {
        double key;
        uint32_t code;
    };
    std::vector<Item> items;
    items.reserve((size_t)(d.rows * groups));
    for (int a = 0; a < d.rows; a++) {
        const int z = -p.cfg.zmax + 2 * (d.i_lo + a);
        for (int64_t g = 0; g < groups; g++)
            items.push_back({(double)z / ((double)(g * per) + 0.5 * (double)per), ((uint32_t)a << 16) | (uint32_t)g});
    }
    std::sort(items.begin(), items.end(),
              [](const Item &x, const Item &y) { return x.key < y.key || (x.key == y.key && x.code < y.code); });
    order.resize(items.size());
    for (size_t k = 0; k < items.size(); k++) order[k] = items[k].code;
    return true;
}

int64_t levels_order_size(const Plan &p) {
    LevelDesc d{};
    level_region(p, 2, false, d);
    const int64_t per = DETECT_WARPS * CPW;
    return (int64_t)d.rows * ((d.chunks + per - 1) / per);
}

cudaError_t upload_levels_order(Plan &p) {
    std::vector<uint32_t> order;
    if (!levels_order(p, order, false)) return cudaErrorInvalidValue;
    p.k4order_n = (int64_t)order.size();
    cudaError_t e = cudaMalloc((void **)&p.d_k4order, sizeof(uint32_t) * order.size());
    if (e == cudaSuccess)
        e = cudaMemcpy(p.d_k4order, order.data(), sizeof(uint32_t) * order.size(), cudaMemcpyHostToDevice);
    // the anchored sums' whole-plane order, for plans that use them
    if (e == cudaSuccess && p.cfg.harm_mode == 1 && levels_order(p, order, true)) {
        p.k4order_a_n = (int64_t)order.size();
        e = cudaMalloc((void **)&p.d_k4order_a, sizeof(uint32_t) * order.size());
        if (e == cudaSuccess)
            e = cudaMemcpy(p.d_k4order_a, order.data(), sizeof(uint32_t) * order.size(), cudaMemcpyHostToDevice);
    }
    return e;
}

cudaError_t launch_peaks(const Plan &p, const void *d_plane, bool bf16, char *ws, fdas_peak *d_peaks,
                         int32_t *d_npeaks, uint32_t series, cudaStream_t st, const uint8_t *l1flag, bool list_cleared) {
    if (bf16)
        return run_peaks<__nv_bfloat16>(p, reinterpret_cast<const __nv_bfloat16 *>(d_plane), ws, d_peaks, d_npeaks,
                                        series, st, l1flag, list_cleared);
    return run_peaks<float>(p, reinterpret_cast<const float *>(d_plane), ws, d_peaks, d_npeaks, series, st, l1flag,
                            list_cleared);
}

}  // namespace fdas
