// K4: harmonic sums and the thresholded peak list (Sec. 2.1: a pulsar shows as peaks at
// integer multiples of f and fdot, and the summed power of the harmonics is the detection
// statistic).
//
// For level H (1, 2, 4, 8, 16): S_H(r, i) = sum_{h=1..H} P(h r, i_h), z_{i_h} = h z_i,
// summed in FP32 in the order h = 1..H (BF16 planes are widened by placing the 16 stored
// bits in the top half of a float, the paper's quick cast of Sec. 3.1), defined where
// |H z_i| <= zmax and H r < Nb.  Peak: S_H > thr and a 3x3 local maximum (strictly above
// earlier neighbours in row-major (i, r) order, >= later ones).
//
// The list comes out in (H, i, r) order without a sort: the work is cut into tiles
// (level, row, chunk of PEAK_TILE bins), enumerated in that order;
//   pass 1 counts the peaks of every tile,
//   pass 2 (one CTA) turns the counts into exclusive offsets and the total,
//   pass 3 recomputes each tile and writes its peaks at offset + rank within the tile.
// A tile stages S_H for its row and the two neighbouring rows, bins r0-1 .. r1+1, in
// shared memory; undefined neighbours hold -inf and never block a peak.
#include <cmath>

#include "fdas_internal.cuh"

namespace fdas {

namespace {

__device__ __forceinline__ float ld_plane(const float *p, int64_t i) { return __ldg(p + i); }
__device__ __forceinline__ float ld_plane(const __nv_bfloat16 *p, int64_t i) {
    const unsigned short bits = __ldg(reinterpret_cast<const unsigned short *>(p) + i);
    return __uint_as_float(((unsigned)bits) << 16);
}

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

struct TileRef {
    int lev, row;
    int64_t r0, r1;
};

__device__ __forceinline__ TileRef locate(const LevelTable &lt, int64_t tile) {
    int l = 0;
#pragma unroll
    for (int k = 1; k < 5; k++)
        if (k < lt.n_levels && tile >= lt.lev[k].tile0) l = k;
    const LevelDesc &d = lt.lev[l];
    const int64_t local = tile - d.tile0;
    TileRef t;
    t.lev = l;
    t.row = d.i_lo + (int)(local / d.chunks);
    t.r0 = (local % d.chunks) * PEAK_TILE;
    t.r1 = min(t.r0 + PEAK_TILE - 1, d.rmax);
    return t;
}

template <typename E, bool WRITE>
__global__ void __launch_bounds__(PEAK_THREADS) k4_tiles(const E *__restrict__ plane, int64_t nb, int zmax, LevelTable lt,
                                                         int32_t *__restrict__ tile_count,
                                                         const int64_t *__restrict__ tile_off,
                                                         fdas_peak *__restrict__ out, int max_peaks, uint32_t series) {
    constexpr int W = PEAK_TILE + 2;
    constexpr int PER = PEAK_TILE / PEAK_THREADS;
    __shared__ float s[3][W];
    __shared__ int warp_tot[PEAK_THREADS / 32];
    const int64_t tile = blockIdx.x;
    const TileRef tr = locate(lt, tile);
    const LevelDesc &d = lt.lev[tr.lev];
    const int H = d.H;
    const int ncol = (int)(tr.r1 - tr.r0 + 3);
    for (int di = 0; di < 3; di++) {
        const int ii = tr.row - 1 + di;
        const bool row_ok = ii >= d.i_lo && ii < d.i_lo + d.rows;
        for (int c = threadIdx.x; c < ncol; c += PEAK_THREADS) {
            const int64_t r = tr.r0 - 1 + c;
            s[di][c] = (row_ok && r >= 0 && r <= d.rmax) ? harm_sum(plane, nb, zmax, H, ii, r) : -INFINITY;
        }
    }
    __syncthreads();
    const float thr = d.thr;
    unsigned mask = 0;
    int cnt = 0;
    const int c0 = threadIdx.x * PER;
#pragma unroll
    for (int e = 0; e < PER; e++) {
        const int c = c0 + e + 1;
        if (tr.r0 + c0 + e > tr.r1) break;
        const float v = s[1][c];
        if (!(v > thr)) continue;
        // earlier neighbours: previous row (all three) and the left cell: strictly greater
        bool pk = v > s[0][c - 1] && v > s[0][c] && v > s[0][c + 1] && v > s[1][c - 1];
        // later neighbours: right cell and next row: greater or equal
        pk = pk && v >= s[1][c + 1] && v >= s[2][c - 1] && v >= s[2][c] && v >= s[2][c + 1];
        if (pk) {
            mask |= 1u << e;
            cnt++;
        }
    }
    // block-wide exclusive scan of cnt (warp shuffles, then warp totals)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    int before = 0, total = 0;
    for (int w = 0; w < PEAK_THREADS / 32; w++) {
        if (w < warp) before += warp_tot[w];
        total += warp_tot[w];
    }
    const int excl = before + incl - cnt;
    if (!WRITE) {
        if (threadIdx.x == 0) tile_count[tile] = total;
        return;
    }
    int64_t pos = tile_off[tile] + excl;
#pragma unroll
    for (int e = 0; e < PER; e++) {
        if (!(mask & (1u << e))) continue;
        if (pos < max_peaks) {
            fdas_peak pk;
            pk.series = series;
            pk.r = (uint32_t)(tr.r0 + c0 + e);
            pk.zi = (int16_t)tr.row;
            pk.harm = (uint8_t)H;
            pk.pad = 0;
            pk.power = s[1][c0 + e + 1];
            out[pos] = pk;
        }
        pos++;
    }
}

// Exclusive scan of the tile counts (one CTA, fixed order) and the total peak count.
__global__ void __launch_bounds__(1024) k4_scan(const int32_t *__restrict__ cnt, int64_t n, int64_t *__restrict__ off,
                                                int32_t *__restrict__ npeaks, int max_peaks,
                                                int32_t *__restrict__ status) {
    __shared__ int64_t warp_tot[32];
    const int64_t per = (n + 1023) / 1024;
    const int64_t b = threadIdx.x * per, e = min(n, b + per);
    int64_t sum = 0;
    for (int64_t k = b; k < e; k++) sum += cnt[k];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    int64_t before = 0, total = 0;
    for (int w = 0; w < 32; w++) {
        if (w < warp) before += warp_tot[w];
        total += warp_tot[w];
    }
    int64_t run = before + incl - sum;
    for (int64_t k = b; k < e; k++) {
        off[k] = run;
        run += cnt[k];
    }
    if (threadIdx.x == 0) {
        *npeaks = (int32_t)(total < 0x7fffffff ? total : 0x7fffffff);
        if (total > max_peaks) atomicOr(status, FDAS_DEV_PEAK_OVERFLOW);
    }
}

template <typename E>
cudaError_t run_peaks(const Plan &p, const E *plane, char *ws, fdas_peak *peaks, int32_t *npeaks, uint32_t series,
                      cudaStream_t st) {
    const LevelTable lt = make_levels(p);
    int32_t *tile_count = reinterpret_cast<int32_t *>(ws + p.ws_tiles);
    int64_t *tile_off = reinterpret_cast<int64_t *>(ws + p.ws_tiles + ((sizeof(int32_t) * p.n_tiles + 255) & ~size_t(255)));
    const int64_t n = p.n_tiles;            // < 2^31: one block per tile on a 1-D grid
    p.prof.begin(FDAS_STAGE_PEAKS, st);
    p.prof.launches += 3;
    k4_tiles<E, false><<<(unsigned)n, PEAK_THREADS, 0, st>>>(plane, p.nb, p.cfg.zmax, lt, tile_count, tile_off,
                                                             peaks, p.cfg.max_peaks, series);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k4_scan<<<1, 1024, 0, st>>>(tile_count, n, tile_off, npeaks, p.cfg.max_peaks, p.d_status);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k4_tiles<E, true><<<(unsigned)n, PEAK_THREADS, 0, st>>>(plane, p.nb, p.cfg.zmax, lt, tile_count, tile_off,
                                                            peaks, p.cfg.max_peaks, series);
    p.prof.end(FDAS_STAGE_PEAKS, st);
    return cudaGetLastError();
}

}  // namespace

LevelTable make_levels(const Plan &p) {
    LevelTable lt{};
    int64_t tile0 = 0;
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
        d.chunks = (d.rmax + 1 + PEAK_TILE - 1) / PEAK_TILE;
        d.tile0 = tile0;
        d.thr = p.cfg.thr[l];
        tile0 += (int64_t)d.rows * d.chunks;
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
