// K6: band maxima of a plane (the paper's harmonic-band analysis, Sec. 4.3 and Table harm_bounds:
// with the pulsar's fundamental f known, the plane is split along frequency into bands and the
// highest cell of band n is taken as harmonic n).
//
// Band b covers bins [lo_b, hi_b] (inclusive) of every template row.  Its result is the largest
// value in the band and the first cell holding it in row-major (zi, r) order.  Each CTA reduces
// a slab of one band and folds its winner into the band's 64-bit slot with one atomicMax on
// (value bits << 32 | ~cell index): plane values are non-negative floats, whose bit patterns
// order like their values, and the inverted index makes the earliest cell win ties.
#include <algorithm>

#include "fdas_internal.cuh"

namespace fdas {

namespace {

constexpr int BAND_THREADS = 256;
constexpr int BAND_SLAB = 8192;                    // cells per CTA

__device__ __forceinline__ float band_ld(const float *p, int64_t i) { return __ldg(p + i); }
__device__ __forceinline__ float band_ld(const __nv_bfloat16 *p, int64_t i) {
    const unsigned short b = __ldg(reinterpret_cast<const unsigned short *>(p) + i);
    return __uint_as_float(((unsigned)b) << 16);
}

__global__ void k6_band_init(unsigned long long *slot, int n) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < n) slot[b] = 0ull;
}

// grid.x: slabs over the largest band, grid.y: bands
template <typename E>
__global__ void __launch_bounds__(BAND_THREADS) k6_band_max(const E *__restrict__ plane, int64_t nb, int K,
                                                            const int64_t *__restrict__ lo,
                                                            const int64_t *__restrict__ hi,
                                                            unsigned long long *__restrict__ slot) {
    const int b = blockIdx.y;
    const int64_t l = lo[b] > 0 ? lo[b] : 0, h = hi[b] < nb - 1 ? hi[b] : nb - 1;
    if (h < l) return;
    const int64_t width = h - l + 1;
    const int64_t cells = width * K;
    const int64_t c0 = (int64_t)blockIdx.x * BAND_SLAB;
    if (c0 >= cells) return;
    const int64_t c1 = min(cells, c0 + BAND_SLAB);
    unsigned long long best = 0ull;
    for (int64_t c = c0 + threadIdx.x; c < c1; c += BAND_THREADS) {
        const int64_t zi = c / width, r = l + (c - zi * width);
        const int64_t idx = zi * nb + r;
        const float v = band_ld(plane, idx);
        const unsigned long long key =
            ((unsigned long long)__float_as_uint(v) << 32) | (unsigned long long)(~(uint32_t)idx);
        best = key > best ? key : best;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long y = __shfl_xor_sync(0xffffffffu, best, o);
        best = y > best ? y : best;
    }
    __shared__ unsigned long long wbest[BAND_THREADS / 32];
    if ((threadIdx.x & 31) == 0) wbest[threadIdx.x >> 5] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < BAND_THREADS / 32; w++) best = wbest[w] > best ? wbest[w] : best;
        atomicMax(slot + b, best);
    }
}

__global__ void k6_band_out(const unsigned long long *__restrict__ slot, int n, int64_t nb, float *__restrict__ value,
                            int64_t *__restrict__ r, int32_t *__restrict__ zi) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n) return;
    const unsigned long long k = slot[b];
    const uint32_t idx = ~(uint32_t)(k & 0xffffffffull);
    const bool empty = k == 0ull;
    value[b] = empty ? -1.0f : __uint_as_float((uint32_t)(k >> 32));
    r[b] = empty ? -1 : (int64_t)(idx % (uint64_t)nb);
    zi[b] = empty ? -1 : (int32_t)(idx / (uint64_t)nb);
}

}  // namespace

cudaError_t launch_band_max(const Plan &p, const void *d_plane, bool bf16, const int64_t *d_lo, const int64_t *d_hi,
                            int n_bands, int64_t max_width, unsigned long long *d_slot, float *d_value,
                            int64_t *d_r, int32_t *d_zi, cudaStream_t st) {
    if (n_bands <= 0) return cudaSuccess;
    const unsigned nb_blocks = (unsigned)((n_bands + 255) / 256);
    k6_band_init<<<nb_blocks, 256, 0, st>>>(d_slot, n_bands);
    const int64_t slabs = std::max<int64_t>(1, (std::min(max_width, p.nb) * p.K + BAND_SLAB - 1) / BAND_SLAB);
    const dim3 grid((unsigned)slabs, (unsigned)n_bands);
    if (bf16)
        k6_band_max<__nv_bfloat16><<<grid, BAND_THREADS, 0, st>>>(static_cast<const __nv_bfloat16 *>(d_plane), p.nb,
                                                                   p.K, d_lo, d_hi, d_slot);
    else
        k6_band_max<float><<<grid, BAND_THREADS, 0, st>>>(static_cast<const float *>(d_plane), p.nb, p.K, d_lo, d_hi,
                                                           d_slot);
    k6_band_out<<<nb_blocks, 256, 0, st>>>(d_slot, n_bands, p.nb, d_value, d_r, d_zi);
    p.prof.launches += 3;
    return cudaGetLastError();
}

}  // namespace fdas
