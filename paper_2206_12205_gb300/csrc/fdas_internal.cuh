// Internal declarations shared by the libfdas translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>
#include <string>
#include <vector>

#include "../../include/fdas.h"

namespace fdas {

// Largest overlap-save / block-FFT length; the block-FFT twiddle table has this many
// entries and a length-L FFT reads every (TW_MAX/L)-th of them.
constexpr int TW_MAX = 8192;
// Two-level twiddle split for the long FFT: W_N^e = hi[e >> TW_LO_BITS] * lo[e & mask].
constexpr int TW_LO_BITS = 13;
// Segment length of the BF16 tensor-core path (64 x 64 four-step DFT) and its largest tap count.
constexpr int TC_S_BF16 = 4096;

// Stage-1 operand order of the tensor path (segment spectra and template banks, S = 64 x 64): per
// segment 16 chunks x 64 columns n2 of four 16-bit pairs; chunk ch of column n2 holds, with
// b = (ch & 1) + 8 (ch >> 1), (Re x[b], Re x[b+2]), (Im x[b], Im x[b+2]), (Re x[b+4], Re x[b+6]),
// (Im x[b+4], Im x[b+6]) of x[n1] = x[64 n1 + n2].  Position, in 16-bit elements, of
// Re x[64 n1 + n2]; Im x follows 2 elements later.
__host__ __device__ constexpr uint32_t tc_s1_pos(int n1, int n2) {
    return (((2u * (uint32_t)(n1 >> 3) + (uint32_t)(n1 & 1)) * 64u + (uint32_t)n2) * 4u +
            2u * (uint32_t)((n1 >> 2) & 1)) * 2u + (uint32_t)((n1 >> 1) & 1);
}
constexpr int TC_MAX_TAPS = 2048;
// Element index of (row, k) in a dense K-major no-swizzle operand image of R rows (8-row x 8-element
// core matrices of 128 bytes; core matrices adjacent along the rows, then along K).
__host__ __device__ constexpr uint32_t tc_kmajor_elem(uint32_t R, uint32_t row, uint32_t k) {
    return ((k >> 3) * (R >> 3) + (row >> 3)) * 64u + (row & 7u) * 8u + (k & 7u);
}

// Per-stage CUDA-event timing (fdas_profile_enable / fdas_profile_read).
constexpr int PROF_STAGES = 6;                   // the four stages, then the two K4 passes
constexpr int PROF_PEAKS_LEVEL1 = 4, PROF_PEAKS_LEVELS = 5;
constexpr int PROF_CAP = 512;
struct Profiler {
    bool on = false;
    cudaEvent_t ev[PROF_STAGES][PROF_CAP][2] = {};
    int n[PROF_STAGES] = {};
    int64_t calls = 0, launches = 0, level1_fused = 0;
    void begin(int stage, cudaStream_t st) {
        if (on && n[stage] < PROF_CAP) cudaEventRecord(ev[stage][n[stage]][0], st);
    }
    void end(int stage, cudaStream_t st) {
        if (on && n[stage] < PROF_CAP) {
            cudaEventRecord(ev[stage][n[stage]][1], st);
            n[stage]++;
        }
    }
};

struct Plan {
    fdas_config cfg;
    int64_t N, nb, n_seg;
    int K, m, S, L;
    int logS;
    // long real FFT split: M = N/2 = M1 * M2 (four-step)
    int64_t M;
    int M1, M2;
    // harmonic-sum levels and peak units (level, row, chunk)
    int n_levels;
    int64_t n_units;
    // workspace layout (byte offsets inside the caller's workspace)
    size_t ws_x, ws_tmp, ws_part, ws_scale, ws_y, ws_segscale, ws_ucount, ws_umask, ws_l1flag,
        ws_k4work, ws_bytes;
    int n_part;
    // plan-owned device memory
    int device;
    float2 *d_tw;          // TW_MAX block-FFT twiddles W_TW_MAX^j
    float2 *d_twn_lo;      // W_N^j, j < 2^TW_LO_BITS
    float2 *d_twn_hi;      // W_N^(j << TW_LO_BITS), j < max(1, N >> TW_LO_BITS)
    float2 *d_G;           // [K][S] FP32 template bank
    __nv_bfloat162 *d_Gbf; // [K][S] BF16 template bank, stage-1 operand order (tensor path)
    void *d_tcF;           // BF16 K-major DFT operand images: split hi, split lo, F1, F2 (4 x 32 KB)
    __half2 *d_Gh;         // [K][S] FP16 template bank times S, stage-1 operand order
    void *d_tcFh;          // FP16 K-major DFT operand images F1, F2 (2 x 32 KB)
    void *d_dimg;          // direct paths: conj(taps) real-ified, K-major operand image (BF16 or E4M3)
    float *d_dsig;         // FP8 direct path: 1 / sigma_z^2 per template (the taps' scales), 32 per group
    float2 *d_tcTw;        // W_4096^{n2 k1}, [k1][n2] (32 KB)
    uint32_t *d_k4order;   // ray order of level 2's (row << 16 | chunk group) blocks for k4_levels_ordered
    int64_t k4order_n;     // its length (rows x chunk groups)
    uint32_t *d_k4order_a; // harm_mode 1: ray order of the whole plane's (row << 16 | 4-chunk group) blocks
    int64_t k4order_a_n;   // its length (K x chunk groups)
    int32_t *d_status;     // sticky device status word
    bool templates_ready;
    bool borrowed;         // template bank and tables belong to another plan (a batch's group leader)
    // launch parameters chosen by the batch autotuner (0: built-in heuristic)
    int tune_zb;           // FP32 path: templates per correlation CTA
    int tune_cta_per_sm;   // split-BF16 path: persistent CTAs per SM
    std::string last_error;
    mutable Profiler prof;
};

// Peak search geometry: tiles of PEAK_ROWS rows x PEAK_CHUNK bins; a unit is one
// (level, row, chunk) with a count and a PEAK_CHUNK-bit mask.
constexpr int PEAK_ROWS = 8;
constexpr int PEAK_CHUNK = 512;
// The non-empty peak units, listed as the level kernels count them: a 4-word header (the list's
// count, then the level search's work count) and up to PEAK_LIST_CAP unit numbers, placed in the
// workspace directly before the unit counts.  When the list holds them all, the output block
// orders and emits them; else it scans every unit's count.
constexpr int PEAK_LIST_CAP = 1024;
constexpr int PEAK_LIST_WORDS = 4 + PEAK_LIST_CAP;

struct LevelDesc {
    int H;          // harmonic count
    int i_lo, rows; // valid rows [i_lo, i_lo + rows)
    int64_t rmax;   // last valid r (H r < nb)
    int64_t chunks; // r-chunks per row
    int64_t unit0;  // first unit index of this level
    float thr;
};
struct LevelTable {
    LevelDesc lev[5];
    int n_levels;
    int anchored;   // 1: highest-harmonic-anchored sums with rounding (every level on the whole plane)
};

LevelTable make_levels(const Plan &p);

// n-point Gauss-Legendre nodes xs and weights ws on [-1, 1] (host, FP64).
void gauss_legendre(int n, double *xs, double *ws);

// ---- launchers (each returns cudaGetLastError() of its launches) ----
cudaError_t launch_make_templates(Plan &p, cudaStream_t st);
cudaError_t launch_spectrum(const Plan &p, const float *d_series, char *ws, cudaStream_t st);
cudaError_t launch_local_norm(const Plan &p, const float2 *d_x, float2 *d_out, cudaStream_t st);
cudaError_t launch_apply_scale(const Plan &p, const char *ws, float *d_xhat, double *d_sigma2,
                               cudaStream_t st);
cudaError_t launch_plane_fp32(const Plan &p, const float2 *d_x, const float *d_scale, char *ws,
                              float *d_plane, cudaStream_t st, uint8_t *l1flag = nullptr);
// The same kernels with the segment spectra (n_seg * S complex64) at d_yhat instead of the workspace.
cudaError_t launch_plane_fp32_scratch(const Plan &p, const float2 *d_x, const float *d_scale, float2 *d_yhat,
                                      float *d_plane, cudaStream_t st);
// l1flag (optional, K x Nb/512 bytes): the plane kernel zeroes it and marks every 512-bin unit of
// a row holding a stored value above the level-1 threshold (the level-1 pass then reads only those).
cudaError_t launch_plane_bf16(const Plan &p, const float2 *d_x, const float *d_scale, char *ws,
                              __nv_bfloat16 *d_plane, cudaStream_t st, uint8_t *l1flag = nullptr);
cudaError_t launch_prepare_bf16(Plan &p, cudaStream_t st);
// FP32 segment spectra for 4096-bin segments (the split-BF16 path's input).
cudaError_t launch_segments_fp32(const Plan &p, const float2 *d_x, const float *d_scale, float2 *d_yhat,
                                 cudaStream_t st);
cudaError_t launch_plane_split(const Plan &p, const float2 *d_x, const float *d_scale, char *ws, float *d_plane,
                               cudaStream_t st);
bool direct_geometry(const Plan &p, int *Kpad, uint32_t *smem_bytes, uint32_t *tmem_cols);
size_t direct_pack_words(const Plan &p);
bool direct_geometry_f8(const Plan &p, int *n_groups, uint32_t *smem_bytes);
cudaError_t launch_plane_direct_f8(const Plan &p, const float2 *d_x, const float *d_scale, char *ws, float *d_plane,
                                   cudaStream_t st, uint8_t *l1flag = nullptr);
cudaError_t launch_plane_direct(const Plan &p, const float2 *d_x, const float *d_scale, char *ws,
                                __nv_bfloat16 *d_plane, cudaStream_t st, uint8_t *l1flag = nullptr);
cudaError_t launch_plane_f16(const Plan &p, const float2 *d_x, const float *d_scale, char *ws, float *d_plane,
                             cudaStream_t st, uint8_t *l1flag = nullptr);
// Whether the plan's plane kernel marks the level-1 units (every precision's plane kernel).
bool level1_fusable(const Plan &p);
// The threshold of the plane kernels' unit marks: a 512-bin unit is marked when it holds a stored
// value above min(thr[0], thr[1] / 2) (thr[0] alone without level 2).  The level-1 pass visits
// only marked units and tests them against thr[0]; the level search skips a chunk outside level
// 4's region whose unit and its second harmonic's two units are unmarked, since there every
// P(r) + P(2 r) rounds to at most 2 (thr[1] / 2) = thr[1] (exact halving, monotone rounding).
inline float mark_threshold(const Plan &p) {
    return p.cfg.max_harm >= 2 ? fminf(p.cfg.thr[0], p.cfg.thr[1] * 0.5f) : p.cfg.thr[0];
}
// The plane of the plan's precision from a spectrum (x: Nb complex; scale: device factor or NULL).
cudaError_t launch_plane_any(const Plan &p, const float2 *x, const float *scale, char *ws, void *d_plane,
                             cudaStream_t st, uint8_t *l1flag = nullptr);
// l1flag: the unit marks of the plane kernel that wrote d_plane (level 1 then visits only the
// marked units), or NULL for the full level-1 pass over the plane.
// The ray order of level 2's blocks (host; false if the region does not fit the 16-bit fields),
// and its upload into p.d_k4order at template time (synchronous copy).
bool levels_order(const Plan &p, std::vector<uint32_t> &order, bool anchored = false);
int64_t levels_order_size(const Plan &p);   // entries of the plain order (level 2's region)
cudaError_t upload_levels_order(Plan &p);
// list_cleared: the peak list's counters (PEAK_LIST_WORDS before the unit counts) were cleared
// earlier on the stream (launch_spectrum does); else the peak search clears them itself.
cudaError_t launch_peaks(const Plan &p, const void *d_plane, bool bf16, char *ws,
                         fdas_peak *d_peaks, int32_t *d_npeaks, uint32_t series, cudaStream_t st,
                         const uint8_t *l1flag = nullptr, bool list_cleared = false);
cudaError_t launch_band_max(const Plan &p, const void *d_plane, bool bf16, const int64_t *d_lo, const int64_t *d_hi,
                            int n_bands, int64_t max_width, unsigned long long *d_slot, float *d_value,
                            int64_t *d_r, int32_t *d_zi, cudaStream_t st);
cudaError_t launch_interp(Plan &p, const float2 *d_x, const fdas_cand *d_pts, const int64_t *d_k0, int n, bool fp64,
                          double *d_out, cudaStream_t st);
cudaError_t launch_refine(Plan &p, const float2 *d_x, const fdas_cand *d_in, int n, int steps, fdas_cand *d_out,
                          double *d_power, int32_t *d_evals, cudaStream_t st);

}  // namespace fdas
