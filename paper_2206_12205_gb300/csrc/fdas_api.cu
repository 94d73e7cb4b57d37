// libfdas C-ABI: plan validation, workspace layout and the entry points of include/fdas.h.
// The entry points only check arguments and enqueue kernels; all numerical work happens
// in the kernels of k0..k4.
#include <algorithm>
#include <cstring>
#include <new>

#include "fdas_internal.cuh"
#include "tc_sm100.cuh"

using fdas::Plan;

struct fdas_plan_s : public fdas::Plan {};

namespace {

Plan *P(fdas_plan_t h) { return static_cast<Plan *>(h); }

constexpr size_t ALIGN = 256;
size_t align_up(size_t x) { return (x + ALIGN - 1) & ~(ALIGN - 1); }
bool is_pow2(int64_t x) { return x > 0 && (x & (x - 1)) == 0; }
int ilog2(int64_t x) {
    int l = 0;
    while ((int64_t(1) << l) < x) l++;
    return l;
}

fdas_status record(Plan *p, cudaError_t e) {
    if (e == cudaSuccess) return FDAS_OK;
    if (p) p->last_error = std::string(cudaGetErrorName(e)) + ": " + cudaGetErrorString(e);
    (void)cudaGetLastError();   // clear a non-sticky error
    return e == cudaErrorMemoryAllocation ? FDAS_E_NOMEM : FDAS_E_CUDA;
}

bool plane_is_bf16(const Plan *p) { return p->cfg.precision == FDAS_BF16 || p->cfg.precision == FDAS_BF16_DIRECT; }
// the DFT-on-tensor-cores paths (segment spectra, DFT operand images and twiddles)
bool uses_tensor_path(const Plan *p) {
    return p->cfg.precision != FDAS_FP32 && p->cfg.precision != FDAS_BF16_DIRECT && p->cfg.precision != FDAS_FP8_DIRECT;
}

// Alignment the kernels' vector accesses rely on (documented in fdas.h).
bool aligned(const void *ptr, uintptr_t a) { return (reinterpret_cast<uintptr_t>(ptr) & (a - 1)) == 0; }
bool args_aligned(const void *series, const void *xhat, const void *ws, const void *plane, const void *peaks) {
    return aligned(series, 8) && aligned(xhat, 8) && aligned(ws, 256) && aligned(plane, 16) && aligned(peaks, 4);
}

}  // namespace

namespace fdas {
// One thread waits on a fresh mbarrier (phase 0 completes only on an arrival that never comes)
// for at most max_cycles, then records the timeout: the bounded wait of the plane kernels.
__global__ void wait_check(int64_t max_cycles, int32_t *status) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        tc::mbar_init(&bar, 1);
        if (!tc::mbar_wait_bounded(&bar, 0, (long long)max_cycles)) atomicOr(status, FDAS_DEV_TIMEOUT);
    }
}

cudaError_t launch_plane_any(const Plan &p, const float2 *x, const float *scale, char *ws, void *d_plane,
                             cudaStream_t st, uint8_t *l1flag) {
    switch (p.cfg.precision) {
        case FDAS_BF16: return launch_plane_bf16(p, x, scale, ws, static_cast<__nv_bfloat16 *>(d_plane), st, l1flag);
        case FDAS_BF16_SPLIT: return launch_plane_split(p, x, scale, ws, static_cast<float *>(d_plane), st);
        case FDAS_FP16_SCALED: return launch_plane_f16(p, x, scale, ws, static_cast<float *>(d_plane), st, l1flag);
        case FDAS_BF16_DIRECT:
            return launch_plane_direct(p, x, scale, ws, static_cast<__nv_bfloat16 *>(d_plane), st, l1flag);
        case FDAS_FP8_DIRECT: return launch_plane_direct_f8(p, x, scale, ws, static_cast<float *>(d_plane), st, l1flag);
        default: return launch_plane_fp32(p, x, scale, ws, static_cast<float *>(d_plane), st, l1flag);
    }
}
}  // namespace fdas

namespace {
cudaError_t launch_plane_any(Plan *p, const float2 *x, const float *scale, char *ws, void *d_plane, cudaStream_t st,
                             uint8_t *l1flag = nullptr) {
    return fdas::launch_plane_any(*p, x, scale, ws, d_plane, st, l1flag);
}
}  // namespace

extern "C" {

static_assert(sizeof(fdas_config) == 72, "fdas_config layout (the Python binding mirrors it)");

int fdas_version(void) { return 106; }

const char *fdas_status_string(fdas_status s) {
    switch (s) {
        case FDAS_OK: return "ok";
        case FDAS_E_INVALID: return "invalid argument";
        case FDAS_E_UNSUPPORTED: return "unsupported configuration";
        case FDAS_E_NOMEM: return "out of memory";
        case FDAS_E_CUDA: return "CUDA error";
        case FDAS_E_OVERFLOW: return "peak list overflow";
        case FDAS_E_TIMEOUT: return "device wait timed out";
        case FDAS_E_STATE: return "call out of order";
    }
    return "unknown status";
}

fdas_status fdas_plan(const fdas_config *cfg, fdas_plan_t *plan, size_t *workspace_bytes) {
    if (!cfg || !plan) return FDAS_E_INVALID;
    *plan = nullptr;
    const fdas_config c = *cfg;
    if (!is_pow2(c.n_samples) || c.n_samples < (int64_t(1) << 11) || c.n_samples > (int64_t(1) << 27))
        return FDAS_E_INVALID;
    if (c.zmax < 0 || c.zmax > 1022 || (c.zmax & 1)) return FDAS_E_INVALID;
    if (!(c.seg_len == 1024 || c.seg_len == 2048 || c.seg_len == 4096 || c.seg_len == 8192)) return FDAS_E_INVALID;
    if (c.taps < 2 || (c.taps & 1) || c.taps > c.seg_len / 2) return FDAS_E_INVALID;
    if (!(c.max_harm == 1 || c.max_harm == 2 || c.max_harm == 4 || c.max_harm == 8 || c.max_harm == 16))
        return FDAS_E_INVALID;
    if (c.max_peaks < 0) return FDAS_E_INVALID;
    if (!(c.sigma2 >= 0.0)) return FDAS_E_INVALID;   // also rejects NaN
    if (c.harm_mode != 0 && c.harm_mode != 1) return FDAS_E_INVALID;
    if (c.norm_block != 0 && (!is_pow2(c.norm_block) || c.norm_block < 64 || c.norm_block > 65536 ||
                              c.sigma2 > 0.0 || c.norm_block > c.n_samples / 2))
        return FDAS_E_INVALID;
    for (int l = 0; l < 5; l++)
        if (c.thr[l] != c.thr[l]) return FDAS_E_INVALID;
    if (c.precision != FDAS_FP32 && c.precision != FDAS_BF16 && c.precision != FDAS_BF16_SPLIT &&
        c.precision != FDAS_FP16_SCALED && c.precision != FDAS_BF16_DIRECT && c.precision != FDAS_FP8_DIRECT)
        return FDAS_E_INVALID;
    if (c.precision != FDAS_FP32 && c.taps > fdas::TC_MAX_TAPS) return FDAS_E_UNSUPPORTED;

    fdas_plan_s *p = new (std::nothrow) fdas_plan_s();
    if (!p) return FDAS_E_NOMEM;
    p->cfg = c;
    p->N = c.n_samples;
    p->nb = p->N / 2;
    p->K = c.zmax + 1;
    p->m = c.taps;
    p->S = c.seg_len;
    // FP32 path: stride a multiple of 32 bins, so each warp's plane stores cover whole 128-byte
    // lines (any L <= S - m + 1 gives the same plane)
    p->L = (p->S - p->m + 1) / 32 * 32;
    if (c.precision != FDAS_FP32) {
        // tensor-core path: 4096-bin segments, stride a multiple of 64 (same plane for any L)
        p->S = fdas::TC_S_BF16;
        p->L = (p->S - p->m + 1) / 64 * 64;
    }
    p->logS = ilog2(p->S);
    p->n_seg = (p->nb + p->L - 1) / p->L;
    p->M = p->nb;
    const int lgM = ilog2(p->M);
    p->M1 = 1 << ((lgM + 1) / 2);
    p->M2 = 1 << (lgM / 2);
    const fdas::LevelTable lt = fdas::make_levels(*p);
    p->n_levels = lt.n_levels;
    p->n_units = lt.lev[lt.n_levels - 1].unit0 + (int64_t)lt.lev[lt.n_levels - 1].rows * lt.lev[lt.n_levels - 1].chunks;
    p->n_part = p->M1 / 2;
    // workspace layout
    size_t off = 0;
    p->ws_x = off;     off = align_up(off + sizeof(float2) * (size_t)p->nb);
    p->ws_tmp = off;   off = align_up(off + sizeof(float2) * (size_t)p->M);
    p->ws_part = off;  off = align_up(off + sizeof(double) * (size_t)p->n_part);
    p->ws_scale = off; off = align_up(off + 16);
    if ((c.precision == FDAS_BF16_DIRECT && !fdas::direct_geometry(*p, nullptr, nullptr, nullptr)) ||
        (c.precision == FDAS_FP8_DIRECT && !fdas::direct_geometry_f8(*p, nullptr, nullptr))) {
        delete p;
        return FDAS_E_UNSUPPORTED;
    }
    // segment spectra, or the BF16 direct path's packed spectrum (the FP8 direct path reads the
    // spectrum itself)
    const size_t ybytes = c.precision == FDAS_BF16_DIRECT ? sizeof(uint32_t) * fdas::direct_pack_words(*p)
                          : c.precision == FDAS_FP8_DIRECT ? 256
                                                           : sizeof(float2) * (size_t)p->n_seg * p->S;
    p->ws_y = off;     off = align_up(off + ybytes);
    p->ws_segscale = off; off = align_up(off + sizeof(float) * (size_t)p->n_seg);
    // the non-empty unit list directly before the counts (the kernels find it from the counts)
    off += sizeof(uint32_t) * fdas::PEAK_LIST_WORDS;
    p->ws_ucount = off; off = align_up(off + sizeof(int32_t) * (size_t)p->n_units);
    p->ws_umask = off;  off = align_up(off + sizeof(uint32_t) * (fdas::PEAK_CHUNK / 32) * (size_t)p->n_units);
    p->ws_l1flag = off; off = align_up(off + (size_t)p->K * (size_t)(p->nb / fdas::PEAK_CHUNK));
    // the level search's work list (the entries of its block order that are not skipped)
    p->ws_k4work = off; off = align_up(off + sizeof(uint32_t) * (size_t)std::max<int64_t>(1, fdas::levels_order_size(*p)));
    p->ws_bytes = off;
    p->device = -1;
    *plan = p;
    if (workspace_bytes) *workspace_bytes = p->ws_bytes;
    return FDAS_OK;
}

fdas_status fdas_levels_order(fdas_plan_t plan, uint32_t *h_order, int64_t capacity, int64_t *n_out) {
    if (!plan || !n_out) return FDAS_E_INVALID;
    std::vector<uint32_t> order;
    if (!fdas::levels_order(*P(plan), order)) return FDAS_E_UNSUPPORTED;
    *n_out = (int64_t)order.size();
    if (!h_order) return FDAS_OK;
    if (capacity < *n_out) return FDAS_E_INVALID;
    std::copy(order.begin(), order.end(), h_order);
    return FDAS_OK;
}

fdas_status fdas_plan_get_info(fdas_plan_t plan, fdas_plan_info *info) {
    if (!plan || !info) return FDAS_E_INVALID;
    const Plan *p = P(plan);
    info->nb = p->nb;
    info->K = p->K;
    info->seg_valid = p->L;
    info->n_seg = p->n_seg;
    info->plane_elem_bytes = plane_is_bf16(p) ? 2 : 4;
    info->cells = (int64_t)p->K * p->nb;
    info->plane_bytes = info->cells * info->plane_elem_bytes;
    info->workspace_bytes = p->ws_bytes;
    return FDAS_OK;
}

fdas_status fdas_make_templates(fdas_plan_t plan, void *stream) {
    if (!plan) return FDAS_E_INVALID;
    Plan *p = P(plan);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (p->templates_ready) return FDAS_OK;
    cudaError_t e = cudaGetDevice(&p->device);
    if (e != cudaSuccess) return record(p, e);
    const size_t nbank = (size_t)p->K * p->S;
    const int64_t nhi = std::max<int64_t>(1, p->N >> fdas::TW_LO_BITS);
    auto alloc = [&](void **ptr, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(ptr, bytes);
    };
    alloc((void **)&p->d_tw, sizeof(float2) * fdas::TW_MAX);
    alloc((void **)&p->d_twn_lo, sizeof(float2) * ((size_t)1 << fdas::TW_LO_BITS));
    alloc((void **)&p->d_twn_hi, sizeof(float2) * (size_t)nhi);
    alloc((void **)&p->d_G, sizeof(float2) * nbank);
    if (uses_tensor_path(p)) {
        if (p->cfg.precision == FDAS_BF16) alloc((void **)&p->d_Gbf, sizeof(__nv_bfloat162) * nbank);
        if (p->cfg.precision == FDAS_FP16_SCALED) {
            alloc((void **)&p->d_Gh, sizeof(__half2) * nbank);
            alloc((void **)&p->d_tcFh, 2 * 2 * 128 * 128);
        }
        alloc((void **)&p->d_tcF, 4 * 2 * 128 * 128);
        alloc((void **)&p->d_tcTw, sizeof(float2) * 64 * 64);
    }
    if (p->cfg.precision == FDAS_BF16_DIRECT) {
        int kp = 0;
        fdas::direct_geometry(*p, &kp, nullptr, nullptr);
        alloc((void **)&p->d_dimg, (size_t)2 * kp * 2 * p->m * 2);
    }
    if (p->cfg.precision == FDAS_FP8_DIRECT) {
        int groups = 0;
        fdas::direct_geometry_f8(*p, &groups, nullptr);
        alloc((void **)&p->d_dimg, (size_t)groups * 64 * 2 * p->m);
        alloc((void **)&p->d_dsig, sizeof(float) * 32 * (size_t)groups);
    }
    alloc((void **)&p->d_status, sizeof(int32_t));
    if (e == cudaSuccess) e = fdas::upload_levels_order(*p);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->d_status, 0, sizeof(int32_t), st);
    if (e == cudaSuccess) e = fdas::launch_make_templates(*p, st);
    if (e == cudaSuccess && uses_tensor_path(p)) e = fdas::launch_prepare_bf16(*p, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return record(p, e);
    p->templates_ready = true;
    return FDAS_OK;
}

static fdas_status ready(Plan *p) {
    if (!p->templates_ready) return FDAS_E_STATE;
    return FDAS_OK;
}

fdas_status fdas_spectrum(fdas_plan_t plan, const float *d_series, void *d_workspace, float *d_xhat,
                          double *d_sigma2, void *stream) {
    if (!plan || !d_series || !d_workspace || !d_xhat) return FDAS_E_INVALID;
    if (!args_aligned(d_series, d_xhat, d_workspace, nullptr, nullptr)) return FDAS_E_INVALID;
    Plan *p = P(plan);
    if (fdas_status s = ready(p)) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    char *ws = static_cast<char *>(d_workspace);
    p->prof.calls++;
    cudaError_t e = fdas::launch_spectrum(*p, d_series, ws, st);
    if (e == cudaSuccess) e = fdas::launch_apply_scale(*p, ws, d_xhat, d_sigma2, st);
    if (e == cudaSuccess && p->cfg.norm_block)        // local normalisation replaces the global scale
        e = fdas::launch_local_norm(*p, reinterpret_cast<const float2 *>(ws + p->ws_x),
                                    reinterpret_cast<float2 *>(d_xhat), st);
    return record(p, e);
}

fdas_status fdas_plane(fdas_plan_t plan, const float *d_xhat, void *d_workspace, void *d_plane, void *stream) {
    if (!plan || !d_xhat || !d_workspace || !d_plane) return FDAS_E_INVALID;
    if (!args_aligned(nullptr, d_xhat, d_workspace, d_plane, nullptr)) return FDAS_E_INVALID;
    Plan *p = P(plan);
    if (fdas_status s = ready(p)) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    char *ws = static_cast<char *>(d_workspace);
    const float2 *x = reinterpret_cast<const float2 *>(d_xhat);
    p->prof.calls++;
    const cudaError_t e = launch_plane_any(p, x, nullptr, ws, d_plane, st);
    return record(p, e);
}

fdas_status fdas_peaks(fdas_plan_t plan, const void *d_plane, void *d_workspace, fdas_peak *d_peaks,
                       int32_t *d_npeaks, void *stream) {
    if (!plan || !d_plane || !d_workspace || !d_npeaks || (!d_peaks && P(plan)->cfg.max_peaks > 0))
        return FDAS_E_INVALID;
    if (!args_aligned(nullptr, nullptr, d_workspace, d_plane, d_peaks) || !aligned(d_npeaks, 4)) return FDAS_E_INVALID;
    Plan *p = P(plan);
    if (fdas_status s = ready(p)) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    p->prof.calls++;
    cudaError_t e = fdas::launch_peaks(*p, d_plane, plane_is_bf16(p), static_cast<char *>(d_workspace), d_peaks,
                                       d_npeaks, 0u, st);
    return record(p, e);
}

fdas_status fdas_search(fdas_plan_t plan, const float *d_series, void *d_workspace, void *d_plane,
                        fdas_peak *d_peaks, int32_t *d_npeaks, void *stream) {
    if (!plan || !d_series || !d_workspace || !d_plane || !d_npeaks || (!d_peaks && P(plan)->cfg.max_peaks > 0))
        return FDAS_E_INVALID;
    if (!args_aligned(d_series, nullptr, d_workspace, d_plane, d_peaks) || !aligned(d_npeaks, 4)) return FDAS_E_INVALID;
    Plan *p = P(plan);
    if (fdas_status s = ready(p)) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    char *ws = static_cast<char *>(d_workspace);
    p->prof.calls++;
    cudaError_t e = fdas::launch_spectrum(*p, d_series, ws, st);
    float2 *x = reinterpret_cast<float2 *>(ws + p->ws_x);
    const float *scale = reinterpret_cast<const float *>(ws + p->ws_scale + 8);
    if (e == cudaSuccess && p->cfg.norm_block) {      // normalised in place, no global scale
        e = fdas::launch_local_norm(*p, x, x, st);
        scale = nullptr;
    }
    // the tensor-core plane kernels mark the level-1 units as they store the plane
    uint8_t *l1flag = fdas::level1_fusable(*p) ? reinterpret_cast<uint8_t *>(ws + p->ws_l1flag) : nullptr;
    if (e == cudaSuccess) e = launch_plane_any(p, x, scale, ws, d_plane, st, l1flag);
    if (e == cudaSuccess)
        e = fdas::launch_peaks(*p, d_plane, plane_is_bf16(p), ws, d_peaks, d_npeaks, 0u, st, l1flag, true);
    return record(p, e);
}

fdas_status fdas_interp_power(fdas_plan_t plan, const float *d_xhat, const fdas_cand *d_pts, const int64_t *d_k0,
                              int32_t n, int32_t fp64, double *d_out, void *stream) {
    if (!plan || n < 0 || (fp64 != 0 && fp64 != 1)) return FDAS_E_INVALID;
    if (n == 0) return FDAS_OK;
    if (!d_xhat || !d_pts || !d_out) return FDAS_E_INVALID;
    if (!aligned(d_xhat, 8) || !aligned(d_pts, 8) || !aligned(d_out, 8) || (d_k0 && !aligned(d_k0, 8)))
        return FDAS_E_INVALID;
    Plan *p = P(plan);
    p->prof.calls++;
    const cudaError_t e = fdas::launch_interp(*p, reinterpret_cast<const float2 *>(d_xhat), d_pts, d_k0, n, fp64 != 0,
                                              d_out, static_cast<cudaStream_t>(stream));
    return record(p, e);
}

fdas_status fdas_refine(fdas_plan_t plan, const float *d_xhat, const fdas_cand *d_in, int32_t n, int32_t steps,
                        fdas_cand *d_out, double *d_power, int32_t *d_evals, void *stream) {
    if (!plan || n < 0 || steps < 0 || steps > FDAS_REFINE_MAX_STEPS) return FDAS_E_INVALID;
    if (n == 0) return FDAS_OK;
    if (!d_xhat || !d_in || !d_out) return FDAS_E_INVALID;
    if (!aligned(d_xhat, 8) || !aligned(d_in, 8) || !aligned(d_out, 8) || (d_power && !aligned(d_power, 8)) ||
        (d_evals && !aligned(d_evals, 4)))
        return FDAS_E_INVALID;
    Plan *p = P(plan);
    p->prof.calls++;
    const cudaError_t e = fdas::launch_refine(*p, reinterpret_cast<const float2 *>(d_xhat), d_in, n, steps, d_out,
                                              d_power, d_evals, static_cast<cudaStream_t>(stream));
    return record(p, e);
}

fdas_status fdas_band_max(fdas_plan_t plan, const void *d_plane, const int64_t *h_lo, const int64_t *h_hi,
                          int32_t n_bands, void *d_scratch, float *d_value, int64_t *d_r, int32_t *d_zi, void *stream) {
    if (!plan || n_bands < 0) return FDAS_E_INVALID;
    if (n_bands == 0) return FDAS_OK;
    if (!d_plane || !h_lo || !h_hi || !d_scratch || !d_value || !d_r || !d_zi) return FDAS_E_INVALID;
    if (!aligned(d_plane, 16) || !aligned(d_scratch, 8) || !aligned(d_value, 4) || !aligned(d_r, 8) ||
        !aligned(d_zi, 4))
        return FDAS_E_INVALID;
    Plan *p = P(plan);
    if ((uint64_t)p->K * (uint64_t)p->nb >= (1ull << 32)) {
        p->last_error = "band maxima index cells with 32 bits: K * Nb must stay below 2^32";
        return FDAS_E_UNSUPPORTED;
    }
    int64_t max_width = 0;
    for (int b = 0; b < n_bands; b++) {
        if (h_lo[b] > h_hi[b]) return FDAS_E_INVALID;
        max_width = std::max(max_width, std::min<int64_t>(h_hi[b], p->nb - 1) - std::max<int64_t>(h_lo[b], 0) + 1);
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned long long *slot = static_cast<unsigned long long *>(d_scratch);
    int64_t *lo = reinterpret_cast<int64_t *>(slot + n_bands);
    int64_t *hi = lo + n_bands;
    p->prof.calls++;
    cudaError_t e = cudaMemcpyAsync(lo, h_lo, sizeof(int64_t) * n_bands, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hi, h_hi, sizeof(int64_t) * n_bands, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = fdas::launch_band_max(*p, d_plane, plane_is_bf16(p), lo, hi, n_bands, max_width, slot, d_value, d_r, d_zi,
                                  st);
    return record(p, e);
}

fdas_status fdas_get_templates(fdas_plan_t plan, float *d_out, void *stream) {
    if (!plan || !d_out) return FDAS_E_INVALID;
    Plan *p = P(plan);
    if (fdas_status s = ready(p)) return s;
    cudaError_t e = cudaMemcpyAsync(d_out, p->d_G, sizeof(float2) * (size_t)p->K * p->S, cudaMemcpyDeviceToDevice,
                                    static_cast<cudaStream_t>(stream));
    return record(p, e);
}

fdas_status fdas_check_timeout(fdas_plan_t plan, int64_t max_cycles, void *stream) {
    if (!plan || max_cycles < 1 || max_cycles > (int64_t{1} << 36)) return FDAS_E_INVALID;
    Plan *p = P(plan);
    if (!p->templates_ready || !p->d_status) return FDAS_E_STATE;
    fdas::wait_check<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(max_cycles, p->d_status);
    return record(p, cudaGetLastError());
}

fdas_status fdas_device_status(fdas_plan_t plan, int32_t *bits, int clear) {
    if (!plan || !bits) return FDAS_E_INVALID;
    Plan *p = P(plan);
    *bits = 0;
    if (!p->d_status) return FDAS_OK;
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(bits, p->d_status, sizeof(int32_t), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && clear) e = cudaMemset(p->d_status, 0, sizeof(int32_t));
    return record(p, e);
}

fdas_status fdas_profile_enable(fdas_plan_t plan, int enable) {
    if (!plan) return FDAS_E_INVALID;
    Plan *p = P(plan);
    fdas::Profiler &pr = p->prof;
    if (enable && !pr.on) {
        for (int s = 0; s < fdas::PROF_STAGES; s++)
            for (int i = 0; i < fdas::PROF_CAP; i++)
                for (int k = 0; k < 2; k++) {
                    if (pr.ev[s][i][k]) continue;
                    cudaError_t e = cudaEventCreate(&pr.ev[s][i][k]);
                    if (e != cudaSuccess) return record(p, e);
                }
        for (int s = 0; s < fdas::PROF_STAGES; s++) pr.n[s] = 0;
    }
    pr.on = enable != 0;
    return FDAS_OK;
}

fdas_status fdas_profile_read(fdas_plan_t plan, fdas_profile *out, int reset) {
    if (!plan || !out) return FDAS_E_INVALID;
    Plan *p = P(plan);
    fdas::Profiler &pr = p->prof;
    std::memset(out, 0, sizeof(*out));
    out->calls = pr.calls;
    out->launches = pr.launches;
    out->level1_fused = pr.level1_fused;
    int any = 0;
    for (int s = 0; s < fdas::PROF_STAGES; s++) any += pr.n[s];
    if (any > 0) {
        cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return record(p, e);
        for (int s = 0; s < fdas::PROF_STAGES; s++) {
            double acc = 0.0;
            for (int i = 0; i < pr.n[s]; i++) {
                float ms = 0.f;
                e = cudaEventElapsedTime(&ms, pr.ev[s][i][0], pr.ev[s][i][1]);
                if (e != cudaSuccess) return record(p, e);
                acc += ms;
            }
            if (s < 4) {
                out->ms[s] = acc;
                out->n_timed[s] = pr.n[s];
            } else {
                out->ms_peaks[s - 4] = acc;
                out->n_timed_peaks[s - 4] = pr.n[s];
            }
        }
    }
    if (reset) {
        pr.calls = pr.launches = pr.level1_fused = 0;
        for (int s = 0; s < fdas::PROF_STAGES; s++) pr.n[s] = 0;
    }
    return FDAS_OK;
}

const char *fdas_last_error(fdas_plan_t plan) {
    if (!plan) return "";
    return P(plan)->last_error.c_str();
}

void fdas_destroy(fdas_plan_t plan) {
    if (!plan) return;
    Plan *p = P(plan);
    if (p->device >= 0 && p->borrowed) {
        cudaDeviceSynchronize();
        cudaFree(p->d_status);
    } else if (p->device >= 0) {
        cudaDeviceSynchronize();
        cudaFree(p->d_tw);
        cudaFree(p->d_twn_lo);
        cudaFree(p->d_twn_hi);
        cudaFree(p->d_G);
        cudaFree(p->d_Gbf);
        cudaFree(p->d_Gh);
        cudaFree(p->d_tcFh);
        cudaFree(p->d_tcF);
        cudaFree(p->d_tcTw);
        cudaFree(p->d_dimg);
        cudaFree(p->d_dsig);
        cudaFree(p->d_k4order);
        cudaFree(p->d_k4order_a);
        cudaFree(p->d_status);
    }
    for (int s = 0; s < fdas::PROF_STAGES; s++)
        for (int i = 0; i < fdas::PROF_CAP; i++)
            for (int k = 0; k < 2; k++)
                if (p->prof.ev[s][i][k]) cudaEventDestroy(p->prof.ev[s][i][k]);
    delete static_cast<fdas_plan_s *>(plan);
}

}  // extern "C"
