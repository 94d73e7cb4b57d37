// Batched search: many series (dispersion-measure trials) of uneven length and zmax in one call.
//
// A batch holds one plan per series.  Series with the same (N, zmax, taps, segment length,
// precision) form a group that shares one template bank and twiddle tables (built once by the
// group's first plan).  fdas_batch_search runs every series through K1 -> K2/K3 -> K4 back to
// back in one CUDA graph: the graph is captured on a library-owned stream the first time a set
// of buffers is seen and relaunched on the caller's stream afterwards, so a batch costs one
// launch on the host.  All series reuse one workspace and one plane buffer (each sized for the
// largest series): stream order keeps a series' peak search ahead of the next series' plane,
// so the device memory is bounded by the largest series, whatever the batch size.
//
// The autotuner (fdas_batch_autotune) times the FP32 path's candidate segment lengths
// S in {1024, 2048, 4096, 8192} (S >= 2 taps) and templates per correlation CTA
// {1, 2, 4, 8, 16} for each group on the current device, keeps the fastest, and caches the
// choices in a small JSON file keyed by the device and the group's shape.  The tensor-core
// paths have no free launch parameters (4096-bin segments, one persistent CTA per SM), so
// their entries record the fixed choice.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "fdas_internal.cuh"

using fdas::Plan;

struct fdas_plan_s : public fdas::Plan {};

struct fdas_batch_s {
    std::vector<fdas_config> cfg;          // per series (seg_len as tuned)
    std::vector<fdas_plan_s *> plan;       // per series
    std::vector<int> group;                // per series: index of its group
    std::vector<int> leader;               // per group: first series
    std::vector<std::string> key;          // per group: shape key
    std::vector<int64_t> sample_off;       // per series: element offset in the packed input
    std::vector<int64_t> peak_off;         // per series: record offset in the peak buffer
    int64_t total_samples = 0, total_peaks = 0, total_cells = 0;
    size_t ws_series = 0, plane_bytes = 0, ws_bytes = 0;
    bool templates_ready = false;
    int device = -1;
    cudaStream_t cap = nullptr;            // capture stream
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    const void *g_series = nullptr, *g_ws = nullptr, *g_peaks = nullptr, *g_npeaks = nullptr;
    std::string last_error;
};

namespace {

constexpr size_t ALIGN = 256;
size_t align_up(size_t x) { return (x + ALIGN - 1) & ~(ALIGN - 1); }
bool aligned(const void *ptr, uintptr_t a) { return (reinterpret_cast<uintptr_t>(ptr) & (a - 1)) == 0; }

fdas_status record(fdas_batch_s *b, cudaError_t e) {
    if (e == cudaSuccess) return FDAS_OK;
    if (b) b->last_error = std::string(cudaGetErrorName(e)) + ": " + cudaGetErrorString(e);
    (void)cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? FDAS_E_NOMEM : FDAS_E_CUDA;
}

fdas_status plan_one(const fdas_config &c, fdas_plan_s **out) {
    fdas_plan_t h = nullptr;
    size_t ws = 0;
    const fdas_status s = fdas_plan(&c, &h, &ws);
    *out = static_cast<fdas_plan_s *>(h);
    return s;
}

std::string group_key(const fdas_config &c) {
    char buf[160];
    std::snprintf(buf, sizeof buf, "p%d:n%lld:z%d:m%d:s%d", c.precision, (long long)c.n_samples, c.zmax, c.taps,
                  c.seg_len);
    return buf;
}

// Shape key of the autotune cache (segment length excluded: it is what gets chosen).
std::string tune_key(const fdas_config &c, int device) {
    cudaDeviceProp prop{};
    cudaGetDeviceProperties(&prop, device);
    char buf[200];
    std::snprintf(buf, sizeof buf, "sm%d%d_x%d:p%d:n%lld:z%d:m%d", prop.major, prop.minor, prop.multiProcessorCount,
                  c.precision, (long long)c.n_samples, c.zmax, c.taps);
    return buf;
}

// (Re)derive the per-series layout: groups, offsets, the shared workspace and plane buffer.
void layout(fdas_batch_s *b) {
    const int n = (int)b->plan.size();
    b->group.assign(n, -1);
    b->leader.clear();
    b->key.clear();
    b->sample_off.assign(n, 0);
    b->peak_off.assign(n, 0);
    std::map<std::string, int> gid;
    int64_t so = 0, po = 0, cells = 0;
    size_t ws = 0, pl = 0;
    for (int i = 0; i < n; i++) {
        const std::string k = group_key(b->cfg[i]);
        auto it = gid.find(k);
        if (it == gid.end()) {
            it = gid.emplace(k, (int)b->leader.size()).first;
            b->leader.push_back(i);
            b->key.push_back(k);
        }
        b->group[i] = it->second;
        b->sample_off[i] = so;
        b->peak_off[i] = po;
        so += b->cfg[i].n_samples;
        po += b->cfg[i].max_peaks;
        fdas_plan_info info{};
        fdas_plan_get_info(b->plan[i], &info);
        cells += info.cells;
        ws = std::max(ws, info.workspace_bytes);
        pl = std::max(pl, (size_t)info.plane_bytes);
    }
    b->total_samples = so;
    b->total_peaks = po;
    b->total_cells = cells;
    b->ws_series = align_up(ws);
    b->plane_bytes = align_up(pl);
    b->ws_bytes = b->ws_series + b->plane_bytes;
}

void drop_graph(fdas_batch_s *b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    b->g_series = b->g_ws = b->g_peaks = b->g_npeaks = nullptr;
}

// ---------------------------------------------------------------- autotune cache (JSON)
struct TuneChoice {
    int seg_len = 0, zb = 0;
    double ms = 0.0;
};

// One entry per line, as written by save_cache: "  \"key\": {\"seg_len\": S, \"zb\": Z, \"ms\": T},"
std::map<std::string, TuneChoice> load_cache(const char *path) {
    std::map<std::string, TuneChoice> m;
    if (!path) return m;
    FILE *f = std::fopen(path, "r");
    if (!f) return m;
    char line[512];
    while (std::fgets(line, sizeof line, f)) {
        char key[256];
        TuneChoice c;
        if (std::sscanf(line, " \"%255[^\"]\": {\"seg_len\": %d, \"zb\": %d, \"ms\": %lf", key, &c.seg_len, &c.zb,
                        &c.ms) == 4)
            m[key] = c;
    }
    std::fclose(f);
    return m;
}

bool save_cache(const char *path, const std::map<std::string, TuneChoice> &m) {
    if (!path) return true;
    const std::string tmp = std::string(path) + ".tmp";
    FILE *f = std::fopen(tmp.c_str(), "w");
    if (!f) return false;
    std::fprintf(f, "{\n \"fdas_autotune\": 1,\n \"entries\": {\n");
    size_t k = 0;
    for (const auto &kv : m) {
        std::fprintf(f, "  \"%s\": {\"seg_len\": %d, \"zb\": %d, \"ms\": %.6f}%s\n", kv.first.c_str(),
                     kv.second.seg_len, kv.second.zb, kv.second.ms, ++k < m.size() ? "," : "");
    }
    std::fprintf(f, " }\n}\n");
    std::fclose(f);
    return std::rename(tmp.c_str(), path) == 0;
}

// Median-free timing: the best of `reps` event-timed fdas_plane calls (after one warm-up).
fdas_status time_plane(const fdas_config &c, int zb, cudaStream_t st, double *ms_out, std::string &err) {
    fdas_plan_s *p = nullptr;
    fdas_status s = plan_one(c, &p);
    if (s != FDAS_OK) return s;
    p->tune_zb = zb;
    s = fdas_make_templates(p, st);
    void *ws = nullptr, *xh = nullptr, *pl = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    fdas_plan_info info{};
    fdas_plan_get_info(p, &info);
    cudaError_t e = cudaSuccess;
    if (s == FDAS_OK) {
        e = cudaMalloc(&ws, info.workspace_bytes);
        if (e == cudaSuccess) e = cudaMalloc(&xh, sizeof(float2) * (size_t)info.nb);
        if (e == cudaSuccess) e = cudaMalloc(&pl, (size_t)info.plane_bytes);
        if (e == cudaSuccess) e = cudaMemsetAsync(xh, 0, sizeof(float2) * (size_t)info.nb, st);
        if (e == cudaSuccess) e = cudaEventCreate(&e0);
        if (e == cudaSuccess) e = cudaEventCreate(&e1);
        double best = 1e30;
        for (int r = 0; r < 4 && e == cudaSuccess && s == FDAS_OK; r++) {
            cudaEventRecord(e0, st);
            s = fdas_plane(p, static_cast<const float *>(xh), ws, pl, st);
            cudaEventRecord(e1, st);
            e = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (r > 0) best = std::min(best, (double)ms);
        }
        *ms_out = best;
    }
    if (e != cudaSuccess) err = std::string(cudaGetErrorName(e)) + ": " + cudaGetErrorString(e);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(ws);
    cudaFree(xh);
    cudaFree(pl);
    fdas_destroy(p);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? FDAS_E_NOMEM : FDAS_E_CUDA;
    return s;
}

}  // namespace

extern "C" {

fdas_status fdas_batch_plan(const fdas_config *cfgs, int32_t n_series, fdas_batch_t *batch, size_t *workspace_bytes) {
    if (!cfgs || !batch || n_series <= 0) return FDAS_E_INVALID;
    *batch = nullptr;
    fdas_batch_s *b = new (std::nothrow) fdas_batch_s();
    if (!b) return FDAS_E_NOMEM;
    b->cfg.assign(cfgs, cfgs + n_series);
    for (int i = 0; i < n_series; i++) {
        fdas_plan_s *p = nullptr;
        const fdas_status s = plan_one(b->cfg[i], &p);
        if (s != FDAS_OK) {
            for (fdas_plan_s *q : b->plan) fdas_destroy(q);
            delete b;
            return s;
        }
        b->plan.push_back(p);
    }
    layout(b);
    *batch = b;
    if (workspace_bytes) *workspace_bytes = b->ws_bytes;
    return FDAS_OK;
}

fdas_status fdas_batch_autotune(fdas_batch_t b, const char *cache_path, void *stream) {
    if (!b) return FDAS_E_INVALID;
    if (b->templates_ready) return FDAS_E_STATE;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return record(b, e);
    std::map<std::string, TuneChoice> cache = load_cache(cache_path);
    bool changed = false;
    for (size_t g = 0; g < b->leader.size(); g++) {
        const fdas_config base = b->cfg[b->leader[g]];
        const std::string k = tune_key(base, dev);
        auto it = cache.find(k);
        TuneChoice choice;
        if (it != cache.end()) {
            choice = it->second;
        } else if (base.precision != FDAS_FP32) {
            choice.seg_len = base.seg_len;   // fixed 4096-bin tensor-core segments; nothing to choose
            choice.zb = 0;
            cache[k] = choice;
            changed = true;
        } else {
            double best = 1e30;
            for (int S = 1024; S <= 8192; S *= 2) {
                if (base.taps > S / 2) continue;
                for (int zb = 1; zb <= 16; zb *= 2) {
                    fdas_config c = base;
                    c.seg_len = S;
                    double ms = 0.0;
                    const fdas_status s = time_plane(c, zb, st, &ms, b->last_error);
                    if (s != FDAS_OK) return s;
                    if (ms < best) {
                        best = ms;
                        choice.seg_len = S;
                        choice.zb = zb;
                        choice.ms = ms;
                    }
                }
            }
            cache[k] = choice;
            changed = true;
        }
        // apply: re-plan the group's series with the chosen segment length and tile
        for (size_t i = 0; i < b->plan.size(); i++) {
            if (b->group[i] != (int)g) continue;
            fdas_config c = b->cfg[i];
            if (choice.seg_len > 0 && base.precision == FDAS_FP32) c.seg_len = choice.seg_len;
            fdas_plan_s *p = nullptr;
            const fdas_status s = plan_one(c, &p);
            if (s != FDAS_OK) return s;
            p->tune_zb = choice.zb;
            fdas_destroy(b->plan[i]);
            b->plan[i] = p;
            b->cfg[i] = c;
        }
    }
    layout(b);
    drop_graph(b);
    if (changed && !save_cache(cache_path, cache)) {
        b->last_error = std::string("cannot write the autotune cache ") + cache_path;
        return FDAS_E_INVALID;
    }
    return FDAS_OK;
}

fdas_status fdas_batch_make_templates(fdas_batch_t b, void *stream) {
    if (!b) return FDAS_E_INVALID;
    if (b->templates_ready) return FDAS_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaGetDevice(&b->device);
    if (e != cudaSuccess) return record(b, e);
    for (size_t g = 0; g < b->leader.size(); g++) {
        const fdas_status s = fdas_make_templates(b->plan[b->leader[g]], st);
        if (s != FDAS_OK) {
            b->last_error = fdas_last_error(b->plan[b->leader[g]]);
            return s;
        }
    }
    for (size_t i = 0; i < b->plan.size(); i++) {
        Plan *p = b->plan[i];
        const Plan *l = b->plan[b->leader[b->group[i]]];
        if (p == l) continue;
        p->device = l->device;
        p->d_tw = l->d_tw;
        p->d_twn_lo = l->d_twn_lo;
        p->d_twn_hi = l->d_twn_hi;
        p->d_G = l->d_G;
        p->d_Gbf = l->d_Gbf;
        p->d_tcF = l->d_tcF;
        p->d_tcTw = l->d_tcTw;
        p->d_Gh = l->d_Gh;
        p->d_tcFh = l->d_tcFh;
        p->d_dimg = l->d_dimg;
        p->d_dsig = l->d_dsig;
        p->d_k4order = l->d_k4order;
        p->k4order_n = l->k4order_n;
        p->borrowed = true;
        e = cudaMalloc((void **)&p->d_status, sizeof(int32_t));
        if (e == cudaSuccess) e = cudaMemsetAsync(p->d_status, 0, sizeof(int32_t), st);
        if (e != cudaSuccess) return record(b, e);
        p->templates_ready = true;
    }
    if (!b->cap) {
        e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
        if (e != cudaSuccess) return record(b, e);
    }
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return record(b, e);
    b->templates_ready = true;
    return FDAS_OK;
}

fdas_status fdas_batch_search(fdas_batch_t b, const float *d_series, void *d_workspace, fdas_peak *d_peaks,
                              int32_t *d_npeaks, void *stream) {
    if (!b || !d_series || !d_workspace || !d_npeaks || (!d_peaks && b->total_peaks > 0)) return FDAS_E_INVALID;
    if (!aligned(d_series, 8) || !aligned(d_workspace, 256) || !aligned(d_peaks, 4) || !aligned(d_npeaks, 4))
        return FDAS_E_INVALID;
    if (!b->templates_ready) return FDAS_E_STATE;
    // every series must start 8-byte aligned inside the packed input
    for (size_t i = 0; i < b->plan.size(); i++)
        if (!aligned(d_series + b->sample_off[i], 8)) return FDAS_E_INVALID;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (!(b->exec && b->g_series == d_series && b->g_ws == d_workspace && b->g_peaks == d_peaks &&
          b->g_npeaks == d_npeaks)) {
        drop_graph(b);
        char *ws = static_cast<char *>(d_workspace);
        void *plane = ws + b->ws_series;
        cudaError_t e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return record(b, e);
        for (size_t i = 0; i < b->plan.size() && e == cudaSuccess; i++) {
            const Plan &p = *b->plan[i];
            e = fdas::launch_spectrum(p, d_series + b->sample_off[i], ws, b->cap);
            float2 *x = reinterpret_cast<float2 *>(ws + p.ws_x);
            const float *scale = reinterpret_cast<const float *>(ws + p.ws_scale + 8);
            if (e == cudaSuccess && p.cfg.norm_block) {
                e = fdas::launch_local_norm(p, x, x, b->cap);
                scale = nullptr;
            }
            uint8_t *l1flag = fdas::level1_fusable(p) ? reinterpret_cast<uint8_t *>(ws + p.ws_l1flag) : nullptr;
            if (e == cudaSuccess) e = fdas::launch_plane_any(p, x, scale, ws, plane, b->cap, l1flag);
            if (e == cudaSuccess)
                e = fdas::launch_peaks(p, plane, p.cfg.precision == FDAS_BF16 || p.cfg.precision == FDAS_BF16_DIRECT,
                                       ws, d_peaks + b->peak_off[i],
                                       d_npeaks + i, (uint32_t)i, b->cap, l1flag);
        }
        cudaGraph_t g = nullptr;
        const cudaError_t e2 = cudaStreamEndCapture(b->cap, &g);
        if (e == cudaSuccess) e = e2;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, g, 0);
        if (e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            b->exec = nullptr;
            return record(b, e);
        }
        b->graph = g;
        b->g_series = d_series;
        b->g_ws = d_workspace;
        b->g_peaks = d_peaks;
        b->g_npeaks = d_npeaks;
    }
    return record(b, cudaGraphLaunch(b->exec, st));
}

fdas_status fdas_batch_get_info(fdas_batch_t b, int32_t *n_series, size_t *workspace_bytes, int64_t *total_samples,
                                int64_t *total_peaks, int64_t *total_cells) {
    if (!b) return FDAS_E_INVALID;
    if (n_series) *n_series = (int32_t)b->plan.size();
    if (workspace_bytes) *workspace_bytes = b->ws_bytes;
    if (total_samples) *total_samples = b->total_samples;
    if (total_peaks) *total_peaks = b->total_peaks;
    if (total_cells) *total_cells = b->total_cells;
    return FDAS_OK;
}

fdas_status fdas_batch_series_info(fdas_batch_t b, int32_t i, fdas_plan_info *info, fdas_config *cfg,
                                   int64_t *sample_offset, int64_t *peak_offset, int32_t *group) {
    if (!b || i < 0 || i >= (int32_t)b->plan.size()) return FDAS_E_INVALID;
    if (info) fdas_plan_get_info(b->plan[i], info);
    if (cfg) *cfg = b->cfg[i];
    if (sample_offset) *sample_offset = b->sample_off[i];
    if (peak_offset) *peak_offset = b->peak_off[i];
    if (group) *group = b->group[i];
    return FDAS_OK;
}

fdas_status fdas_batch_device_status(fdas_batch_t b, int32_t *bits, int clear) {
    if (!b || !bits) return FDAS_E_INVALID;
    int32_t acc = 0;
    for (fdas_plan_s *p : b->plan) {
        int32_t v = 0;
        const fdas_status s = fdas_device_status(p, &v, clear);
        if (s != FDAS_OK) return s;
        acc |= v;
    }
    *bits = acc;
    return FDAS_OK;
}

const char *fdas_batch_last_error(fdas_batch_t b) { return b ? b->last_error.c_str() : ""; }

void fdas_batch_destroy(fdas_batch_t b) {
    if (!b) return;
    if (b->device >= 0) cudaDeviceSynchronize();
    drop_graph(b);
    if (b->cap) cudaStreamDestroy(b->cap);
    // followers first: they borrow their group leader's device memory
    for (size_t i = 0; i < b->plan.size(); i++)
        if (b->plan[i]->borrowed) fdas_destroy(b->plan[i]);
    for (size_t i = 0; i < b->plan.size(); i++)
        if (!b->plan[i]->borrowed) fdas_destroy(b->plan[i]);
    delete b;
}

}  // extern "C"
